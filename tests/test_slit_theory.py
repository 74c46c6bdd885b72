"""The slit theory the transport checks compare with (Sec. 4, Eq.
theomassflow and Eq. theo, as derived from the model in the Debye-Hueckel
limit) against direct quadrature of the profiles it comes from:

  psi(z)   = psi_w cosh(k z) / cosh(k h),  psi_w = 4 pi l_B sigma / (k tanh(k h))
             (psi'' = k^2 psi, psi'(+-h) = +-4 pi l_B sigma: Gauss at a wall of
             charge sigma per unit area),
  rho_e(z) = -psi'' / (4 pi l_B) = -k^2 psi / (4 pi l_B)   (Eq. Poisson),
  u_x(z)   = E (psi(z) - psi_w) / (4 pi l_B nu)   (Stokes with the force
             rho_e E, no slip at the walls),

  I_m = int rho u_x dz (unit density), I_eo = int rho_e u_x dz.

The same closed forms sit in bench.py and the GPU slit test; both are
checked here."""

import math

import pytest
from scipy.integrate import quad

import bench
from tests import test_gpu_slit_transport as gpu_slit

L_B = 0.7


def profiles(e, sigma, debye, width, nu, lb=L_B):
    k, h = 1.0 / debye, 0.5 * width
    psi_w = 4 * math.pi * lb * sigma / (k * math.tanh(k * h))
    psi = lambda z: psi_w * math.cosh(k * z) / math.cosh(k * h)
    rho_e = lambda z: -k * k * psi(z) / (4 * math.pi * lb)
    u = lambda z: e * (psi(z) - psi_w) / (4 * math.pi * lb * nu)
    return k, h, psi, rho_e, u


@pytest.mark.parametrize("ratio", [0.4, 0.2, 0.1])
@pytest.mark.parametrize("sigma", [-1e-4, 2e-3])
def test_closed_forms_equal_the_integrals_of_the_profiles(ratio, sigma):
    W, e, nu = 50.0, 1e-4, 1.0 / 6.0
    debye = ratio * W
    k, h, psi, rho_e, u = profiles(e, sigma, debye, W, nu)
    # the profiles satisfy what they are built from
    dz = 1e-3
    for z in (-0.7 * h, 0.0, 0.3 * h):
        d2 = (psi(z + dz) - 2 * psi(z) + psi(z - dz)) / dz ** 2
        assert d2 == pytest.approx(k * k * psi(z), rel=1e-5)
    slope = (psi(h + dz) - psi(h - dz)) / (2 * dz)
    assert slope == pytest.approx(4 * math.pi * L_B * sigma, rel=1e-6)
    # total charge of the fluid neutralises both walls
    q, _ = quad(rho_e, -h, h, epsabs=0, epsrel=1e-12)
    assert q == pytest.approx(-2 * sigma, rel=1e-9)
    im_q, _ = quad(u, -h, h, epsabs=0, epsrel=1e-12)
    ieo_q, _ = quad(lambda z: rho_e(z) * u(z), -h, h, epsabs=0, epsrel=1e-12)
    for im, ieo in (bench.slit_theory(e, sigma, debye, W, nu),
                    gpu_slit.theory(e, sigma, debye, W, nu)):
        assert im == pytest.approx(im_q, rel=1e-9)
        assert ieo == pytest.approx(ieo_q, rel=1e-9)


def test_mass_flow_tends_to_helmholtz_smoluchowski_plug_flow():
    """Thin double layers: I_m -> 2 h u_HS with u_HS = -E psi_w/(4 pi l_B nu)
    = -E sigma lambda_D / nu (the wall potential psi_w -> 4 pi l_B sigma
    lambda_D): the relative difference is lambda_D / h."""
    W, e, nu, sigma = 50.0, 1e-4, 1.0 / 6.0, -1e-4
    for ratio in (0.02, 0.005):
        debye = ratio * W
        im, _ = bench.slit_theory(e, sigma, debye, W, nu)
        plug = W * (-e * sigma * debye / nu)
        assert im / plug - 1 == pytest.approx(-debye / (0.5 * W), rel=1e-6)
