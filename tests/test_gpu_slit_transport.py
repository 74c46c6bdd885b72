"""Charged slit under a field parallel to the walls (Sec. 4): the mass flow
rate, the convective (electro-osmotic) current and the ohmic current
against the theory the paper compares with, at two drag frequencies.

Theory (unit density, wall charge sigma per wall node, h = W / 2,
k = 1 / lambda_D), derived from the model in the Debye-Hueckel limit:
u_x(z) = E (psi(z) - psi_w) / (4 pi l_B nu) with psi = psi_w cosh(k z) /
cosh(k h), psi_w = 4 pi l_B sigma / (k tanh(k h)), so
  I_m  = (E sigma / nu)(2 / k^2)(1 - k h / tanh(k h))     (Eq. theomassflow)
  I_eo = -(E sigma^2 / (nu k tanh^2(k h)))
         [(k h + sinh(2 k h) / 2) / cosh^2(k h) - 2 tanh(k h)]   (Eq. theo)
The wall potential here is ~1e-2 (Debye-Hueckel holds) and lambda_D spans
10 cells, so both hold to a fraction of a percent; the paper's finding that
the solvent moves with the barycentric velocity at large omega_drag and
departs from it at small omega_drag is checked through their difference
(set by the ion drift, of order D, so 1000 times smaller at Sc 1000); the
ohmic current I - I_eo is proportional to D (the ion profiles are the
equilibrium ones at every D)."""

import math

import numpy as np
import pytest

from paper_1507_04891_gb300 import lbm, transport
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


def theory(e, sigma, debye, width, nu):
    k, h = 1.0 / debye, 0.5 * width
    kh = k * h
    im = (e * sigma / nu) * (2.0 / k ** 2) * (1.0 - kh / math.tanh(kh))
    ieo = -(e * sigma ** 2 / (nu * k * math.tanh(kh) ** 2)) * (
        (kh + 0.5 * math.sinh(2 * kh)) / math.cosh(kh) ** 2 - 2.0 * math.tanh(kh))
    return im, ieo


def test_slit_currents_against_theory_at_two_drag_frequencies():
    W, sigma, e, debye = 50, -1e-4, 1e-4, 10.0
    nu = CS2 * (1.0 - 0.5)
    wl = WL.slit(nx=32, ny=8, width=W, sigma=sigma, debye=debye, e_field=e, schmidt=1.0)
    lat = lbm.Lattice(32, 8, W + 2, 3, omega_drag=1.0, bjerrum=wl.bjerrum, e_ext=wl.e_ext,
                      poisson="fft", step_graph=True)
    lat.set_walls(wl.solid, wl.sigma)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
    im_th, ieo_th = theory(e, sigma, debye, W, nu)
    res = {}
    # the double layer forms at Sc = 1; at Sc = 1000 only the drift and the
    # flow readjust (20000 steps: ~13 e-folds of the slowest viscous mode)
    for sc in (1.0, 1000.0):
        od = lbm.omega_drag_for_schmidt(1.0, sc)
        lat.set_plane_omega_drag(np.full(W + 2, od))
        lat.step(20000)
        c = transport.slit_currents(lat, wl.valence, wl.solid)
        assert lat.diagnostics()["poisson_residual"] <= 1e-8
        assert abs(c["I_m"] / im_th - 1) <= 0.01, (sc, c["I_m"], im_th)
        assert abs(c["I_eo"] / ieo_th - 1) <= 0.02, (sc, c["I_eo"], ieo_th)
        res[sc] = (c, CS2 * (1.0 / od - 0.5))
    (c1, d1), (c3, d3) = res[1.0], res[1000.0]
    # solvent and barycentric velocities: close at large omega_drag, apart at
    # small (their difference comes from the ion drift, of order D)
    assert c3["solvent_vs_barycentric"] < 1e-4 < c1["solvent_vs_barycentric"]
    assert c1["solvent_vs_barycentric"] >= 100 * c3["solvent_vs_barycentric"]
    # ohmic current proportional to D
    ohm1, ohm3 = c1["I"] - c1["I_eo"], c3["I"] - c3["I_eo"]
    assert abs((ohm1 / ohm3) / (d1 / d3) - 1) <= 0.02
