"""GPU parity at the method's hard edge and of the FP64 diagnostics.

High Schmidt number: omega_drag = 1.980 (Sc = 100) and 1.998 (Sc = 1000),
where the drag relaxes the species velocities almost completely every step
and alternates the sign of the ion flux.  The charged ternary mixture runs
200 steps in a charged slit with an applied field and in a periodic box,
with the spectral and the multigrid Poisson solvers, and must match the
FP64 oracle node by node within 1e-5 (the FP32 bound: relative density
error, momentum error relative to n c_s).

Diagnostics: the FP64 sums of lbm_diagnostics (species masses, total
momentum, net fluid charge) against the oracle's sums of the same state
(Sec. 3: species continuity, total momentum), on a charged slit with a
flowing electrolyte, after 60 steps.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-5
CS = 1.0 / math.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


def _pair(wl, od, solver, solid=None, sigma=None, u0=None):
    nz, ny, nx = wl.shape
    lat = lbm.Lattice(nx, ny, nz, wl.nspecies, omega_visc=wl.omega_visc, omega_drag=od,
                      bjerrum=wl.bjerrum, e_ext=wl.e_ext, poisson=solver, poisson_tol=1e-8,
                      poisson_maxit=500)
    if solid is not None:
        lat.set_walls(solid, sigma)
    for s in range(wl.nspecies):
        n0 = wl.n0[s] if solid is None else np.where(solid, 1.0, wl.n0[s])
        lat.set_species(s, wl.mass[s], wl.valence[s], n0, None if u0 is None else u0[s])
    p = O.Params(wl.omega_visc, od, wl.mass, wl.valence, bjerrum=wl.bjerrum, e_ext=wl.e_ext,
                 solid=solid, sigma=sigma)
    o = O.Oracle(p, wl.shape)
    o.initialise(wl.n0 if solid is None else np.where(solid[None], 0.0, wl.n0), u0)
    return lat, o


def _worst(lat, o, fluid):
    n_o, u_o = o.fields()
    worst = 0.0
    for s in range(n_o.shape[0]):
        n_g, u_g = lat.get_moments(s)
        en = (np.abs(n_g - n_o[s])[fluid] / n_o[s][fluid]).max()
        ej = (np.abs(n_g * u_g - n_o[s] * u_o[s])[:, fluid] / (n_o[s][fluid] * CS)).max()
        worst = max(worst, en, ej)
    return worst


@pytest.mark.parametrize("solver", ["fft", "mg"])
@pytest.mark.parametrize("schmidt", [100.0, 1000.0])
def test_charged_slit_high_schmidt_200_steps(solver, schmidt):
    wl = WL.slit(nx=16, ny=8, width=14, sigma=-0.01, debye=4.0, e_field=1e-4, schmidt=schmidt)
    od = lbm.omega_drag_for_schmidt(1.0, schmidt)
    lat, o = _pair(wl, od, solver, wl.solid, wl.sigma)
    for _ in range(4):
        lat.step(50)
        o.run(50)
        assert lat.diagnostics()["poisson_residual"] <= 1e-8
    err = _worst(lat, o, ~wl.solid)
    assert err <= TOL, (solver, schmidt, err)


@pytest.mark.parametrize("solver", ["fft", "mg"])
@pytest.mark.parametrize("schmidt", [100.0, 1000.0])
def test_charged_bulk_high_schmidt_200_steps(solver, schmidt):
    wl = WL.ternary_bulk(shape=(12, 16, 16), seed=34, spread=3e-3)
    wl.e_ext = (2e-4, -1e-4, 5e-5)
    od = lbm.omega_drag_for_schmidt(1.0, schmidt)
    lat, o = _pair(wl, od, solver)
    lat.step(200)
    o.run(200)
    assert lat.diagnostics()["poisson_residual"] <= 1e-8
    err = _worst(lat, o, np.ones(wl.shape, bool))
    assert err <= TOL, (solver, schmidt, err)


def test_fp64_diagnostics_against_oracle_sums():
    """Species masses, total momentum and net fluid charge of lbm_diagnostics
    against the oracle's FP64 sums of the same state: charged walls, applied
    field, a flowing electrolyte, 60 steps.  A wrong factor or a dropped
    species in any sum fails (the momentum is ~2% of M c_s, the charge ~1%
    of the ion mass)."""
    wl = WL.slit(nx=16, ny=8, width=14, sigma=-0.01, debye=4.0, e_field=1e-4, schmidt=10.0)
    g = np.random.Generator(np.random.PCG64(58))
    u0 = np.zeros((3, 3) + wl.shape)
    u0[:, 0] = 0.02
    u0 += g.uniform(-0.005, 0.005, size=u0.shape)
    u0 = np.where(wl.solid[None, None], 0.0, u0)
    od = lbm.omega_drag_for_schmidt(1.0, 10.0)
    lat, o = _pair(wl, od, "mg", wl.solid, wl.sigma, u0=u0)
    lat.step(60)
    o.run(60)
    d = lat.diagnostics()
    fl = ~wl.solid
    n_o, u_o = o.fields()
    M = n_o[:, fl].sum(axis=1)
    P = (wl.mass[:, None, None] * n_o[:, None][:, :, fl] * u_o[:, :, fl]).sum(axis=(0, 2))
    Q = (wl.valence[:, None] * n_o[:, fl]).sum()
    assert d["steps"] == 60 and not d["unstable"]
    assert np.all(np.abs(d["mass"] - M) <= 1e-6 * M), (d["mass"], M)
    scale = M.sum() * CS
    assert np.abs(P[0]) > 1e-3 * scale      # the comparison below can see a factor
    assert np.all(np.abs(d["momentum"] - P) <= 1e-6 * scale), (d["momentum"], P)
    qscale = (np.abs(wl.valence) * M).sum()
    assert abs(Q) > 1e-2 * qscale
    assert abs(d["charge"] - Q) <= 1e-6 * qscale, (d["charge"], Q)
