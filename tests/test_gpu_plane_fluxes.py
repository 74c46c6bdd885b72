"""lbm_plane_fluxes against the FP64 oracle: per z-plane and species, the sums
of n^a and of the mid-step flux n^a (u^a + F^a / 2) (Eq. ourforc's velocity,
F^a the drag on force-shifted velocities and the electric force of Sec. 2),
with the potential of the last solve (the oracle's StepInfo.psi of the last
step).  A charged slit with a field along the walls, and a periodic charged
mixture with a field in every direction."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1507_04891_gb300 import lbm, transport
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
CS = 1.0 / math.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


def oracle_plane_sums(o, info, half_force=True):
    p = o.p
    n, ua = o.fields()
    grad = O.potential_gradient(info.psi, p)
    fel = O.electric_acceleration(p.valence, grad, p.e_ext)
    fd = O.drag_acceleration(n, O.drag_velocity(ua, fel), p.omega_drag)
    F = np.where(o.fluid[None, None], fel + fd, 0.0)
    flux = n[:, None] * (ua + (0.5 * F if half_force else 0.0))
    out = np.zeros((o.shape[0], n.shape[0], 4))
    out[:, :, 0] = n.sum(axis=(2, 3)).T
    out[:, :, 1:] = flux.sum(axis=(3, 4)).transpose(2, 0, 1)
    return out


def run_pair(wl, od, solver, steps, solid=None, sigma=None):
    nz, ny, nx = wl.shape
    lat = lbm.Lattice(nx, ny, nz, 3, omega_drag=od, bjerrum=wl.bjerrum, e_ext=wl.e_ext,
                      poisson=solver)
    if solid is not None:
        lat.set_walls(solid, sigma)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s] if solid is None else np.where(solid, 1.0, wl.n0[s]))
    p = O.Params(1.0, od, wl.mass, wl.valence, bjerrum=wl.bjerrum, e_ext=wl.e_ext, solid=solid,
                 sigma=sigma)
    o = O.Oracle(p, wl.shape)
    o.initialise(wl.n0 if solid is None else np.where(solid[None], 0.0, wl.n0))
    lat.step(steps)
    info = o.run(steps)
    return lat, o, info


def check(lat, o, info):
    g = lat.plane_fluxes()
    ref = oracle_plane_sums(o, info)
    area = o.shape[1] * o.shape[2]
    # densities to FP32 parity; fluxes relative to the plane's n c_s
    scale = ref[:, :, :1] + 1e-300
    assert np.all(np.abs(g[:, :, 0] - ref[:, :, 0]) <= 1e-5 * scale[:, :, 0])
    # a plane sum of per-node errors within the FP32 bound (1e-5 n c_s)
    # whose signs vary: within 2e-6 n c_s summed over the plane
    tol = 2e-6 * CS * ref[:, :, :1] + 1e-12 * area
    assert np.all(np.abs(g[:, :, 1:] - ref[:, :, 1:]) <= tol), np.abs(g[:, :, 1:] - ref[:, :, 1:]).max()
    # the half-force part of the flux is well above the tolerance: a dropped
    # or wrong force term fails the comparison above
    bare = oracle_plane_sums(o, info, half_force=False)
    assert np.abs(ref[:, :, 1:] - bare[:, :, 1:]).max() > 5 * tol.max()
    return g, ref


@pytest.mark.parametrize("solver", ["fft", "mg"])
def test_slit_plane_fluxes_against_oracle(solver):
    wl = WL.slit(nx=16, ny=8, width=14, sigma=-0.01, debye=4.0, e_field=2e-3, schmidt=10.0)
    od = lbm.omega_drag_for_schmidt(1.0, 10.0)
    lat, o, info = run_pair(wl, od, solver, 40, wl.solid, wl.sigma)
    g, _ = check(lat, o, info)
    # the slit analysis sums the library's plane values over the fluid planes
    c = transport.slit_currents(lat, wl.valence, wl.solid)
    fl = ~wl.solid.any(axis=(1, 2))
    assert abs(c["I_m"] - g[fl, :, 1].sum() / 128) <= 1e-12 * abs(c["I_m"])


def test_periodic_plane_fluxes_against_oracle():
    wl = WL.ternary_bulk(shape=(12, 8, 16), seed=61, spread=3e-3)
    wl.e_ext = (2e-3, -1e-3, 5e-4)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    lat, o, info = run_pair(wl, od, "fft", 30)
    check(lat, o, info)
