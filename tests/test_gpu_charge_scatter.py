"""The charge density from the previous step's stream/collide.

On periodic FP32 lattices without walls (nx a multiple of 32) the library
does not compute rho_e(t) = sum_a z_a sum_p f_p^a(r, t) of Eq. (Poisson) by a
pass over the pulled populations: the stream/collide of step t - 1 adds each
stored charged population f*_p(r) to the node r + c_p that pulls it, in
64-bit fixed point (the same quantity, summed in another order).  These
tests hold that path to the FP64 oracle node by node over 200 steps (the
FP32 bound 1e-5), to the separate charge pass (LBM_FLAG_CHARGE_PASS) within
FP32 rounding of the source, and check that the source is recomputed when
the populations come from elsewhere (lbm_set_species, lbm_set_state) and
after a step graph's rerun branch.
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


def _lattice(wl, od, **kw):
    nz, ny, nx = wl.shape
    lat = lbm.Lattice(nx, ny, nz, wl.nspecies, omega_visc=wl.omega_visc, omega_drag=od,
                      bjerrum=wl.bjerrum, e_ext=wl.e_ext, poisson_tol=1e-8, poisson_maxit=500,
                      **kw)
    for s in range(wl.nspecies):
        lat.set_species(s, wl.mass[s], wl.valence[s], wl.n0[s])
    return lat


def _oracle(wl, od):
    p = O.Params(wl.omega_visc, od, wl.mass, wl.valence, bjerrum=wl.bjerrum, e_ext=wl.e_ext)
    o = O.Oracle(p, wl.shape)
    o.initialise(wl.n0)
    return o


def _fields(lat, S):
    return [lat.get_moments(s) for s in range(S)]


def _rel_diff(fa, fb):
    worst = 0.0
    for (na, ua), (nb, ub) in zip(fa, fb):
        worst = max(worst, float((np.abs(na - nb) / nb).max()),
                    float((np.abs(na * ua - nb * ub) / (nb * CS)).max()))
    return worst


def _against_oracle(lat, o, S):
    n_o, u_o = o.fields()
    return _rel_diff(_fields(lat, S), [(n_o[s], u_o[s]) for s in range(S)])


@pytest.mark.parametrize("solver,graph", [("fft", False), ("fft", True), ("mg", False)])
def test_scattered_charge_matches_oracle_200_steps(solver, graph):
    """Charged ternary, 32 x 16 x 12 periodic (a row is one warp, its x wrap
    stays inside the warp), Sc 3 and an applied field: per node within 1e-5
    of the oracle after 200 steps, and within 1e-7 of the same lattice with
    the charge pass."""
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=52, spread=3e-3)
    wl.e_ext = (1e-4, -5e-5, 0.0)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    kw = dict(poisson=solver, step_graph=graph)
    lat = _lattice(wl, od, **kw)
    ref = _lattice(wl, od, charge_pass=True, **kw)
    o = _oracle(wl, od)
    for _ in range(4):
        lat.step(50)
        ref.step(50)
        o.run(50)
        assert lat.diagnostics()["poisson_residual"] <= 1e-8
    assert _against_oracle(lat, o, 3) <= TOL
    assert _rel_diff(_fields(lat, 3), _fields(ref, 3)) <= 1e-7


@pytest.mark.parametrize("nx,ny", [(64, 8), (128, 8), (256, 8)])
def test_scatter_row_layouts_match_the_charge_pass(nx, ny):
    """Rows of 2, 4 and 8 warps (nx = 64, 128, 256: the x-neighbours of a
    warp's first and last lane sit in the next warps, and the last warp's
    wrap to the first), periodic wrap along y over 8 rows and along z over
    4 planes: 40 graph steps within 1e-7 of the charge pass, the species
    masses equal."""
    wl = WL.ternary_bulk(shape=(4, ny, nx), seed=53, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 10.0)
    lat = _lattice(wl, od, poisson="fft", step_graph=True)
    ref = _lattice(wl, od, poisson="fft", step_graph=True, charge_pass=True)
    lat.step(40)
    ref.step(40)
    assert _rel_diff(_fields(lat, 3), _fields(ref, 3)) <= 1e-7
    a = np.array(lat.diagnostics()["mass"])
    b = np.array(ref.diagnostics()["mass"])
    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("graph", [False, True])
def test_source_recomputed_after_new_populations(graph):
    """lbm_set_species and lbm_set_state replace the populations: the next
    step must not take the source the last stream/collide scattered (that
    of the old populations).  The run after the replacement equals a fresh
    lattice started from the same state (up to the Poisson tolerance)."""
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=55, spread=3e-3)
    wl2 = WL.ternary_bulk(shape=(12, 16, 32), seed=56, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    kw = dict(poisson="fft", step_graph=graph)
    lat = _lattice(wl, od, **kw)
    lat.step(7)
    for s in range(3):
        lat.set_species(s, wl2.mass[s], wl2.valence[s], wl2.n0[s])
    lat.step(9)
    fresh = _lattice(wl2, od, **kw)
    fresh.step(9)
    assert _rel_diff(_fields(lat, 3), _fields(fresh, 3)) <= 1e-7
    # set_state back to the state after 9 steps of the fresh lattice
    state, step = fresh.get_state()
    fresh.step(6)
    lat.step(11)
    lat.set_state(state, step)
    lat.step(6)
    assert _rel_diff(_fields(lat, 3), _fields(fresh, 3)) <= 1e-7
