"""Batched slit instances stacked along z in one lattice, whole-step CUDA
graphs with a device-side Poisson loop, per-plane drag frequency, and the
autotuner.  Checked against independent runs of each instance and the
FP64 oracle."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
CS = 1.0 / math.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


def _instances():
    return [WL.slit(nx=16, ny=8, width=w, sigma=sg, debye=4.0, e_field=1e-4, schmidt=sc)
            for w, sg, sc in [(6, -0.01, 1.0), (11, -0.004, 30.0), (9, -0.02, 300.0)]]


def _single(wl, storage="fp32", step_graph=False):
    nz, ny, nx = wl.shape
    lat = lbm.Lattice(nx, ny, nz, 3, omega_visc=wl.omega_visc,
                      omega_drag=lbm.omega_drag_for_schmidt(wl.omega_visc, wl.schmidt),
                      bjerrum=wl.bjerrum, e_ext=wl.e_ext, storage=storage, poisson="fft",
                      step_graph=step_graph)
    lat.set_walls(wl.solid, wl.sigma)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
    return lat


def test_step_graph_matches_host_driven_steps():
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=35, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    lats = []
    for graph in (False, True):
        lat = lbm.Lattice(32, 16, 12, 3, omega_drag=od, bjerrum=0.7, poisson="fft",
                          step_graph=graph)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
        lats.append(lat)
    lats[0].step(30)
    st = lats[1].step(30)
    assert st == lbm.LBM_OK
    d = lats[1].diagnostics()
    assert d["steps"] == 30 and d["poisson_residual"] <= 1e-8 and 1 <= d["poisson_iters"] <= 3
    for s in range(3):
        a, ua = lats[0].get_moments(s)
        b, ub = lats[1].get_moments(s)
        assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max()
        assert np.abs(a * ua - b * ub).max() <= 1e-9


def test_stacked_slits_equal_independent_instances():
    insts = _instances()
    lat, z0 = lbm.stack_slits(insts, storage="fp32", step_graph=True)
    assert z0 == [0, insts[0].shape[0], insts[0].shape[0] + insts[1].shape[0]]
    assert lat.step(60) == lbm.LBM_OK
    for i, wl in enumerate(insts):
        one = _single(wl)
        one.step(60)
        nz = wl.shape[0]
        for s in range(3):
            n1, u1 = one.get_moments(s)
            nb, ub = lat.get_moments(s)
            nb, ub = nb[z0[i]:z0[i] + nz], ub[:, z0[i]:z0[i] + nz]
            fl = ~wl.solid
            # the stack stores deviations from one reference density per
            # species (the mean over all channels), a single channel from its
            # own: the same arithmetic rounds differently, so the two agree to
            # FP32 accuracy (the 1e-5 parity bar), not to the last bit
            assert (np.abs(nb - n1)[fl] / n1[fl]).max() <= 1e-5
            assert (np.abs(nb * ub - n1 * u1)[:, fl] / (n1[fl] * CS)).max() <= 1e-5


def test_stacked_slit_against_oracle():
    insts = _instances()
    lat, z0 = lbm.stack_slits(insts, storage="fp32", step_graph=True)
    lat.step(40)
    wl = insts[1]
    od = lbm.omega_drag_for_schmidt(wl.omega_visc, wl.schmidt)
    p = O.Params(wl.omega_visc, od, wl.mass, wl.valence, bjerrum=wl.bjerrum, e_ext=wl.e_ext,
                 solid=wl.solid, sigma=wl.sigma)
    o = O.Oracle(p, wl.shape)
    o.initialise(np.where(wl.solid[None], 0.0, wl.n0))
    o.run(40)
    n_o, u_o = o.fields()
    nz = wl.shape[0]
    fl = ~wl.solid
    for s in range(3):
        nb, ub = lat.get_moments(s)
        nb, ub = nb[z0[1]:z0[1] + nz], ub[:, z0[1]:z0[1] + nz]
        assert (np.abs(nb - n_o[s])[fl] / n_o[s][fl]).max() <= 1e-5
        assert (np.abs(nb * ub - n_o[s] * u_o[s])[:, fl] / (n_o[s][fl] * CS)).max() <= 1e-5


def test_stacked_fp16_within_1e3_of_fp32():
    insts = _instances()
    a, _ = lbm.stack_slits(insts, storage="fp32", step_graph=True)
    b, _ = lbm.stack_slits(insts, storage="fp16", step_graph=True)
    a.step(100)
    b.step(100)
    solid = np.concatenate([w.solid for w in insts])
    fl = ~solid
    for s in range(3):
        na, ua = a.get_moments(s)
        nb, ub = b.get_moments(s)
        assert (np.abs(na - nb)[fl] / na[fl]).max() <= 1e-3
        assert (np.abs(na * ua - nb * ub)[:, fl] / (na[fl] * CS)).max() <= 1e-3


def test_autotune_keeps_state_and_picks_a_size():
    wl = WL.ternary_bulk(shape=(16, 16, 32), seed=36)
    lat = lbm.Lattice(32, 16, 16, 3, omega_drag=1.2, bjerrum=0.7, poisson="fft")
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    lat.step(3)
    before, _ = lat.get_state()
    r = lat.autotune()
    after, _ = lat.get_state()
    assert np.array_equal(before, after)
    assert r["collide_threads"] in (64, 128, 256) and r["charge_threads"] in (64, 128, 256)
    lat.step(2)  # still steps with the chosen sizes
    assert not lat.diagnostics()["unstable"]


def test_stack_rejects_mismatched_instances():
    ok = lbm.Lattice.create_stack(16, 8, [8, 8], [1.0, 1.2], 3, bjerrum=0.7, poisson="fft",
                                  step_graph=True)
    assert ok.shape == (16, 8, 16) and ok.instance_z0(1) == 8 and ok.instance_z0(2) == -1
    cfgs = [lbm.make_config(16, 8, 8, 3, bjerrum=0.7, poisson="fft"),
            lbm.make_config(16, 8, 8, 3, bjerrum=0.5, poisson="fft")]
    with pytest.raises(lbm.LBMError):
        lbm.Lattice(16, 8, 16, 3, _stack=cfgs)


def test_step_graph_with_steps_needing_more_applications_than_baked():
    """The step graph bakes k applications and runs the stream/collide beside
    the final test; a step that needs more runs the while loop and the
    stream/collide again.  A standalone solve capped at one application
    primes the prediction to k = 1 while the steps need two: the graph path
    must still equal the host-driven one.  The solves start from the previous
    potential (no extrapolation), so every step needs two."""
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=36, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    rho0 = (wl.valence[:, None, None, None] * wl.n0).sum(0)
    lats = []
    for graph in (False, True):
        lat = lbm.Lattice(32, 16, 12, 3, omega_drag=od, bjerrum=0.7, poisson="fft",
                          step_graph=graph, extrapolate=False)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
        lat.solve_poisson(rho0, tol=1e-8, maxit=1)    # one application: k = 1 next
        lats.append(lat)
    lats[0].step(20)
    assert lats[1].step(20) == lbm.LBM_OK
    d = lats[1].diagnostics()
    assert d["steps"] == 20 and d["poisson_residual"] <= 1e-8 and d["poisson_iters"] >= 2
    for s in range(3):
        a, ua = lats[0].get_moments(s)
        b, ub = lats[1].get_moments(s)
        assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max()
        assert np.abs(a * ua - b * ub).max() <= 1e-9


def test_step_graph_rerun_uses_refined_potential():
    """A step that needs more applications than the graph bakes runs the
    stream/collide again on the refined potential, from the step's input
    populations into the step's output: the populations then equal the
    host-driven step's exactly (same kernels, same potential).  Keeping the
    speculative result instead (collided on the potential after the baked
    application) changes them by far more than this bound."""
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=36, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    rho0 = (wl.valence[:, None, None, None] * wl.n0).sum(0)
    lats = []
    for graph in (False, True):
        lat = lbm.Lattice(32, 16, 12, 3, omega_drag=od, bjerrum=0.7, poisson="fft",
                          step_graph=graph, extrapolate=False)
        for s in range(3):
            lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
        lat.solve_poisson(rho0, tol=1e-8, maxit=1)    # one application: k = 1 next
        lats.append(lat)
    lats[0].step(3)
    assert lats[1].step(3) == lbm.LBM_OK
    assert lats[1].diagnostics()["poisson_iters"] >= 2
    for s in range(3):
        a = lats[0].get_populations(s)
        b = lats[1].get_populations(s)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
