"""Learned Poisson initial guess: GPU forward/backward against an FP64 CPU
reference (central finite differences), training on solver-generated
residuals, and the gain over the solver without it."""

import numpy as np
import pytest

from oracle import nn_oracle
from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


@pytest.mark.parametrize("walls", [False, True])
def test_gradient_matches_fp64_finite_differences(walls):
    shape = (5, 6, 7)
    C = 3
    lat = lbm.Lattice(7, 6, 5, 1, bjerrum=0.7, poisson="mg")
    fluid = np.ones(shape, bool)
    if walls:
        solid, sigma = WL.random_solid(shape, seed=3, fraction=0.15)
        lat.set_walls(solid, sigma)
        fluid = ~solid
    lat.nn_init(hidden=C, seed=11)
    g = np.random.Generator(np.random.PCG64(12))
    params = g.uniform(-0.4, 0.4, size=lat.nn_params().size).astype(np.float32)
    lat.nn_params(params)
    x0 = np.where(fluid, g.standard_normal(shape), 0.0).astype(np.float32)
    L_gpu, grad = lat.nn_loss_grad(x0)
    p64 = params.astype(np.float64)
    L_cpu = nn_oracle.loss(p64, x0.astype(np.float64), fluid, C)
    assert abs(L_gpu - L_cpu) <= 1e-5 * L_cpu
    h = 1e-5
    idx = g.choice(p64.size, size=40, replace=False)
    for k in idx:
        pp, pm = p64.copy(), p64.copy()
        pp[k] += h
        pm[k] -= h
        fd = (nn_oracle.loss(pp, x0, fluid, C) - nn_oracle.loss(pm, x0, fluid, C)) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-3 * np.abs(grad).max() + 1e-4 * abs(fd), (k, grad[k], fd)


@pytest.mark.parametrize("hidden,walls", [(8, False), (8, True), (3, True)])
def test_inference_matches_fp64_forward(hidden, walls):
    """The solver's inference pass (FP16 weights and activations, channel
    pairs for even widths, the generic kernels for odd ones) against the
    FP64 forward pass of the oracle network, on random parameters and a
    random normalised residual.  FP16 keeps about three digits: the bound is
    3% of the largest output, far below what matters for an initial guess
    whose solve iterates to the same tolerance."""
    shape = (6, 8, 10)
    lat = lbm.Lattice(10, 8, 6, 1, bjerrum=0.7, poisson="mg")
    fluid = np.ones(shape, bool)
    if walls:
        solid, sigma = WL.random_solid(shape, seed=13, fraction=0.15)
        lat.set_walls(solid, sigma)
        fluid = ~solid
    lat.nn_init(hidden=hidden, seed=14)
    g = np.random.Generator(np.random.PCG64(15))
    params = g.uniform(-0.3, 0.3, size=lat.nn_params().size).astype(np.float32)
    lat.nn_params(params)
    x0 = np.where(fluid, g.standard_normal(shape), 0.0).astype(np.float32)
    y = lat.nn_infer(x0)
    ref = nn_oracle.forward(params.astype(np.float64), x0.astype(np.float64), fluid, hidden)
    assert np.all(y[~fluid] == 0.0)
    assert np.abs(y - ref).max() <= 3e-2 * np.abs(ref).max(), np.abs(y - ref).max()
    assert np.corrcoef(y[fluid], ref[fluid])[0, 1] > 0.999


def _porous_lattice(n, extrapolate=True):
    wl = WL.porous_spheres(n=n, seed=1238)
    lat = lbm.Lattice(n, n, n, 3, omega_drag=1.0, bjerrum=0.7, poisson="mg", poisson_maxit=200,
                      extrapolate=extrapolate)
    lat.set_walls(wl.solid, wl.sigma)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
    return lat


def test_training_on_solver_residuals_lowers_the_loss():
    lat = _porous_lattice(32)
    lat.step(4)
    lat.nn_init(hidden=8, seed=5)
    lat.nn_collect(16)
    lat.step(16)
    assert lat.nn_stats()["collected"] == 16
    losses = lat.nn_train(epochs=30, lr=5e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0]


def test_learned_guess_gains_over_the_history_start():
    """The network, trained on the residuals the history start leaves (16
    steps of a training run), then used on the same trajectory from the
    same initial state as a run without it: every solve still ends at 1e-8
    and the network lowers the start residual by more than a third.  (The
    V-cycles are not asserted: over 32 held-out steps they come out a few
    cycles either side of the run without the network from one run to the
    next, so the network gains in start residual but not robustly in
    cycles.)"""
    base = _porous_lattice(64)
    base.step(4)
    base.nn_init(hidden=8, seed=3)
    base.nn_collect(16)
    base.step(16)
    base.nn_train(epochs=40, lr=5e-3)
    params = base.nn_params()
    base.destroy()
    cycles, starts = {}, {}
    for use in (False, True):
        lat = _porous_lattice(64)
        if use:
            lat.nn_init(hidden=8, seed=3)
            lat.nn_params(params)
            lat.nn_use(True)
        lat.step(20)
        lat.set_timing(True)
        lat.step(32)
        cycles[use] = lat.get_timing()["poisson_iters"]
        starts[use] = lat.poisson_stats()["start_residual_geomean"]
        assert lat.diagnostics()["poisson_residual"] <= 1e-8
        if use:
            st = lat.nn_stats()
            assert st["tried"] >= 40 and st["kept"] >= 0.8 * st["tried"] and st["mean_ratio"] < 0.66
        lat.destroy()
    assert starts[True] < 0.66 * starts[False], (starts, cycles)
