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


def _charged_lattice(n, seed, poisson="mg"):
    wl = WL.ternary_bulk(shape=(n, n, n), seed=seed, schmidt=1.0)
    # both arms of the comparison start each solve from the previous potential
    lat = lbm.Lattice(n, n, n, 3, omega_drag=1.0, bjerrum=0.7, poisson=poisson, poisson_maxit=100,
                      extrapolate=False)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    return lat


def test_training_on_solver_residuals_lowers_the_loss():
    lat = _charged_lattice(24, 41)
    lat.nn_init(hidden=8, seed=5)
    lat.nn_collect(16)
    lat.step(16)
    assert lat.nn_stats()["collected"] == 16
    losses = lat.nn_train(epochs=30, lr=5e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0]


def test_learned_guess_cuts_multigrid_cycles_on_held_out_steps():
    """Train on the first steps of a run, then compare the held-out steps
    from the same state with and without the guess: every solve still ends
    at the 1e-8 residual, the guess lowers the initial residual and the
    number of V-cycles."""
    base = _charged_lattice(32, 42)
    base.nn_init(hidden=8, seed=7)
    base.nn_collect(24)
    base.step(24)
    base.nn_train(epochs=60, lr=5e-3)
    params = base.nn_params()
    state, step = base.get_state()
    psi = base.get_potential()
    cycles = {}
    for use in (False, True):
        lat = _charged_lattice(32, 42)
        lat.set_state(state, step)
        # warm start from the same potential
        rho = sum(z * lat.get_moments(s)[0] for s, z in ((1, 1.0), (2, -1.0)))
        lat.solve_poisson(rho, psi, tol=1e-12)
        if use:
            lat.nn_init(hidden=8, seed=7)
            lat.nn_params(params)
            lat.nn_use(True)
        lat.set_timing(True)
        lat.step(12)
        cycles[use] = lat.get_timing()["poisson_iters"]
        assert lat.diagnostics()["poisson_residual"] <= 1e-8
        if use:
            st = lat.nn_stats()
            assert st["tried"] == 12 and st["kept"] >= 6 and st["mean_ratio"] < 0.9
    assert cycles[True] <= cycles[False]
