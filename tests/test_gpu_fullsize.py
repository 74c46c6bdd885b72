"""Full-size checks in the configuration the benchmark times (charged
ternary 128^3, spectral Poisson to 1e-8, FP32): one step against the FP64
oracle at every node, and properties that hold at any size over 50 steps."""

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


def _bench_lattice(wl, storage="fp32"):
    od = lbm.omega_drag_for_schmidt(wl.omega_visc, wl.schmidt)
    lat = lbm.Lattice(128, 128, 128, 3, omega_visc=wl.omega_visc, omega_drag=od, bjerrum=wl.bjerrum,
                      storage=storage, poisson="fft", poisson_tol=1e-8, poisson_maxit=500)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    return lat, od


def test_one_full_size_step_matches_oracle_everywhere():
    wl = WL.ternary_bulk(n=128, seed=1235, schmidt=1.0)
    lat, od = _bench_lattice(wl)
    lat.step(1)
    p = O.Params(wl.omega_visc, od, wl.mass, wl.valence, bjerrum=wl.bjerrum)
    o = O.Oracle(p, wl.shape)
    o.initialise(wl.n0)
    o.step()
    n_o = O.number_density(o.f)
    for s in range(3):
        n_g, u_g = lat.get_moments(s)
        assert (np.abs(n_g - n_o[s]) / n_o[s]).max() <= 1e-5
        j_o = np.einsum("pzyx,pd->dzyx", o.f[s], O.C.astype(float))
        assert (np.abs(n_g * u_g - j_o) / (n_o[s] * CS)).max() <= 1e-5


def test_full_size_invariants_over_50_steps():
    wl = WL.ternary_bulk(n=128, seed=1235, schmidt=1.0)
    lat, _ = _bench_lattice(wl)
    d0 = lat.diagnostics()
    lat.step(50)
    d1 = lat.diagnostics()
    # species mass (FP64 sums of FP32 state) and total momentum
    assert np.all(np.abs(d1["mass"] / d0["mass"] - 1) <= 1e-6)
    assert np.all(np.abs(d1["momentum"]) <= 1e-6 * d0["mass"].sum() * CS)
    # every solve of the run reached the tolerance
    assert d1["poisson_residual"] <= 1e-8 and not d1["unstable"]


def test_full_size_potential_residual_under_oracle_operator():
    wl = WL.ternary_bulk(n=128, seed=1236, schmidt=100.0)
    lat, _ = _bench_lattice(wl)
    lat.step(10)
    rho = lat.get_moments(1)[0] - lat.get_moments(2)[0]
    psi, iters, res, st = lat.solve_poisson(rho, lat.get_potential(), tol=1e-8)
    assert st == lbm.LBM_OK and res <= 1e-8
    fluid = np.ones(wl.shape, bool)
    A, _ = O.poisson_matrix(fluid)
    s = 4 * math.pi * wl.bjerrum * (rho - rho.mean())
    r = s.ravel() - A @ psi.ravel()
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(s)
