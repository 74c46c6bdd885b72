"""The general drag of Sec. 2 on the GPU: a symmetric matrix of pair
frequencies omega^{ab} (gamma^{ab} = omega^{ab} n_b / n for equal masses)
against the FP64 oracle's drag_acceleration (pinned in
tests/test_oracle_pair_drag.py), per node within 1e-5 after 200 steps, and
the diffusion of a dilute tracer at the closed-form rate of its pair
frequencies."""

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


def compare(lat, o, fluid):
    n_o, u_o = o.fields()
    for s in range(n_o.shape[0]):
        n_g, u_g = lat.get_moments(s)
        en = (np.abs(n_g - n_o[s])[fluid] / n_o[s][fluid]).max()
        ej = (np.abs(n_g * u_g - n_o[s] * u_o[s])[:, fluid] / (n_o[s][fluid] * CS)).max()
        assert en <= 1e-5 and ej <= 1e-5, (s, en, ej)


@pytest.mark.parametrize("solver", ["fft", "mg"])
def test_charged_ternary_with_diameter_pair_frequencies(solver):
    """Solvent, cation and anion of diameters 1.0, 0.8, 1.3 (Sec. 2's
    gamma^{ab} with the arithmetic-mean contact diameter), charged slit with
    a field along the walls."""
    W = O.pair_drag_frequencies([1.0, 0.8, 1.3], 1.0)
    wl = WL.slit(nx=16, ny=8, width=14, sigma=-0.01, debye=4.0, e_field=2e-4, schmidt=1.0)
    lat = lbm.Lattice(16, 8, 16, 3, omega_drag=1.0, bjerrum=wl.bjerrum, e_ext=wl.e_ext, poisson=solver)
    lat.set_walls(wl.solid, wl.sigma)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], np.where(wl.solid, 1.0, wl.n0[s]))
    lat.set_drag_matrix(W)
    p = O.Params(1.0, W, wl.mass, wl.valence, bjerrum=wl.bjerrum, e_ext=wl.e_ext, solid=wl.solid,
                 sigma=wl.sigma)
    o = O.Oracle(p, wl.shape)
    o.initialise(np.where(wl.solid[None], 0.0, wl.n0))
    lat.step(200)
    o.run(200)
    compare(lat, o, ~wl.solid)


def test_quaternary_random_symmetric_matrix_with_velocities():
    g = np.random.Generator(np.random.PCG64(81))
    A = g.uniform(0.3, 1.7, size=(4, 4))
    W = 0.5 * (A + A.T)
    shape = (8, 10, 12)
    n0 = g.uniform(0.15, 0.35, size=(4,) + shape)
    u0 = g.uniform(-0.02, 0.02, size=(4, 3) + shape)
    lat = lbm.Lattice(12, 10, 8, 4, omega_drag=1.0)
    for s in range(4):
        lat.set_species(s, 1.0, 0.0, n0[s], u0[s])
    lat.set_drag_matrix(W)
    p = O.Params(1.0, W, np.ones(4), np.zeros(4))
    o = O.Oracle(p, shape)
    o.initialise(n0, u0)
    lat.step(200)
    o.run(200)
    compare(lat, o, np.ones(shape, bool))
    d = lat.diagnostics()
    assert np.abs(d["momentum"] - (n0[:, None] * u0).sum(axis=(0, 2, 3, 4))).max() <= 1e-8 * n0.sum()


def test_tracer_diffuses_with_its_effective_pair_frequency():
    """A dilute third species in a 60/40 mixture feels omega_eff =
    omega^{31} x1 + omega^{32} x2: its concentration mode decays at D q^2,
    D = c_s^2 (1/omega_eff - 1/2) (Sec. 4's lattice diffusivity)."""
    W = np.array([[1.0, 1.2, 0.8], [1.2, 1.0, 1.6], [0.8, 1.6, 1.0]])
    L, x1, eps = 64, 0.6, 1e-3
    basis = np.sin(2 * math.pi * np.arange(L) / L)
    n3 = eps * (1.0 + 0.9 * basis)
    n0 = np.stack([np.full(L, x1), 1.0 - x1 - n3, n3]).reshape((3, 1, 1, L))
    lat = lbm.Lattice(L, 1, 1, 3, omega_drag=1.0)
    for s in range(3):
        lat.set_species(s, 1.0, 0.0, n0[s])
    lat.set_drag_matrix(W)
    amps = []
    for t in range(0, 601, 25):
        if t:
            lat.step(25)
        m = lat.get_moments(2)[0][0, 0]
        amps.append(2.0 / L * ((m - m.mean()) * basis).sum())
    ts = np.arange(0, 601, 25)
    sel = ts >= 100
    rate = -np.polyfit(ts[sel], np.log(np.abs(amps)[sel]), 1)[0]
    w_eff = W[2, 0] * x1 + W[2, 1] * (1.0 - x1 - eps)
    D = (1.0 / w_eff - 0.5) / 3.0
    assert abs(rate / (D * (2 * math.pi / L) ** 2) - 1) < 0.01, (rate, D)


def test_binary_matrix_is_its_cross_frequency():
    wl = WL.binary_random((6, 8, 10), seed=82, schmidt=3.0)
    a = lbm.Lattice(10, 8, 6, 2, omega_drag=1.37)
    b = lbm.Lattice(10, 8, 6, 2, omega_drag=0.5)
    for lat in (a, b):
        for s in range(2):
            lat.set_species(s, 1.0, 0.0, wl.n0[s], wl.u0[s])
    b.set_drag_matrix([[0.1, 1.37], [1.37, 1.9]])
    a.step(20)
    b.step(20)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    b.set_drag_matrix(None)


def test_drag_matrix_argument_errors():
    lat = lbm.Lattice(4, 4, 4, 3, omega_drag=1.0)
    for bad in ([[1, 1.2, 0.8], [1.1, 1, 1.0], [0.8, 1.0, 1]],      # asymmetric
                [[1, 2.0, 0.8], [2.0, 1, 1.0], [0.8, 1.0, 1]],      # out of range
                [[1, 0.0, 0.8], [0.0, 1, 1.0], [0.8, 1.0, 1]]):
        with pytest.raises(lbm.LBMError) as e:
            lat.set_drag_matrix(bad)
        assert e.value.status == lbm.LBM_EINVAL
    lat.set_plane_omega_drag(np.full(4, 1.2))
    with pytest.raises(lbm.LBMError):
        lat.set_drag_matrix(np.full((3, 3), 1.0))
