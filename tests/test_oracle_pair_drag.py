"""Pins of the oracle's general drag (Sec. 2, gamma^{alpha beta} for equal
masses and species diameters sigma_alpha): the matrix of pair frequencies
reduces to the paper's single omega_drag, conserves momentum when it is
symmetric, follows the paper's diameter dependence, and a tracer species
diffuses with the closed-form coefficient of its pair frequencies."""

import math

import numpy as np
import pytest

from oracle import lbm_oracle as O


def fields(seed, S=3, shape=(3, 4, 5)):
    rng = np.random.default_rng(seed)
    n = rng.uniform(0.1, 1.0, size=(S,) + shape)
    u = rng.uniform(-0.05, 0.05, size=(S, 3) + shape)
    return n, u


def test_equal_pair_frequencies_are_the_single_drag_frequency():
    n, u = fields(1)
    F1 = O.drag_acceleration(n, u, 1.3)
    F2 = O.drag_acceleration(n, u, np.full((3, 3), 1.3))
    assert np.array_equal(F1, F2)


def test_symmetric_matrix_conserves_momentum():
    n, u = fields(2)
    rng = np.random.default_rng(3)
    A = rng.uniform(0.2, 1.8, size=(3, 3))
    W = 0.5 * (A + A.T)
    F = O.drag_acceleration(n, u, W)
    np.testing.assert_allclose((n[:, None] * F).sum(0), 0.0, atol=1e-15)
    # an asymmetric matrix breaks the third principle: the check is not vacuous
    Fa = O.drag_acceleration(n, u, A)
    assert np.abs((n[:, None] * Fa).sum(0)).max() > 1e-4


def test_binary_depends_on_the_cross_frequency_only():
    n, u = fields(4, S=2)
    W = np.array([[0.3, 1.1], [1.1, 1.7]])
    np.testing.assert_array_equal(O.drag_acceleration(n, u, W), O.drag_acceleration(n, u, 1.1))
    np.testing.assert_allclose(O.drag_acceleration(n, u, W)[0],
                               -1.1 * n[1] / n.sum(0) * (u[0] - u[1]), rtol=1e-13)


def test_pair_frequencies_follow_the_contact_diameter():
    """Equal diameters give the paper's omega_drag = (8/3) sigma^2 n
    sqrt(k_B T / (pi m)) g for every pair; sigma_ab is the arithmetic mean,
    entering squared; g_ab multiplies; the matrix is symmetric."""
    n_tot, sig, cs2 = 1.0, 0.9, 1.0 / 3.0
    W = O.pair_drag_frequencies([sig, sig, sig], n_tot)
    ref = 8.0 / 3.0 * sig ** 2 * n_tot * math.sqrt(cs2 / math.pi)
    np.testing.assert_allclose(W, ref, rtol=1e-15)
    W2 = O.pair_drag_frequencies([1.0, 3.0], 2.0, g_contact=[[1.0, 1.5], [1.5, 2.0]], kT_over_m=0.5)
    c = 8.0 / 3.0 * 2.0 * math.sqrt(0.5 / math.pi)
    np.testing.assert_allclose(W2, [[c * 1.0, c * 4.0 * 1.5], [c * 4.0 * 1.5, c * 9.0 * 2.0]], rtol=1e-14)
    assert np.array_equal(W2, W2.T)


def _tracer_rate(W, L=32, eps=1e-3, x1=0.6, steps=200):
    shape = (1, 1, L)
    x = np.arange(L)
    basis = np.sin(2 * math.pi * x / L)
    n3 = eps * (1.0 + 0.9 * basis)
    n0 = np.stack([np.full(L, x1), 1.0 - x1 - n3, n3]).reshape((3,) + shape)
    p = O.Params(1.0, W, [1.0, 1.0, 1.0], [0.0, 0.0, 0.0])
    o = O.Oracle(p, shape)
    o.initialise(n0)
    amp = []
    for t in range(steps + 1):
        m = O.number_density(o.f)[2, 0, 0]
        amp.append(2.0 / L * ((m - m.mean()) * basis).sum())
        if t < steps:
            o.step()
    amp = np.array(amp)
    t = np.arange(len(amp))
    sel = t >= 50
    return -np.polyfit(t[sel], np.log(np.abs(amp[sel])), 1)[0]


def test_tracer_diffuses_with_its_effective_pair_frequency():
    """A dilute third species in a uniform mixture of fractions x1, x2 feels
    the drag omega_eff = omega^{31} x1 + omega^{32} x2 (the background is at
    rest to first order in its dilution), so its concentration mode decays at
    D k^2 with D = v_T^2 (1/omega_eff - 1/2), as the binary diffusivity of
    Sec. 4 with omega_eff for omega_drag."""
    W = np.array([[1.0, 1.2, 0.8],
                  [1.2, 1.0, 1.6],
                  [0.8, 1.6, 1.0]])
    x1, x2 = 0.6, 0.4
    q2 = (2 * math.pi / 32) ** 2
    rate = _tracer_rate(W, x1=x1)
    w_eff = W[2, 0] * x1 + W[2, 1] * x2
    D = O.diffusivity(w_eff)
    assert abs(rate / (D * q2) - 1) < 0.005, (rate, D * q2)
    # weighting by the tracer's own pair frequencies in the other order
    # (omega^{31} with x2, omega^{32} with x1) is 25% off: the pin separates them
    D_wrong = O.diffusivity(W[2, 0] * x2 + W[2, 1] * x1)
    assert abs(D_wrong / D - 1) > 0.2
