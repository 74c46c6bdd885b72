"""Pins of the FP64 reference of the learned Poisson initial guess
(oracle/nn_oracle.py) to facts outside its own code: the centre tap reduces
the network to y = b tanh(a x0); a single off-centre tap moves a delta input
by the documented offset; the output is linear in the second layer and
periodic-translation equivariant; solid cells give zero; and the loss on a
Fourier mode of the 7-point finite-volume operator, whose eigenvalue is
2 (1 - cos(2 pi / n)), reaches 0 and 1 where that closed form says."""

import math

import numpy as np
import pytest

from oracle import nn_oracle as NN

SHAPE = (4, 5, 6)


def params_of(C, W1=None, b1=None, W2=None):
    W1 = np.zeros((C, 2, 27)) if W1 is None else W1
    b1 = np.zeros(C) if b1 is None else b1
    W2 = np.zeros((C, 27)) if W2 is None else W2
    return np.concatenate([W1.ravel(), b1.ravel(), W2.ravel()])


def centre():
    return 13    # (dz, dy, dx) = (0, 0, 0)


def test_offset_table_is_the_documented_enumeration():
    offs = NN.offsets()
    assert len(offs) == 27 and len(set(offs)) == 27
    assert offs[centre()] == (0, 0, 0)
    assert offs[0] == (-1, -1, -1) and offs[26] == (1, 1, 1)
    assert offs[14] == (0, 0, 1) and offs[16] == (0, 1, 0) and offs[22] == (1, 0, 0)


def test_centre_taps_reduce_to_a_pointwise_tanh():
    rng = np.random.default_rng(5)
    x0 = rng.uniform(-2, 2, SHAPE)
    fluid = np.ones(SHAPE, bool)
    a, b, c0 = 0.7, -1.3, 0.2
    W1 = np.zeros((1, 2, 27)); W1[0, 0, centre()] = a; W1[0, 1, centre()] = c0
    W2 = np.zeros((1, 27)); W2[0, centre()] = b
    y = NN.forward(params_of(1, W1=W1, W2=W2), x0, fluid, 1)
    # the fluid channel is 1 everywhere: it adds c0 like a bias
    assert np.allclose(y, b * np.tanh(a * x0 + c0), rtol=0, atol=1e-15)


@pytest.mark.parametrize("layer", [1, 2])
@pytest.mark.parametrize("o", [14, 16, 22, 0, 26])
def test_single_tap_reads_the_neighbour_at_the_offset(layer, o):
    """A delta at r0 reaches the output at r0 - d (the tap reads x[r + d]),
    wrapping periodically."""
    dz, dy, dx = NN.offsets()[o]
    x0 = np.zeros(SHAPE)
    r0 = (1, 2, 3)
    x0[r0] = 1.0
    fluid = np.ones(SHAPE, bool)
    W1 = np.zeros((1, 2, 27)); W2 = np.zeros((1, 27))
    if layer == 1:
        W1[0, 0, o] = 0.5; W2[0, centre()] = 1.0
    else:
        W1[0, 0, centre()] = 0.5; W2[0, o] = 1.0
    y = NN.forward(params_of(1, W1=W1, W2=W2), x0, fluid, 1)
    want = np.zeros(SHAPE)
    want[(r0[0] - dz) % SHAPE[0], (r0[1] - dy) % SHAPE[1], (r0[2] - dx) % SHAPE[2]] = math.tanh(0.5)
    assert np.allclose(y, want, rtol=0, atol=1e-15)


def test_linear_in_the_second_layer_and_translation_equivariant():
    rng = np.random.default_rng(6)
    C = 3
    x0 = rng.standard_normal(SHAPE)
    fluid = np.ones(SHAPE, bool)
    W1 = rng.standard_normal((C, 2, 27)) * 0.3
    b1 = rng.standard_normal(C) * 0.1
    W2a = rng.standard_normal((C, 27))
    W2b = rng.standard_normal((C, 27))
    f = lambda W2, x: NN.forward(params_of(C, W1, b1, W2), x, fluid, C)
    assert np.allclose(f(2 * W2a - W2b, x0), 2 * f(W2a, x0) - f(W2b, x0), atol=1e-12)
    shift = (1, -2, 3)
    assert np.allclose(f(W2a, np.roll(x0, shift, (0, 1, 2))),
                       np.roll(f(W2a, x0), shift, (0, 1, 2)), atol=1e-12)
    # each hidden channel contributes separately
    one = [f(np.where(np.arange(C)[:, None] == c, W2a, 0.0), x0) for c in range(C)]
    assert np.allclose(sum(one), f(W2a, x0), atol=1e-12)


def test_solid_cells_are_zero_and_the_mask_is_an_input_channel():
    rng = np.random.default_rng(7)
    x0 = rng.standard_normal(SHAPE)
    fluid = np.ones(SHAPE, bool)
    fluid[2, 3, 1] = False
    W1 = np.zeros((1, 2, 27)); W1[0, 1, 14] = 1.0     # reads the mask at x + 1
    W2 = np.zeros((1, 27)); W2[0, centre()] = 1.0
    y = NN.forward(params_of(1, W1=W1, W2=W2), x0, fluid, 1)
    want = np.where(fluid, math.tanh(1.0), 0.0)
    want[2, 3, 0] = 0.0                                # its x + 1 is the solid cell
    assert np.allclose(y, want, rtol=0, atol=1e-15)


def test_loss_on_a_fourier_mode_of_the_operator():
    """x0 = cos(2 pi x / n) on a periodic all-fluid box is an eigenvector of
    the 7-point operator with eigenvalue 2 (1 - cos(2 pi / n)).  With a tiny
    centre tap a and an output tap b the guess is y = b tanh(a x0) ~ a b x0,
    so the loss is (1 - a b lam)^2 up to O(a^2): 1 at b = 0, 0 at
    b = 1/(a lam), 1/4 at half that."""
    nz, ny, nx = 3, 4, 8
    x = np.arange(nx)
    x0 = np.broadcast_to(np.cos(2 * math.pi * x / nx), (nz, ny, nx)).copy()
    fluid = np.ones((nz, ny, nx), bool)
    lam = 2.0 * (1.0 - math.cos(2 * math.pi / nx))
    a = 1e-4
    W1 = np.zeros((1, 2, 27)); W1[0, 0, centre()] = a
    for b, want in ((0.0, 1.0), (1.0 / (a * lam), 0.0), (0.5 / (a * lam), 0.25),
                    (2.0 / (a * lam), 1.0)):
        W2 = np.zeros((1, 27)); W2[0, centre()] = b
        L = NN.loss(params_of(1, W1=W1, W2=W2), x0, fluid, 1)
        assert L == pytest.approx(want, abs=1e-7), b
