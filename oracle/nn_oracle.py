"""FP64 CPU reference of the learned Poisson initial guess (forward pass and
loss), for checking the GPU network's gradients by central finite
differences.

TEST INFRASTRUCTURE ONLY.  The network is not part of the paper's method; it
is this library's addition (an initial guess for the Poisson solve, after
which the plain solver iterates to the same tolerance).  Layout of the
parameter vector: W1[c][ci][o] (c < C, ci < 2, o < 27), b1[c], W2[c][o], with
o = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1).
"""

import numpy as np

from .lbm_oracle import poisson_matrix


def _shift(a, dz, dy, dx):
    """out[z, y, x] = a[z + dz, y + dy, x + dx] on the periodic lattice."""
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def offsets():
    return [(o // 9 - 1, (o // 3) % 3 - 1, o % 3 - 1) for o in range(27)]


def forward(params, x0, fluid, C):
    """y (correction in units of the residual rms) of the two-layer network."""
    params = np.asarray(params, dtype=np.float64)
    W1 = params[:C * 54].reshape(C, 2, 27)
    b1 = params[C * 54:C * 54 + C]
    W2 = params[C * 54 + C:].reshape(C, 27)
    x = [np.asarray(x0, dtype=np.float64), fluid.astype(np.float64)]
    pre = np.zeros((C,) + x0.shape)
    for c in range(C):
        pre[c] += b1[c]
        for o, (dz, dy, dx) in enumerate(offsets()):
            for ci in range(2):
                pre[c] += W1[c, ci, o] * _shift(x[ci], dz, dy, dx)
    hid = np.tanh(pre)
    y = np.zeros(x0.shape)
    for c in range(C):
        for o, (dz, dy, dx) in enumerate(offsets()):
            y += W2[c, o] * _shift(hid[c], dz, dy, dx)
    return np.where(fluid, y, 0.0)


def loss(params, x0, fluid, C):
    """||x0 - A y||^2 / ||x0||^2 over fluid cells, A the finite-volume
    operator of the Poisson solve."""
    A, _ = poisson_matrix(fluid)
    y = forward(params, x0, fluid, C)
    xf = np.asarray(x0, dtype=np.float64)[fluid]
    res = xf - A @ y[fluid]
    return float(res @ res / (xf @ xf))
