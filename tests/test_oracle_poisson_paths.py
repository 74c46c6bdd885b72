"""Pins of the oracle's Poisson paths that the small-lattice pins do not
reach: the conjugate-gradient path used above the direct-solve limit (full
128^3 parity runs take it), and the per-component neutralising background
(a neutralising mean per connected fluid domain) on lattices whose fluid
splits into known pieces."""

import math

import numpy as np
import pytest

from oracle import lbm_oracle as O


def fourier_case(shape):
    z, y, x = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    k = (2 * math.pi / shape[2], 2 * math.pi * 2 / shape[1], 2 * math.pi / shape[0])
    s = np.sin(k[0] * x + 0.4) * np.cos(k[1] * y) + np.cos(k[2] * z - 0.1)
    lam_xy = (2 - 2 * math.cos(k[0])) + (2 - 2 * math.cos(k[1]))
    lam_z = 2 - 2 * math.cos(k[2])
    psi = np.sin(k[0] * x + 0.4) * np.cos(k[1] * y) / lam_xy + np.cos(k[2] * z - 0.1) / lam_z
    return s, psi


def test_cg_path_solves_a_sum_of_fourier_modes():
    """A psi = s for a sum of two eigenvectors of the periodic 7-point
    operator: psi = sum of mode / eigenvalue, both paths, zero mean."""
    shape = (8, 6, 10)
    s, want = fourier_case(shape)
    fluid = np.ones(shape, bool)
    cg = O.PoissonSolver(fluid, direct_limit=0)
    lu = O.PoissonSolver(fluid)
    assert not cg.direct and lu.direct
    for solver in (cg, lu):
        psi = solver.solve(s)
        np.testing.assert_allclose(psi, want, atol=1e-11)
        assert abs(psi.mean()) < 1e-12
        assert solver.residual(psi, s) < 1e-12


def stacked_slits(widths, ny=3, nx=4):
    """Solid planes between slits of the given widths (one plane each side)."""
    nz = sum(w + 1 for w in widths)
    solid = np.zeros((nz, ny, nx), bool)
    z = 0
    for w in widths:
        solid[z] = True
        z += w + 1
    return solid


def test_fluid_components_of_stacked_slits_and_an_enclosed_cell():
    solid = stacked_slits([3, 5, 2])
    ncomp, lab = O.fluid_components(~solid)
    assert ncomp == 3
    fl = ~solid
    labels = np.full(solid.shape, -1)
    labels[fl] = lab
    # each slit is one component, different slits are different ones
    firsts = [labels[1, 0, 0], labels[5, 0, 0], labels[11, 0, 0]]
    assert len(set(firsts)) == 3
    for z0, w, l in ((1, 3, firsts[0]), (5, 5, firsts[1]), (11, 2, firsts[2])):
        assert (labels[z0:z0 + w] == l).all()
    # a fluid cell with six solid face neighbours is a component of its own
    box = np.zeros((5, 5, 5), bool)
    box[1:4, 1:4, 1:4] = True
    box[2, 2, 2] = False
    ncomp, lab = O.fluid_components(~box)
    assert ncomp == 2
    # diagonal contact does not connect (face neighbours only)
    diag = np.ones((4, 4, 4), bool)
    diag[1, 1, 1] = diag[2, 2, 2] = False
    assert O.fluid_components(~diag)[0] == 2


@pytest.mark.parametrize("direct_limit", [70000, 0])
def test_each_component_is_neutralised_and_zero_mean(direct_limit):
    """Charge confined to the second slit of three: the source of every slit
    has zero sum, the first and third slits get psi = 0, and the second gets
    the slit solution of a uniform-plus-mode charge with zero mean."""
    widths = [3, 6, 4]
    solid = stacked_slits(widths, ny=4, nx=6)
    shape = solid.shape
    rho = np.zeros(shape)
    x = np.arange(shape[2])
    rho[5:11] = 0.2 + 0.05 * np.cos(2 * math.pi * x / shape[2])     # slit 2 only
    p = O.Params(1.0, 1.0, [1.0], [0.0], bjerrum=0.7, solid=solid)
    s = O.poisson_source(rho, p, shape)
    fl = ~solid
    for z0, w in ((1, 3), (5, 6), (12, 4)):
        assert abs(s[z0:z0 + w].sum()) < 1e-12
    assert np.abs(s[1:4]).max() == 0 and np.abs(s[12:16]).max() == 0
    # the uniform part is removed: what is left is the x-mode, 4 pi l_B times it
    mode = np.broadcast_to(np.cos(2 * math.pi * x / shape[2]), s[5:11].shape)
    np.testing.assert_allclose(s[5:11], 4 * math.pi * 0.7 * 0.05 * mode, atol=1e-13)
    solver = O.PoissonSolver(fl, direct_limit=direct_limit)
    psi = solver.solve(s)
    assert np.abs(psi[1:4]).max() < 1e-13 and np.abs(psi[12:16]).max() < 1e-13
    # inside the slit the x-mode is uniform in z and y, and the walls are
    # Neumann: psi = s / (2 - 2 cos(2 pi / nx))
    lam = 2 - 2 * math.cos(2 * math.pi / shape[2])
    np.testing.assert_allclose(psi[5:11], s[5:11] / lam, atol=1e-11)
    assert abs(psi[5:11].mean()) < 1e-13
