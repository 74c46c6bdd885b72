"""Host analysis of slit currents (paper_1507_04891_gb300/transport.py) on
synthetic moments with a known answer, and the bulk-conductivity input.

A stand-in lattice returns prescribed densities and bare velocities; the
currents must follow from the mid-step velocities u + F/2 with
F = z E - omega_drag (u + z E / 2 - v): computed here independently per
node, in a loop, and compared with the vectorised analysis."""

import numpy as np

from paper_1507_04891_gb300 import transport
from paper_1507_04891_gb300 import workloads as WL


class FakeLattice:
    def __init__(self, n, u):
        self.n, self.u = n, u

    def get_moments(self, s):
        return self.n[s].copy(), self.u[s].copy()


def test_slit_currents_match_a_direct_loop():
    rng = np.random.default_rng(3)
    S, shape = 3, (6, 2, 3)
    solid = np.zeros(shape, bool)
    solid[0] = solid[-1] = True
    n = rng.uniform(0.001, 0.02, size=(S,) + shape)
    n[0] = 1.0 - n[1] - n[2]
    u = rng.normal(0, 1e-4, size=(S, 3) + shape)
    n[:, solid] = 0.0
    u[:, :, solid] = 0.0
    valence, E, om = np.array([0.0, 1.0, -1.0]), 2e-4, 1.7
    c = transport.slit_currents(FakeLattice(n, u), valence, E, om, solid)
    # direct per-node computation
    Im = I = Ieo = 0.0
    nz, ny, nx = shape
    prof_n = np.zeros((S, nz))
    prof_j = np.zeros((S, nz))
    for zz in range(1, nz - 1):
        for yy in range(ny):
            for xx in range(nx):
                nn = n[:, zz, yy, xx]
                ux = u[:, 0, zz, yy, xx]
                v = sum(nn[b] * (ux[b] + 0.5 * valence[b] * E) for b in range(S)) / nn.sum()
                for a in range(S):
                    F = valence[a] * E - om * (ux[a] + 0.5 * valence[a] * E - v)
                    prof_n[a, zz] += nn[a] / (nx * ny)
                    prof_j[a, zz] += nn[a] * (ux[a] + 0.5 * F) / (nx * ny)
    for zz in range(1, nz - 1):
        rho = prof_n[:, zz].sum()
        uxb = prof_j[:, zz].sum() / rho
        Im += prof_j[:, zz].sum()
        I += sum(valence[a] * prof_j[a, zz] for a in range(S))
        Ieo += sum(valence[a] * prof_n[a, zz] for a in range(S)) * uxb
    np.testing.assert_allclose([c["I_m"], c["I"], c["I_eo"]], [Im, I, Ieo], rtol=1e-12, atol=1e-20)


def test_half_force_shift_of_a_uniform_drift():
    """A neutral pair drifting at the Einstein velocity in its bare moments:
    the drag on force-shifted velocities leaves the mid-step current equal to
    the bare one plus half the field's push, which cancels for +/- ions."""
    shape = (4, 1, 1)
    solid = np.zeros(shape, bool)
    solid[0] = solid[-1] = True
    n = np.zeros((3,) + shape)
    n[:, 1:-1] = np.array([0.98, 0.01, 0.01])[:, None, None, None]
    u = np.zeros((3, 3) + shape)
    u[1, 0, 1:-1], u[2, 0, 1:-1] = 3e-5, -3e-5
    c = transport.slit_currents(FakeLattice(n, u), np.array([0.0, 1.0, -1.0]), 1e-4, 1.5, solid)
    assert abs(c["I_m"]) < 1e-18
    assert c["I"] > 0 and abs(c["I_eo"]) < 1e-18


def test_bulk_conductivity_input_is_neutral_and_uniform():
    wl = WL.bulk_conductivity(n=8, fraction=0.02, e_field=3e-3)
    assert wl.n0.shape == (3, 8, 8, 8)
    np.testing.assert_allclose(wl.n0.sum(0), 1.0)
    np.testing.assert_allclose((wl.valence[:, None, None, None] * wl.n0).sum(0), 0.0)
    assert np.ptp(wl.n0[1]) == 0.0 and wl.e_ext == (3e-3, 0.0, 0.0)
