"""Host analysis of slit currents (paper_1507_04891_gb300/transport.py) on
prescribed plane sums, and the bulk-conductivity input.

A stand-in lattice returns prescribed plane sums of n and of the mid-step
flux (what lbm_plane_fluxes returns); the currents must be the sums over the
fluid planes of the plane averages, computed here independently in a loop.
The mid-step flux itself is computed on the GPU and checked against the
oracle in tests/test_gpu_plane_fluxes.py."""

import numpy as np

from paper_1507_04891_gb300 import transport
from paper_1507_04891_gb300 import workloads as WL


class FakeLattice:
    def __init__(self, sums):
        self.sums = sums

    def plane_fluxes(self):
        return self.sums.copy()


def test_slit_currents_match_a_direct_loop():
    rng = np.random.default_rng(3)
    S, shape = 3, (6, 2, 3)
    nz, ny, nx = shape
    solid = np.zeros(shape, bool)
    solid[0] = solid[-1] = True
    sums = np.zeros((nz, S, 4))
    for z in range(1, nz - 1):
        n = rng.uniform(0.001, 0.02, size=S)
        n[0] = 1.0 - n[1] - n[2]
        sums[z, :, 0] = n * nx * ny
        sums[z, :, 1:] = rng.normal(0, 1e-4, size=(S, 3)) * nx * ny
    valence = np.array([0.0, 1.0, -1.0])
    c = transport.slit_currents(FakeLattice(sums), valence, solid)
    Im = I = Ieo = 0.0
    for z in range(1, nz - 1):
        n = sums[z, :, 0] / (nx * ny)
        j = sums[z, :, 1] / (nx * ny)
        ux = j.sum() / n.sum()
        Im += j.sum()
        I += sum(valence[a] * j[a] for a in range(S))
        Ieo += sum(valence[a] * n[a] for a in range(S)) * ux
    np.testing.assert_allclose([c["I_m"], c["I"], c["I_eo"]], [Im, I, Ieo], rtol=1e-12, atol=1e-20)
    u0 = sums[1:-1, 0, 1] / sums[1:-1, 0, 0]
    uxb = sums[1:-1, :, 1].sum(1) / sums[1:-1, :, 0].sum(1)
    assert abs(c["solvent_vs_barycentric"] - np.abs(u0 - uxb).max() / np.abs(uxb).max()) < 1e-12


def test_only_whole_fluid_planes_count():
    """A plane with any wall node is not part of the channel."""
    S, shape = 2, (4, 2, 2)
    solid = np.zeros(shape, bool)
    solid[0] = True
    solid[2, 0, 0] = True
    sums = np.zeros((4, S, 4))
    sums[:, :, 0] = 4.0
    sums[:, 0, 1] = [0.0, 1.0, 100.0, 2.0]
    c = transport.slit_currents(FakeLattice(sums), np.array([0.0, 0.0]), solid)
    assert c["I_m"] == (1.0 + 2.0) / 4


def test_bulk_conductivity_input_is_neutral_and_uniform():
    wl = WL.bulk_conductivity(n=8, fraction=0.02, e_field=3e-3)
    assert wl.n0.shape == (3, 8, 8, 8)
    np.testing.assert_allclose(wl.n0.sum(0), 1.0)
    np.testing.assert_allclose((wl.valence[:, None, None, None] * wl.n0).sum(0), 0.0)
    assert np.ptp(wl.n0[1]) == 0.0 and wl.e_ext == (3e-3, 0.0, 0.0)
