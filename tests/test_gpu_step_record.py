"""Per-step diagnostics read back during a multi-step call (lbm_step_record)
against single steps each followed by lbm_diagnostics, for graph-replayed
and host-driven steps, charged with walls and without."""

import numpy as np
import pytest

from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


def _pair(graph, walls):
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=51, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    solid = sigma = None
    if walls:
        solid = np.zeros(wl.shape, bool)
        solid[0] = solid[-1] = True
        sigma = np.where(solid, -0.005, 0.0)
    lats = []
    for _ in range(2):
        lat = lbm.Lattice(32, 16, 12, 3, omega_drag=od, bjerrum=0.7, poisson="fft",
                          step_graph=graph)
        if walls:
            lat.set_walls(solid, sigma)
        for s in range(3):
            n0 = wl.n0[s] if solid is None else np.where(solid, 1.0, wl.n0[s])
            lat.set_species(s, 1.0, wl.valence[s], n0)
        lats.append(lat)
    return lats


@pytest.mark.parametrize("graph,walls", [(True, False), (False, False), (False, True), (True, True)])
def test_step_record_rows_equal_single_step_diagnostics(graph, walls):
    a, b = _pair(graph, walls)
    a.step(2)
    b.step(2)
    K = 12
    rows = b.step_record(K)
    assert rows.shape == (K, 3 + 7)
    for k in range(K):
        a.step(1)
        ref = a.diagnostics()["raw"]
        # same kernels on the same state: the sums agree to rounding of the
        # final FP64 combination at most
        np.testing.assert_allclose(rows[k][:7], ref[:7], rtol=1e-13, atol=1e-13)
        assert rows[k][7] == ref[7]                 # Poisson applications
        assert rows[k][8] == pytest.approx(ref[8], rel=1e-6, abs=1e-14)
        assert rows[k][9] == ref[9] == 2 + k + 1    # steps taken
    # the last row is what lbm_diagnostics reports after the call
    np.testing.assert_allclose(b.diagnostics()["raw"][:7], rows[-1][:7], rtol=1e-13, atol=1e-13)
    # both lattices advanced identically
    for s in range(3):
        na, _ = a.get_moments(s)
        nb, _ = b.get_moments(s)
        assert np.array_equal(na, nb)


def test_step_record_zero_steps_and_chunks():
    a, b = _pair(False, False)
    assert b.step_record(0).shape == (0, 10)
    rows = b.step_record(3)
    assert [int(r[9]) for r in rows] == [1, 2, 3]
