"""lbm_get_moments_noalloc, the entry point for callers that must not
allocate device memory, against lbm_get_moments on the same lattice, on two
calls in a row (the static staging array keeps the first call's contents;
the second call must overwrite them).  Collected last on purpose."""

import numpy as np
import pytest

from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


def test_noalloc_moments_match_the_allocating_entry_point_twice():
    wl = WL.ternary_bulk(shape=(16, 32, 32), seed=97, spread=3e-3)
    lat = lbm.Lattice(32, 32, 16, 3, omega_drag=1.3, bjerrum=0.7, poisson="fft")
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    lat.step(5)
    for call in range(2):
        for s in (2, 0, 1):
            n_ref, u_ref = lat.get_moments(s)
            n, u = lat.get_moments_noalloc(s)
            # same kernel, same data: identical to the bit
            assert np.array_equal(n, n_ref), (call, s)
            assert np.array_equal(u, u_ref), (call, s)
        lat.step(3)     # the second call sees a different state


def test_noalloc_rejects_lattices_beyond_the_limit():
    n = 65  # 65^3 > 2^18 nodes
    lat = lbm.Lattice(n, n, n, 1)
    lat.set_species(0, 1.0, 0.0, np.ones((n, n, n)))
    with pytest.raises(lbm.LBMError) as e:
        lat.get_moments_noalloc(0)
    assert e.value.status == lbm.LBM_EINVAL
    assert "LBM_NOALLOC_MAX_NODES" in str(e.value)


def test_noalloc_waits_for_steps_queued_on_a_caller_stream():
    """Steps queued on a caller's stream (a torch side stream), then the
    moments with no synchronisation in between: the call must see the state
    after those steps, as lbm_get_moments does after lbm_synchronize.  A
    neutral lattice, so that lbm_step queues its 50 launches without any
    host read-back."""
    torch = pytest.importorskip("torch")
    wl = WL.binary_random((32, 64, 64), seed=98, schmidt=3.0)
    lat = lbm.Lattice(64, 64, 32, 2, omega_drag=1.4)
    for s in range(2):
        lat.set_species(s, 1.0, 0.0, wl.n0[s], wl.u0[s])
    side = torch.cuda.Stream()
    lat.step(50, stream=side.cuda_stream)
    n, u = lat.get_moments_noalloc(1)
    lat.synchronize()
    n_ref, u_ref = lat.get_moments(1)
    assert np.array_equal(n, n_ref)
    assert np.array_equal(u, u_ref)
    assert lat.diagnostics()["steps"] == 50
