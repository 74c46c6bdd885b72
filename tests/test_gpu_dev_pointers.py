"""The device-pointer entry points with torch tensors: lbm_set_species_dev
(initial fields in caller device memory, checked on the device) gives the
same state as lbm_set_species from host memory, lbm_get_moments_dev writes
the same moments as lbm_get_moments into caller device memory on a caller
stream, and invalid fields are rejected."""

import numpy as np
import pytest

from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


@pytest.mark.parametrize("walls", [False, True])
def test_set_species_dev_equals_host_and_moments_dev(walls):
    torch = pytest.importorskip("torch")
    wl = WL.ternary_bulk(shape=(10, 12, 16), seed=71, spread=3e-3)
    g = np.random.Generator(np.random.PCG64(72))
    u0 = g.uniform(-0.01, 0.01, size=(3, 3) + wl.shape)
    solid = sigma = None
    if walls:
        solid, sigma = WL.random_solid(wl.shape, seed=73, fraction=0.1)
    od = lbm.omega_drag_for_schmidt(1.0, 5.0)

    def make():
        lat = lbm.Lattice(16, 12, 10, 3, omega_drag=od, bjerrum=0.7, poisson="mg")
        if walls:
            lat.set_walls(solid, sigma)
        return lat

    n0 = wl.n0 if not walls else np.where(solid[None], 1.0, wl.n0)
    host, devl = make(), make()
    for s in range(3):
        host.set_species(s, 1.0, wl.valence[s], n0[s], u0[s])
    side = torch.cuda.Stream()
    keep = []
    for s in range(3):
        tn = torch.from_numpy(np.ascontiguousarray(n0[s])).cuda()
        tu = torch.from_numpy(np.ascontiguousarray(u0[s])).cuda()
        keep += [tn, tu]
        torch.cuda.synchronize()
        devl.set_species_dev(s, 1.0, wl.valence[s], tn.data_ptr(), tu.data_ptr(), stream=side.cuda_stream)
    # the reference density n_ref is summed in another order on the device:
    # the states agree to FP32 rounding of the stored deviations
    a, _ = host.get_state()
    b, _ = devl.get_state()
    assert np.abs(a - b).max() <= 1e-6
    host.step(7)
    devl.step(7, stream=side.cuda_stream)
    N = host.N
    for s in range(3):
        tn = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
        tu = torch.full((3 * N,), -1.0, dtype=torch.float64, device="cuda")
        devl.get_moments_dev(s, tn.data_ptr(), tu.data_ptr(), stream=side.cuda_stream)
        side.synchronize()
        n_ref, u_ref = host.get_moments(s)
        n_dev = tn.cpu().numpy().reshape(host.shape)
        u_dev = tu.cpu().numpy().reshape((3,) + host.shape)
        fl = np.ones(host.shape, bool) if solid is None else ~solid
        assert np.abs(n_dev - n_ref)[fl].max() <= 1e-6 * n_ref[fl].max()
        assert np.abs(n_dev * u_dev - n_ref * u_ref)[:, fl].max() <= 1e-7
        if solid is not None:
            assert np.all(n_dev[solid] == 0.0)


def test_set_species_dev_rejects_invalid_fields():
    torch = pytest.importorskip("torch")
    lat = lbm.Lattice(8, 8, 8, 2)
    bad = torch.full((512,), 0.5, dtype=torch.float64, device="cuda")
    bad[77] = -0.1
    with pytest.raises(lbm.LBMError) as e:
        lat.set_species_dev(0, 1.0, 0.0, bad.data_ptr())
    assert e.value.status == lbm.LBM_EINVAL
    bad[77] = float("nan")
    with pytest.raises(lbm.LBMError):
        lat.set_species_dev(0, 1.0, 0.0, bad.data_ptr())
    ok = torch.full((512,), 0.5, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * 512, dtype=torch.float64, device="cuda")
    u[5] = float("inf")
    with pytest.raises(lbm.LBMError):
        lat.set_species_dev(0, 1.0, 0.0, ok.data_ptr(), u.data_ptr())
    lat.set_species_dev(0, 1.0, 0.0, ok.data_ptr())
    lat.set_species_dev(1, 1.0, 0.0, ok.data_ptr())
    d = lat.diagnostics()
    assert abs(d["mass"][0] - 256.0) < 1e-9 and not d["unstable"]


def test_moments_into_pinned_host_memory_and_refusals():
    """lbm_get_moments_dev writes pinned host buffers directly (the same
    values as through device buffers); pageable host memory is refused before
    any kernel runs."""
    torch = pytest.importorskip("torch")
    wl = WL.ternary_bulk(shape=(10, 8, 16), seed=61, spread=3e-3)
    lat = lbm.Lattice(16, 8, 10, 3, omega_drag=1.0, bjerrum=0.7, poisson="fft")
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    lat.step(3)
    N = 16 * 8 * 10
    dn = torch.empty(N, dtype=torch.float64, device="cuda")
    du = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    pn = torch.empty(N, dtype=torch.float64).pin_memory()
    pu = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    lat.get_moments_dev(1, dn.data_ptr(), du.data_ptr())
    lat.get_moments_dev(1, pn.data_ptr(), pu.data_ptr())
    lat.synchronize()
    torch.cuda.synchronize()
    assert np.array_equal(dn.cpu().numpy(), pn.numpy())
    assert np.array_equal(du.cpu().numpy(), pu.numpy())
    n_ref, u_ref = lat.get_moments(1)
    assert np.array_equal(n_ref.ravel(), pn.numpy())
    pageable = np.empty(N)
    with pytest.raises(lbm.LBMError):
        lat.get_moments_dev(1, pageable.ctypes.data, None)
    with pytest.raises(lbm.LBMError):
        lat.set_species_dev(0, 1.0, 0.0, pageable.ctypes.data)
