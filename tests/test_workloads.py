"""The seeded input generators produce the workloads they state: shapes,
densities, charges and parameter ranges of the benchmark recipes, seeded
reproducibility, and overall charge neutrality.  (Input generation only:
the module holds none of the method's arithmetic.)"""

import math

import numpy as np
import pytest

from paper_1507_04891_gb300 import workloads as WL


def neutral(wl):
    q = (wl.valence[:, None, None, None] * wl.n0).sum()
    if wl.sigma is not None:
        q += wl.sigma.sum()
    return abs(q)


def test_binary_sinusoid_recipe():
    wl = WL.binary_sinusoid(n=32)
    assert wl.shape == (32, 32, 32) and wl.nspecies == 2
    x = np.arange(32)
    np.testing.assert_allclose(wl.n0[0][5, 7], 0.5 + 0.01 * np.sin(2 * math.pi * x / 32), rtol=0, atol=1e-15)
    np.testing.assert_allclose(wl.n0.sum(0), 1.0, rtol=0, atol=1e-15)
    assert wl.u0 is None and wl.schmidt == 10.0 and wl.omega_visc == 1.0 and wl.steps == 200


def test_ternary_bulk_recipe_and_seed():
    wl = WL.ternary_bulk(shape=(32, 32, 32), seed=1235)
    a, b = wl.n0[1], wl.n0[2]
    assert a.min() >= 0.009 and a.max() <= 0.011 and b.min() >= 0.009 and b.max() <= 0.011
    np.testing.assert_allclose(wl.n0.sum(0), 1.0, rtol=0, atol=1e-15)
    # i.i.d. uniform on [0.009, 0.011]: mean and standard deviation
    assert abs(a.mean() - 0.01) < 5e-6 and abs(a.std() - 2e-3 / math.sqrt(12)) < 5e-6
    assert abs(np.corrcoef(a.ravel(), b.ravel())[0, 1]) < 0.01
    assert list(wl.valence) == [0.0, 1.0, -1.0] and wl.bjerrum == 0.7
    again = WL.ternary_bulk(shape=(32, 32, 32), seed=1235)
    other = WL.ternary_bulk(shape=(32, 32, 32), seed=1236)
    assert np.array_equal(wl.n0, again.n0) and not np.array_equal(wl.n0, other.n0)
    # the benchmark lattice: 128^3 by default
    assert WL.ternary_bulk.__defaults__[0] == 128


def test_slit_defaults_are_the_slit_benchmark():
    """64 x 64 in-plane, 64 fluid planes between two wall planes, -0.01 per
    wall node, Debye length 8, field 1e-4 along x."""
    wl = WL.slit()
    assert wl.shape == (66, 64, 64)
    assert wl.solid[0].all() and wl.solid[-1].all() and not wl.solid[1:-1].any()
    assert np.all(wl.sigma[0] == -0.01) and np.all(wl.sigma[-1] == -0.01)
    assert wl.meta["debye"] == 8.0 and wl.e_ext == (1e-4, 0.0, 0.0)
    assert 1 / math.sqrt(4 * math.pi * wl.bjerrum * wl.meta["nbulk"]) == pytest.approx(8.0, rel=1e-12)
    assert neutral(wl) < 1e-10
    assert np.all(wl.n0[:, 0] == 0) and np.all(wl.n0[:, -1] == 0)


def test_batched_slits_ranges_and_seed():
    insts = WL.batched_slits()
    assert len(insts) == 64
    widths = [w.shape[0] - 2 for w in insts]
    assert min(widths) >= 16 and max(widths) <= 128 and len(set(widths)) > 20
    assert all(w.shape[1:] == (32, 32) for w in insts)
    scs = np.array([w.schmidt for w in insts])
    assert scs.min() >= 1.0 and scs.max() <= 1000.0
    # log-uniform: about half the instances below sqrt(1000)
    assert 20 <= (scs < math.sqrt(1000.0)).sum() <= 44
    sig = np.array([w.meta["sigma"] for w in insts])
    assert sig.min() >= -0.02 and sig.max() <= -0.002
    assert all(neutral(w) < 1e-9 for w in insts)
    again = WL.batched_slits()
    assert [w.shape for w in again] == [w.shape for w in insts]
    assert [w.schmidt for w in again] == [w.schmidt for w in insts]


def test_porous_spheres_recipe_small_box():
    wl = WL.porous_spheres(n=48, rmin=3, rmax=6)
    solid, sig = wl.solid, wl.sigma
    f = solid.mean()
    # stops at the first sphere that reaches the target fraction
    assert 0.20 <= f < 0.20 + (4 / 3) * math.pi * 6 ** 3 / 48 ** 3
    fluid = ~solid
    surface = np.zeros_like(solid)
    for ax in range(3):
        for sh in (1, -1):
            surface |= solid & np.roll(fluid, sh, axis=ax)
    # every surface node carries +/- 0.01, nothing else is charged
    assert np.all(np.abs(sig[surface]) == 0.01) and np.all(sig[~surface] == 0)
    assert (sig > 0).any() and (sig < 0).any()
    # ions neutralise the walls uniformly over the fluid; solid nodes are empty
    assert neutral(wl) < 1e-9
    assert np.all(wl.n0[:, solid] == 0)
    np.testing.assert_allclose(wl.n0[:, fluid].sum(0), 1.0, rtol=0, atol=1e-15)
    assert np.ptp(wl.n0[1][fluid]) == 0 and np.ptp(wl.n0[2][fluid]) == 0


def test_porous_spheres_bounding_boxes_equal_the_whole_grid_recipe():
    """The generator places each sphere through its bounding box; the same
    draws applied to the whole grid (distance of every node to the centre,
    nearest periodic image) give the same solid mask and charges."""
    n, seed = 40, 77
    wl = WL.porous_spheres(n=n, seed=seed, rmin=3, rmax=9)
    rng = np.random.Generator(np.random.PCG64(seed))
    solid = np.zeros((n, n, n), bool)
    sign = np.zeros((n, n, n))
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    while solid.mean() < 0.20:
        c = rng.integers(0, n, size=3)
        r = int(rng.integers(3, 9 + 1))
        s = 1.0 if rng.random() < 0.5 else -1.0
        d2 = sum(((g - ci + n // 2) % n - n // 2) ** 2 for g, ci in zip((zz, yy, xx), c))
        inside = d2 <= r * r
        sign[inside & ~solid] = s
        solid |= inside
    assert np.array_equal(wl.solid, solid)
    assert np.array_equal(np.sign(wl.sigma), np.where(wl.sigma != 0, sign, 0.0))
