"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, node by node.

Tolerance (FP32 arithmetic, 1e-5 relative per node after 200 steps):
  |n_gpu - n_oracle| / n_oracle <= 1e-5,
  |j_gpu - j_oracle| / (n_oracle c_s) <= 1e-5  (j = n u, c_s = 1/sqrt 3).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-5
CS = 1.0 / math.sqrt(3.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_04891_gb300.build import build_library
    build_library()


def make_oracle(wl, omega_drag, solid=None, sigma=None):
    p = O.Params(wl.omega_visc, omega_drag, wl.mass, wl.valence, bjerrum=wl.bjerrum,
                 e_ext=wl.e_ext, solid=solid, sigma=sigma)
    o = O.Oracle(p, wl.shape)
    n0 = wl.n0 if solid is None else np.where(solid[None], 0.0, wl.n0)
    o.initialise(n0, wl.u0)
    return o


def make_gpu(wl, omega_drag, solid=None, sigma=None, **kw):
    nz, ny, nx = wl.shape
    lat = lbm.Lattice(nx, ny, nz, wl.nspecies, omega_visc=wl.omega_visc, omega_drag=omega_drag,
                      bjerrum=wl.bjerrum, e_ext=wl.e_ext, **kw)
    if solid is not None:
        lat.set_walls(solid, sigma)
    for s in range(wl.nspecies):
        n0 = wl.n0[s] if solid is None else np.where(solid, 1.0, wl.n0[s])
        lat.set_species(s, wl.mass[s], wl.valence[s], n0, None if wl.u0 is None else wl.u0[s])
    return lat


def compare_fields(lat, o, fluid=None, tol=TOL):
    n_o, u_o = o.fields()
    fluid = np.ones(o.shape, bool) if fluid is None else fluid
    worst = 0.0
    for s in range(n_o.shape[0]):
        n_g, u_g = lat.get_moments(s)
        en = np.abs(n_g - n_o[s])[fluid] / n_o[s][fluid]
        ej = np.abs(n_g * u_g - n_o[s] * u_o[s])[:, fluid] / (n_o[s][fluid] * CS)
        assert en.max() <= tol, ("density", s, en.max())
        assert ej.max() <= tol, ("momentum", s, ej.max())
        worst = max(worst, en.max(), ej.max())
    return worst


def test_binary_sinusoid_32cubed_200_steps():
    """Neutral binary mixture, 32^3 periodic, Sc = 10, 200 steps."""
    wl = WL.binary_sinusoid(n=32, schmidt=10.0)
    od = lbm.omega_drag_for_schmidt(1.0, 10.0)
    lat = make_gpu(wl, od)
    o = make_oracle(wl, od)
    lat.step(200)
    o.run(200)
    compare_fields(lat, o)


def test_random_binary_ragged_lattice_populations():
    """Ragged extents (not multiples of any tile) and random velocities:
    every population of every node."""
    wl = WL.binary_random((7, 9, 13), seed=31, schmidt=3.0)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    lat = make_gpu(wl, od)
    o = make_oracle(wl, od)
    lat.step(60)
    o.run(60)
    compare_fields(lat, o)
    for s in range(2):
        fg = lat.get_populations(s)
        ref = o.f[s]
        scale = O.W[:, None, None, None] * O.number_density(o.f)[s][None]
        assert (np.abs(fg - ref) / scale).max() <= TOL


@pytest.mark.parametrize("solver", ["mg", "sor"])
def test_charged_ternary_random_walls(solver):
    """Charged walls with random geometry, applied field, Poisson each step."""
    wl = WL.ternary_bulk(shape=(9, 10, 11), seed=32, spread=3e-3)
    wl.e_ext = (2e-4, -1e-4, 5e-5)
    solid, sigma = WL.random_solid(wl.shape, seed=33, fraction=0.12)
    od = lbm.omega_drag_for_schmidt(1.0, 5.0)
    lat = make_gpu(wl, od, solid, sigma, poisson=solver, poisson_tol=1e-8, poisson_maxit=5000)
    o = make_oracle(wl, od, solid, sigma)
    for _ in range(200):
        lat.step(1)
        info = o.step()
        d = lat.diagnostics()
        assert d["poisson_residual"] <= 1e-8
    compare_fields(lat, o, fluid=~solid)
    psi_g = lat.get_potential()
    psi_o = info.psi
    fl = ~solid
    dg = psi_g[fl] - psi_g[fl].mean()
    do = psi_o[fl] - psi_o[fl].mean()
    assert np.abs(dg - do).max() <= 1e-5 * np.abs(do).max()


@pytest.mark.parametrize("solver", ["mg", "fft"])
def test_charged_slit_with_field(solver):
    """Slit between charged walls (MG: trimmed non-periodic Poisson box;
    FFT: x-y transform with a Neumann chain along z)."""
    wl = WL.slit(nx=16, ny=8, width=14, sigma=-0.01, debye=4.0, e_field=1e-4, schmidt=10.0)
    od = lbm.omega_drag_for_schmidt(1.0, 10.0)
    lat = make_gpu(wl, od, wl.solid, wl.sigma, poisson=solver)
    o = make_oracle(wl, od, wl.solid, wl.sigma)
    lat.step(200)
    o.run(200)
    compare_fields(lat, o, fluid=~wl.solid)


@pytest.mark.parametrize("solver", ["mg", "sor", "fft"])
@pytest.mark.parametrize("geometry", ["periodic", "slit", "random"])
def test_standalone_poisson_against_oracle(solver, geometry):
    shape = (16, 8, 32) if solver == "fft" else (16, 12, 20)
    if solver == "fft" and geometry == "random":
        pytest.skip("the spectral solver needs whole fluid or wall planes (checked below)")
    g = np.random.Generator(np.random.PCG64(41))
    solid = sigma = None
    if geometry == "slit":
        solid = np.zeros(shape, bool)
        solid[0] = solid[-1] = True
        sigma = np.where(solid, -0.01, 0.0)
    elif geometry == "random":
        solid, sigma = WL.random_solid(shape, seed=42, fraction=0.1)
    rho = g.uniform(-0.01, 0.01, size=shape)
    nz, ny, nx = shape
    lat = lbm.Lattice(nx, ny, nz, 1, bjerrum=0.7, poisson=solver, poisson_maxit=20000)
    if solid is not None:
        lat.set_walls(solid, sigma)
    psi, iters, res, st = lat.solve_poisson(rho, tol=1e-9)
    assert st == lbm.LBM_OK and res <= 1e-9 and iters >= 1
    p = O.Params(1.0, 1.0, [1.0], [1.0], bjerrum=0.7, solid=solid, sigma=sigma)
    fluid = O.fluid_mask(shape, p)
    s = O.poisson_source(np.where(fluid, rho, 0.0), p, shape)
    solver_o = O.PoissonSolver(fluid)
    # residual of the GPU potential under the oracle's FP64 operator
    assert solver_o.residual(psi, s) <= 2e-9
    ref = solver_o.solve(s)
    d = (psi - psi[fluid].mean())[fluid] - ref[fluid]
    assert np.abs(d).max() <= 1e-7 * np.abs(ref).max()


def test_mass_and_momentum_conservation_fp64_diagnostics():
    wl = WL.binary_random((16, 16, 16), seed=51, schmidt=10.0)
    lat = make_gpu(wl, lbm.omega_drag_for_schmidt(1.0, 10.0))
    d0 = lat.diagnostics()
    lat.step(200)
    d1 = lat.diagnostics()
    assert np.all(np.abs(d1["mass"] / d0["mass"] - 1) <= 1e-6)
    assert np.all(np.abs(d1["momentum"] - d0["momentum"]) <= 1e-6 * d0["mass"].sum() * CS)
    assert d1["steps"] == 200 and not d1["unstable"]


def test_checkpoint_resume_is_bitwise():
    wl = WL.binary_random((8, 10, 12), seed=61)
    od = lbm.omega_drag_for_schmidt(1.0, 10.0)
    lat = make_gpu(wl, od)
    lat.step(7)
    state, step = lat.get_state()
    assert step == 7
    lat.step(9)
    a, _ = lat.get_state()
    lat.set_state(state, step)
    lat.step(9)
    b, stepb = lat.get_state()
    assert stepb == 16
    assert np.array_equal(a, b)


def test_argument_errors():
    lat = lbm.Lattice(6, 5, 4, 2)
    with pytest.raises(lbm.LBMError) as e:
        lat.step(1)
    assert e.value.status == lbm.LBM_EINVAL
    n0 = np.full((4, 5, 6), 0.5)
    lat.set_species(0, 1.0, 0.0, n0)
    with pytest.raises(lbm.LBMError):
        lat.set_species(1, 2.0, 0.0, n0)          # unequal mass
    bad = n0.copy()
    bad[1, 2, 3] = -0.1
    with pytest.raises(lbm.LBMError):
        lat.set_species(1, 1.0, 0.0, bad)         # negative density
    with pytest.raises(lbm.LBMError):
        lat.set_walls(np.zeros((4, 5, 6), bool))  # walls after species
    with pytest.raises(lbm.LBMError):
        lat.set_species(2, 1.0, 0.0, n0)          # index out of range
    with pytest.raises(lbm.LBMError):
        lat.get_potential()                       # neutral lattice
    with pytest.raises(lbm.LBMError):
        lbm.Lattice(4, 4, 4, 1).set_walls(np.ones((4, 4, 4), bool))   # all solid


def test_nan_population_reports_unstable():
    wl = WL.binary_random((4, 4, 4), seed=71)
    lat = make_gpu(wl, 1.0)
    state, step = lat.get_state()
    state[123] = np.nan
    lat.set_state(state, step)
    assert lat.diagnostics()["unstable"]


def test_poisson_iteration_cap_reports_noconv():
    wl = WL.ternary_bulk(shape=(16, 16, 16), seed=81)
    lat = make_gpu(wl, 1.0, poisson="sor", poisson_tol=1e-14, poisson_maxit=10)
    st = lat.step(3, allow_noconv=True)
    assert st == lbm.LBM_ENOCONV
    assert lat.diagnostics()["steps"] == 1


def test_fft_rejects_geometry_it_cannot_solve():
    lat = lbm.Lattice(8, 8, 6, 1, bjerrum=0.7, poisson="fft")
    solid, sigma = WL.random_solid((6, 8, 8), seed=5, fraction=0.1)
    with pytest.raises(lbm.LBMError) as e:
        lat.set_walls(solid, sigma)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError):
        lbm.Lattice(12, 8, 6, 1, bjerrum=0.7, poisson="fft")   # nx not a power of two


def test_fft_stacked_slits_each_neutralised_separately():
    """Three slits of different widths and wall charges stacked along z:
    independent fluid domains, each with its own source mean (oracle reading
    of the neutralising background per connected component)."""
    nx, ny = 16, 8
    widths, sigmas = [5, 9, 12], [-0.01, -0.004, -0.02]
    nz = sum(w + 1 for w in widths)
    solid = np.zeros((nz, ny, nx), bool)
    sigma = np.zeros((nz, ny, nx))
    z = 0
    for w, sg in zip(widths, sigmas):
        solid[z] = True
        sigma[z] = sg
        z += w + 1
    g = np.random.Generator(np.random.PCG64(77))
    rho = np.where(solid, 0.0, g.uniform(-0.003, 0.003, size=solid.shape))
    lat = lbm.Lattice(nx, ny, nz, 1, bjerrum=0.7, poisson="fft", poisson_maxit=50)
    lat.set_walls(solid, sigma)
    psi, iters, res, st = lat.solve_poisson(rho, tol=1e-10)
    assert st == lbm.LBM_OK and res <= 1e-10 and iters <= 4
    p = O.Params(1.0, 1.0, [1.0], [1.0], bjerrum=0.7, solid=solid, sigma=sigma)
    s = O.poisson_source(rho, p, solid.shape)
    so = O.PoissonSolver(~solid)
    assert so.ncomp == 3
    ref = so.solve(s)
    assert so.residual(psi, s) <= 2e-10
    # compare with the per-component means removed
    d = so._zero_mean(psi[~solid]) - ref[~solid]
    assert np.abs(d).max() <= 1e-8 * np.abs(ref).max()


def test_fft_charged_ternary_periodic_steps():
    wl = WL.ternary_bulk(shape=(12, 16, 32), seed=34, spread=3e-3)
    od = lbm.omega_drag_for_schmidt(1.0, 3.0)
    lat = make_gpu(wl, od, poisson="fft")
    o = make_oracle(wl, od)
    for _ in range(200):
        lat.step(1)
        d = lat.diagnostics()
        assert d["poisson_residual"] <= 1e-8 and d["poisson_iters"] <= 3
        o.step()
    compare_fields(lat, o)


@pytest.mark.parametrize("solver", ["mg", "sor"])
def test_poisson_with_isolated_fluid_pockets(solver):
    """Walls that close off single fluid cells: every connected fluid
    component is its own Poisson domain with its own neutralising mean."""
    shape = (12, 10, 16)
    solid, sigma = WL.random_solid(shape, seed=42, fraction=0.1)
    # wall in two single cells completely
    for (z, y, x) in [(3, 4, 5), (8, 2, 11)]:
        solid[z, y, x] = False
        for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            solid[(z + dz) % 12, (y + dy) % 10, (x + dx) % 16] = True
    sigma = np.where(solid, sigma, 0.0)
    g = np.random.Generator(np.random.PCG64(43))
    rho = g.uniform(-0.01, 0.01, size=shape)
    lat = lbm.Lattice(16, 10, 12, 1, bjerrum=0.7, poisson=solver, poisson_maxit=20000)
    lat.set_walls(solid, sigma)
    psi, iters, res, st = lat.solve_poisson(rho, tol=1e-10)
    assert st == lbm.LBM_OK and res <= 1e-10
    p = O.Params(1.0, 1.0, [1.0], [1.0], bjerrum=0.7, solid=solid, sigma=sigma)
    so = O.PoissonSolver(~solid)
    assert so.ncomp >= 3
    s = O.poisson_source(np.where(solid, 0.0, rho), p, shape)
    assert so.residual(psi, s) <= 2e-10
    d = so._zero_mean(psi[~solid]) - so.solve(s)[~solid]
    assert np.abs(d).max() <= 1e-7 * np.abs(so.solve(s)).max()
