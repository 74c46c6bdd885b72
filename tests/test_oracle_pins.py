"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a textbook identity or a brute-force computation.  The
tests are chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand anywhere in the oracle fails at least one of them (the
coverage table is in the design notes).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1507_04891_gb300 import workloads as WL

CS2 = 1.0 / 3.0


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_fields(seed, S=3, shape=(3, 4, 5), umax=0.05):
    g = rng(seed)
    n = g.uniform(0.05, 1.0, size=(S,) + shape)
    ua = g.uniform(-umax, umax, size=(S, 3) + shape)
    u = g.uniform(-umax, umax, size=(3,) + shape)
    F = g.uniform(-umax, umax, size=(S, 3) + shape)
    return n, ua, u, F


def cdot(v):
    """(v . c_p) computed with explicit loops over the velocity list of the
    D3Q19 lattice, independent of the oracle's vectorised helper."""
    out = np.zeros((19,) + v.shape[1:])
    for p in range(19):
        for d in range(3):
            out[p] += O.C[p, d] * v[d]
    return out


# ---------------------------------------------------------------------------
# Lattice tables: textbook D3Q19 isotropy (pins C, W, OPP)
# ---------------------------------------------------------------------------
def test_d3q19_isotropy_and_opposites():
    c = O.C.astype(float)
    w = O.W
    assert c.shape == (19, 3)
    assert len({tuple(v) for v in O.C}) == 19
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("p,pi->i", w, c), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("p,pi,pj->ij", w, c, c), CS2 * np.eye(3), atol=1e-16)
    np.testing.assert_allclose(np.einsum("p,pi,pj,pk->ijk", w, c, c, c), 0, atol=1e-16)
    d = np.eye(3)
    iso4 = CS2 ** 2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                       + np.einsum("il,jk->ijkl", d, d))
    np.testing.assert_allclose(np.einsum("p,pi,pj,pk,pl->ijkl", w, c, c, c, c), iso4, atol=1e-16)
    for p in range(19):
        np.testing.assert_array_equal(O.C[O.OPP[p]], -O.C[p])
    # speeds: 1 rest, 6 of |c|^2 = 1 (w = 1/18), 12 of |c|^2 = 2 (w = 1/36)
    sp2 = (c * c).sum(1)
    assert sp2[0] == 0 and np.all(sp2[1:7] == 1) and np.all(sp2[7:] == 2)
    assert np.all(w[1:7] == 1 / 18) and np.all(w[7:] == 1 / 36)


# ---------------------------------------------------------------------------
# P1: the literal orthogonalised equilibrium equals the textbook second-order
# equilibrium at the species velocity (algebraic identity derived by hand)
# ---------------------------------------------------------------------------
def test_phi_perp_is_equilibrium_at_species_velocity():
    n, ua, u, _ = random_fields(1)
    phi = O.phi_perp(n, ua, u)
    for a in range(n.shape[0]):
        vc = cdot(ua[a])
        vv = (ua[a] ** 2).sum(0)
        ref = n[a] * O.W[:, None, None, None] * (
            1 + 3 * vc + 4.5 * vc ** 2 - 1.5 * vv)
        np.testing.assert_allclose(phi[a], ref, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------------------
# P2: velocity moments of phi_perp and of g_p (Appendix integrals S^1, S^2)
# ---------------------------------------------------------------------------
def test_moments_of_phi_perp_and_forcing():
    n, ua, u, F = random_fields(2)
    c = O.C.astype(float)
    phi = O.phi_perp(n, ua, u)
    g = O.forcing_term(n, F, u)
    for a in range(n.shape[0]):
        np.testing.assert_allclose(phi[a].sum(0), n[a], rtol=1e-14)
        m1 = np.einsum("pzyx,pd->dzyx", phi[a], c)
        np.testing.assert_allclose(m1, n[a] * ua[a], rtol=1e-12, atol=1e-16)
        m2 = np.einsum("pzyx,pi,pj->ijzyx", phi[a], c, c)
        ref2 = n[a] * (CS2 * np.eye(3)[:, :, None, None, None] + ua[a][:, None] * ua[a][None])
        np.testing.assert_allclose(m2, ref2, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(g[a].sum(0), 0, atol=1e-15)
        g1 = np.einsum("pzyx,pd->dzyx", g[a], c)
        np.testing.assert_allclose(g1, n[a] * F[a], rtol=1e-12, atol=1e-16)
        g2 = np.einsum("pzyx,pi,pj->ijzyx", g[a], c, c)
        ref = n[a] * (F[a][:, None] * u[None] + u[:, None] * F[a][None])
        np.testing.assert_allclose(g2, ref, rtol=1e-11, atol=1e-16)


def test_species_and_barycentric_moments():
    """n, u^alpha and u of a hand-built distribution with known moments."""
    n, ua, u, _ = random_fields(3, S=2)
    mass = np.array([1.0, 1.0])
    f = O.phi_perp(n, ua, u)
    fluid = np.ones(n.shape[1:], bool)
    nn = O.number_density(f)
    uu = O.species_velocity(f, nn, fluid)
    np.testing.assert_allclose(nn, n, rtol=1e-14)
    np.testing.assert_allclose(uu, ua, rtol=1e-11, atol=1e-16)
    ub = O.barycentric_velocity(nn, uu, mass)
    ref = (n[0] * ua[0] + n[1] * ua[1]) / (n[0] + n[1])
    np.testing.assert_allclose(ub, ref, rtol=1e-11, atol=1e-16)


def test_drag_closed_forms():
    """Equal masses: sum_beta (n_beta/n)(u^a-u^b) = u^a - u (number mean);
    the drag forces sum to zero (third principle, Eq. globalmomentumcont);
    the binary case reduces to Eq. (gammaab)."""
    n, ua, _, _ = random_fields(4, S=3)
    F = O.drag_acceleration(n, ua, 1.3)
    ubar = (n[:, None] * ua).sum(0) / n.sum(0)
    for a in range(3):
        np.testing.assert_allclose(F[a], -1.3 * (ua[a] - ubar), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose((n[:, None] * F).sum(0), 0, atol=1e-15)
    n2, u2, _, _ = random_fields(5, S=2)
    F2 = O.drag_acceleration(n2, u2, 0.7)
    np.testing.assert_allclose(F2[0], -0.7 * n2[1] / n2.sum(0) * (u2[0] - u2[1]), rtol=1e-12)


# ---------------------------------------------------------------------------
# Streaming and bounce-back: brute force on a delta function
# ---------------------------------------------------------------------------
def test_streaming_moves_delta_by_c_and_bounces_back():
    shape = (5, 6, 7)
    p = O.Params(1.0, 1.0, [1.0], [0.0])
    for q in range(19):
        fs = np.zeros((1, 19) + shape)
        fs[0, q, 2, 3, 4] = 1.0
        out = O.stream(fs, p)
        cz, cy, cx = O.C[q, 2], O.C[q, 1], O.C[q, 0]
        assert out[0, q, (2 + cz) % 5, (3 + cy) % 6, (4 + cx) % 7] == 1.0
        assert out.sum() == 1.0
    # a wall node at r + c_q sends the population back into direction opp(q)
    for q in range(1, 19):
        solid = np.zeros(shape, bool)
        cz, cy, cx = O.C[q, 2], O.C[q, 1], O.C[q, 0]
        solid[(2 + cz) % 5, (3 + cy) % 6, (4 + cx) % 7] = True
        pw = O.Params(1.0, 1.0, [1.0], [0.0], solid=solid)
        fs = np.zeros((1, 19) + shape)
        fs[0, q, 2, 3, 4] = 1.0
        out = O.stream(fs, pw)
        assert out[0, O.OPP[q], 2, 3, 4] == 1.0
        assert out.sum() == 1.0


# ---------------------------------------------------------------------------
# P3 / P4: conservation invariants
# ---------------------------------------------------------------------------
def _oracle_from(wl, omega_drag=None, solid=None, sigma=None, bjerrum=None, e_ext=None):
    od = omega_drag if omega_drag is not None else O.omega_drag_for_schmidt(wl.omega_visc, wl.schmidt)
    p = O.Params(wl.omega_visc, od, wl.mass, wl.valence,
                 bjerrum=wl.bjerrum if bjerrum is None else bjerrum,
                 e_ext=wl.e_ext if e_ext is None else e_ext,
                 solid=wl.solid if solid is None else solid,
                 sigma=wl.sigma if sigma is None else sigma)
    o = O.Oracle(p, wl.shape)
    o.initialise(wl.n0, wl.u0)
    return o


@pytest.mark.parametrize("walls", [False, True])
def test_species_mass_conserved(walls):
    wl = WL.binary_random((6, 5, 7), seed=11)
    solid = sigma = None
    if walls:
        solid, sigma = WL.random_solid(wl.shape, seed=12)
    o = _oracle_from(wl, solid=solid, sigma=sigma)
    m0 = O.number_density(o.f).sum(axis=(1, 2, 3))
    o.run(25)
    m1 = O.number_density(o.f).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(m1, m0, rtol=1e-13)


def test_total_momentum_conserved_neutral():
    wl = WL.binary_random((6, 5, 7), seed=13, schmidt=50.0)
    o = _oracle_from(wl)
    n, u = o.fields()
    p0 = (n[:, None] * u).sum(axis=(0, 2, 3, 4))
    o.run(25)
    n, u = o.fields()
    p1 = (n[:, None] * u).sum(axis=(0, 2, 3, 4))
    np.testing.assert_allclose(p1, p0, atol=1e-13)
    # species momenta do change (drag acts), so the check is not vacuous
    assert np.abs((n[0, None] * u[0]).sum(axis=(1, 2, 3))).max() > 1e-6


def test_total_momentum_conserved_charged():
    """sum_r rho_e grad psi = 0 for the periodic problem: the circulant
    Laplacian and the antisymmetric central difference commute."""
    wl = WL.ternary_bulk(shape=(6, 7, 8), seed=14, spread=3e-3)
    o = _oracle_from(wl)
    n, u = o.fields()
    p0 = (n[:, None] * u).sum(axis=(0, 2, 3, 4))
    o.run(15)
    n, u = o.fields()
    p1 = (n[:, None] * u).sum(axis=(0, 2, 3, 4))
    np.testing.assert_allclose(p1, p0, atol=1e-13)
    assert np.abs((n[1, None] * u[1]).sum(axis=(1, 2, 3))).max() > 1e-9


# ---------------------------------------------------------------------------
# P5: diffusive decay of a concentration mode, D = v_T^2 (1/omega_drag - 1/2)
# ---------------------------------------------------------------------------
def _decay_rate(series, t0, t1):
    t = np.arange(len(series))
    sel = (t >= t0) & (t <= t1)
    slope = np.polyfit(t[sel], np.log(np.abs(series[sel])), 1)[0]
    return -slope


@pytest.mark.parametrize("schmidt", [1.0, 10.0, 100.0])
def test_mutual_diffusion_decay_rate(schmidt):
    L = 32
    wl = WL.binary_sinusoid(n=L, ny=1, nz=1, schmidt=schmidt)
    o = _oracle_from(wl)
    x = np.arange(L)
    basis = np.sin(2 * math.pi * x / L)
    amp = []
    for t in range(201):
        nA = O.number_density(o.f)[0, 0, 0]
        amp.append(2.0 / L * ((nA - nA.mean()) * basis).sum())
        if t < 200:
            o.step()
    amp = np.array(amp)
    D = O.diffusivity(o.p.omega_drag)
    assert abs(D - 1.0 / 6.0 / schmidt) < 1e-15
    rate = _decay_rate(amp, 50, 200)
    q2 = (2 * math.pi / L) ** 2
    assert abs(rate / (D * q2) - 1) < 0.01, (rate, D * q2)


# ---------------------------------------------------------------------------
# P8: shear-wave decay gives nu = v_T^2 (1/omega_visc - 1/2) for any omega_drag
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("omega_visc,omega_drag", [(1.0, 1.0), (1.0, 1.8181818), (1.0, 1.98),
                                                   (1.6, 0.7)])
def test_shear_wave_viscosity_independent_of_drag(omega_visc, omega_drag):
    L = 32
    shape = (L, 1, 1)
    z = np.arange(L)
    u0 = np.zeros((2, 3) + shape)
    u0[:, 0, :, 0, 0] = 1e-3 * np.sin(2 * math.pi * z / L)
    n0 = np.stack([np.full(shape, 0.3), np.full(shape, 0.7)])
    p = O.Params(omega_visc, omega_drag, [1.0, 1.0], [0.0, 0.0])
    o = O.Oracle(p, shape)
    o.initialise(n0, u0)
    basis = np.sin(2 * math.pi * z / L)
    amp = []
    for t in range(161):
        n, u = o.fields()
        jx = (n[:, None] * u).sum(0)[0, :, 0, 0] / n.sum(0)[:, 0, 0]
        amp.append(2.0 / L * (jx * basis).sum())
        o.step()
    rate = _decay_rate(np.array(amp), 10, 160)
    nu = O.viscosity(omega_visc)
    q2 = (2 * math.pi / L) ** 2
    assert abs(rate / (nu * q2) - 1) < 0.01, (rate, nu * q2)


# ---------------------------------------------------------------------------
# P6: omega_drag = omega_visc reduces to the standard mixture BGK up to the
# second-order diffusion-velocity term (derived by hand)
# ---------------------------------------------------------------------------
def test_bgk_limit_closed_form_difference():
    n, ua, _, _ = random_fields(6, S=3)
    mass = np.ones(3)
    f = O.phi_perp(n, ua, O.barycentric_velocity(n, ua, mass))
    f = f * (1 + 0.05 * rng(7).uniform(-1, 1, size=f.shape))   # off-equilibrium
    om = 1.37
    fluid = np.ones(n.shape[1:], bool)
    nn = O.number_density(f)
    uu = O.species_velocity(f, nn, fluid)
    ub = O.barycentric_velocity(nn, uu, mass)
    F = O.drag_acceleration(nn, uu, om)
    ours = O.collide(f, O.phi_perp(nn, uu, ub), O.forcing_term(nn, F, ub), om)
    ubc = cdot(ub)
    ub2 = (ub ** 2).sum(0)
    for a in range(3):
        eq_u = nn[a] * O.W[:, None, None, None] * (1 + 3 * ubc + 4.5 * ubc ** 2 - 1.5 * ub2)
        bgk = f[a] - om * (f[a] - eq_u)
        d = uu[a] - ub
        dc = cdot(d)
        extra = om * nn[a] * O.W[:, None, None, None] * (dc ** 2 - CS2 * (d ** 2).sum(0)) / (2 * CS2 ** 2)
        np.testing.assert_allclose(ours[a] - bgk, extra, atol=1e-15)


# ---------------------------------------------------------------------------
# P7: indifferentiability of identical species
# ---------------------------------------------------------------------------
def test_indifferentiability_proportional_split():
    wl = WL.binary_random((5, 4, 6), seed=8)
    ntot = wl.n0.sum(0, keepdims=True)
    u1 = (wl.n0[:, None] * wl.u0).sum(0, keepdims=True) / ntot[:, None]
    p1 = O.Params(0.9, 1.3, [1.0], [0.0])
    one = O.Oracle(p1, wl.shape)
    one.initialise(ntot, u1)
    x = 0.37
    p2 = O.Params(0.9, 1.3, [1.0, 1.0], [0.0, 0.0])
    two = O.Oracle(p2, wl.shape)
    two.initialise(np.concatenate([x * ntot, (1 - x) * ntot]), np.concatenate([u1, u1]))
    for _ in range(20):
        one.step()
        two.step()
    np.testing.assert_allclose(two.f.sum(0), one.f[0], rtol=1e-12, atol=1e-15)


def test_indifferentiability_one_step_identity():
    """Arbitrary split: after one collision the summed distribution differs
    from the one-species BGK by omega_visc sum_a n^a w [(d.c)^2 - cs^2 d^2]/(2cs^4),
    d = u^a - u (derived by hand from the Appendix form)."""
    n, ua, _, _ = random_fields(9, S=2)
    mass = np.ones(2)
    om_v, om_d = 0.8, 1.6
    fluid = np.ones(n.shape[1:], bool)
    ub = O.barycentric_velocity(n, ua, mass)
    f = O.phi_perp(n, ua, ub) * (1 + 0.03 * rng(10).uniform(-1, 1, size=(2, 19) + n.shape[1:]))
    nn = O.number_density(f)
    uu = O.species_velocity(f, nn, fluid)
    ub = O.barycentric_velocity(nn, uu, mass)
    F = O.drag_acceleration(nn, uu, om_d)
    two = O.collide(f, O.phi_perp(nn, uu, ub), O.forcing_term(nn, F, ub), om_v).sum(0)
    ft = f.sum(0, keepdims=True)
    nt = nn.sum(0, keepdims=True)
    one = O.collide(ft, O.phi_perp(nt, ub[None], ub), 0.0, om_v)[0]
    extra = 0
    for a in range(2):
        d = uu[a] - ub
        dc = cdot(d)
        extra = extra + om_v * nn[a] * O.W[:, None, None, None] * (dc ** 2 - CS2 * (d ** 2).sum(0)) / (2 * CS2 ** 2)
    np.testing.assert_allclose(two - one, extra, atol=1e-15)


# ---------------------------------------------------------------------------
# P12: uniform electrolyte under a field reaches the drift of the Einstein
# relation, u^a - u = z^a E D / v_T^2 with the lattice D (steady state of the
# species momentum balance: drag balances the field exactly)
# ---------------------------------------------------------------------------
def test_uniform_drift_velocity():
    shape = (2, 2, 2)
    n0 = np.stack([np.full(shape, 0.98), np.full(shape, 0.01), np.full(shape, 0.01)])
    E = np.array([1e-4, -2e-5, 3e-5])
    om_d = 1.3
    p = O.Params(1.0, om_d, [1.0] * 3, [0.0, 1.0, -1.0], e_ext=E)
    o = O.Oracle(p, shape)
    o.initialise(n0)
    o.run(80)
    n, u = o.fields()
    ub = O.barycentric_velocity(n, u, p.mass)
    for a, z in enumerate([0.0, 1.0, -1.0]):
        for d in range(3):
            D = CS2 * (1 / om_d - 0.5)
            np.testing.assert_allclose(u[a, d] - ub[d], z * E[d] * D / CS2, rtol=1e-9, atol=1e-18)
    np.testing.assert_allclose(ub, 0, atol=1e-18)


# ---------------------------------------------------------------------------
# P9: Poisson solver and potential gradient, closed forms and brute force
# ---------------------------------------------------------------------------
def test_poisson_periodic_fourier_mode():
    shape = (6, 8, 10)
    z, y, x = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    k = (2 * math.pi * 2 / 10, 2 * math.pi * 1 / 8, 2 * math.pi * 1 / 6)
    s = np.cos(k[0] * x + k[1] * y + k[2] * z + 0.3)
    lam = sum(2 - 2 * math.cos(kk) for kk in k)
    solver = O.PoissonSolver(np.ones(shape, bool))
    psi = solver.solve(s)
    np.testing.assert_allclose(psi, s / lam, atol=1e-12)
    assert solver.residual(psi, s) < 1e-12


def test_poisson_slit_quadratic_and_wall_gradient():
    """Uniform charge rho between two walls of charge sigma per node,
    2 sigma + rho W = 0: psi(z) = -2 pi l_B rho (z - c)^2 + const,
    c = (W + 1)/2, solves the finite-volume problem exactly, and the cell
    gradient at every fluid cell is psi'(z) = -4 pi l_B rho (z - c)."""
    Wd, lB = 9, 0.7
    shape = (Wd + 2, 3, 4)
    solid = np.zeros(shape, bool)
    solid[0] = solid[-1] = True
    sig = np.where(solid, -0.013, 0.0)
    rho = -2 * -0.013 / Wd
    p = O.Params(1.0, 1.0, [1.0, 1.0], [1.0, -1.0], bjerrum=lB, solid=solid, sigma=sig)
    rho_e = np.where(solid, 0.0, rho)
    s = O.poisson_source(rho_e, p, shape)
    psi = O.PoissonSolver(~solid).solve(s)
    zc = np.arange(Wd + 2) - (Wd + 1) / 2.0
    exact = -2 * math.pi * lB * rho * zc ** 2
    sel = ~solid[:, 0, 0]
    exact = exact - exact[sel].mean()
    np.testing.assert_allclose(psi[sel, 1, 2], exact[sel], atol=1e-12)
    g = O.potential_gradient(psi, p)
    np.testing.assert_allclose(g[2][sel, 1, 2], -4 * math.pi * lB * rho * zc[sel], atol=1e-12)
    np.testing.assert_allclose(g[0][sel], 0, atol=1e-12)
    np.testing.assert_allclose(g[1][sel], 0, atol=1e-12)


def test_poisson_neumann_cosine_mode():
    """DCT-II modes cos(pi m (z - 1/2)/W) are exact eigenvectors of the
    zero-charge Neumann problem between walls."""
    Wd = 8
    shape = (Wd + 2, 4, 6)
    solid = np.zeros(shape, bool)
    solid[0] = solid[-1] = True
    z, y, x = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    m = 3
    s = np.cos(2 * math.pi * x / 6) * np.cos(math.pi * m * (z - 0.5) / Wd)
    s = np.where(solid, 0.0, s)
    lam = (2 - 2 * math.cos(2 * math.pi / 6)) + (2 - 2 * math.cos(math.pi * m / Wd))
    psi = O.PoissonSolver(~solid).solve(s)
    np.testing.assert_allclose(psi[~solid], (s / lam)[~solid], atol=1e-12)


def test_poisson_bruteforce_dense_random_walls():
    """Brute force: dense least-squares solve of the operator assembled
    cell by cell with explicit loops, on a tiny lattice with random walls."""
    shape = (4, 3, 5)
    solid, sig = WL.random_solid(shape, seed=21, fraction=0.2)
    solid[1, 1, 2] = False
    fluid = ~solid
    # keep the largest connected fluid component only (one free constant)
    lab = np.full(shape, -1)
    comp = 0
    for start in zip(*np.nonzero(fluid)):
        if lab[start] >= 0:
            continue
        stack = [start]
        lab[start] = comp
        while stack:
            zc, yc, xc = stack.pop()
            for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
                nb = ((zc + dz) % 4, (yc + dy) % 3, (xc + dx) % 5)
                if fluid[nb] and lab[nb] < 0:
                    lab[nb] = comp
                    stack.append(nb)
        comp += 1
    big = np.argmax(np.bincount(lab[lab >= 0]))
    solid = solid | (lab != big)
    fluid = ~solid
    cells = list(zip(*np.nonzero(fluid)))
    index = {c: i for i, c in enumerate(cells)}
    A = np.zeros((len(cells), len(cells)))
    for c, i in index.items():
        for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            nb = ((c[0] + dz) % 4, (c[1] + dy) % 3, (c[2] + dx) % 5)
            if nb in index:
                A[i, i] += 1
                A[i, index[nb]] -= 1
    g = rng(22)
    b = g.uniform(-1, 1, size=len(cells))
    b -= b.mean()
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    x -= x.mean()
    s = np.zeros(shape)
    for c, i in index.items():
        s[c] = b[i]
    psi = O.PoissonSolver(fluid).solve(s)
    got = np.array([psi[c] for c in cells])
    np.testing.assert_allclose(got, x, atol=1e-11)


def test_wall_charge_split_between_faces():
    """A wall node with k fluid face neighbours gives sigma/k to each; the
    total wall charge handed to the fluid equals the total wall charge."""
    shape = (5, 4, 6)
    solid, sig = WL.random_solid(shape, seed=31, fraction=0.3)
    p = O.Params(1.0, 1.0, [1.0], [1.0], bjerrum=1.0, solid=solid, sigma=sig)
    w = O.wall_charge_per_cell(p, shape)
    fluid = ~solid
    has_fluid_nb = np.zeros(shape, bool)
    for ax in range(3):
        for sh in (1, -1):
            has_fluid_nb |= np.roll(fluid, sh, axis=ax)
    np.testing.assert_allclose(w[fluid].sum(), sig[solid & has_fluid_nb].sum(), atol=1e-15)
    # a single isolated wall node with all 6 neighbours fluid
    solid1 = np.zeros(shape, bool)
    solid1[2, 2, 3] = True
    p1 = O.Params(1.0, 1.0, [1.0], [1.0], bjerrum=1.0, solid=solid1, sigma=np.where(solid1, 0.6, 0))
    w1 = O.wall_charge_per_cell(p1, shape)
    for dz, dy, dx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
        assert abs(w1[2 + dz, 2 + dy, 3 + dx] - 0.1) < 1e-15
    assert abs(w1.sum() - 0.6) < 1e-15


# ---------------------------------------------------------------------------
# P10: charged slit at rest relaxes to the Poisson-Boltzmann profile
# (ideal-gas chemical potential, Eq. chemdef, with Eq. Poisson); the
# equilibrium does not depend on the diffusivity
# ---------------------------------------------------------------------------
def _discrete_pb(Np, Nn, Wd, sigma, lB, guess):
    """1-D finite-volume Poisson-Boltzmann problem between two walls of
    charge sigma per node, canonical ion numbers Np, Nn: Newton via fsolve."""
    from scipy.optimize import fsolve

    def resid(x):
        ep, en = np.exp(-x), np.exp(x)
        rho = Np * ep / ep.sum() - Nn * en / en.sum()
        w = np.zeros(Wd)
        w[0] += sigma
        w[-1] += sigma
        tot = rho + w
        tot = tot - tot.mean()
        A = np.zeros(Wd)
        A[1:] += x[1:] - x[:-1]
        A[:-1] += x[:-1] - x[1:]
        r = A - 4 * math.pi * lB * tot
        r[0] = x.mean()
        return r
    return fsolve(resid, guess, xtol=1e-12)


@pytest.mark.parametrize("schmidt,steps", [(1.0, 1500), (4.0, 6000)])
def test_slit_equilibrium_is_poisson_boltzmann(schmidt, steps):
    Wd, lB, sig, debye = 16, 0.7, -0.01, 4.0
    wl = WL.slit(nx=1, ny=1, width=Wd, sigma=sig, debye=debye, bjerrum=lB,
                 e_field=0.0, schmidt=schmidt)
    o = _oracle_from(wl)
    info = o.run(steps)
    n = info.n
    psi = info.psi[1:-1, 0, 0]
    psi = psi - psi.mean()
    x = _discrete_pb(n[1, 1:-1].sum(), n[2, 1:-1].sum(), Wd, sig, lB, psi)
    assert np.ptp(x) > 0.2
    assert np.abs(psi - x).max() < 0.005 * np.ptp(x)
    # ions follow n ~ exp(-z psi) to the lattice's O(h^2) accuracy
    for a, z in ((1, 1.0), (2, -1.0)):
        dev = np.log(n[a, 1:-1, 0, 0]) + z * psi
        assert np.ptp(dev) < 0.03 * np.ptp(psi)
    assert info.poisson_rel_residual < 1e-12


def test_poisson_components_are_independent():
    """Two slits stacked along z (separated by wall planes) are independent
    domains: the solve on the stack equals the exact quadratic of each slit
    (per-component neutralising background and zero mean)."""
    lB = 0.7
    W1, W2, s1, s2 = 5, 8, -0.011, -0.004
    nz = W1 + W2 + 2
    shape = (nz, 2, 3)
    solid = np.zeros(shape, bool)
    solid[0] = True
    solid[W1 + 1] = True
    sig = np.zeros(shape)
    sig[0] = s1
    sig[W1 + 1] = s2
    # uniform charge in each slit; each slit sees its two walls
    rho = np.zeros(shape)
    rho[1:W1 + 1] = 0.002
    rho[W1 + 2:] = -0.001
    p = O.Params(1.0, 1.0, [1.0], [1.0], bjerrum=lB, solid=solid, sigma=sig)
    so = O.PoissonSolver(~solid)
    assert so.ncomp == 2
    psi = so.solve(O.poisson_source(rho, p, shape))
    for lo, W, sa, sb, r0 in [(1, W1, s1, s2, 0.002), (W1 + 2, W2, s2, s1, -0.001)]:
        # net charge density with the component mean removed: each wall plane
        # has fluid on both sides and hands half its charge to each
        q = np.full(W, r0)
        q[0] += 0.5 * sa
        q[-1] += 0.5 * sb
        q -= q.mean()
        # exact 1-D finite-volume solve (Neumann chain), zero mean
        A = np.diag(np.r_[1, np.full(W - 2, 2), 1].astype(float)) - np.eye(W, k=1) - np.eye(W, k=-1)
        x = np.linalg.lstsq(A, 4 * math.pi * lB * q, rcond=None)[0]
        x -= x.mean()
        np.testing.assert_allclose(psi[lo:lo + W, 1, 2], x, atol=1e-12)


# ---------------------------------------------------------------------------
# P11: electro-osmotic flow in the charged slit follows Helmholtz-
# Smoluchowski: the mixture momentum balance nu rho u'' = -rho_e E with
# Poisson psi'' = -4 pi l_B rho_e and no slip gives
# u_x(z) = E (psi(z) - psi_wall) / (4 pi l_B rho nu)  (Eq. globalmomentumcontc)
# ---------------------------------------------------------------------------
def test_slit_electroosmotic_profile_helmholtz_smoluchowski():
    Wd, lB, sig, debye, E = 12, 0.7, -0.01, 4.0, 1e-5
    wl = WL.slit(nx=1, ny=1, width=Wd, sigma=sig, debye=debye, bjerrum=lB, e_field=0.0,
                 schmidt=1.0)
    eq = _oracle_from(wl)
    eq.run(1500)                         # ions at rest reach equilibrium first
    p = O.Params(1.0, O.omega_drag_for_schmidt(1.0, 100.0), wl.mass, wl.valence, bjerrum=lB,
                 e_ext=(E, 0.0, 0.0), solid=wl.solid, sigma=wl.sigma)
    o = O.Oracle(p, wl.shape)
    o.f = eq.f.copy()
    info = o.run(2000)                   # flow develops in ~ W^2 / (pi^2 nu) steps
    n, u = info.n[:, 1:-1, 0, 0], info.u[:, :, 1:-1, 0, 0]
    psi = info.psi[1:-1, 0, 0]
    rho = n.sum(0)
    rho_e = (wl.valence[:, None] * n).sum(0)
    # mid-step (force-shifted) barycentric velocity
    ux = ((n * u[:, 0]).sum(0) + 0.5 * rho_e * E) / rho
    psi_wall = psi[0] + 2 * math.pi * lB * sig   # half a cell out, Neumann slope
    nu = O.viscosity(1.0)
    pred = E * (psi - psi_wall) / (4 * math.pi * lB * rho * nu)
    assert pred.max() > 1e-6
    assert np.abs(ux - pred).max() <= 0.02 * np.abs(pred).max()
