"""Plain FP64 restatement of the two-timescale multicomponent LB update.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Slow on purpose:
whole-array numpy operations in the order the paper states the steps, no
fusion, no blocking, no precision tricks.

Conventions (readings of the paper, each listed in the design notes):

* D3Q19 (Sec. 4, text after Eq. latboeq); direction 0 is rest, 1..6 are
  +x,-x,+y,-y,+z,-z, 7..18 are the 12 edge vectors in opposite pairs
  (2k-1, 2k).  Lattice sound speed v_T^2 = c_s^2 = 1/3 and the weights
  Gamma_0(c_p) = w_p = 1/3, 1/18, 1/36 (Appendix, Eq. ourforc).
* Arrays: f has shape (S, 19, nz, ny, nx), x fastest.  The lattice is a
  3-torus; walls are solid nodes given by a boolean mask.
* f(t) is the pre-collision (post-streaming) state at time t.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ---------------------------------------------------------------------------
# D3Q19 velocity set (Sec. 4: "D3Q19 velocity discretization")
# ---------------------------------------------------------------------------
C = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
], dtype=np.int64)
Q = 19
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
OPP = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17])
CS2 = 1.0 / 3.0          # v_T^2 in lattice units (k_B T / m with m = 1)


class Params:
    """Model parameters of Eq. (evolution) and Eq. (latboeq).

    omega_visc : BGK frequency of the non-hydrodynamic modes, Eq. (dufty1).
    omega_drag : drag frequency, Sec. 2 ("omega_drag ... used to tune the
                 diffusion coefficient"); or a symmetric (S, S) matrix of
                 pair frequencies omega^{alpha beta} for the general
                 gamma^{alpha beta} of Sec. 2 (see pair_drag_frequencies).
    mass       : (S,) particle masses m^alpha (all equal on one lattice).
    valence    : (S,) z^alpha.
    bjerrum    : l_B of Eq. (Poisson); 0 switches the electrostatics off.
    e_ext      : (3,) applied field as an acceleration per unit valence.
    solid      : (nz, ny, nx) bool mask of wall nodes, or None.
    sigma      : (nz, ny, nx) surface charge per solid node (units of e), or None.
    """

    def __init__(self, omega_visc, omega_drag, mass, valence, bjerrum=0.0,
                 e_ext=(0.0, 0.0, 0.0), solid=None, sigma=None):
        self.omega_visc = float(omega_visc)
        od = np.asarray(omega_drag, dtype=np.float64)
        self.omega_drag = float(od) if od.ndim == 0 else od.copy()
        self.mass = np.asarray(mass, dtype=np.float64)
        self.valence = np.asarray(valence, dtype=np.float64)
        self.bjerrum = float(bjerrum)
        self.e_ext = np.asarray(e_ext, dtype=np.float64)
        self.solid = None if solid is None else np.asarray(solid, dtype=bool)
        self.sigma = None if sigma is None else np.asarray(sigma, dtype=np.float64)


def _shift(a, c):
    """out[r] = a[r - c] on the periodic lattice, c = (cx, cy, cz)."""
    return np.roll(a, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(-3, -2, -1))


def fluid_mask(shape, p: Params):
    if p.solid is None:
        return np.ones(shape, dtype=bool)
    return ~p.solid


# ---------------------------------------------------------------------------
# Macroscopic fields, Sec. 3 (definitions of n^alpha, u^alpha, u)
# ---------------------------------------------------------------------------
def number_density(f):
    """n^alpha = sum_p f_p^alpha (discrete form of the zeroth moment)."""
    return f.sum(axis=1)


def species_velocity(f, n, fluid):
    """u^alpha = (1/n^alpha) sum_p c_p f_p^alpha (bare first moment)."""
    j = np.einsum("spzyx,pd->sdzyx", f, C.astype(np.float64))
    u = np.zeros_like(j)
    safe = np.where(fluid, n, 1.0)[:, None]
    u[:] = np.where(fluid[None, None], j / safe, 0.0)
    return u


def barycentric_velocity(n, u, mass):
    """u = sum_alpha rho^alpha u^alpha / rho with rho^alpha = m^alpha n^alpha."""
    rho_a = mass[:, None, None, None] * n
    rho = rho_a.sum(axis=0)
    num = (rho_a[:, None] * u).sum(axis=0)
    safe = np.where(rho != 0.0, rho, 1.0)
    return np.where(rho[None] != 0.0, num / safe[None], 0.0)


# ---------------------------------------------------------------------------
# Forces (accelerations per particle), Sec. 2 drag force and Eq. (Poisson)
# ---------------------------------------------------------------------------
def drag_acceleration(n, u, omega_drag):
    """F^{alpha,drag}/m = -sum_beta omega^{alpha beta} (n_beta/n) (u^alpha - u^beta).

    omega_drag is the paper's single drag frequency (Sec. 2, the equal-mass,
    equal-diameter form gamma^{alpha beta} = omega_drag n_beta / n), or a
    symmetric (S, S) matrix of pair frequencies (the general gamma^{alpha
    beta} of Sec. 2 for equal masses, gamma^{alpha beta} = omega^{alpha
    beta} n_beta / n).  Written as the literal double sum over the species
    pair (alpha, beta), with n = sum_beta n_beta.
    """
    S = n.shape[0]
    W = np.asarray(omega_drag, dtype=np.float64)
    if W.ndim == 0:
        W = np.full((S, S), float(W))
    ntot = n.sum(axis=0)
    safe = np.where(ntot != 0.0, ntot, 1.0)
    F = np.zeros_like(u)
    for a in range(S):
        for b in range(S):
            F[a] += -W[a, b] * (n[b] / safe)[None] * (u[a] - u[b])
    return F


def pair_drag_frequencies(diameters, n_total, g_contact=None, kT_over_m=None):
    """omega^{alpha beta} of the general drag coefficient of Sec. 2 for
    species of equal mass m and diameters sigma_alpha:
    gamma^{alpha beta} = (8/3) sigma_ab^2 n_beta sqrt(k_B T / (pi m)) g_ab
    with sigma_ab = (sigma_a + sigma_b)/2 and g_ab the pair correlation at
    contact (the paper's expression with m_alpha = m_beta), written as
    omega^{alpha beta} n_beta / n, so
    omega^{alpha beta} = (8/3) sigma_ab^2 n sqrt(k_B T / (pi m)) g_ab.
    k_B T / m defaults to v_T^2 of the lattice; g_ab to 1."""
    d = np.asarray(diameters, dtype=np.float64)
    S = d.size
    g = np.ones((S, S)) if g_contact is None else np.asarray(g_contact, dtype=np.float64)
    kt = CS2 if kT_over_m is None else float(kT_over_m)
    sab = 0.5 * (d[:, None] + d[None, :])
    return (8.0 / 3.0) * sab ** 2 * float(n_total) * np.sqrt(kt / np.pi) * g


def drag_velocity(ua, Fel):
    """Species velocities that enter the drag force: the bare moments
    u^alpha shifted by half of the electric/applied acceleration,
    u^alpha + F^{alpha,el}/2 (the mid-step velocity of the external force).

    Reading of the paper (which leaves the discretisation to "the standard
    procedure"): the drag itself stays explicit, so a neutral mixture keeps
    the lattice diffusivity D = v_T^2 (1/omega_drag - 1/2) of Sec. 4, while
    the electric force does not feed back into the drag through the
    force-induced shift of the bare moment.  With it the charged steady
    state is the Boltzmann/Poisson-Boltzmann one for every omega_drag and
    the field-driven drift obeys the Einstein relation u = z E D / v_T^2
    that the Drude-Lorentz formula, Eq. (Drude), assumes.
    """
    return ua + 0.5 * Fel


def wall_face_charge(p: Params, shape):
    """Charge carried by each wall face: a solid node with k fluid face
    neighbours hands sigma/k to each of them (boundary condition of
    Eq. (Poisson), surface charge per wall node)."""
    nz, ny, nx = shape
    q = np.zeros(shape)
    if p.solid is None or p.sigma is None:
        return q
    fluid = ~p.solid
    k = np.zeros(shape)
    for d in range(1, 7):
        k += _shift(fluid, -C[d])            # neighbour r + c_d is fluid
    has = p.solid & (k > 0)
    q[has] = p.sigma[has] / k[has]
    return q


def wall_charge_per_cell(p: Params, shape):
    """w_i = sum over the solid face neighbours j of cell i of q_j."""
    q = wall_face_charge(p, shape)
    fluid = fluid_mask(shape, p)
    w = np.zeros(shape)
    if p.solid is None:
        return w
    for d in range(1, 7):
        qn = _shift(q, -C[d])                # q at r + c_d
        sn = _shift(p.solid, -C[d])
        w += np.where(fluid & sn, qn, 0.0)
    return w


def poisson_matrix(fluid):
    """Finite-volume 7-point operator A on the fluid cells of the torus:
    (A psi)_i = sum_{fluid face neighbours j} (psi_i - psi_j).

    A psi = 4 pi l_B (rho_e + w) is the cell-integrated form of
    nabla^2 psi = -4 pi l_B rho_e with the wall-charge Neumann condition
    [nabla psi]_perp = -4 pi l_B Sigma / e (Eq. (Poisson) and the boundary
    condition after it), normal pointing into the fluid.
    Returns (A over fluid cells, index map full -> fluid cell or -1).
    """
    shape = fluid.shape
    N = fluid.size
    idx = -np.ones(N, dtype=np.int64)
    fl = fluid.ravel()
    nf = int(fl.sum())
    idx[fl] = np.arange(nf)
    full = np.arange(N).reshape(shape)
    rows, cols, vals = [], [], []
    for d in range(1, 7):
        nb = _shift(full, -C[d]).ravel()     # index of r + c_d
        ok = fl & fl[nb]
        i = idx[np.nonzero(ok)[0]]
        j = idx[nb[ok]]
        rows += [i, i]
        cols += [i, j]
        vals += [np.ones(len(i)), -np.ones(len(i))]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nf, nf))
    return A, idx


def fluid_components(fluid):
    """Connected components of the fluid cells (face neighbours, periodic):
    (number of components, label per fluid cell in the order of fluid.ravel())."""
    from scipy.sparse.csgraph import connected_components
    A, _ = poisson_matrix(fluid)
    return connected_components(A, directed=False)


def poisson_source(rho_e, p: Params, shape):
    """s = 4 pi l_B (rho_e + w - mean), the right-hand side of A psi = s.
    The mean is taken over each connected fluid component (a neutralising
    background per isolated fluid domain), which makes every component's
    Neumann/periodic problem solvable."""
    fluid = fluid_mask(shape, p)
    tot = rho_e + wall_charge_per_cell(p, shape)
    ncomp, lab = fluid_components(fluid)
    vals = tot[fluid]
    means = np.bincount(lab, weights=vals, minlength=ncomp) / np.bincount(lab, minlength=ncomp)
    s = np.zeros(shape)
    s[fluid] = 4.0 * np.pi * p.bjerrum * (vals - means[lab])
    return s


class PoissonSolver:
    """Solves A psi = s on the fluid cells with zero mean on every connected
    fluid component (the constant of each is free for the periodic /
    Neumann problem).  Sparse LU of the bordered
    system [[A, 1], [1^T, 0]] for small lattices, conjugate gradients with a
    1e-13 relative tolerance for large ones; either is far tighter than the
    1e-8 the GPU iterates to."""

    def __init__(self, fluid, direct_limit=70000):
        self.fluid = fluid
        self.A, self.idx = poisson_matrix(fluid)
        nf = self.A.shape[0]
        self.nf = nf
        self.ncomp, self.lab = fluid_components(fluid)
        self.direct = nf <= direct_limit
        if self.direct:
            # one zero-mean constraint per connected component
            E = sp.csr_matrix((np.ones(nf), (np.arange(nf), self.lab)), shape=(nf, self.ncomp))
            B = sp.bmat([[self.A, E], [E.T, None]], format="csc")
            self.lu = spla.splu(B)

    def _zero_mean(self, x):
        cnt = np.bincount(self.lab, minlength=self.ncomp)
        means = np.bincount(self.lab, weights=x, minlength=self.ncomp) / cnt
        return x - means[self.lab]

    def solve(self, s):
        b = s[self.fluid]
        if self.direct:
            x = self.lu.solve(np.concatenate([b, np.zeros(self.ncomp)]))[:self.nf]
        else:
            x, info = spla.cg(self.A, b, rtol=1e-13, atol=0.0, maxiter=20000)
            if info != 0:
                raise RuntimeError("oracle CG did not converge")
            x = self._zero_mean(x)
        psi = np.zeros(self.fluid.shape)
        psi[self.fluid] = x
        return psi

    def residual(self, psi, s):
        b = s[self.fluid]
        return np.linalg.norm(b - self.A @ psi[self.fluid]) / max(np.linalg.norm(b), 1e-300)


def potential_gradient(psi, p: Params):
    """Cell gradient of psi: the mean of the two face gradients along each
    axis (second-order central difference in the bulk).  A wall face takes
    the Neumann value of the boundary condition after Eq. (Poisson):
    d psi/dn_out = 4 pi l_B q for the face charge q."""
    shape = psi.shape
    fluid = fluid_mask(shape, p)
    q = wall_face_charge(p, shape)
    g = np.zeros((3,) + shape)
    for axis in range(3):
        e = np.zeros(3, dtype=np.int64)
        e[axis] = 1
        plus_fluid = _shift(fluid, -e)
        minus_fluid = _shift(fluid, e)
        gp = np.where(plus_fluid, _shift(psi, -e) - psi, 4.0 * np.pi * p.bjerrum * _shift(q, -e))
        gm = np.where(minus_fluid, psi - _shift(psi, e), -4.0 * np.pi * p.bjerrum * _shift(q, e))
        g[axis] = np.where(fluid, 0.5 * (gp + gm), 0.0)
    return g


def electric_acceleration(valence, grad_psi, e_ext):
    """F^{alpha,el}/m = z^alpha (-v_T^2 grad psi~ + E_ext): the mean-field
    term of Eq. (equilproc2) with psi~ = e psi / k_B T and k_B T / m = v_T^2,
    plus an applied field given as acceleration per unit valence."""
    S = valence.shape[0]
    F = np.zeros((S,) + grad_psi.shape)
    for a in range(S):
        for d in range(3):
            F[a, d] = valence[a] * (-CS2 * grad_psi[d] + e_ext[d])
    return F


# ---------------------------------------------------------------------------
# Discrete equilibrium and forcing, Appendix
# ---------------------------------------------------------------------------
def _dot_c(v):
    """(v . c_p) for every p: v has shape (..., 3, nz, ny, nx) -> (..., 19, ...)."""
    return np.einsum("pd,...dzyx->...pzyx", C.astype(np.float64), v)


def phi_perp(n, ua, u):
    """Discrete orthogonalised equilibrium phi_perp,p^alpha, the final
    expression of the Appendix, written term by term (not simplified):

      n w_p { 1 + u^a.c/vT^2 + 1/(2 vT^4) [ 2(u^a.c)(u.c) - 2 vT^2 (u^a.u)
              - (u.c)^2 + vT^2 |u|^2 + ((u^a - u).c)^2 - vT^2 |u^a - u|^2 ] }
    """
    S = n.shape[0]
    out = np.zeros((S, Q) + n.shape[1:])
    uc = _dot_c(u)                                  # (19, ...)
    uu = (u * u).sum(axis=0)
    for a in range(S):
        uac = _dot_c(ua[a])
        dc = _dot_c(ua[a] - u)
        uau = (ua[a] * u).sum(axis=0)
        dd = ((ua[a] - u) ** 2).sum(axis=0)
        bracket = (2.0 * uac * uc - 2.0 * CS2 * uau - uc ** 2 + CS2 * uu
                   + dc ** 2 - CS2 * dd)
        out[a] = n[a] * W[:, None, None, None] * (
            1.0 + uac / CS2 + bracket / (2.0 * CS2 * CS2))
    return out


def forcing_term(n, F, u):
    """g_p^alpha of Eq. (ourforc):
       n^a w_p [ F.c/vT^2 + ((F.c)(u.c) - vT^2 F.u)/vT^4 ]."""
    S = n.shape[0]
    out = np.zeros((S, Q) + n.shape[1:])
    uc = _dot_c(u)
    for a in range(S):
        Fc = _dot_c(F[a])
        Fu = (F[a] * u).sum(axis=0)
        out[a] = n[a] * W[:, None, None, None] * (
            Fc / CS2 + (Fc * uc - CS2 * Fu) / (CS2 * CS2))
    return out


# ---------------------------------------------------------------------------
# Collision and streaming, Eq. (latboeq)
# ---------------------------------------------------------------------------
def collide(f, phi, g, omega_visc):
    """f* = f - omega_visc (f - phi_perp) + g   (right side of Eq. latboeq)."""
    return f - omega_visc * (f - phi) + g


def stream(fstar, p: Params):
    """f_p(r + c_p, t + 1) = f*_p(r, t) (left side of Eq. latboeq) on the
    torus.  When r - c_p is a wall node the population returns by halfway
    bounce-back: f_p(r, t + 1) = f*_{opp(p)}(r, t).  Wall nodes hold zeros."""
    out = np.zeros_like(fstar)
    shape = fstar.shape[2:]
    fluid = fluid_mask(shape, p)
    for q in range(Q):
        pulled = _shift(fstar[:, q], C[q])
        if p.solid is not None:
            src_solid = _shift(p.solid, C[q])
            pulled = np.where(src_solid[None], fstar[:, OPP[q]], pulled)
        out[:, q] = np.where(fluid[None], pulled, 0.0)
    return out


# ---------------------------------------------------------------------------
# Whole step and initialisation
# ---------------------------------------------------------------------------
class StepInfo:
    def __init__(self):
        self.n = None
        self.u = None
        self.ubar = None
        self.psi = None
        self.poisson_rel_residual = None


class Oracle:
    """Time stepper: holds f(t) and applies, per step, the operations in the
    order of Eq. (latboeq): moments -> (Poisson) -> forces -> phi_perp, g_p
    -> collision -> streaming."""

    def __init__(self, p: Params, shape):
        self.p = p
        self.shape = tuple(shape)
        self.fluid = fluid_mask(self.shape, p)
        self.poisson = PoissonSolver(self.fluid) if p.bjerrum > 0 else None
        self.f = None
        self.t = 0

    def initialise(self, n0, u0=None):
        """f_p^alpha(0) = phi_perp,p(n0^alpha, u0^alpha, u0) (local equilibrium)."""
        S = n0.shape[0]
        n0 = np.where(self.fluid[None], n0, 0.0)
        if u0 is None:
            u0 = np.zeros((S, 3) + self.shape)
        u0 = np.where(self.fluid[None, None], u0, 0.0)
        ubar = barycentric_velocity(n0, u0, self.p.mass)
        self.f = phi_perp(n0, u0, ubar)
        self.t = 0

    def fields(self, f=None):
        f = self.f if f is None else f
        n = number_density(f)
        u = species_velocity(f, n, self.fluid)
        return n, u

    def potential(self, n):
        rho_e = (self.p.valence[:, None, None, None] * n).sum(axis=0)
        s = poisson_source(rho_e, self.p, self.shape)
        psi = self.poisson.solve(s)
        return psi, s

    def step(self):
        p = self.p
        info = StepInfo()
        f = self.f
        n = number_density(f)
        ua = species_velocity(f, n, self.fluid)
        u = barycentric_velocity(n, ua, p.mass)
        if self.poisson is not None:
            psi, s = self.potential(n)
            grad = potential_gradient(psi, p)
            info.psi = psi
            info.poisson_rel_residual = self.poisson.residual(psi, s)
        else:
            grad = np.zeros((3,) + self.shape)
        Fel = electric_acceleration(p.valence, grad, p.e_ext)
        Fdrag = drag_acceleration(n, drag_velocity(ua, Fel), p.omega_drag)
        F = np.where(self.fluid[None, None], Fel + Fdrag, 0.0)
        phi = phi_perp(n, ua, u)
        g = forcing_term(n, F, u)
        fstar = collide(f, phi, g, p.omega_visc)
        self.f = stream(fstar, p)
        self.t += 1
        info.n, info.u, info.ubar = n, ua, u
        return info

    def run(self, steps):
        info = None
        for _ in range(steps):
            info = self.step()
        return info


def diffusivity(omega_drag):
    """D = v_T^2 (1/omega_drag - 1/2), Sec. 4 (Chapman-Enskog result)."""
    return CS2 * (1.0 / omega_drag - 0.5)


def viscosity(omega_visc):
    """nu = v_T^2 (1/omega_visc - 1/2), Sec. 4."""
    return CS2 * (1.0 / omega_visc - 0.5)


def omega_drag_for_schmidt(omega_visc, sc):
    """omega_drag giving Sc = nu / D at fixed omega_visc."""
    D = viscosity(omega_visc) / sc
    return 1.0 / (0.5 + D / CS2)


__all__ = [
    "C", "Q", "W", "OPP", "CS2", "Params", "number_density", "species_velocity",
    "barycentric_velocity", "drag_acceleration", "pair_drag_frequencies", "drag_velocity",
    "wall_face_charge",
    "wall_charge_per_cell", "poisson_matrix", "poisson_source", "fluid_components", "PoissonSolver",
    "potential_gradient", "electric_acceleration", "phi_perp", "forcing_term",
    "collide", "stream", "Oracle", "StepInfo",
    "diffusivity", "viscosity", "omega_drag_for_schmidt", "fluid_mask",
]
