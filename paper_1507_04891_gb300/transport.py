"""Slit transport diagnostics from the moments of a lattice (Sec. 4, the
charged slit under a field parallel to the walls).

For a slit with walls normal to z and a field E along x, the state is
uniform in x and y; the plane averages give z-profiles, and the paper's
currents per unit wall area are sums over the fluid planes:

* mass flow rate       I_m  = sum_z sum_a m n^a u^a_x        (Eq. currmass)
* electric current     I    = sum_z sum_a z_a n^a u^a_x
* convective current   I_eo = sum_z rho_e(z) u_x(z)          (Eq. curreo)

with u_x the barycentric velocity.  The velocities are the mid-step
(force-shifted) ones, u^a + F^a / 2, as for the second-order forcing of
Eq. ourforc: F^a_x = z_a E - omega_drag (u^a_x + z_a E / 2 - v_x), v the
number-weighted mean of u^b + z_b E / 2 (the drag on force-shifted
velocities); the field inside the slit has no x component.  Host analysis
of lbm.Lattice.get_moments output; nothing here runs on the GPU.
"""

from __future__ import annotations

import numpy as np


def slit_profiles(lat, valence, e_field, omega_drag, solid):
    """Plane-averaged profiles over the fluid planes of a slit: density per
    species n[a, z], mid-step velocities ux[a, z], barycentric rho and u_x."""
    S = len(valence)
    mom = [lat.get_moments(s) for s in range(S)]
    n = np.stack([m[0] for m in mom])                                # (S, nz, ny, nx)
    u = np.stack([m[1][0] for m in mom])                             # bare u_x
    z = np.asarray(valence, dtype=float)[:, None, None, None]
    ntot = n.sum(0)
    fl = ~solid
    ntot_safe = np.where(fl, ntot, 1.0)
    vx = (n * (u + 0.5 * z * e_field)).sum(0) / ntot_safe
    F = z * e_field - omega_drag * (u + 0.5 * z * e_field - vx[None])
    uphys = u + 0.5 * F
    planes = np.where(fl.all(axis=(1, 2)))[0]
    nz_prof = n[:, planes].mean(axis=(2, 3))
    jx_prof = (n * uphys)[:, planes].mean(axis=(2, 3))
    return planes, nz_prof, jx_prof


def slit_currents(lat, valence, e_field, omega_drag, solid):
    """I_m, I, I_eo per unit wall area, and the largest difference between
    the solvent (species 0) and the barycentric velocity relative to the
    largest barycentric velocity."""
    planes, n, j = slit_profiles(lat, valence, e_field, omega_drag, solid)
    z = np.asarray(valence, dtype=float)[:, None]
    rho = n.sum(0)
    ux = j.sum(0) / rho
    rho_e = (z * n).sum(0)
    Im = float(j.sum())
    I = float((z * j).sum())
    Ieo = float((rho_e * ux).sum())
    u0 = j[0] / n[0]
    dev = float(np.abs(u0 - ux).max() / max(np.abs(ux).max(), 1e-300))
    return {"I_m": Im, "I": I, "I_eo": Ieo, "solvent_vs_barycentric": dev,
            "u_x_max": float(np.abs(ux).max())}
