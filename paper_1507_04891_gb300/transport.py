"""Slit transport diagnostics from the library's plane sums (Sec. 4, the
charged slit under a field parallel to the walls).

For a slit with walls normal to z and a field E along x, the state is
uniform in x and y; lbm_plane_fluxes gives, per z-plane and species, the sums
of n^a and of the mid-step flux n^a (u^a + F^a / 2) (the velocity of the
second-order forcing of Eq. ourforc, F^a the drag and electric force the
collision applies).  The paper's currents per unit wall area are sums of the
plane averages over the fluid planes:

* mass flow rate       I_m  = sum_z sum_a m n^a u^a_x        (Eq. currmass)
* electric current     I    = sum_z sum_a z_a n^a u^a_x
* convective current   I_eo = sum_z rho_e(z) u_x(z)          (Eq. curreo)

with u_x the barycentric velocity of the plane.  All node arithmetic runs on
the GPU; this module only sums the returned plane values.
"""

from __future__ import annotations

import numpy as np


def slit_profiles(lat, solid):
    """Plane-averaged profiles over the fluid planes of a slit: the indices
    of the fluid planes, density per species n[a, z] and mid-step flux
    jx[a, z] along x."""
    sums = lat.plane_fluxes()                      # (nz, S, 4)
    planes = np.where(~solid.any(axis=(1, 2)))[0]
    area = float(solid.shape[1] * solid.shape[2])
    n = sums[planes, :, 0].T / area
    jx = sums[planes, :, 1].T / area
    return planes, n, jx


def slit_currents(lat, valence, solid):
    """I_m, I, I_eo per unit wall area, and the largest difference between
    the solvent (species 0) and the barycentric velocity relative to the
    largest barycentric velocity."""
    planes, n, j = slit_profiles(lat, solid)
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
