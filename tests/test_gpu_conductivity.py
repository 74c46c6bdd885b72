"""Bulk electric conductivity (Sec. 4, the current against D; Eq. Drude).

A uniform neutral electrolyte in a uniform field: once the species
velocities relax, the total current J = sum_a z_a n_a u_a must equal the
Drude-Lorentz value (e^2 D / v_T^2) sum_a z_a^2 n_a E with the lattice
diffusivity D = c_s^2 (1/omega_drag - 1/2) and v_T^2 = c_s^2, so J is
proportional to D; the barycentric velocity stays zero (no net force).
The oracle reaches this exactly (test_uniform_drift_velocity); here the
CUDA path is held to it in FP32 across Schmidt numbers, including the
BGK limit omega_drag = omega_visc (Sc = 1 at omega_visc = 1)."""

import math

import numpy as np
import pytest

from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

CS2 = 1.0 / 3.0


def drude(fraction, e, omega_drag):
    D = CS2 * (1.0 / omega_drag - 0.5)
    return D / CS2 * 2 * fraction * e       # z = +1 and -1, n = fraction each


def relax_steps(omega_drag, target=1e-9):
    # the relative velocity relaxes by |1 - omega_drag| per step
    q = abs(1.0 - omega_drag)
    return 200 if q < 1e-3 else 200 + int(math.log(target) / math.log(q))


def measure(schmidt, n=16, e=1e-3, fraction=0.01, storage="fp32"):
    wl = WL.bulk_conductivity(n=n, e_field=e, schmidt=schmidt, fraction=fraction)
    od = lbm.omega_drag_for_schmidt(wl.omega_visc, schmidt)
    lat = lbm.Lattice(n, n, n, 3, omega_visc=wl.omega_visc, omega_drag=od, bjerrum=wl.bjerrum,
                      e_ext=wl.e_ext, storage=storage, poisson="fft", step_graph=True)
    for s in range(3):
        lat.set_species(s, 1.0, wl.valence[s], wl.n0[s])
    lat.step(relax_steps(od))
    J = np.zeros(3)
    mom = np.zeros(3)
    for s in range(3):
        ns, us = lat.get_moments(s)
        J += wl.valence[s] * (ns * us).reshape(3, -1).sum(1) / ns.size
        mom += (ns * us).reshape(3, -1).sum(1) / ns.size
    d = lat.diagnostics()
    lat.destroy()
    return J, mom, od, d


@pytest.mark.parametrize("schmidt", [1.0, 10.0, 100.0, 1000.0])
def test_bulk_current_is_drude(schmidt):
    e, fraction = 1e-3, 0.01
    J, mom, od, d = measure(schmidt, e=e, fraction=fraction)
    Jd = drude(fraction, e, od)
    # The populations carry the half-force shift z E / 2 of the bare velocity;
    # the drift is the fraction 2 (1/omega_drag - 1/2) ~ 1/Sc of it, and in a
    # uniform box every node rounds alike (nothing averages out), so FP32
    # deviations resolve the current to about 1e-7 Sc.
    tol = max(1e-6, 3e-7 * schmidt)
    assert abs(J[0] / Jd - 1) <= tol, (J, Jd)
    assert abs(J[1]) <= tol * abs(Jd) and abs(J[2]) <= tol * abs(Jd)
    # no net force on the neutral mixture: the barycentric momentum stays at
    # round-off, far below the ion momenta n u ~ J / 2
    assert np.abs(mom).max() <= 1e-3 * abs(Jd) + 1e-11
    assert d["poisson_residual"] <= 1e-8


def test_current_proportional_to_diffusivity():
    """Fig. sigvsdiff: the current at fixed field scales with D."""
    Js, Ds = [], []
    for sc in (1.0, 3.0, 30.0, 300.0):
        J, _, od, _ = measure(sc)
        Js.append(J[0])
        Ds.append(CS2 * (1.0 / od - 0.5))
    ratio = np.array(Js) / np.array(Ds)
    assert np.ptp(ratio) <= 2e-4 * ratio.mean()
