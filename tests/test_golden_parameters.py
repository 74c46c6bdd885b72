"""The paper's printed Sec. 4 parameters (tests/golden/sec4_parameters.json,
each value with its citation) against the seeded input generators: the
workloads reproduce the slit's wall charge and Debye lengths through the
paper's own definition of lambda_D, and the bulk electrolyte's ion density.
The paper prints its results only as figures, so these parameter values are
its only printed numbers."""

import json
import math
import os

import numpy as np
import pytest

from paper_1507_04891_gb300 import workloads as WL

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "sec4_parameters.json")) as fh:
    G = {k: v["value"] for k, v in json.load(fh).items() if isinstance(v, dict)}

CS2 = 1.0 / 3.0      # v_T^2 of D3Q19


def test_wall_charge_per_node_reproduces_the_printed_total():
    """Sigma Lx Ly / e = -0.04 on one 40 x 10 wall: -1e-4 per wall node; the
    slit generator puts exactly that charge on every node of both walls."""
    lx, ly, lz = G["slit_mesh"]
    sigma = G["wall_charge_total"] / (lx * ly)
    assert sigma == pytest.approx(-1e-4, rel=1e-12)
    wl = WL.slit(nx=lx, ny=ly, width=lz, sigma=sigma, debye=0.2 * lz)
    assert wl.sigma[0].sum() == pytest.approx(G["wall_charge_total"], rel=1e-12)
    assert wl.sigma[-1].sum() == pytest.approx(G["wall_charge_total"], rel=1e-12)
    assert not wl.sigma[1:-1].any()
    # the fluid carries the opposite of both walls' charge: neutral overall
    rho_e = (wl.valence[:, None, None, None] * wl.n0).sum(0)
    assert rho_e.sum() + wl.sigma.sum() == pytest.approx(0.0, abs=1e-12)   # 2e4 summands


@pytest.mark.parametrize("ratio", G["debye_over_Lz"])
def test_slit_bulk_density_gives_the_printed_debye_length(ratio):
    """lambda_D = 1/sqrt(4 pi l_B (n+_b + n-_b)) (Sec. 4) equals ratio * L_z
    for the bulk ion density the generator derives from it."""
    lx, ly, lz = G["slit_mesh"]
    sigma = G["wall_charge_total"] / (lx * ly)
    wl = WL.slit(nx=lx, ny=ly, width=lz, sigma=sigma, debye=ratio * lz)
    nb = wl.meta["nbulk"]
    assert 1.0 / math.sqrt(4 * math.pi * wl.bjerrum * nb) == pytest.approx(ratio * lz, rel=1e-12)
    # fluid ion densities: bulk sum plus the counter-ion excess, both positive
    npos, nneg = wl.n0[1, 1, 0, 0], wl.n0[2, 1, 0, 0]
    assert npos + nneg == pytest.approx(nb, rel=1e-12)
    assert npos - nneg == pytest.approx(-2 * sigma / lz, rel=1e-12)
    assert nneg > 0
    assert wl.n0[:, 1:-1].sum(0) == pytest.approx(np.ones((lz, ly, lx)), abs=1e-15)


def test_bulk_electrolyte_ion_to_solvent_ratio():
    """n^+/n^0 = n^-/n^0 = 1e-2 (Sec. 4); the generator takes ion fractions
    of a total density 1, within 3% of that ratio at fraction 0.01 and
    exactly equal at fraction r/(1 + 2r)."""
    r = G["ion_to_solvent_density"]
    wl = WL.bulk_conductivity(shape=G["bulk_mesh"][::-1], fraction=0.01)
    ratio = wl.n0[1] / wl.n0[0]
    assert np.allclose(ratio, r, rtol=0.03)
    exact = WL.bulk_conductivity(shape=(4, 4, 4), fraction=r / (1 + 2 * r))
    assert np.allclose(exact.n0[1] / exact.n0[0], r, rtol=1e-12)
    assert np.allclose(exact.n0[2] / exact.n0[0], r, rtol=1e-12)


def test_printed_frequency_ratios_are_stable_at_the_printed_viscosity():
    """nu = v_T^2 (1/omega_visc - 1/2) = 1 (Sec. 4) gives omega_visc = 2/7;
    the two limiting omega_drag/omega_visc of the velocity-difference
    figure then give omega_drag = 0.1 and 1.5, both inside (0, 2), with
    D = v_T^2 (1/omega_drag - 1/2) = 19/6 and 1/18 (Sc = 6/19 and 18).  At
    omega_visc = 1 the ratio 5.25 would leave (0, 2): the printed ratios
    belong to nu = 1."""
    omega_visc = 1.0 / (G["nu"] / CS2 + 0.5)
    assert omega_visc == pytest.approx(2.0 / 7.0, rel=1e-14)
    od = [q * omega_visc for q in G["omega_drag_over_omega_visc"]]
    assert od == pytest.approx([0.1, 1.5], rel=1e-14)
    assert all(0.0 < w < 2.0 for w in od)
    D = [CS2 * (1.0 / w - 0.5) for w in od]
    assert D == pytest.approx([19.0 / 6.0, 1.0 / 18.0], rel=1e-13)
    assert [G["nu"] / d for d in D] == pytest.approx([6.0 / 19.0, 18.0], rel=1e-13)
    assert G["omega_drag_over_omega_visc"][1] * 1.0 > 2.0
