"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only input generation (initial densities, wall masks, wall
charges, parameter sets): none of the lattice Boltzmann arithmetic.  Both the
CUDA path (through the C ABI) and the FP64 oracle take their inputs from
here, as plain numpy arrays.  Random numbers come from numpy's PCG64 with a
stated seed.

Shapes follow the (nz, ny, nx) layout with x fastest; species densities have
shape (S, nz, ny, nx).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    shape: tuple                      # (nz, ny, nx)
    n0: np.ndarray                    # (S, nz, ny, nx) initial number densities
    mass: np.ndarray                  # (S,)
    valence: np.ndarray               # (S,)
    omega_visc: float
    schmidt: float
    bjerrum: float = 0.0
    e_ext: tuple = (0.0, 0.0, 0.0)
    solid: np.ndarray | None = None   # (nz, ny, nx) bool
    sigma: np.ndarray | None = None   # (nz, ny, nx) charge per solid node
    u0: np.ndarray | None = None      # (S, 3, nz, ny, nx)
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nspecies(self):
        return self.n0.shape[0]

    @property
    def sites(self):
        return int(np.prod(self.shape))


def binary_sinusoid(n=32, ny=None, nz=None, amplitude=0.01, schmidt=10.0,
                    omega_visc=1.0, steps=200):
    """Neutral binary mixture, total density 1, species-A fraction
    0.5 + amplitude*sin(2 pi x / n), zero velocity (bulk mutual diffusion
    experiment of the paper, 32^3 periodic here)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    x = np.arange(n, dtype=np.float64)
    a = 0.5 + amplitude * np.sin(2.0 * math.pi * x / n)
    nA = np.broadcast_to(a, (nz, ny, n)).copy()
    n0 = np.stack([nA, 1.0 - nA])
    return Workload("binary_sinusoid_%dx%dx%d" % (n, ny, nz), (nz, ny, n), n0,
                    np.ones(2), np.zeros(2), omega_visc, schmidt, steps=steps)


def binary_random(shape, seed, schmidt=10.0, omega_visc=1.0, amplitude=0.02,
                  velocity=0.02):
    """Binary mixture with i.i.d. uniform density and velocity perturbations
    (parity and invariant tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    a = 0.5 + rng.uniform(-amplitude, amplitude, size=shape)
    b = 0.5 + rng.uniform(-amplitude, amplitude, size=shape)
    u0 = rng.uniform(-velocity, velocity, size=(2, 3) + tuple(shape))
    return Workload("binary_random", tuple(shape), np.stack([a, b]), np.ones(2),
                    np.zeros(2), omega_visc, schmidt, u0=u0)


def ternary_bulk(n=128, seed=1235, schmidt=1.0, omega_visc=1.0, bjerrum=0.7,
                 fraction=0.01, spread=1e-3, steps=1000, shape=None):
    """Charged ternary mixture (solvent z=0, cation z=+1, anion z=-1), ion
    number fractions `fraction` plus i.i.d. uniform +/- `spread`, solvent
    fills total density 1, zero velocity, periodic."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n) if shape is None else tuple(shape)
    xp = fraction + rng.uniform(-spread, spread, size=shape)
    xm = fraction + rng.uniform(-spread, spread, size=shape)
    n0 = np.stack([1.0 - xp - xm, xp, xm])
    return Workload("ternary_bulk_%dx%dx%d" % shape[::-1], shape, n0, np.ones(3),
                    np.array([0.0, 1.0, -1.0]), omega_visc, schmidt,
                    bjerrum=bjerrum, steps=steps, meta={"seed": seed})


def bulk_conductivity(n=64, fraction=0.01, e_field=1e-3, schmidt=1.0, omega_visc=1.0,
                      bjerrum=0.7, shape=None):
    """Uniform neutral ternary electrolyte (solvent z=0, cation z=+1, anion
    z=-1, ion number fractions `fraction`, solvent fills total density 1)
    in a uniform field along x: the bulk conductivity experiment (Sec. 4,
    current against D, Eq. Drude).  No random numbers."""
    shape = (n, n, n) if shape is None else tuple(shape)
    ones = np.ones(shape)
    n0 = np.stack([(1.0 - 2 * fraction) * ones, fraction * ones, fraction * ones])
    return Workload("bulk_conductivity_%dx%dx%d" % shape[::-1], shape, n0, np.ones(3),
                    np.array([0.0, 1.0, -1.0]), omega_visc, schmidt, bjerrum=bjerrum,
                    e_ext=(e_field, 0.0, 0.0), meta={"fraction": fraction})


def slit(nx=64, ny=64, width=64, sigma=-0.01, debye=8.0, bjerrum=0.7,
         e_field=1e-4, schmidt=1.0, omega_visc=1.0, steps=20000):
    """Charged slit channel: solid planes z = 0 and z = width + 1, each wall
    node carrying charge `sigma`; electrolyte with bulk ion density fixed by
    the Debye length, lambda_D = 1/sqrt(4 pi l_B (n+ + n-)); counter-ion
    excess spread uniformly so that fluid + wall charge is zero; applied
    field along x."""
    nz = width + 2
    shape = (nz, ny, nx)
    solid = np.zeros(shape, dtype=bool)
    solid[0] = True
    solid[-1] = True
    sig = np.zeros(shape)
    sig[0] = sigma
    sig[-1] = sigma
    nbulk = 1.0 / (4.0 * math.pi * bjerrum * debye * debye)
    excess = -2.0 * sigma / width           # n+ - n- needed for neutrality
    npos = 0.5 * (nbulk + excess)
    nneg = 0.5 * (nbulk - excess)
    if nneg <= 0:
        raise ValueError("wall charge too large for this Debye length")
    n0 = np.zeros((3,) + shape)
    n0[1, 1:-1] = npos
    n0[2, 1:-1] = nneg
    n0[0, 1:-1] = 1.0 - npos - nneg
    return Workload("slit_%dx%dx%d" % (nx, ny, nz), shape, n0, np.ones(3),
                    np.array([0.0, 1.0, -1.0]), omega_visc, schmidt,
                    bjerrum=bjerrum, e_ext=(e_field, 0.0, 0.0), solid=solid,
                    sigma=sig, steps=steps,
                    meta={"nbulk": nbulk, "sigma": sigma, "debye": debye})


def porous_spheres(n=256, seed=1238, solid_fraction=0.20, rmin=4, rmax=12,
                   surface_charge=0.01, bjerrum=0.7, fraction=0.01,
                   schmidt=1.0, omega_visc=1.0):
    """Periodic box with seeded random spheres (radius U{rmin..rmax}, overlaps
    allowed) placed until the solid fraction reaches the target; every solid
    node with a fluid face neighbour carries +/- surface_charge, the sign
    drawn per sphere; ions neutralise the total wall charge uniformly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, n, n)
    solid = np.zeros(shape, dtype=bool)
    sign = np.zeros(shape)
    nsolid, target = 0, solid_fraction * n ** 3
    while nsolid < target:
        c = rng.integers(0, n, size=3)
        r = int(rng.integers(rmin, rmax + 1))
        s = 1.0 if rng.random() < 0.5 else -1.0
        # the nodes within distance r of c (periodic, nearest image), taken
        # from the bounding box of the sphere only (the whole axis when the
        # box would wrap onto itself)
        def offsets(ci):
            if 2 * r + 1 <= n:
                return np.arange(-r, r + 1)
            return (np.arange(n) - ci + n // 2) % n - n // 2
        oz, oy, ox = offsets(c[0]), offsets(c[1]), offsets(c[2])
        iz, iy, ix = (c[0] + oz) % n, (c[1] + oy) % n, (c[2] + ox) % n
        inside = (oz[:, None, None] ** 2 + oy[None, :, None] ** 2 + ox[None, None, :] ** 2) <= r * r
        box = np.ix_(iz, iy, ix)
        new = inside & ~solid[box]
        sub = sign[box]
        sub[new] = s
        sign[box] = sub
        solid[box] |= inside
        nsolid += int(new.sum())
    fluid = ~solid
    surface = np.zeros(shape, dtype=bool)
    for ax in range(3):
        for sh in (1, -1):
            surface |= solid & np.roll(fluid, sh, axis=ax)
    sig = np.where(surface, surface_charge * sign, 0.0)
    qwall = sig.sum()
    nfl = fluid.sum()
    excess = -qwall / nfl
    npos = fraction + 0.5 * excess
    nneg = fraction - 0.5 * excess
    n0 = np.zeros((3,) + shape)
    n0[1][fluid] = npos
    n0[2][fluid] = nneg
    n0[0][fluid] = 1.0 - npos - nneg
    return Workload("porous_%d" % n, shape, n0, np.ones(3), np.array([0.0, 1.0, -1.0]),
                    omega_visc, schmidt, bjerrum=bjerrum, solid=solid, sigma=sig,
                    meta={"seed": seed, "solid_fraction": float(solid.mean())})


def random_solid(shape, seed, fraction=0.15):
    """I.i.d. random wall nodes with charges U[-0.02, 0.02] (edge-case tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    solid = rng.random(shape) < fraction
    sig = np.where(solid, rng.uniform(-0.02, 0.02, size=shape), 0.0)
    return solid, sig


def batched_slits(count=64, seed=1237, nx=32, ny=32, wmin=16, wmax=128,
                  sc_min=1.0, sc_max=1000.0, sig_min=-0.02, sig_max=-0.002,
                  debye=8.0, bjerrum=0.7, e_field=1e-4):
    """Parameters of the batched slit sweep: widths U{wmin..wmax}, Schmidt
    number log-uniform, wall charge per node uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    widths = rng.integers(wmin, wmax + 1, size=count)
    scs = np.exp(rng.uniform(math.log(sc_min), math.log(sc_max), size=count))
    sigs = rng.uniform(sig_min, sig_max, size=count)
    return [slit(nx=nx, ny=ny, width=int(w), sigma=float(s), debye=debye,
                 bjerrum=bjerrum, e_field=e_field, schmidt=float(sc))
            for w, sc, s in zip(widths, scs, sigs)]
