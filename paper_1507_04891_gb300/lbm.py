"""Python binding of the C ABI in include/lbm.h (ctypes; marshalling only).

Every numerical step runs in the CUDA library liblbm_gb300.so.  There is no
fallback: if the library is missing or no GPU is present, the calls raise.
Array layouts follow the C ABI: fields are (nz, ny, nx) with x fastest,
velocities (3, nz, ny, nx), populations (19, nz, ny, nx).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENOCONV, LBM_EUNSTABLE, LBM_ETIMEOUT = range(7)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                4: "LBM_ENOCONV", 5: "LBM_EUNSTABLE", 6: "LBM_ETIMEOUT"}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
LBM_FLAG_STEP_GRAPH = 1
LBM_FLAG_NO_EXTRAPOLATION = 2
LBM_FLAG_CHARGE_PASS = 4
POISSON = {"mg": 0, "sor": 1, "fft": 2}

# every symbol include/lbm.h declares
EXPORTED = [
    "lbm_config_default", "lbm_create", "lbm_destroy", "lbm_set_walls", "lbm_set_species",
    "lbm_step", "lbm_synchronize", "lbm_get_moments", "lbm_get_populations",
    "lbm_get_potential", "lbm_solve_poisson", "lbm_diagnostics", "lbm_get_state",
    "lbm_set_state", "lbm_set_timing", "lbm_get_timing", "lbm_num_nodes",
    "lbm_create_stack", "lbm_instance_z0", "lbm_set_plane_omega_drag", "lbm_autotune",
    "lbm_nn_init", "lbm_nn_collect", "lbm_nn_train", "lbm_nn_use", "lbm_nn_params",
    "lbm_nn_loss_grad", "lbm_nn_stats", "lbm_get_moments_noalloc", "lbm_state_len", "lbm_stream", "lbm_last_error",
    "lbm_set_species_dev", "lbm_get_moments_dev", "lbm_plane_fluxes", "lbm_omega_drag_for_schmidt",
    "lbm_set_drag_matrix", "lbm_poisson_stats", "lbm_nn_infer", "lbm_step_record",
]


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("nspecies", ctypes.c_int),
        ("omega_visc", ctypes.c_double), ("omega_drag", ctypes.c_double),
        ("bjerrum", ctypes.c_double), ("e_ext", ctypes.c_double * 3),
        ("storage", ctypes.c_int), ("poisson", ctypes.c_int),
        ("poisson_tol", ctypes.c_double), ("poisson_maxit", ctypes.c_int),
        ("device", ctypes.c_int), ("flags", ctypes.c_int),
    ]


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbm_gb300.so not found at %s: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')" % path)
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.lbm_config_default.argtypes = [ctypes.POINTER(LbmConfig)]
    lib.lbm_config_default.restype = None
    lib.lbm_create.argtypes = [ctypes.POINTER(LbmConfig), ctypes.POINTER(P)]
    lib.lbm_create.restype = I
    lib.lbm_destroy.argtypes = [P]
    lib.lbm_destroy.restype = None
    lib.lbm_set_walls.argtypes = [P, P, P]
    lib.lbm_set_walls.restype = I
    lib.lbm_set_species.argtypes = [P, I, D, D, P, P]
    lib.lbm_set_species.restype = I
    lib.lbm_step.argtypes = [P, I, V]
    lib.lbm_step.restype = I
    lib.lbm_step_record.argtypes = [P, I, P, V]
    lib.lbm_step_record.restype = I
    lib.lbm_synchronize.argtypes = [P]
    lib.lbm_synchronize.restype = I
    lib.lbm_get_moments.argtypes = [P, I, P, P]
    lib.lbm_get_moments.restype = I
    lib.lbm_get_moments_noalloc.argtypes = [P, I, P, P]
    lib.lbm_get_moments_noalloc.restype = I
    lib.lbm_get_populations.argtypes = [P, I, P]
    lib.lbm_get_populations.restype = I
    lib.lbm_get_potential.argtypes = [P, P]
    lib.lbm_get_potential.restype = I
    lib.lbm_solve_poisson.argtypes = [P, P, P, D, I, ctypes.POINTER(I), dp]
    lib.lbm_solve_poisson.restype = I
    lib.lbm_diagnostics.argtypes = [P, P]
    lib.lbm_diagnostics.restype = I
    lib.lbm_get_state.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
    lib.lbm_get_state.restype = I
    lib.lbm_set_state.argtypes = [P, P, ctypes.c_int64]
    lib.lbm_set_state.restype = I
    lib.lbm_set_timing.argtypes = [P, I]
    lib.lbm_set_timing.restype = I
    lib.lbm_get_timing.argtypes = [P, P]
    lib.lbm_get_timing.restype = I
    lib.lbm_create_stack.argtypes = [I, ctypes.POINTER(LbmConfig), ctypes.POINTER(P)]
    lib.lbm_create_stack.restype = I
    lib.lbm_instance_z0.argtypes = [P, I]
    lib.lbm_instance_z0.restype = I
    lib.lbm_set_plane_omega_drag.argtypes = [P, P]
    lib.lbm_set_plane_omega_drag.restype = I
    lib.lbm_autotune.argtypes = [P, P]
    lib.lbm_autotune.restype = I
    lib.lbm_nn_init.argtypes = [P, I, ctypes.c_uint64]
    lib.lbm_nn_init.restype = I
    lib.lbm_nn_collect.argtypes = [P, I]
    lib.lbm_nn_collect.restype = I
    lib.lbm_nn_train.argtypes = [P, I, D, P]
    lib.lbm_nn_train.restype = I
    lib.lbm_nn_use.argtypes = [P, I]
    lib.lbm_nn_use.restype = I
    lib.lbm_nn_params.argtypes = [P, P, P, ctypes.POINTER(I)]
    lib.lbm_nn_params.restype = I
    lib.lbm_nn_loss_grad.argtypes = [P, P, ctypes.POINTER(D), P]
    lib.lbm_nn_loss_grad.restype = I
    lib.lbm_nn_stats.argtypes = [P, P]
    lib.lbm_nn_stats.restype = I
    lib.lbm_num_nodes.argtypes = [P]
    lib.lbm_num_nodes.restype = ctypes.c_int64
    lib.lbm_state_len.argtypes = [P]
    lib.lbm_state_len.restype = ctypes.c_int64
    lib.lbm_stream.argtypes = [P]
    lib.lbm_stream.restype = P
    lib.lbm_last_error.argtypes = [P]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_set_species_dev.argtypes = [P, I, D, D, P, P, V]
    lib.lbm_set_species_dev.restype = I
    lib.lbm_get_moments_dev.argtypes = [P, I, P, P, V]
    lib.lbm_get_moments_dev.restype = I
    lib.lbm_plane_fluxes.argtypes = [P, P]
    lib.lbm_plane_fluxes.restype = I
    lib.lbm_omega_drag_for_schmidt.argtypes = [D, D]
    lib.lbm_omega_drag_for_schmidt.restype = D
    lib.lbm_set_drag_matrix.argtypes = [P, P]
    lib.lbm_set_drag_matrix.restype = I
    lib.lbm_poisson_stats.argtypes = [P, P]
    lib.lbm_poisson_stats.restype = I
    lib.lbm_nn_infer.argtypes = [P, P, P]
    lib.lbm_nn_infer.restype = I
    _lib = lib
    return lib


def make_config(nx, ny, nz, nspecies, omega_visc=1.0, omega_drag=1.0, bjerrum=0.0,
                e_ext=(0.0, 0.0, 0.0), storage="fp32", poisson="mg", poisson_tol=1e-8,
                poisson_maxit=200, device=0, step_graph=False, extrapolate=True, charge_pass=False):
    lib = load_library()
    cfg = LbmConfig()
    lib.lbm_config_default(ctypes.byref(cfg))
    cfg.nx, cfg.ny, cfg.nz, cfg.nspecies = int(nx), int(ny), int(nz), int(nspecies)
    cfg.omega_visc, cfg.omega_drag, cfg.bjerrum = float(omega_visc), float(omega_drag), float(bjerrum)
    for d in range(3):
        cfg.e_ext[d] = float(e_ext[d])
    cfg.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    cfg.poisson = POISSON[poisson] if isinstance(poisson, str) else int(poisson)
    cfg.poisson_tol, cfg.poisson_maxit, cfg.device = float(poisson_tol), int(poisson_maxit), int(device)
    cfg.flags = (LBM_FLAG_STEP_GRAPH if step_graph else 0) | \
                (0 if extrapolate else LBM_FLAG_NO_EXTRAPOLATION) | \
                (LBM_FLAG_CHARGE_PASS if charge_pass else 0)
    return cfg


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def omega_drag_for_schmidt(omega_visc: float, schmidt: float) -> float:
    """lbm_omega_drag_for_schmidt: omega_drag with Sc = nu/D (Sec. 4 of the
    paper); raises for omega_visc outside (0, 2) or Sc <= 0."""
    od = float(load_library().lbm_omega_drag_for_schmidt(float(omega_visc), float(schmidt)))
    if od == 0.0:
        raise ValueError("omega_visc must lie in (0, 2) and the Schmidt number be positive")
    return od


class Lattice:
    """One lattice handle (lbm_t).  Methods carry the names of the C calls.

    Constructor arguments are the fields of lbm_config: storage "fp32",
    "fp16" or "bf16"; poisson "mg", "sor" or "fft"; step_graph sets
    LBM_FLAG_STEP_GRAPH (spectral solver only); extrapolate=False sets
    LBM_FLAG_NO_EXTRAPOLATION (each solve starts from the previous potential
    instead of its extrapolation in time); charge_pass=True sets
    LBM_FLAG_CHARGE_PASS (the charge density by a separate pass each step,
    not scattered by the previous stream/collide)."""

    def __init__(self, nx, ny, nz, nspecies, omega_visc=1.0, omega_drag=1.0,
                 bjerrum=0.0, e_ext=(0.0, 0.0, 0.0), storage="fp32", poisson="mg",
                 poisson_tol=1e-8, poisson_maxit=200, device=0, step_graph=False,
                 extrapolate=True, charge_pass=False, _stack=None):
        self._lib = load_library()
        cfg = make_config(nx, ny, nz, nspecies, omega_visc, omega_drag, bjerrum, e_ext, storage,
                          poisson, poisson_tol, poisson_maxit, device, step_graph, extrapolate,
                          charge_pass)
        self.cfg = cfg
        self.S = int(nspecies)
        h = ctypes.c_void_p()
        if _stack is None:
            st = self._lib.lbm_create(ctypes.byref(cfg), ctypes.byref(h))
        else:
            arr = (LbmConfig * len(_stack))(*_stack)
            st = self._lib.lbm_create_stack(len(_stack), arr, ctypes.byref(h))
            nz = sum(c.nz for c in _stack)
        if st != LBM_OK:
            raise LBMError(st, self._lib.lbm_last_error(None).decode())
        self.shape = (int(nz), int(ny), int(nx))
        self.h = h
        self.N = int(self._lib.lbm_num_nodes(h))

    @classmethod
    def create_stack(cls, nx, ny, nzs, omega_drags, nspecies, **kw):
        """lbm_create_stack: instances of extents nzs[i] and drag
        frequencies omega_drags[i] stacked along z."""
        cfgs = [make_config(nx, ny, nz_i, nspecies, kw.get("omega_visc", 1.0), od,
                            kw.get("bjerrum", 0.0), kw.get("e_ext", (0.0, 0.0, 0.0)),
                            kw.get("storage", "fp32"), kw.get("poisson", "fft"),
                            kw.get("poisson_tol", 1e-8), kw.get("poisson_maxit", 200),
                            kw.get("device", 0), kw.get("step_graph", False),
                            kw.get("extrapolate", True))
                for nz_i, od in zip(nzs, omega_drags)]
        return cls(nx, ny, sum(nzs), nspecies, _stack=cfgs)

    def instance_z0(self, i):
        return int(self._lib.lbm_instance_z0(self.h, int(i)))

    def set_drag_matrix(self, omega):
        """lbm_set_drag_matrix: symmetric (S, S) matrix of pair drag
        frequencies, or None for the config's single omega_drag."""
        w = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
        if w is not None and w.shape != (self.S, self.S):
            raise ValueError("the drag matrix must be (S, S)")
        self._check(self._lib.lbm_set_drag_matrix(self.h, _ptr(w)))

    def set_plane_omega_drag(self, omega):
        om = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
        if om is not None and om.shape != (self.shape[0],):
            raise ValueError("one omega per z-plane")
        self._check(self._lib.lbm_set_plane_omega_drag(self.h, _ptr(om)))

    # -- learned Poisson initial guess --------------------------------------
    def nn_init(self, hidden=8, seed=1):
        self._check(self._lib.lbm_nn_init(self.h, int(hidden), int(seed)))

    def nn_collect(self, capacity):
        self._check(self._lib.lbm_nn_collect(self.h, int(capacity)))

    def nn_train(self, epochs, lr=1e-2):
        losses = np.zeros(max(1, int(epochs)))
        self._check(self._lib.lbm_nn_train(self.h, int(epochs), float(lr), _ptr(losses)))
        return losses[:int(epochs)]

    def nn_use(self, enable=True):
        self._check(self._lib.lbm_nn_use(self.h, int(bool(enable))))

    def nn_params(self, set_to=None):
        n = ctypes.c_int(0)
        self._check(self._lib.lbm_nn_params(self.h, None, None, ctypes.byref(n)))
        out = np.empty(n.value, dtype=np.float32)
        src = None if set_to is None else np.ascontiguousarray(set_to, dtype=np.float32)
        self._check(self._lib.lbm_nn_params(self.h, _ptr(out), _ptr(src), ctypes.byref(n)))
        return out

    def nn_loss_grad(self, x0, grad=True):
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
        if x0.shape != self.shape:
            raise ValueError("x0 must have the lattice shape")
        loss = ctypes.c_double(0.0)
        n = ctypes.c_int(0)
        self._check(self._lib.lbm_nn_params(self.h, None, None, ctypes.byref(n)))
        g = np.zeros(n.value, dtype=np.float32) if grad else None
        self._check(self._lib.lbm_nn_loss_grad(self.h, _ptr(x0), ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def nn_infer(self, x0):
        """lbm_nn_infer: the solver's FP16 inference pass on x0 (lattice
        shape); returns y, the correction in units of the residual rms."""
        x0 = np.ascontiguousarray(x0, dtype=np.float32)
        if x0.shape != self.shape:
            raise ValueError("x0 must have the lattice shape")
        y = np.empty(self.shape, dtype=np.float32)
        self._check(self._lib.lbm_nn_infer(self.h, _ptr(x0), _ptr(y)))
        return y

    def nn_stats(self):
        out = np.zeros(5)
        self._check(self._lib.lbm_nn_stats(self.h, _ptr(out)))
        return {"tried": int(out[0]), "kept": int(out[1]), "mean_ratio": out[2],
                "collected": int(out[3]), "nparams": int(out[4])}

    def autotune(self):
        out = np.zeros(4)
        self._check(self._lib.lbm_autotune(self.h, _ptr(out)))
        return {"collide_threads": int(out[0]), "collide_ms": out[1],
                "charge_threads": int(out[2]), "charge_ms": out[3]}

    # -- helpers -----------------------------------------------------------
    def _check(self, st, allow=()):
        if st != LBM_OK and st not in allow:
            raise LBMError(st, self._lib.lbm_last_error(self.h).decode())
        return st

    def _field(self, a, comps=None):
        a = np.ascontiguousarray(a, dtype=np.float64)
        want = self.shape if comps is None else (comps,) + self.shape
        if a.shape != want:
            raise ValueError("expected shape %s, got %s" % (want, a.shape))
        return a

    # -- C calls -------------------------------------------------------------
    def set_walls(self, solid, sigma=None):
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        if solid.shape != self.shape:
            raise ValueError("solid must have shape %s" % (self.shape,))
        sig = None if sigma is None else self._field(sigma)
        self._check(self._lib.lbm_set_walls(self.h, _ptr(solid), _ptr(sig)))

    def set_species(self, s, mass, valence, n0, u0=None):
        n0 = self._field(n0)
        u0 = None if u0 is None else self._field(u0, 3)
        self._check(self._lib.lbm_set_species(self.h, int(s), float(mass), float(valence),
                                              _ptr(n0), _ptr(u0)))

    def step(self, nsteps=1, stream=None, allow_noconv=False):
        return self._check(self._lib.lbm_step(self.h, int(nsteps),
                                              ctypes.c_void_p(stream) if stream else None),
                           allow=(LBM_ENOCONV,) if allow_noconv else ())

    def synchronize(self):
        self._check(self._lib.lbm_synchronize(self.h))

    def get_moments(self, s):
        n = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self._check(self._lib.lbm_get_moments(self.h, int(s), _ptr(n), _ptr(u)))
        return n, u

    def set_species_dev(self, s, mass, valence, n0_ptr, u0_ptr=None, stream=None):
        """lbm_set_species_dev: n0_ptr / u0_ptr are device addresses (for
        example torch tensors' data_ptr()) of N and 3N doubles."""
        self._check(self._lib.lbm_set_species_dev(
            self.h, int(s), float(mass), float(valence), ctypes.c_void_p(int(n0_ptr)),
            ctypes.c_void_p(int(u0_ptr)) if u0_ptr else None,
            ctypes.c_void_p(int(stream)) if stream else None))

    def get_moments_dev(self, s, n_ptr, u_ptr=None, stream=None):
        """lbm_get_moments_dev: queues the moments of species s into device
        memory at n_ptr (N doubles) and u_ptr (3N doubles) on `stream`."""
        self._check(self._lib.lbm_get_moments_dev(
            self.h, int(s), ctypes.c_void_p(int(n_ptr)) if n_ptr else None,
            ctypes.c_void_p(int(u_ptr)) if u_ptr else None,
            ctypes.c_void_p(int(stream)) if stream else None))

    def plane_fluxes(self):
        """lbm_plane_fluxes: array (nz, S, 4) of plane sums of n and of the
        mid-step flux n (u + F/2) (x, y, z)."""
        out = np.empty((self.shape[0], self.S, 4))
        self._check(self._lib.lbm_plane_fluxes(self.h, _ptr(out)))
        return out

    def get_moments_noalloc(self, s):
        """lbm_get_moments_noalloc: no device allocation (static staging)."""
        n = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self._check(self._lib.lbm_get_moments_noalloc(self.h, int(s), _ptr(n), _ptr(u)))
        return n, u

    def get_populations(self, s):
        f = np.empty((19,) + self.shape)
        self._check(self._lib.lbm_get_populations(self.h, int(s), _ptr(f)))
        return f

    def get_potential(self):
        psi = np.empty(self.shape)
        self._check(self._lib.lbm_get_potential(self.h, _ptr(psi)))
        return psi

    def solve_poisson(self, rho_e, psi0=None, tol=1e-8, maxit=0):
        rho = self._field(rho_e)
        psi = np.zeros(self.shape) if psi0 is None else self._field(psi0).copy()
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        st = self._check(self._lib.lbm_solve_poisson(self.h, _ptr(rho), _ptr(psi), float(tol),
                                                     int(maxit), ctypes.byref(it), ctypes.byref(res)),
                         allow=(LBM_ENOCONV,))
        return psi, it.value, res.value, st

    def diagnostics(self):
        out = np.empty(self.S + 7)
        st = self._check(self._lib.lbm_diagnostics(self.h, _ptr(out)), allow=(LBM_EUNSTABLE,))
        S = self.S
        return {"mass": out[:S].copy(), "momentum": out[S:S + 3].copy(), "charge": out[S + 3],
                "poisson_iters": int(out[S + 4]), "poisson_residual": out[S + 5],
                "steps": int(out[S + 6]), "unstable": st == LBM_EUNSTABLE, "raw": out}

    def step_record(self, nsteps, stream=None):
        """nsteps steps, each with its diagnostics read back (lbm_step_record):
        an array of nsteps rows in the layout of diagnostics()["raw"]."""
        out = np.empty((max(0, int(nsteps)), self.S + 7))
        self._check(self._lib.lbm_step_record(self.h, int(nsteps), _ptr(out),
                                              ctypes.c_void_p(stream) if stream else None))
        return out

    def get_state(self):
        n = int(self._lib.lbm_state_len(self.h))
        buf = np.empty(n, dtype=np.float32)
        step = ctypes.c_int64(0)
        self._check(self._lib.lbm_get_state(self.h, _ptr(buf), ctypes.byref(step)))
        return buf, step.value

    def set_state(self, buf, step):
        buf = np.ascontiguousarray(buf, dtype=np.float32)
        if buf.size != int(self._lib.lbm_state_len(self.h)):
            raise ValueError("state has the wrong length")
        self._check(self._lib.lbm_set_state(self.h, _ptr(buf), int(step)))

    def set_timing(self, enable=True):
        self._check(self._lib.lbm_set_timing(self.h, int(bool(enable))))

    def get_timing(self):
        out = np.zeros(7)
        self._check(self._lib.lbm_get_timing(self.h, _ptr(out)))
        return {"charge_ms": out[0], "poisson_ms": out[1], "collide_ms": out[2],
                "charge_launches": int(out[3]), "poisson_iters": int(out[4]),
                "collide_launches": int(out[5]), "kernel_launches": int(out[6])}

    def poisson_stats(self):
        """lbm_poisson_stats: iterations, start and end relative residuals of
        the last solve, and the geometric-mean start residual since
        set_timing."""
        out = np.zeros(5)
        self._check(self._lib.lbm_poisson_stats(self.h, _ptr(out)))
        return {"iters": int(out[0]), "start_residual": out[1], "final_residual": out[2],
                "solves": int(out[3]), "start_residual_geomean": 10.0 ** out[4] if out[3] else None}

    @property
    def stream(self):
        return int(self._lib.lbm_stream(self.h) or 0)

    def destroy(self):
        if getattr(self, "h", None):
            self._lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def from_workload(wl, storage="fp32", poisson="mg", poisson_tol=1e-8, poisson_maxit=200,
                  omega_drag=None, device=0):
    """Creates and initialises a lattice from a workloads.Workload."""
    nz, ny, nx = wl.shape
    od = omega_drag if omega_drag is not None else omega_drag_for_schmidt(wl.omega_visc, wl.schmidt)
    lat = Lattice(nx, ny, nz, wl.nspecies, omega_visc=wl.omega_visc, omega_drag=od,
                  bjerrum=wl.bjerrum, e_ext=wl.e_ext, storage=storage, poisson=poisson,
                  poisson_tol=poisson_tol, poisson_maxit=poisson_maxit, device=device)
    if wl.solid is not None:
        lat.set_walls(wl.solid, wl.sigma)
    for s in range(wl.nspecies):
        u0 = None if wl.u0 is None else wl.u0[s]
        lat.set_species(s, wl.mass[s], wl.valence[s], wl.n0[s], u0)
    return lat


def stack_slits(instances, storage="fp16", step_graph=True, poisson_tol=1e-8, device=0,
                extrapolate=True):
    """Batched independent slit channels (workloads.slit instances sharing
    nx, ny, omega_visc, l_B and the applied field) stacked along z in one
    lattice: each instance keeps its own walls, wall charge and drag
    frequency.  Returns (lattice, list of first planes)."""
    nx = instances[0].shape[2]
    ny = instances[0].shape[1]
    nzs = [w.shape[0] for w in instances]
    ods = [omega_drag_for_schmidt(w.omega_visc, w.schmidt) for w in instances]
    w0 = instances[0]
    lat = Lattice.create_stack(nx, ny, nzs, ods, w0.nspecies, omega_visc=w0.omega_visc,
                               bjerrum=w0.bjerrum, e_ext=w0.e_ext, storage=storage, poisson="fft",
                               poisson_tol=poisson_tol, device=device, step_graph=step_graph,
                               extrapolate=extrapolate)
    solid = np.concatenate([w.solid for w in instances], axis=0)
    sigma = np.concatenate([w.sigma for w in instances], axis=0)
    lat.set_walls(solid, sigma)
    for s in range(w0.nspecies):
        n0 = np.concatenate([np.where(w.solid, 1.0, w.n0[s]) for w in instances], axis=0)
        lat.set_species(s, w0.mass[s], w0.valence[s], n0)
    z0 = [lat.instance_z0(i) for i in range(len(instances))]
    return lat, z0
