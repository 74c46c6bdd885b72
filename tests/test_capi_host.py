"""Host-side checks of the C ABI library (no GPU): it builds, loads and
exports every symbol include/lbm.h declares."""

import ctypes
import os
import re
import subprocess

import pytest

from paper_1507_04891_gb300 import lbm
from paper_1507_04891_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return build_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)) - {"lbm_t"})


def test_header_declares_the_binding_list():
    assert declared_symbols() == sorted(lbm.EXPORTED)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(lbm_[a-z_0-9]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for s in declared_symbols():
        assert getattr(lib, s) is not None


def test_config_default_is_host_only(libpath):
    lib = lbm.load_library(libpath)
    cfg = lbm.LbmConfig()
    lib.lbm_config_default(ctypes.byref(cfg))
    assert (cfg.nx, cfg.ny, cfg.nz, cfg.nspecies) == (1, 1, 1, 1)
    assert cfg.omega_visc == 1.0 and cfg.poisson_tol == 1e-8 and cfg.poisson_maxit == 200


def test_create_rejects_bad_arguments_before_touching_a_device(libpath):
    lib = lbm.load_library(libpath)
    cfg = lbm.LbmConfig()
    lib.lbm_config_default(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    for field, value in [("nx", 0), ("nspecies", 5), ("omega_visc", 2.0), ("omega_drag", 0.0),
                         ("storage", 7), ("poisson", 9)]:
        bad = lbm.LbmConfig.from_buffer_copy(cfg)
        setattr(bad, field, value)
        assert lib.lbm_create(ctypes.byref(bad), ctypes.byref(h)) == lbm.LBM_EINVAL
        assert h.value is None
        assert lib.lbm_last_error(None)
    assert lib.lbm_create(None, ctypes.byref(h)) == lbm.LBM_EINVAL


def test_null_handle_calls_are_rejected(libpath):
    lib = lbm.load_library(libpath)
    assert lib.lbm_step(None, 1, None) == lbm.LBM_EINVAL
    assert lib.lbm_get_moments(None, 0, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_diagnostics(None, None) == lbm.LBM_EINVAL
    assert lib.lbm_num_nodes(None) == 0
    lib.lbm_destroy(None)


def test_omega_for_schmidt_matches_paper_relations():
    # nu = cs^2 (1/w_v - 1/2), D = cs^2 (1/w_d - 1/2), Sc = nu / D
    for wv, sc in [(1.0, 10.0), (1.0, 1.0), (0.8, 1000.0)]:
        wd = lbm.omega_drag_for_schmidt(wv, sc)
        nu = (1 / wv - 0.5) / 3
        D = (1 / wd - 0.5) / 3
        assert abs(nu / D - sc) < 1e-9 * sc
    assert abs(lbm.omega_drag_for_schmidt(1.0, 10.0) - 1 / 0.55) < 1e-12


def test_config_layout_matches_c_compiler(tmp_path):
    """ctypes mirror of lbm_config has the C compiler's size and offsets."""
    fields = [f for f, _ in lbm.LbmConfig._fields_]
    src = tmp_path / "layout.c"
    body = "".join('printf("%%s %%zu\\n", "%s", offsetof(lbm_config, %s));' % (f, f) for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                   'int main(void){printf("size %zu\\n", sizeof(lbm_config));' + body + 'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(lbm.LbmConfig)
    for f in fields:
        assert int(out[f]) == getattr(lbm.LbmConfig, f).offset, f


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, storage and solver codes and flag bits of the binding
    are the values the C compiler sees in include/lbm.h."""
    names = {"LBM_OK": lbm.LBM_OK, "LBM_EINVAL": lbm.LBM_EINVAL, "LBM_ENOMEM": lbm.LBM_ENOMEM,
             "LBM_ECUDA": lbm.LBM_ECUDA, "LBM_ENOCONV": lbm.LBM_ENOCONV,
             "LBM_EUNSTABLE": lbm.LBM_EUNSTABLE, "LBM_ETIMEOUT": lbm.LBM_ETIMEOUT,
             "LBM_FP32": lbm.STORAGE["fp32"], "LBM_FP16_SHIFT": lbm.STORAGE["fp16"],
             "LBM_BF16_SHIFT": lbm.STORAGE["bf16"], "LBM_POISSON_MG": lbm.POISSON["mg"],
             "LBM_POISSON_SOR": lbm.POISSON["sor"], "LBM_POISSON_FFT": lbm.POISSON["fft"],
             "LBM_FLAG_STEP_GRAPH": lbm.LBM_FLAG_STEP_GRAPH,
             "LBM_FLAG_NO_EXTRAPOLATION": lbm.LBM_FLAG_NO_EXTRAPOLATION,
             "LBM_FLAG_CHARGE_PASS": lbm.LBM_FLAG_CHARGE_PASS}
    src = tmp_path / "consts.c"
    body = "".join('printf("%s %%d\\n", (int)(%s));' % (n, n) for n in names)
    src.write_text('#include <stdio.h>\n#include "lbm.h"\nint main(void){' + body + 'return 0;}\n')
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for n, v in names.items():
        assert int(out[n]) == v, n
    # flag bits are distinct powers of two
    flags = [lbm.LBM_FLAG_STEP_GRAPH, lbm.LBM_FLAG_NO_EXTRAPOLATION, lbm.LBM_FLAG_CHARGE_PASS]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)
    cfg = lbm.make_config(8, 8, 8, 1, step_graph=True, extrapolate=False)
    assert cfg.flags == lbm.LBM_FLAG_STEP_GRAPH | lbm.LBM_FLAG_NO_EXTRAPOLATION
    cfg = lbm.make_config(8, 8, 8, 1, charge_pass=True)
    assert cfg.flags == lbm.LBM_FLAG_CHARGE_PASS


def test_omega_drag_for_schmidt_inverts_the_lattice_transport_coefficients(libpath):
    """lbm_omega_drag_for_schmidt is host arithmetic: the drag frequency it
    returns must give back Sc = nu / D with the lattice nu and D of Sec. 4,
    and the frequencies of the benchmark's Schmidt numbers at omega_visc = 1."""
    lib = lbm.load_library(libpath)
    f = lib.lbm_omega_drag_for_schmidt
    for ov in (0.3, 1.0, 1.7):
        for sc in (0.5, 1.0, 10.0, 100.0, 1000.0):
            od = f(ov, sc)
            assert 0.0 < od < 2.0
            nu = (1.0 / ov - 0.5) / 3.0
            D = (1.0 / od - 0.5) / 3.0
            assert abs(nu / D / sc - 1.0) < 1e-12
    assert f(1.0, 1.0) == 1.0
    for sc, od in ((10.0, 20.0 / 11.0), (100.0, 200.0 / 101.0), (1000.0, 2000.0 / 1001.0)):
        assert abs(f(1.0, sc) - od) < 1e-15
    for ov, sc in ((0.0, 1.0), (2.0, 1.0), (1.0, 0.0), (1.0, -3.0), (1.0, float("inf"))):
        assert f(ov, sc) == 0.0
