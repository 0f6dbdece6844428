"""The C-ABI library builds for sm_103a, loads on a machine without a GPU and
exports every entry point include/sr3d.h declares; argument validation that
happens before any CUDA call is checked here too."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sr3d.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(sr3d_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_2010_15491_gb300.build import build
    return build()


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for need in ("sr3d_plan", "sr3d_tikhonov", "sr3d_admm_tv", "sr3d_destroy"):
        assert need in syms


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sr3d_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(built)
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_binding_covers_the_header(built):
    import paper_2010_15491_gb300 as sr3d
    assert sorted(sr3d.EXPORTED) == declared_symbols()
    sr3d.load()


def test_library_is_built_for_sm_103a(built):
    out = subprocess.run(["cuobjdump", "--list-elf", built], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def _plan_rc(**kw):
    import paper_2010_15491_gb300 as sr3d
    L = sr3d.load()
    psf = np.ones((3, 3, 3)) / 27.0
    base = dict(m_h=64, n_h=64, s_h=64, dr=2, dc=2, ds=2, p_m=3, p_n=3, p_s=3, dtype=0)
    base.update(kw)
    d = sr3d.Desc(base["m_h"], base["n_h"], base["s_h"], base["dr"], base["dc"], base["ds"],
                  psf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), base["p_m"], base["p_n"], base["p_s"],
                  base["dtype"], None)
    h = ctypes.c_void_p()
    rc = L.sr3d_plan(ctypes.byref(h), ctypes.byref(d))
    if rc == 0:
        L.sr3d_destroy(h)
    return rc, L.sr3d_last_error().decode()


@pytest.mark.parametrize("kw,code", [
    (dict(m_h=0), -1), (dict(dr=0), -1), (dict(dtype=7), -1), (dict(p_m=99), -1),
    (dict(m_h=96, dr=5), -2), (dict(n_h=64, dc=3), -2),
    (dict(m_h=80, dr=1), -3), (dict(m_h=48, dr=1), -3), (dict(n_h=12, dc=1), -3),
    (dict(m_h=64, dr=4, n_h=64, dc=4), -3), (dict(m_h=32, dr=32), -3), (dict(s_h=2, ds=1, p_s=1), -3),
])
def test_plan_rejects_bad_descriptors_before_touching_the_gpu(built, kw, code):
    rc, msg = _plan_rc(**kw)
    assert rc == code, (rc, msg)
    assert msg


def test_null_arguments_are_rejected(built):
    import paper_2010_15491_gb300 as sr3d
    L = sr3d.load()
    assert L.sr3d_plan(None, None) == -1
    assert L.sr3d_tikhonov(None, None, None, 1.0, None) == -1
    assert L.sr3d_admm_tv(None, None, None, None, 1e-3, 1e-2, 10, 0.0, 0.0, None) == -1
    assert L.sr3d_destroy(None) == 0
    assert "NULL" in L.sr3d_last_error().decode()
