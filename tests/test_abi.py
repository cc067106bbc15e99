"""The C-ABI library builds, loads and exports every symbol include/ctfmm.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fmm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2305_17867_gb300 import build_ext

    path = build_ext.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_2305_17867_gb300 import _lib

    assert set(_lib.EXPORTS) <= set(declared_symbols())


def test_status_strings_without_gpu():
    from paper_2305_17867_gb300 import _lib

    L = _lib.load()
    assert L.fmm_status_string(0) == b"ok"
    assert L.fmm_status_string(-6).startswith(b"point outside")


def test_plan_validation_without_gpu():
    # descriptions that fmm_plan_create rejects before any CUDA call
    from paper_2305_17867_gb300 import _lib

    L = _lib.load()

    def create(**kw):
        d = _lib.PlanDesc()
        d.kernel, d.d, d.p, d.levels, d.root_size = 0, 3, 8, 3, 1.0
        for k, v in kw.items():
            setattr(d, k, v)
        h = ctypes.c_void_p()
        rc = L.fmm_plan_create(ctypes.byref(h), ctypes.byref(d))
        assert not h.value
        return rc

    for prec in (2, 3, 4, 5):  # tensor-core formats have no FFT form
        assert create(precision=prec, m2l=1) == -2
    assert create(precision=5, levels=-4, max_leaf=64) == -2  # F16X3: uniform trees
    assert create(m2l=3) == -1
    assert create(precision=7) == -1
    assert create(p=0) == -1
    assert create(levels=1) == -1
    assert create(kernel=1, lam=0.0) == -1  # Yukawa needs lambda > 0
    assert create(kernel=3, d=2, lam=1.0) == -2  # Helmholtz only in 3D
    assert create(kernel=3, lam=1.0, levels=-4, max_leaf=64) == -2  # Helmholtz: uniform trees


def test_dw_selftest_validation_without_gpu():
    # argument checks come before any CUDA call
    from paper_2305_17867_gb300 import _lib

    L = _lib.load()
    x = (ctypes.c_double * 2)(1.0, 2.0)
    assert L.fmm_selftest_dw(3, 2, x, x, x) == -1  # FMM_ERR_ARG
    assert L.fmm_selftest_dw(-1, 2, x, x, x) == -1  # FMM_ERR_ARG
    assert L.fmm_selftest_dw(0, -1, x, x, x) == -1  # FMM_ERR_ARG
    assert L.fmm_selftest_dw(0, 2, None, x, x) == -1  # FMM_ERR_ARG
    assert L.fmm_selftest_dw(1, 0, None, None, None) == _lib.FMM_OK
