"""Python view of the CPU FP64 oracle (``fmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports this module, and this module imports nothing
from the product package.

Every function is argument marshalling around the C oracle; the arithmetic
and the paper citations live in ``fmm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_SO = os.path.join(_HERE, "_build", "libfmm_oracle.so")
_LOCK = threading.Lock()
_LIB = None

LAPLACE, YUKAWA, BIHARMONIC, HELM_RE, HELM_IM = 0, 1, 2, 3, 4
# "helmholtz_re" / "helmholtz_im": cos(kappa r)/r and sin(kappa r)/r (lam = kappa),
# the real and imaginary parts of the Helmholtz kernel e^{i kappa r}/r; the
# complex "helmholtz" results below are composed from the two real FMMs.
KERNELS = {"laplace": LAPLACE, "yukawa": YUKAWA, "biharmonic": BIHARMONIC,
           "helmholtz_re": HELM_RE, "helmholtz_im": HELM_IM}


def _quadlib():
    import platform
    return ["-lquadmath"] if platform.machine() in ("x86_64", "AMD64") else []


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, OpenMP)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC] + _quadlib() + ["-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = build()
            L = ctypes.CDLL(path)
            i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            vp = ctypes.c_void_p
            L.or_num_terms.argtypes = [i32, i32]
            L.or_num_terms.restype = i32
            L.or_multi_indices.argtypes = [i32, i32, vp]
            L.or_mi_index.argtypes = [i32, vp]
            L.or_mi_index.restype = i32
            L.or_pde_for_kernel.argtypes = [i32, i32, f64, vp]
            L.or_pde_for_kernel.restype = i32
            L.or_expansion_new.argtypes = [i32, i32, i32, vp, i32]
            L.or_expansion_new.restype = vp
            L.or_expansion_free.argtypes = [vp]
            L.or_expansion_info.argtypes = [vp, vp, vp]
            L.or_expansion_info.restype = i32
            L.or_expansion_stored.argtypes = [vp, vp]
            L.or_expansion_matrix.argtypes = [vp, vp]
            L.or_decompress.argtypes = [vp, vp, vp]
            L.or_compress.argtypes = [vp, vp, vp]
            L.or_derivatives.argtypes = [i32, i32, f64, i32, vp, vp]
            L.or_derivatives.restype = i32
            L.or_derivatives_batch.argtypes = [i32, i32, f64, i32, i64, vp, vp]
            L.or_derivatives_batch.restype = i32
            L.or_direct.argtypes = [i32, i32, f64, i64, vp, vp, i64, vp, vp, vp]
            L.or_p2m.argtypes = [vp, vp, i64, vp, vp, vp]
            L.or_m2p.argtypes = [vp, i32, f64, vp, vp, vp]
            L.or_m2p.restype = f64
            L.or_m2m_full.argtypes = [vp, vp, vp, vp]
            L.or_m2m.argtypes = [vp, vp, vp, vp]
            L.or_m2l.argtypes = [vp, vp, vp, vp]
            L.or_m2l_naive.argtypes = [i32, i32, vp, vp, vp]
            L.or_l2l.argtypes = [vp, vp, vp, vp]
            L.or_l2p.argtypes = [vp, vp, vp, vp, vp]
            L.or_l2p.restype = f64
            L.or_p2l.argtypes = [vp, i32, f64, vp, i64, vp, vp, vp]
            L.or_fmm_uniform.argtypes = [i32, i32, f64, i32, i32, i32, vp, f64,
                                         i64, vp, vp, i64, vp, i64, vp, vp, vp]
            L.or_fmm_uniform.restype = i32
            L.or_fmm_adaptive.argtypes = [i32, i32, f64, i32, i32, i32, vp, f64,
                                          i64, vp, vp, i64, vp, i64, vp, vp, vp, vp]
            L.or_fmm_adaptive.restype = i32
            L.or_num_threads.restype = i32
            L.or_set_num_threads.argtypes = [i32]
            _LIB = L
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_terms(d: int, p: int) -> int:
    return lib().or_num_terms(d, p)


def multi_indices(d: int, p: int) -> np.ndarray:
    n = num_terms(d, p)
    out = np.zeros((n, d), dtype=np.int32)
    lib().or_multi_indices(d, p, _p(out))
    return out


def mi_index(d: int, m) -> int:
    a = np.ascontiguousarray(m, dtype=np.int32)
    return lib().or_mi_index(d, _p(a))


def pde_for_kernel(kernel: str, d: int, lam: float = 0.0):
    a = np.zeros(64, dtype=np.float64)
    c = lib().or_pde_for_kernel(KERNELS[kernel], d, lam, _p(a))
    return c, a[: num_terms(d, c)].copy()


class Expansion:
    """Oracle expansion of order p for a PDE (compressed or plain Taylor)."""

    def __init__(self, d: int, p: int, kernel: str = "laplace", lam: float = 0.0,
                 compressed: bool = True, pde=None):
        self.d, self.p, self.kernel, self.lam = d, p, kernel, lam
        if pde is None:
            c, a = pde_for_kernel(kernel, d, lam)
        else:
            c, a = pde
            a = _f64(a)
        self._a = a
        self.c = c
        self._h = lib().or_expansion_new(d, p, c, _p(a), int(compressed))
        nf = ctypes.c_int()
        nj = ctypes.c_int()
        lib().or_expansion_info(self._h, ctypes.byref(nf), ctypes.byref(nj))
        self.nfull, self.nj = nf.value, nj.value
        self.j = np.zeros(self.nj, dtype=np.int32)
        lib().or_expansion_stored(self._h, _p(self.j))
        self.mi = multi_indices(d, p)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _LIB is not None:
            _LIB.or_expansion_free(h)
            self._h = None

    @property
    def M(self) -> np.ndarray:
        out = np.zeros((self.nfull, self.nj), dtype=np.float64)
        lib().or_expansion_matrix(self._h, _p(out))
        return out

    def decompress(self, s):
        s = _f64(s)
        out = np.zeros(self.nfull)
        lib().or_decompress(self._h, _p(s), _p(out))
        return out

    def compress(self, a):
        a = _f64(a)
        out = np.zeros(self.nj)
        lib().or_compress(self._h, _p(a), _p(out))
        return out

    def p2m(self, c, y, w):
        c, y, w = _f64(c), _f64(y), _f64(w)
        out = np.zeros(self.nj)
        lib().or_p2m(self._h, _p(c), len(w), _p(y), _p(w), _p(out))
        return out

    def m2p(self, c, beta, x):
        return lib().or_m2p(self._h, KERNELS[self.kernel], self.lam, _p(_f64(c)),
                            _p(_f64(beta)), _p(_f64(x)))

    def m2m_full(self, h, a):
        out = np.zeros(self.nfull)
        lib().or_m2m_full(self._h, _p(_f64(h)), _p(_f64(a)), _p(out))
        return out

    def m2m(self, h, beta):
        out = np.zeros(self.nj)
        lib().or_m2m(self._h, _p(_f64(h)), _p(_f64(beta)), _p(out))
        return out

    def m2l(self, hvec, beta):
        D2 = derivatives(self.kernel, self.d, 2 * self.p, hvec, self.lam)
        out = np.zeros(self.nj)
        lib().or_m2l(self._h, _p(D2), _p(_f64(beta)), _p(out))
        return out

    def l2l(self, h, L1):
        out = np.zeros(self.nj)
        lib().or_l2l(self._h, _p(_f64(h)), _p(_f64(L1)), _p(out))
        return out

    def l2p(self, c, L, x, grad: bool = False):
        g = np.zeros(self.d) if grad else None
        v = lib().or_l2p(self._h, _p(_f64(c)), _p(_f64(L)), _p(_f64(x)), _p(g))
        return (v, g) if grad else v

    def p2l(self, c, y, w):
        out = np.zeros(self.nj)
        y, w = _f64(y), _f64(w)
        lib().or_p2l(self._h, KERNELS[self.kernel], self.lam, _p(_f64(c)), len(w),
                     _p(y), _p(w), _p(out))
        return out


def m2l_naive(d: int, p: int, D2, alpha):
    out = np.zeros(num_terms(d, p))
    lib().or_m2l_naive(d, p, _p(_f64(D2)), _p(_f64(alpha)), _p(out))
    return out


def _complex(fn, kernel, *args, **kw):
    """Helmholtz as the real FMM of each part of G, composed re + i im."""
    re = fn("helmholtz_re", *args, **kw)
    im = fn("helmholtz_im", *args, **kw)
    if isinstance(re, tuple):
        return tuple(None if a is None else a + 1j * b for a, b in zip(re, im))
    return re + 1j * im


def derivatives(kernel: str, d: int, pmax: int, x, lam: float = 0.0) -> np.ndarray:
    if kernel == "helmholtz":
        return _complex(derivatives, kernel, d, pmax, x, lam)
    out = np.zeros(num_terms(d, pmax))
    rc = lib().or_derivatives(KERNELS[kernel], d, lam, pmax, _p(_f64(x)), _p(out))
    if rc != 0:
        raise ValueError("derivative at the origin")
    return out


def derivatives_batch(kernel: str, d: int, pmax: int, x, lam: float = 0.0) -> np.ndarray:
    if kernel == "helmholtz":
        return _complex(derivatives_batch, kernel, d, pmax, x, lam)
    x = _f64(x).reshape(-1, d)
    out = np.zeros((x.shape[0], num_terms(d, pmax)))
    rc = lib().or_derivatives_batch(KERNELS[kernel], d, lam, pmax, x.shape[0], _p(x), _p(out))
    if rc != 0:
        raise ValueError("derivative at the origin")
    return out


def direct(kernel: str, d: int, src, w, tgt, lam: float = 0.0, grad: bool = False):
    if kernel == "helmholtz":
        return _complex(direct, kernel, d, src, w, tgt, lam=lam, grad=grad)
    src, w, tgt = _f64(src), _f64(w), _f64(tgt)
    nt = tgt.shape[0]
    phi = np.zeros(nt)
    g = np.zeros((nt, d)) if grad else None
    lib().or_direct(KERNELS[kernel], d, lam, src.shape[0], _p(src), _p(w), nt,
                    _p(tgt), _p(phi), _p(g))
    return (phi, g) if grad else phi


def fmm_uniform(kernel: str, d: int, p: int, L: int, src, w, tgt, lo=None,
                size: float = 1.0, lam: float = 0.0, compressed: bool = True,
                sample=None, grad: bool = False):
    """Uniform-tree FMM; with ``sample`` only those target indices are evaluated."""
    if kernel == "helmholtz":
        return _complex(fmm_uniform, kernel, d, p, L, src, w, tgt, lo=lo, size=size, lam=lam, compressed=compressed, sample=sample, grad=grad)
    src, w, tgt = _f64(src), _f64(w), _f64(tgt)
    lo = _f64(np.zeros(d) if lo is None else lo)
    ns = 0 if sample is None else len(sample)
    samp = None if sample is None else np.ascontiguousarray(sample, dtype=np.int64)
    nout = ns if ns else tgt.shape[0]
    phi = np.zeros(nout)
    g = np.zeros((nout, d)) if grad else None
    rc = lib().or_fmm_uniform(KERNELS[kernel], d, lam, p, L, int(compressed), _p(lo),
                              float(size), src.shape[0], _p(src), _p(w), tgt.shape[0],
                              _p(tgt), ns, _p(samp), _p(phi), _p(g))
    if rc != 0:
        raise ValueError(f"oracle FMM failed with status {rc}")
    return (phi, g) if grad else phi


def fmm_adaptive(kernel: str, d: int, p: int, src, w, tgt, max_leaf: int = 64,
                 max_depth: int = 10, lo=None, size: float = 1.0, lam: float = 0.0,
                 sample=None, want_stats: bool = False):
    """Adaptive-tree FMM (U/V/W/X lists).  Returns phi, or (phi, stats, cover)
    with stats = dict(boxes, leaves, depth, U, V, W, X, WX_direct) and cover =
    sources reached per evaluated target (with multiplicity); WX_direct counts
    the W and X pairs summed directly (boxes of at most |j| points)."""
    src, w, tgt = _f64(src), _f64(w), _f64(tgt)
    lo = _f64(np.zeros(d) if lo is None else lo)
    ns = 0 if sample is None else len(sample)
    samp = None if sample is None else np.ascontiguousarray(sample, dtype=np.int64)
    nout = ns if ns else tgt.shape[0]
    phi = np.zeros(nout)
    st = np.zeros(8, dtype=np.int64)
    cov = np.zeros(nout)
    rc = lib().or_fmm_adaptive(KERNELS[kernel], d, lam, p, max_leaf, max_depth, _p(lo),
                               float(size), src.shape[0], _p(src), _p(w), tgt.shape[0],
                               _p(tgt), ns, _p(samp), _p(phi), _p(st), _p(cov))
    if rc != 0:
        raise ValueError(f"oracle adaptive FMM failed with status {rc}")
    if not want_stats:
        return phi
    keys = ["boxes", "leaves", "depth", "U", "V", "W", "X", "WX_direct"]
    return phi, dict(zip(keys, [int(v) for v in st[:8]])), cov


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(n)
