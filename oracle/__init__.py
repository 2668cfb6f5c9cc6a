"""FP64 CPU oracle for the per-SNP GLS sequence (Eq. 1 / Eq. 2 / Listing 1).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use this package; the library and its Python binding
never import it.  It shares no code with the CUDA path.  The arithmetic lives
in gls_oracle.c (plain C loops, FP64); this module only marshals numpy arrays.

Every function here has a mathematical pin in tests/test_oracle.py (brute
force on tiny inputs, closed forms, invariants).  Functions without one say
"parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gls_oracle.c")
_LIB = os.path.join(_HERE, "_gls_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gls_oracle.c into _gls_oracle.so with gcc (-O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        lib.oracle_form_m.argtypes = [i64, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_form_m.restype = None
        lib.oracle_potrf.argtypes = [i64, dp]
        lib.oracle_potrf.restype = i64
        lib.oracle_trsm_lower.argtypes = [i64, dp, i64, dp]
        lib.oracle_trsm_lower.restype = None
        lib.oracle_gls.argtypes = [i64, ctypes.c_int, dp, dp, dp, i64, dp, dp, dp, dp, ip]
        lib.oracle_gls.restype = ctypes.c_int
        lib.oracle_gls_grad.argtypes = [i64, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, i64,
                                         dp, dp, dp, dp]
        lib.oracle_gls_grad.restype = ctypes.c_int
        lib.oracle_reml.argtypes = [i64, ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_reml.restype = i64
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def form_m(phi, h: float, sigma2: float) -> np.ndarray:
    """M = sigma2 (h Phi + (1 - h) I)  (variance-component form; Sec. 1.3 leaves M open)."""
    phi = _f64(phi)
    n = phi.shape[0]
    M = np.empty((n, n), dtype=np.float64, order="F")
    _load().oracle_form_m(n, _p(phi), float(h), float(sigma2), _p(M))
    return M


class NotSPD(ValueError):
    def __init__(self, index: int):
        super().__init__(f"matrix is not positive definite (pivot {index})")
        self.index = index


def potrf(M) -> np.ndarray:
    """Lower Cholesky factor L, L L^T = M (Sec. 2.1, "potrf M").  Raises NotSPD."""
    L = np.array(M, dtype=np.float64, order="F", copy=True)
    bad = _load().oracle_potrf(L.shape[0], _p(L))
    if bad >= 0:
        raise NotSPD(int(bad))
    return L


def trsm_lower(L, X) -> np.ndarray:
    """L^-1 X by forward substitution (Eq. 2's X~ = L^-1 X; Sec. 2.2's trsm)."""
    L = _f64(L)
    X = np.array(X, dtype=np.float64, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    _load().oracle_trsm_lower(L.shape[0], _p(L), X.shape[1], _p(X))
    return X


def gls(L, XL, y, XR):
    """Per-SNP GLS (Eq. 1 through Eq. 2, in the order of Listing 1).

    L: n x n lower factor of M; XL: n x (p-1); y: n; XR: n x m SNP columns.
    Returns (r, se, chi2, status): r and se are p x m (row p-1 = SNP effect),
    chi2 the Wald statistic r_{p-1}^2 / (S^-1)_{p-1,p-1}, status 1 marks a
    numerically collinear design (NaN outputs).
    """
    L = _f64(L)
    n = L.shape[0]
    XL = _f64(XL).reshape(n, -1, order="F") if np.size(XL) else np.zeros((n, 0), order="F")
    y = _f64(y).reshape(n)
    XR = _f64(XR).reshape(n, -1, order="F")
    p = XL.shape[1] + 1
    m = XR.shape[1]
    r = np.empty((p, m), dtype=np.float64, order="F")
    se = np.empty((p, m), dtype=np.float64, order="F")
    chi2 = np.empty(m, dtype=np.float64)
    status = np.empty(m, dtype=np.int32)
    XLp = XL if XL.size else np.zeros((n, 1), order="F")
    rc = _load().oracle_gls(n, p, _p(L), _p(XLp), _p(y), m, _p(XR), _p(r), _p(se), _p(chi2),
                            _p(status, ctypes.c_int))
    if rc != 0:
        raise ValueError("oracle_gls: bad arguments")
    return r, se, chi2, status


def gls_grad(L, phi, h: float, sigma2: float, XL, y, XR):
    """Wald chi2 per SNP, d chi2 / dh per SNP, and sum over SNPs of d chi2 / dy.

    Dense form with D = dM/dh = sigma2 (Phi - I) (not in the paper; the
    differentiation form).  Returns (chi2, dchi2_dh, dy)."""
    L, phi = _f64(L), _f64(phi)
    n = L.shape[0]
    XL = _f64(XL).reshape(n, -1, order="F") if np.size(XL) else np.zeros((n, 0), order="F")
    y = _f64(y).reshape(n)
    XR = _f64(XR).reshape(n, -1, order="F")
    p, m = XL.shape[1] + 1, XR.shape[1]
    chi2 = np.empty(m)
    dh = np.empty(m)
    dy = np.empty(n)
    XLp = XL if XL.size else np.zeros((n, 1), order="F")
    rc = _load().oracle_gls_grad(n, p, _p(L), _p(phi), float(h), float(sigma2), _p(XLp), _p(y), m, _p(XR),
                                 _p(chi2), _p(dh), _p(dy))
    if rc != 0:
        raise ValueError("oracle_gls_grad: bad arguments")
    return chi2, dh, dy


def reml(phi, XL, y, h: float, grad: bool = True):
    """REML log-likelihood of the null model y ~ N(X_L beta, s2 (h Phi + (1-h) I)),
    s2 profiled out; returns (l, dl/dh or None, s2_hat).  Dense evaluation."""
    phi = _f64(phi)
    n = phi.shape[0]
    XL = _f64(XL).reshape(n, -1, order="F")
    y = _f64(y).reshape(n)
    out = np.zeros(3)
    rc = _load().oracle_reml(n, XL.shape[1], _p(phi), _p(XL), _p(y), float(h), int(bool(grad)), _p(out))
    if rc != 0:
        raise NotSPD(int(rc) - 1)
    return out[0], (out[1] if grad else None), out[2]


def reml_argmax(phi, XL, y, lo: float = 1e-4, hi: float = 1.0 - 1e-4, grid: int = 41, tol: float = 1e-7):
    """argmax of the REML log-likelihood over h: a dense grid, then
    golden-section search in the bracket around the best grid point."""
    hs = np.linspace(lo, hi, grid)
    vals = [reml(phi, XL, y, h, grad=False)[0] for h in hs]
    i = int(np.argmax(vals))
    a, b = hs[max(i - 1, 0)], hs[min(i + 1, grid - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = reml(phi, XL, y, c, grad=False)[0], reml(phi, XL, y, d, grad=False)[0]
    while b - a > tol:
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = reml(phi, XL, y, c, grad=False)[0]
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = reml(phi, XL, y, d, grad=False)[0]
    return 0.5 * (a + b)


def gls_from_phi(phi, XL, y, XR, h: float, sigma2: float):
    """form_m -> potrf -> gls, the whole sequence from Phi."""
    return gls(potrf(form_m(phi, h, sigma2)), XL, y, XR)
