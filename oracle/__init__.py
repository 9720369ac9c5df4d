"""CPU FP64 oracle for the matricized least-square-errors polynomial fit.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never calls it; the library never calls this.

The arithmetic lives in ``lsefit_oracle.c`` (plain sequential C, FP64, every
operation separately rounded), which follows Section II of Dasgupta,
arXiv 1512.08017: the power sums S_k = sum x^k (k <= 2m) and
T_k = sum x^k y (k <= m), the Hankel normal matrix A[j][k] = S_{j+k},
B[j] = T_j, and Gaussian elimination of AX = B.  Two independent validators
sit beside it: ``exact`` (the same definition in exact rational arithmetic)
and ``householder`` (the Vandermonde QR least-squares solve that Section III
describes for MATLAB's polyfit).  ``fit_general`` generalises the objective
to per-point weights and to the Chebyshev basis, from the definition of its
normal equations.

Readings where the paper is silent or misprinted are listed at the top of
``lsefit_oracle.c``.  Parity unpinned: the correlation coefficient "R" of
Tables II-IV (the paper does not define it) is not part of the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LSEFIT_ORACLE_SOURCE lets the mutation tests build the oracle from a copy of
# lsefit_oracle.c with a planted mistake (in a separate process and build dir).
_SRC = os.environ.get("LSEFIT_ORACLE_SOURCE") or os.path.join(_HERE, "lsefit_oracle.c")
_BUILD_DIR = os.environ.get("LSEFIT_ORACLE_BUILD_DIR") or os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblsefit_oracle.so")

# Machine epsilons of the arithmetic that formed the sums (singularity threshold).
EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23

# Oracle status values, as numbered in lsefit_oracle.c.
STATUS_NAMES = {0: "ok", 1: "n_too_small", 2: "singular", 3: "nonfinite",
                4: "bad_interval", 5: "bad_arg"}

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile lsefit_oracle.c into a shared library (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["cc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", "-pthread",
           "-Wall", "-Werror", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.orc_map_constants.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
        lib.orc_map_constants.restype = ctypes.c_int
        lib.orc_powersums.argtypes = [dp, dp, i64, ctypes.c_int, dp, dp, dp]
        lib.orc_powersums.restype = None
        lib.orc_solve.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_solve_cholesky.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
        lib.orc_solve_cholesky.restype = ctypes.c_int
        lib.orc_unmap.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_unmap.restype = None
        lib.orc_fit.argtypes = [dp, dp, i64, ctypes.c_int, dp, ctypes.c_double, dp, dp, dp, dp]
        lib.orc_fit.restype = ctypes.c_int
        lib.orc_eval.argtypes = [ctypes.c_int, dp, dp, i64, dp]
        lib.orc_eval.restype = None
        lib.orc_sse.argtypes = [ctypes.c_int, dp, dp, dp, i64]
        lib.orc_sse.restype = ctypes.c_double
        lib.orc_backward.argtypes = [dp, dp, i64, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, dp, dp]
        lib.orc_backward.restype = ctypes.c_int
        lib.orc_fit_general.argtypes = [dp, dp, dp, i64, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                        dp, dp, dp, dp]
        lib.orc_fit_general.restype = ctypes.c_int
        lib.orc_cheb_to_mono.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_cheb_to_mono.restype = None
        lib.orc_residuals_general.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, i64, dp, dp]
        lib.orc_residuals_general.restype = ctypes.c_double
        lib.orc_powersums_threads.argtypes = [dp, dp, i64, ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.orc_powersums_threads.restype = ctypes.c_int
        lib.orc_max_degree.argtypes = []
        lib.orc_max_degree.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_degree() -> int:
    return _load().orc_max_degree()


def map_constants(lo: float, hi: float, fp32: bool):
    """(c, s) of the affine map t = s(x - c) onto [-1, 1]; rounded to FP32 if fp32.

    Returns (status_name, c, s)."""
    c = ctypes.c_double(0.0)
    s = ctypes.c_double(0.0)
    st = _load().orc_map_constants(float(lo), float(hi), int(bool(fp32)),
                                   ctypes.byref(c), ctypes.byref(s))
    return STATUS_NAMES[st], c.value, s.value


def powersums(x, y, m: int, cs=None):
    """S[0..2m], T[0..m] of Section II (t = s(x - c) when cs = (c, s) is given)."""
    x = _f64(x)
    y = _f64(y)
    assert x.shape == y.shape and x.ndim == 1
    S = np.zeros(2 * m + 1)
    T = np.zeros(m + 1)
    mp = _f64(cs) if cs is not None else None
    _load().orc_powersums(_ptr(x), _ptr(y), x.size, m, _ptr(mp) if mp is not None else None,
                          _ptr(S), _ptr(T))
    return S, T


def host_threads() -> int:
    """Threads the all-core variant uses by default: the host's online CPUs."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1)


def powersums_threads(x, y, m: int, cs=None, threads: int | None = None):
    """powersums on all host cores, for timing only: fixed equal point ranges,
    one per thread, each summed by the sequential routine; the per-thread sums
    added in thread order (one thread: identical to powersums)."""
    x = _f64(x)
    y = _f64(y)
    assert x.shape == y.shape and x.ndim == 1
    S = np.zeros(2 * m + 1)
    T = np.zeros(m + 1)
    mp = _f64(cs) if cs is not None else None
    nt = host_threads() if threads is None else int(threads)
    st = _load().orc_powersums_threads(_ptr(x), _ptr(y), x.size, m, _ptr(mp) if mp is not None else None, nt,
                                       _ptr(S), _ptr(T))
    if st != 0:
        raise ValueError(f"orc_powersums_threads: {STATUS_NAMES[st]} (threads={nt})")
    return S, T


def fit_threads(x, y, m: int, cs=None, eps: float = EPS64, threads: int | None = None) -> dict:
    """The fit of ``fit`` with the power sums taken by powersums_threads (timing
    the oracle on all host cores); the elimination and the un-map are the same."""
    S, T = powersums_threads(x, y, m, cs, threads)
    st, Xt = solve(S, T, m, eps)
    X = unmap(Xt, cs[0], cs[1]) if (cs is not None and st == "ok") else Xt.copy()
    return {"status": st, "X": X, "Xt": Xt, "S": S, "T": T}


def solve(S, T, m: int, eps: float = EPS64):
    """Gaussian elimination (partial pivoting) of A X = B built from S, T.

    eps: machine epsilon of the arithmetic that formed the sums.
    Returns (status_name, X)."""
    S = _f64(S)
    T = _f64(T)
    X = np.full(m + 1, np.nan)
    st = _load().orc_solve(m, _ptr(S), _ptr(T), float(eps), _ptr(X))
    return STATUS_NAMES[st], X


def solve_cholesky(S, T, m: int, eps: float = EPS64):
    """Cholesky factorisation of the Hankel normal matrix, then two triangular solves.

    Returns (status_name, X)."""
    S = _f64(S)
    T = _f64(T)
    X = np.full(m + 1, np.nan)
    st = _load().orc_solve_cholesky(m, _ptr(S), _ptr(T), float(eps), _ptr(X))
    return STATUS_NAMES[st], X


def unmap(Xt, c: float, s: float):
    """x-basis coefficients of sum_k Xt[k] (s(x - c))^k."""
    Xt = _f64(Xt)
    X = np.zeros_like(Xt)
    _load().orc_unmap(Xt.size - 1, float(c), float(s), _ptr(Xt), _ptr(X))
    return X


def fit(x, y, m: int, cs=None, eps: float = EPS64) -> dict:
    """The paper's fit.  eps: machine epsilon of the arithmetic the sums are
    formed in (singularity threshold).  Returns dict(status, X, Xt, S, T)."""
    x = _f64(x)
    y = _f64(y)
    assert x.shape == y.shape and x.ndim == 1
    X = np.zeros(m + 1)
    Xt = np.zeros(m + 1)
    S = np.zeros(2 * m + 1)
    T = np.zeros(m + 1)
    mp = _f64(cs) if cs is not None else None
    st = _load().orc_fit(_ptr(x), _ptr(y), x.size, m, _ptr(mp) if mp is not None else None,
                         float(eps), _ptr(X), _ptr(Xt), _ptr(S), _ptr(T))
    return {"status": STATUS_NAMES[st], "X": X, "Xt": Xt, "S": S, "T": T}


def fit_interval(x, y, m: int, lo: float, hi: float, fp32: bool) -> dict:
    """Fit on t = s(x - c) for the map of [lo, hi] onto [-1, 1], coefficients mapped back.

    fp32: the points are mapped and powered in FP32 (map constants rounded to
    FP32, FP32 singularity threshold); otherwise FP64."""
    st, c, s = map_constants(lo, hi, fp32)
    if st != "ok":
        n = m + 1
        return {"status": st, "X": np.full(n, np.nan), "Xt": np.full(n, np.nan),
                "S": None, "T": None, "c": np.nan, "s": np.nan}
    out = fit(x, y, m, (c, s), eps=EPS32 if fp32 else EPS64)
    out["c"] = c
    out["s"] = s
    return out


def evaluate(X, x):
    """f(x_i) = sum_j X[j] x_i^j."""
    X = _f64(X)
    x = _f64(x)
    f = np.zeros_like(x)
    _load().orc_eval(X.size - 1, _ptr(X), _ptr(x), x.size, _ptr(f))
    return f


def sse(X, x, y) -> float:
    """sum_i (y_i - f(x_i))^2."""
    X = _f64(X)
    x = _f64(x)
    y = _f64(y)
    return float(_load().orc_sse(X.size - 1, _ptr(X), _ptr(x), _ptr(y), x.size))


def backward(x, y, m: int, cs, S, Xt, gX, eps: float = EPS64):
    """Adjoint of ``fit`` for dL/dX = gX.  Returns (status_name, dx, dy)."""
    x = _f64(x)
    y = _f64(y)
    S = _f64(S)
    Xt = _f64(Xt)
    gX = _f64(gX)
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    mp = _f64(cs) if cs is not None else None
    st = _load().orc_backward(_ptr(x), _ptr(y), x.size, m, _ptr(mp) if mp is not None else None,
                              _ptr(S), _ptr(Xt), _ptr(gX), float(eps), _ptr(dx), _ptr(dy))
    return STATUS_NAMES[st], dx, dy


BASES = {"monomial": 0, "chebyshev": 1}


def cheb_to_mono(a):
    """Monomial coefficients of sum_k a[k] T_k(t)."""
    a = _f64(a)
    out = np.zeros_like(a)
    _load().orc_cheb_to_mono(a.size - 1, _ptr(a), _ptr(out))
    return out


def fit_general(x, y, m: int, w=None, basis: str = "monomial", cs=None, eps: float = EPS64) -> dict:
    """Weighted and/or Chebyshev-basis fit: minimises sum_i w_i (y_i - f(t_i))^2
    with f = sum_k Xb[k] phi_k(t), phi_k = t^k or T_k(t); t = s(x - c) when
    cs = (c, s).  Returns dict(status, X (x monomials), Xb, G, b)."""
    x = _f64(x)
    y = _f64(y)
    assert x.shape == y.shape and x.ndim == 1
    wa = _f64(w) if w is not None else None
    if wa is not None:
        assert wa.shape == x.shape
    n1 = m + 1
    X = np.zeros(n1)
    Xb = np.zeros(n1)
    G = np.zeros(n1 * n1)
    b = np.zeros(n1)
    mp = _f64(cs) if cs is not None else None
    st = _load().orc_fit_general(_ptr(x), _ptr(y), _ptr(wa) if wa is not None else None, x.size, m,
                                 BASES[basis], _ptr(mp) if mp is not None else None, float(eps),
                                 _ptr(X), _ptr(Xb), _ptr(G), _ptr(b))
    return {"status": STATUS_NAMES[st], "X": X, "Xb": Xb, "G": G.reshape(n1, n1), "b": b}


def fit_general_interval(x, y, m: int, lo: float, hi: float, fp32: bool, w=None,
                         basis: str = "monomial") -> dict:
    """fit_general on the map of [lo, hi] onto [-1, 1] (constants and threshold as fit_interval)."""
    st, c, s = map_constants(lo, hi, fp32)
    if st != "ok":
        n1 = m + 1
        return {"status": st, "X": np.full(n1, np.nan), "Xb": np.full(n1, np.nan), "G": None, "b": None,
                "c": np.nan, "s": np.nan}
    out = fit_general(x, y, m, w=w, basis=basis, cs=(c, s), eps=EPS32 if fp32 else EPS64)
    out["c"] = c
    out["s"] = s
    return out


def residuals_general(x, y, Xb, basis: str = "monomial", cs=None):
    """Residuals of the fit f = sum_k Xb[k] phi_k(t), t = s(x - c) when cs = (c, s):
    returns (SSE, V^T r with (V^T r)_k = sum_i phi_k(t_i) r_i, r)."""
    x = _f64(x)
    y = _f64(y)
    Xb = _f64(Xb)
    m = Xb.size - 1
    r = np.zeros_like(x)
    vtr = np.zeros(m + 1)
    mp = _f64(cs) if cs is not None else None
    sse = _load().orc_residuals_general(m, BASES[basis], _ptr(Xb), _ptr(mp) if mp is not None else None,
                                        _ptr(x), _ptr(y), x.size, _ptr(r), _ptr(vtr))
    return float(sse), vtr, r
