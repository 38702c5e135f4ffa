"""Python access to the plain FP64 CPU oracle (``grbk_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product library never imports this
package, and this package never imports the product library.

``build()`` compiles the C file with gcc (-O2 -ffp-contract=off) into
``oracle/_build/libgrbk_oracle.so``; ``lib()`` loads it, building on demand.
``build_omp()`` compiles the same source with -fopenmp into
``libgrbk_oracle_omp.so`` for timing the oracle on every host core
(``solve(..., omp=True)``); it computes the same bits as the single-thread
build and no test of the oracle's values uses it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grbk_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libgrbk_oracle.so")
_SO_OMP = os.path.join(_OUT_DIR, "libgrbk_oracle_omp.so")

GRBK, RGRBK, MWRBK, RBK, BK = 0, 1, 2, 3, 4
VARIANTS = {"grbk": GRBK, "rgrbk": RGRBK, "mwrbk": MWRBK, "rbk": RBK, "bk": BK}
MODE_GRAM, MODE_FACTORED, MODE_LITERAL = 0, 1, 2
STOP_NONE, STOP_RELRES, STOP_RSE = 0, 1, 2
RAN_MAXIT, TOL_MET, EXACT, NOT_CONVERGED = 0, 1, 2, 3

_libs = {}
_override = None


def compile_c(src: str, so: str, openmp: bool = False) -> str:
    """gcc -O2 -ffp-contract=off a C source into a shared object (atomic rename)."""
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared"]
                          + (["-fopenmp"] if openmp else []) + ["-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        compile_c(_SRC, _SO)
    return _SO


def build_omp(force: bool = False) -> str:
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < os.path.getmtime(_SRC):
        compile_c(_SRC, _SO_OMP, openmp=True)
    return _SO_OMP


class use_library:
    """Context manager: route every oracle call through another build of the
    oracle source (the tests use it to check that a planted mistake is caught)."""

    def __init__(self, so_path):
        self.so_path = so_path

    def __enter__(self):
        global _override
        self._prev, _override = _override, self.so_path
        return self

    def __exit__(self, *exc):
        global _override
        _override = self._prev


def lib(omp: bool = False):
    # GRBK_ORACLE_SO lets the mutation test point a child process at a build of
    # a deliberately broken copy of the oracle source.
    path = build_omp() if omp else (_override or os.environ.get("GRBK_ORACLE_SO") or build())
    if path not in _libs:
        L = ctypes.CDLL(path)
        i64, u64, dbl, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        L.oracle_philox4x64_10.argtypes = [vp, vp, vp]
        L.oracle_philox4x64_10.restype = None
        L.oracle_uniform.argtypes = [u64, u64, u64]
        L.oracle_uniform.restype = dbl
        L.oracle_residual.argtypes = [i64, i64, i64, i64, vp, vp, vp, vp, vp]
        L.oracle_residual.restype = None
        L.oracle_row_sqnorms.argtypes = [i64, i64, vp, vp]
        L.oracle_row_sqnorms.restype = None
        L.oracle_spectral_norm_sq.argtypes = [i64, i64, vp, i64]
        L.oracle_spectral_norm_sq.restype = dbl
        L.oracle_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, dbl, dbl, u64, u64, i64,
                                   ctypes.c_int, ctypes.c_int, dbl, vp, vp, vp, vp, vp, vp, vp,
                                   vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, vp]
        L.oracle_uniform_column.argtypes = [u64, u64, u64]
        L.oracle_uniform_column.restype = dbl
        L.oracle_solve.restype = i64
        L.oracle_last_loop_seconds.argtypes = []
        L.oracle_last_loop_seconds.restype = dbl
        L.oracle_threads.argtypes = []
        L.oracle_threads.restype = ctypes.c_int
        _libs[path] = L
    return _libs[path]


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().oracle_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed, k, sys=0):
    return lib().oracle_uniform(int(seed), int(k), int(sys))


def uniform_column(seed, k, sys=0):
    return lib().oracle_uniform_column(int(seed), int(k), int(sys))


def residual(A, X, B, C):
    A, X, B, C = map(_f64, (A, X, B, C))
    m, p = A.shape
    q, n = B.shape
    R = np.empty((m, n))
    lib().oracle_residual(m, p, q, n, _ptr(A), _ptr(X), _ptr(B), _ptr(C), _ptr(R))
    return R


def row_sqnorms(A):
    A = _f64(A)
    a = np.empty(A.shape[0])
    lib().oracle_row_sqnorms(A.shape[0], A.shape[1], _ptr(A), _ptr(a))
    return a


def spectral_norm_sq(B, iters=500):
    B = _f64(B)
    return lib().oracle_spectral_norm_sq(B.shape[0], B.shape[1], _ptr(B), int(iters))


def threads(omp: bool = False) -> int:
    """Threads the oracle's row loops run on (1 for the tests' build)."""
    return int(lib(omp).oracle_threads())


def solve(A, B, C, variant="grbk", theta=0.5, alpha=None, X0=None, seed=0, sys=0, maxit=1000,
          mode=MODE_GRAM, stop=STOP_NONE, tol=0.0, Xref=None, trace=True, want_R=False, omp=False,
          extended=False):
    """Run the oracle; returns a dict with X, iters, status and (if trace) the
    per-iteration traces rows, S, t, margin_adm, margin_pick, err2.  omp=True
    runs the OpenMP build (same results, every host core; timing only).
    extended=True: the least-squares extension (column steps on Y; want_R
    also returns the final Y)."""
    A, B, C = map(_f64, (A, B, C))
    m, p = A.shape
    q, n = B.shape
    assert C.shape == (m, n)
    if alpha is None:
        alpha = 1.0 / spectral_norm_sq(B)
    X = np.zeros((p, q)) if X0 is None else _f64(X0).copy()
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    dims = np.array([m, p, q, n], dtype=np.int64)
    T = max(int(maxit), 1)
    rows = np.full(T, -1, dtype=np.int64) if trace else None
    S = np.full(T, np.nan) if trace else None
    t = np.full(T, np.nan) if trace else None
    madm = np.full(T, np.nan) if trace else None
    mpick = np.full(T, np.nan) if trace else None
    err2 = np.full(T + 1, np.nan) if (trace and Xref is not None) else None
    Xr = None if Xref is None else _f64(Xref)
    R = np.empty((m, n)) if want_R else None
    s = np.empty(m) if want_R else None
    Y = np.empty((m, n)) if (want_R and extended) else None
    st = ctypes.c_int(0)
    it = lib(omp).oracle_solve(_ptr(dims), _ptr(A), _ptr(B), _ptr(C), _ptr(X), v, float(theta),
                            float(alpha), int(seed), int(sys), int(maxit), int(mode), int(stop),
                            float(tol), _ptr(Xr), _ptr(rows), _ptr(S), _ptr(t), _ptr(madm),
                            _ptr(mpick), _ptr(err2), _ptr(R), _ptr(s), ctypes.byref(st), int(bool(extended)),
                            _ptr(Y))
    out = dict(X=X, iters=int(it), status=int(st.value), alpha=float(alpha),
               loop_seconds=float(lib(omp).oracle_last_loop_seconds()))
    if trace:
        out.update(rows=rows[:it], S=S[:it], t=t[:it], margin_adm=madm[:it],
                   margin_pick=mpick[:it])
        if err2 is not None:
            out["err2"] = err2[:it + 1]
    if want_R:
        out.update(R=R, s=s)
        if extended:
            out["Y"] = Y
    return out
