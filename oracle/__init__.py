"""Plain FP64 CPU oracle for the pivoted skew-symmetric LTL^T factorization.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU
baseline are the only callers.  The GPU product path never imports this package, and
this package imports nothing from the GPU package.

The arithmetic lives in ``skew_oracle.c`` (plain C, compiled here with gcc and
``-ffp-contract=off``); this module only builds it and marshals numpy arrays.
Paper: "Performant Tridiagonal Factorization of Skew-Symmetric Matrices"
(arXiv 2411.09859); each C function cites the passage it follows.

Every function takes and returns numpy float64 arrays indexed ``A[i, j]``.  Only the
strictly lower triangle of a skew input is read.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "skew_oracle.c")
_LIB_PATH = os.path.join(HERE, "_liboracle.so")
_lock = threading.Lock()
_default = None

ERR_NONFINITE = -100
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC"]


def compile_source(src: str, out: str) -> str:
    """Compile one C source of the oracle into a shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``skew_oracle.c`` into ``_liboracle.so`` beside it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)):
        return _LIB_PATH
    return compile_source(SOURCE, _LIB_PATH)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _fortran_copy(A: np.ndarray) -> np.ndarray:
    return np.array(A, dtype=np.float64, order="F", copy=True)


class OracleLib:
    """ctypes view of one compiled oracle library (the default one, or a test build)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        i64, dbl, p = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.oracle_ltlt_steps.argtypes = [i64, p, i64, p, i64, p, p, i64]
        lib.oracle_ltlt_steps.restype = ctypes.c_int
        lib.oracle_pfaffian.argtypes = [i64, p, p, p, p]
        lib.oracle_pfaffian.restype = None
        lib.oracle_skew_rank2k.argtypes = [i64, i64, dbl, p, i64, p, i64, dbl, p, i64]
        lib.oracle_skew_rank2k.restype = None
        lib.oracle_skew_tridiag_rankk.argtypes = [i64, i64, dbl, p, i64, p, dbl, p, i64]
        lib.oracle_skew_tridiag_rankk.restype = None
        lib.oracle_pfaffian_twostep.argtypes = [i64, p, i64, p, p, p, p]
        lib.oracle_pfaffian_twostep.restype = ctypes.c_int
        lib.oracle_ltlt_setup.argtypes = [i64, p, i64, p, i64, p, p]
        lib.oracle_ltlt_setup.restype = ctypes.c_int
        lib.oracle_ltlt_range.argtypes = [i64, p, i64, p, i64, p, p, i64, i64]
        lib.oracle_ltlt_range.restype = ctypes.c_int
        lib.oracle_ltlt_many.argtypes = [i64, p, p, p, p, p, p, p, p]
        lib.oracle_ltlt_many.restype = None
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def threads(self) -> int:
        """Host threads the update loop uses (OpenMP; OMP_NUM_THREADS)."""
        return int(self.lib.oracle_threads())

    def ltlt(self, A: np.ndarray, nsteps: int | None = None, overwrite: bool = False):
        """Unblocked right-looking pivoted LTL^T of the skew matrix ``A``.

        Returns ``(L, t, piv, info)``: L n x n unit lower (Fortran order), t length
        n-1, piv int32 length n (absolute, piv[0] = 0), info as returned by the C
        routine (0, 1 + first zero pivot, or a negative error).  ``nsteps`` stops
        after that many elimination steps (bounded timing samples only).  With
        ``overwrite`` and a Fortran-ordered float64 ``A``, ``A`` is the workspace.
        """
        n = int(A.shape[0])
        if A.shape != (n, n):
            raise ValueError("A must be square")
        if overwrite and A.dtype == np.float64 and A.flags.f_contiguous:
            X = A
        else:
            X = _fortran_copy(A)
        L = np.zeros((n, n), dtype=np.float64, order="F")
        t = np.zeros(max(n - 1, 1), dtype=np.float64)
        piv = np.zeros(max(n, 1), dtype=np.int32)
        steps = n if nsteps is None else int(nsteps)
        ld = max(n, 1)
        if n == 0:
            X = np.zeros((1, 1), order="F")
            L = np.zeros((1, 1), order="F")
        info = self.lib.oracle_ltlt_steps(n, _ptr(X), ld, _ptr(L), ld, _ptr(t),
                                          _ptr(piv), steps)
        if n == 0:
            return (np.zeros((0, 0), order="F"), np.zeros(0), np.zeros(0, np.int32),
                    int(info))
        return L, t[: n - 1], piv, int(info)

    def ltlt_begin(self, A: np.ndarray):
        """Set up the factorization of ``A`` for :meth:`ltlt_continue` (the state of
        ``oracle_ltlt_setup``).  Returns a dict holding the workspace X, L, t, piv,
        the order, the next step and info."""
        n = int(A.shape[0])
        if A.shape != (n, n) or n < 2:
            raise ValueError("A must be square of order >= 2")
        st = {"n": n, "X": _fortran_copy(A),
              "L": np.zeros((n, n), dtype=np.float64, order="F"),
              "t": np.zeros(n - 1, dtype=np.float64),
              "piv": np.zeros(n, dtype=np.int32), "k": 0, "info": 0}
        info = self.lib.oracle_ltlt_setup(n, _ptr(st["X"]), n, _ptr(st["L"]), n,
                                          _ptr(st["t"]), _ptr(st["piv"]))
        if info != 0:
            raise ValueError(f"oracle_ltlt_setup failed with {info}")
        return st

    def ltlt_continue(self, st: dict, kend: int) -> int:
        """Elimination steps st["k"] .. kend-1 of the factorization begun by
        :meth:`ltlt_begin` (``oracle_ltlt_range``); the results after the last step
        (n-1) are those of :meth:`ltlt`.  Returns the next step."""
        n = st["n"]
        kend = min(int(kend), n - 1)
        info = self.lib.oracle_ltlt_range(n, _ptr(st["X"]), n, _ptr(st["L"]), n,
                                          _ptr(st["t"]), _ptr(st["piv"]), st["k"], kend)
        if info and not st["info"]:
            st["info"] = int(info)
        st["k"] = max(st["k"], kend)
        return st["k"]

    def ltlt_many(self, As):
        """Whole factorizations and Pfaffians of the matrices ``As`` (a list), one
        matrix per host thread (``oracle_ltlt_many``).  The inputs are copied first;
        returns ``(logabs, sign, info, ts, pivs, seconds)`` with ``seconds`` the wall
        time of the C call alone."""
        import time
        count = len(As)
        ns = np.array([A.shape[0] for A in As], dtype=np.int64)
        Xs = [_fortran_copy(A) if A.shape[0] > 0 else np.zeros((1, 1), order="F") for A in As]
        Ls = [np.zeros((max(n, 1), max(n, 1)), dtype=np.float64, order="F") for n in ns]
        ts = [np.zeros(max(n - 1, 1), dtype=np.float64) for n in ns]
        pivs = [np.zeros(max(n, 1), dtype=np.int32) for n in ns]

        def table(arrs):
            return (ctypes.c_void_p * max(count, 1))(*[a.ctypes.data for a in arrs])

        tX, tL, tt, tp = table(Xs), table(Ls), table(ts), table(pivs)
        info = np.zeros(max(count, 1), dtype=np.int32)
        logabs = np.zeros(max(count, 1), dtype=np.float64)
        sign = np.zeros(max(count, 1), dtype=np.int32)
        t0 = time.perf_counter()
        self.lib.oracle_ltlt_many(count, _ptr(ns), tX, tL, tt, tp, _ptr(info),
                                  _ptr(logabs), _ptr(sign))
        seconds = time.perf_counter() - t0
        return (logabs[:count], sign[:count], info[:count],
                [t[: max(int(n) - 1, 0)] for t, n in zip(ts, ns)],
                [p[: int(n)] for p, n in zip(pivs, ns)], seconds)

    def pfaffian_from_factors(self, n: int, t: np.ndarray, piv: np.ndarray):
        """``(log|Pf|, sign)`` read off T and P (sign in {-1, 0, 1})."""
        tt = np.zeros(max(len(t), 1))
        tt[: len(t)] = t
        pp = np.zeros(max(len(piv), 1), dtype=np.int32)
        pp[: len(piv)] = piv
        logabs = np.zeros(1, dtype=np.float64)
        sign = np.zeros(1, dtype=np.int32)
        self.lib.oracle_pfaffian(int(n), _ptr(tt), _ptr(pp), _ptr(logabs), _ptr(sign))
        return float(logabs[0]), int(sign[0])

    def pfaffian(self, A: np.ndarray):
        """``(log|Pf(A)|, sign)`` via :meth:`ltlt` then :meth:`pfaffian_from_factors`."""
        L, t, piv, info = self.ltlt(A)
        if info < 0:
            raise ValueError(f"oracle_ltlt failed with {info}")
        return self.pfaffian_from_factors(A.shape[0], t, piv)

    def pfaffian_twostep(self, A: np.ndarray):
        """Pf(A) by the two-step elimination with pivoting at even steps only.

        Returns ``(log|Pf|, sign, a, piv, info)``: ``a`` the floor(n/2) pivot-block
        entries, ``piv`` int32 length n (piv[k+1] at even k, identity elsewhere),
        ``info`` as returned by the C routine.
        """
        n = int(A.shape[0])
        X = _fortran_copy(A) if n > 0 else np.zeros((1, 1), order="F")
        a = np.zeros(max(n // 2, 1), dtype=np.float64)
        piv = np.zeros(max(n, 1), dtype=np.int32)
        logabs = np.zeros(1, dtype=np.float64)
        sign = np.zeros(1, dtype=np.int32)
        info = self.lib.oracle_pfaffian_twostep(n, _ptr(X), max(n, 1), _ptr(a), _ptr(piv),
                                                _ptr(logabs), _ptr(sign))
        return float(logabs[0]), int(sign[0]), a[: n // 2], piv[:n], int(info)

    def skew_rank2k(self, alpha, A, B, beta, C):
        """Copy of C with its strictly lower part := beta C + alpha (A B^T - B A^T)."""
        m, k = A.shape
        Af, Bf, Cf = _fortran_copy(A), _fortran_copy(B), _fortran_copy(C)
        ld = max(m, 1)
        self.lib.oracle_skew_rank2k(m, k, float(alpha), _ptr(Af), ld, _ptr(Bf), ld,
                                    float(beta), _ptr(Cf), ld)
        return Cf

    def skew_tridiag_rankk(self, alpha, A, t, beta, C):
        """Copy of C with its strictly lower part := beta C + alpha A T A^T."""
        m, b = A.shape
        Af, Cf = _fortran_copy(A), _fortran_copy(C)
        tt = np.zeros(max(b - 1, 1))
        tt[: max(b - 1, 0)] = np.asarray(t, dtype=np.float64)[: max(b - 1, 0)]
        ld = max(m, 1)
        self.lib.oracle_skew_tridiag_rankk(m, b, float(alpha), _ptr(Af), ld, _ptr(tt),
                                           float(beta), _ptr(Cf), ld)
        return Cf


def default() -> OracleLib:
    """The oracle built from ``skew_oracle.c`` (compiled on first use)."""
    global _default
    with _lock:
        if _default is None:
            try:
                _default = OracleLib(build())
            except OSError:
                # a library left by a build on another architecture: rebuild here
                _default = OracleLib(build(force=True))
        return _default


def threads() -> int:
    return default().threads()


def ltlt(A, nsteps=None, overwrite=False):
    return default().ltlt(A, nsteps=nsteps, overwrite=overwrite)


def pfaffian_from_factors(n, t, piv):
    return default().pfaffian_from_factors(n, t, piv)


def ltlt_begin(A):
    return default().ltlt_begin(A)


def ltlt_continue(st, kend):
    return default().ltlt_continue(st, kend)


def ltlt_many(As):
    return default().ltlt_many(As)


def pfaffian(A):
    return default().pfaffian(A)


def pfaffian_twostep(A):
    return default().pfaffian_twostep(A)


def skew_rank2k(alpha, A, B, beta, C):
    return default().skew_rank2k(alpha, A, B, beta, C)


def skew_tridiag_rankk(alpha, A, t, beta, C):
    return default().skew_tridiag_rankk(alpha, A, t, beta, C)
