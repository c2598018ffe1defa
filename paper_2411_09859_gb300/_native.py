"""ctypes declarations of libskewltlt.so and torch-tensor marshalling."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libskewltlt.so")

STATUS = {
    0: "SKEW_OK",
    -100: "SKEW_ERR_NONFINITE",
    -101: "SKEW_ERR_NOMEM",
    -102: "SKEW_ERR_CUDA",
    -103: "SKEW_ERR_TIMEOUT",
    -104: "SKEW_ERR_NODEVICE",
    -105: "SKEW_ERR_SCRATCH_LIMIT",
    -106: "SKEW_ERR_BUSY",
}

_lock = threading.Lock()
_lib = None

_i64, _i32, _dbl, _vp, _sz = (ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                              ctypes.c_void_p, ctypes.c_size_t)

SIGNATURES = {
    "skew_version": ([], _i32),
    "skew_last_error": ([], ctypes.c_char_p),
    "skew_kernel_launches": ([], ctypes.c_uint64),
    "skew_trim_memory": ([], _i32),
    "skew_pool_usage": ([_vp, _vp, _i32], _i32),
    "skew_selftest_bounded_wait": ([_dbl, _vp], _i32),
    "skew_selftest_mbarrier_wait": ([_dbl, _vp], _i32),
    "skew_profile_enable": ([_i32], _i32),
    "skew_profile_read": ([_vp], _i32),
    "skew_default_nb": ([_i64], _i32),
    "skew_set_nb_table": ([_i32, _vp, _vp], _i32),
    "skew_set_batched_nb_table": ([_i32, _vp, _vp], _i32),
    "skew_get_batched_nb": ([_i32], _i32),
    "skew_set_batched_tiles": ([_i32, _vp, _vp, _vp], _i32),
    "skew_get_batched_warp_tile": ([_i32], _i32),
    "skew_set_batched_threads": ([_i32], _i32),
    "skew_workspace_bytes": ([_i64, _i32, _i32], _sz),
    "skew_workspace_bytes_lookahead": ([_i64, _i32, _i32], _sz),
    "skew_set_lookahead": ([_i32], _i32),
    "skew_set_cluster_panel": ([_i32], _i32),
    "skew_set_lookahead_switch": ([ctypes.c_longlong], ctypes.c_longlong),
    "skew_set_nb_table_ex": ([_i32, _vp, _vp, _vp], _i32),
    "skew_lookahead_used": ([_i64, _i32, _i32], _i32),
    "skew_ltlt": ([_i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _i32, _vp, _sz, _vp], _i32),
    "skew_pfaffian": ([_i64, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp], _i32),
    "skew_pfaffian_from_factors": ([_i64, _vp, _vp, _vp, _vp, _vp], _i32),
    "skew_pfaffian_noalloc": ([_i64, _vp, _i64, _vp, _vp, _vp, _i32, _vp], _i32),
    "skew_rank2k": ([_i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _vp], _i32),
    "skew_tridiag_rankk": ([_i64, _i64, _dbl, _vp, _i64, _vp, _dbl, _vp, _i64, _vp], _i32),
    "skew_ltlt_host": ([_i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i32], _i32),
    "skew_ltlt_host_timing": ([_vp, _vp, _vp], _i32),
    "skew_batched_workspace_bytes": ([_i32, _i32], _sz),
    "skew_ltlt_ex": ([_i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _i32, _i32, _vp, _sz, _vp], _i32),
    "skew_pfaffian_ex": ([_i64, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _sz, _vp], _i32),
    "skew_workspace_bytes_ex": ([_i64, _i32, _i32, _i32], _sz),
    "skew_rank2k_ex": ([_i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _i32, _vp], _i32),
    "skew_ltlt_batched": ([_i32, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp], _i32),
    "skew_pfaffian_batched": ([_i32, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp], _i32),
    "skew_pfaffian_twostep": ([_i64, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _sz, _vp], _i32),
    "skew_workspace_bytes_twostep": ([_i64, _i32, _i32], _sz),
    "skew_server_create": ([_sz, _i32, _i32, _vp], _i32),
    "skew_server_submit": ([_vp, _i64, _vp, _i64, _i32, _vp], _i32),
    "skew_server_poll": ([_vp, ctypes.c_uint64, _vp], _i32),
    "skew_server_wait": ([_vp, ctypes.c_uint64, _dbl, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "skew_server_release": ([_vp, ctypes.c_uint64], _i32),
    "skew_server_stats": ([_vp, _vp, _vp, _vp], _i32),
    "skew_server_timing": ([_vp, ctypes.c_uint64, _vp, _vp, _vp], _i32),
    "skew_server_copy_factors": ([_vp, ctypes.c_uint64, _vp, _vp, _vp, _i64], _i32),
    "skew_server_destroy": ([_vp], _i32),
}


class SkewError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        if status < 0 and -status < 100:
            what = f"argument {-status} is invalid"
        else:
            what = STATUS.get(status, str(status))
        detail = ""
        if status == -102 and _lib is not None:
            detail = ": " + _lib.skew_last_error().decode()
        super().__init__(f"{fn} failed with {status} ({what}){detail}")


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_2411_09859_gb300.build`")
            try:
                import torch  # noqa: F401  (loads the CUDA runtime torch uses first)
            except ImportError:
                pass
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _install_saved_nb_table(L)
            _lib = L
        return _lib


def _install_saved_nb_table(L):
    """Install the autotuner's saved panel-width table (nb_table.json), if present."""
    import json
    path = os.path.join(_HERE, "nb_table.json")
    if not os.path.exists(path):
        return
    with open(path) as f:
        saved = json.load(f)
    table = saved.get("table", [])
    nu = (ctypes.c_int64 * max(len(table), 1))(*[int(e[0]) for e in table])
    nbs = (ctypes.c_int32 * max(len(table), 1))(*[int(e[1]) for e in table])
    las = (ctypes.c_int32 * max(len(table), 1))(*[int(e[2]) if len(e) > 2 else -1 for e in table])
    L.skew_set_nb_table_ex(len(table), ctypes.cast(nu, ctypes.c_void_p), ctypes.cast(nbs, ctypes.c_void_p),
                           ctypes.cast(las, ctypes.c_void_p))
    bt = saved.get("batched_table", [])
    bu = (ctypes.c_int32 * max(len(bt), 1))(*[int(e[0]) for e in bt])
    bn = (ctypes.c_int32 * max(len(bt), 1))(*[int(e[1]) for e in bt])
    bw = (ctypes.c_int32 * max(len(bt), 1))(*[int(e[2]) if len(e) > 2 else 32 for e in bt])
    L.skew_set_batched_tiles(len(bt), ctypes.cast(bu, ctypes.c_void_p), ctypes.cast(bn, ctypes.c_void_p),
                             ctypes.cast(bw, ctypes.c_void_p))
    L.skew_set_batched_threads(int(saved.get("batched_threads", 256)))


def _check(fn: str, status: int):
    if status != 0:
        raise SkewError(fn, status)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def fortran_empty(rows: int, cols: int, device=None, dtype=None):
    """Uninitialised column-major (rows x cols) CUDA tensor (stride(0) == 1)."""
    import torch
    dtype = dtype or torch.float64
    device = device or "cuda"
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def _colmajor(name: str, M, rows: int):
    import torch
    if not M.is_cuda or M.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if M.dim() != 2 or M.shape[0] != rows:
        raise ValueError(f"{name} must have {rows} rows")
    if M.shape[1] > 1 and M.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return max(M.stride(1) if M.shape[1] > 1 else rows, 1)


KIND_NAMES = ["prologue", "panel", "pivot_rows", "skr2k", "finish", "batched"]


class KernelStat(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("launches", ctypes.c_uint64)]


def profile_enable(on: bool = True):
    """Bracket every library kernel launch with CUDA events (see profile_read)."""
    _check("skew_profile_enable", lib().skew_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """Per kernel kind: summed event ms, algorithmic flops and bytes, launch count
    since the last read (waits for the recorded events)."""
    stats = (KernelStat * len(KIND_NAMES))()
    _check("skew_profile_read", lib().skew_profile_read(ctypes.cast(stats, ctypes.c_void_p)))
    return {name: {"ms": s.ms, "flops": s.flops, "bytes": s.bytes, "launches": int(s.launches)}
            for name, s in zip(KIND_NAMES, stats)}


def kernel_launches() -> int:
    return int(lib().skew_kernel_launches())


def default_nb(n: int) -> int:
    return int(lib().skew_default_nb(n))


def set_batched_nb_table(table):
    """Install ``[(n_upper, nb), ...]`` or ``[(n_upper, nb, warp_tile), ...]`` (nb in 8,
    16, 32; warp_tile in 16, 32, default 32) as the batched kernels' panel width and
    update warp tile per order bucket; an empty list restores width 16, tile 32."""
    count = len(table)
    nu = (ctypes.c_int32 * max(count, 1))(*[int(e[0]) for e in table])
    nbs = (ctypes.c_int32 * max(count, 1))(*[int(e[1]) for e in table])
    wts = (ctypes.c_int32 * max(count, 1))(*[int(e[2]) if len(e) > 2 else 32 for e in table])
    _check("skew_set_batched_tiles",
           lib().skew_set_batched_tiles(count, ctypes.cast(nu, ctypes.c_void_p),
                                        ctypes.cast(nbs, ctypes.c_void_p),
                                        ctypes.cast(wts, ctypes.c_void_p)))


def batched_nb(n: int) -> int:
    return int(lib().skew_get_batched_nb(n))


def batched_warp_tile(n: int) -> int:
    return int(lib().skew_get_batched_warp_tile(n))


def set_batched_threads(threads: int) -> int:
    """Threads per CTA of the blocked batched kernels (256 or 128); returns the old value."""
    old = int(lib().skew_set_batched_threads(int(threads)))
    if old < 0:
        raise SkewError("skew_set_batched_threads", old)
    return old


def set_nb_table(table):
    """Install ``[(n_upper, nb), ...]`` or ``[(n_upper, nb, lookahead), ...]`` (increasing
    n_upper; lookahead 1 / 0 / -1 = look-ahead / plain / built-in choice, default -1) as
    the default panel widths and paths; an empty list restores the built-in rules."""
    count = len(table)
    nu = (ctypes.c_int64 * max(count, 1))(*[int(e[0]) for e in table])
    nbs = (ctypes.c_int32 * max(count, 1))(*[int(e[1]) for e in table])
    las = (ctypes.c_int32 * max(count, 1))(*[int(e[2]) if len(e) > 2 else -1 for e in table])
    _check("skew_set_nb_table_ex",
           lib().skew_set_nb_table_ex(count, ctypes.cast(nu, ctypes.c_void_p),
                                      ctypes.cast(nbs, ctypes.c_void_p),
                                      ctypes.cast(las, ctypes.c_void_p)))


def workspace_bytes(n: int, nb: int = 0, with_L: bool = True, lookahead: bool = False) -> int:
    """Workspace bytes of ltlt / pfaffian at order n and width nb; with `lookahead`, the
    size that lets the call take the look-ahead path (see set_lookahead)."""
    fn = lib().skew_workspace_bytes_lookahead if lookahead else lib().skew_workspace_bytes
    return int(fn(n, nb, 1 if with_L else 0))


def set_lookahead(mode) -> int:
    """Path of later ltlt / pfaffian calls (skew_set_lookahead): False / 0 plain, True / 1
    the look-ahead where the panel-width table (or the built-in rule) picks it for the
    order, 2 wherever it applies, 32 / 64 as 2 with that many rows per panel CTA.
    Returns the old setting."""
    m = int(mode) if not isinstance(mode, bool) else (1 if mode else 0)
    return int(lib().skew_set_lookahead(m))


def set_cluster_panel(on: bool) -> bool:
    """Use the cluster panel for narrow trailing blocks on the plain path (default on);
    returns the old setting."""
    return bool(lib().skew_set_cluster_panel(1 if on else 0))


def set_lookahead_switch(rows: int) -> int:
    """Trailing order below which a look-ahead factorization goes on without the
    look-ahead (skew_set_lookahead_switch; -1: the default, 2560 rows).
    Returns the old setting."""
    return int(lib().skew_set_lookahead_switch(int(rows)))


def lookahead_used(n: int, nb: int = 0, precision: int = 0) -> bool:
    """Whether a call at order n, width nb takes the look-ahead path on this device."""
    return bool(lib().skew_lookahead_used(n, nb, precision))


def pool_usage(reset_high: bool = False):
    """(bytes in use, most bytes in use at once since the last reset) of the library's
    own device allocations on the current device."""
    now, high = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check("skew_pool_usage", lib().skew_pool_usage(ctypes.byref(now), ctypes.byref(high),
                                                    1 if reset_high else 0))
    return int(now.value), int(high.value)


def trim_memory():
    _check("skew_trim_memory", lib().skew_trim_memory())


PRECISION_FP64 = 0
PRECISION_SPLIT_BF16 = 1


def ltlt(A, nb: int = 0, stream=None, L=None, t=None, piv=None, info=None, workspace=None,
         precision: int = PRECISION_FP64):
    """P A P^T = L T L^T of the column-major float64 CUDA tensor ``A`` (destroyed).

    Returns ``(L, t, piv, info)`` as CUDA tensors (L column-major n x n, t (n-1,),
    piv int32 (n,), info int32 (1,)).  Asynchronous on ``stream``.
    """
    import torch
    n = A.shape[0]
    lda = _colmajor("A", A, n)
    L = fortran_empty(n, n, A.device) if L is None else L
    ldl = _colmajor("L", L, n)
    t = torch.empty(max(n - 1, 0), dtype=torch.float64, device=A.device) if t is None else t
    piv = torch.empty(n, dtype=torch.int32, device=A.device) if piv is None else piv
    info = torch.empty(1, dtype=torch.int32, device=A.device) if info is None else info
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    st = lib().skew_ltlt_ex(n, _ptr(A), lda, _ptr(L), ldl, _ptr(t) if n > 1 else None,
                            _ptr(piv), _ptr(info), nb, precision, ws, wsb, _stream_handle(stream))
    _check("skew_ltlt_ex", st)
    return L, t, piv, info


def pfaffian(A, nb: int = 0, stream=None, t=None, piv=None, info=None, workspace=None,
             precision: int = PRECISION_FP64):
    """log|Pf(A)| and sign through the factorization (A destroyed).

    Returns ``(logabs, sign, t, piv, info)`` CUDA tensors (logabs float64 (1,),
    sign int32 (1,)).
    """
    import torch
    n = A.shape[0]
    lda = _colmajor("A", A, n)
    dev = A.device
    logabs = torch.empty(1, dtype=torch.float64, device=dev)
    sign = torch.empty(1, dtype=torch.int32, device=dev)
    t = torch.empty(max(n - 1, 0), dtype=torch.float64, device=dev) if t is None else t
    piv = torch.empty(n, dtype=torch.int32, device=dev) if piv is None else piv
    info = torch.empty(1, dtype=torch.int32, device=dev) if info is None else info
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    st = lib().skew_pfaffian_ex(n, _ptr(A), lda, _ptr(logabs), _ptr(sign),
                                _ptr(t) if n > 1 else None, _ptr(piv) if n > 0 else None,
                                _ptr(info), nb, precision, ws, wsb, _stream_handle(stream))
    _check("skew_pfaffian_ex", st)
    return logabs, sign, t, piv, info


def pfaffian_twostep(A, nb: int = 0, stream=None, a=None, piv=None, info=None,
                     workspace=None, precision: int = PRECISION_FP64):
    """log|Pf(A)| and sign by the two-step (Pfaffian-only) elimination (A destroyed).

    Returns ``(logabs, sign, a, piv, info)`` CUDA tensors: ``a`` the n/2 pivot-block
    entries, ``piv`` int32 (n,) with the even-step exchanges.
    """
    import torch
    n = A.shape[0]
    lda = _colmajor("A", A, n)
    dev = A.device
    logabs = torch.empty(1, dtype=torch.float64, device=dev)
    sign = torch.empty(1, dtype=torch.int32, device=dev)
    a = torch.empty(max(n // 2, 1), dtype=torch.float64, device=dev) if a is None else a
    piv = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if piv is None else piv
    info = torch.empty(1, dtype=torch.int32, device=dev) if info is None else info
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    st = lib().skew_pfaffian_twostep(n, _ptr(A) if n > 0 else None, lda, _ptr(logabs),
                                     _ptr(sign), _ptr(a), _ptr(piv), _ptr(info), nb, precision,
                                     ws, wsb, _stream_handle(stream))
    _check("skew_pfaffian_twostep", st)
    return logabs, sign, a[: n // 2], piv[:n], info


def pfaffian_from_factors(t, piv, n: int, stream=None):
    import torch
    dev = piv.device
    logabs = torch.empty(1, dtype=torch.float64, device=dev)
    sign = torch.empty(1, dtype=torch.int32, device=dev)
    st = lib().skew_pfaffian_from_factors(n, _ptr(t) if n > 1 else None,
                                          _ptr(piv) if n > 0 else None, _ptr(logabs),
                                          _ptr(sign), _stream_handle(stream))
    _check("skew_pfaffian_from_factors", st)
    return logabs, sign


def rank2k(alpha: float, X, Y, beta: float, C, stream=None, precision: int = PRECISION_FP64):
    """C := beta C + alpha (X Y^T - Y X^T) on the strictly lower triangle (in place)."""
    m = C.shape[0]
    k = X.shape[1]
    ldx = _colmajor("X", X, m)
    ldy = _colmajor("Y", Y, m)
    ldc = _colmajor("C", C, m)
    st = lib().skew_rank2k_ex(m, k, float(alpha), _ptr(X), ldx, _ptr(Y), ldy, float(beta),
                              _ptr(C), ldc, precision, _stream_handle(stream))
    _check("skew_rank2k_ex", st)
    return C


def tridiag_rankk(alpha: float, A, t, beta: float, C, stream=None):
    """C := beta C + alpha A T A^T on the strictly lower triangle (in place)."""
    m = C.shape[0]
    b = A.shape[1]
    lda = _colmajor("A", A, m)
    ldc = _colmajor("C", C, m)
    st = lib().skew_tridiag_rankk(m, b, float(alpha), _ptr(A), lda,
                                  _ptr(t) if b > 1 else None, float(beta), _ptr(C), ldc,
                                  _stream_handle(stream))
    _check("skew_tridiag_rankk", st)
    return C


def ltlt_host(A: np.ndarray, want_L: bool = True, nb: int = 0, L_out=None, t_out=None,
              piv_out=None):
    """Host-buffer convenience call: returns numpy (L or None, t, piv, logabs, sign, info).

    ``A`` is a float64 numpy array (any order; its strictly lower triangle is read).
    ``L_out`` (n x n Fortran-ordered float64), ``t_out`` (n-1 float64) and
    ``piv_out`` (n int32) may be given to receive the results (e.g. page-locked).
    """
    n = A.shape[0]
    Af = np.asfortranarray(A, dtype=np.float64)
    if want_L:
        L = np.zeros((n, n), dtype=np.float64, order="F") if L_out is None else L_out
        if not (L.flags.f_contiguous and L.dtype == np.float64 and L.shape == (n, n)):
            raise ValueError("L_out must be an n x n Fortran-ordered float64 array")
    else:
        L = None
    t = np.zeros(max(n - 1, 1), dtype=np.float64) if t_out is None else t_out
    piv = np.zeros(max(n, 1), dtype=np.int32) if piv_out is None else piv_out
    logabs = ctypes.c_double(0.0)
    sign = ctypes.c_int32(0)
    info = ctypes.c_int32(0)
    ld = max(n, 1)
    st = lib().skew_ltlt_host(n, ctypes.c_void_p(Af.ctypes.data), ld,
                              None if L is None else ctypes.c_void_p(L.ctypes.data), ld,
                              ctypes.c_void_p(t.ctypes.data), ctypes.c_void_p(piv.ctypes.data),
                              ctypes.byref(logabs), ctypes.byref(sign), ctypes.byref(info), nb)
    _check("skew_ltlt_host", st)
    return L, t[: max(n - 1, 0)], piv[:n], logabs.value, sign.value, info.value


def ltlt_host_timing():
    """(h2d_ms, device_ms, d2h_ms) of the last completed :func:`ltlt_host` call on the
    current device, or None if there is none."""
    v = [ctypes.c_float(0.0) for _ in range(3)]
    st = lib().skew_ltlt_host_timing(*[ctypes.byref(x) for x in v])
    if st == -1:
        return None
    _check("skew_ltlt_host_timing", st)
    return tuple(float(x.value) for x in v)


BATCH_MAX_N = 8192


def problem_table(As, Ls, ts, pivs, device):
    """Device array of skew_problem descriptors (n, A, lda, L, ldl, t, piv).  Checks
    that every A is a column-major float64 CUDA tensor."""
    import torch
    rows = []
    for A, L, t, piv in zip(As, Ls, ts, pivs):
        n = A.shape[0]
        _colmajor("A", A, n)
        lda = max(A.stride(1) if n > 1 else 1, 1)
        ldl = 0 if L is None else max(L.stride(1) if n > 1 else 1, 1)
        rows.append([n, A.data_ptr() if n > 0 else 0, lda,
                     0 if L is None else L.data_ptr(), ldl,
                     t.data_ptr() if n > 1 else 0, piv.data_ptr() if n > 0 else 0])
    host = torch.tensor(rows, dtype=torch.int64).reshape(-1, 7)
    return host.to(device)


def batched_workspace_bytes(count: int, max_n: int) -> int:
    return int(lib().skew_batched_workspace_bytes(count, max_n))


def ltlt_batched(As, want_L: bool = False, stream=None, max_n: int | None = None,
                 table=None, outs=None, workspace=None):
    """Factor every column-major float64 CUDA tensor of the list ``As`` (destroyed) in
    one batched launch.  Returns ``(logabs, sign, info, ts, pivs, Ls)``: per-problem
    CUDA tensors (logabs float64 (count,), sign/info int32 (count,)) and lists of the
    factors (``Ls`` entries are None unless ``want_L``).  A ``table`` from
    :func:`problem_table` (built, and checked, once for the same tensors) skips the
    per-tensor work on the host."""
    import torch
    count = len(As)
    dev = As[0].device if count else torch.device("cuda")
    if outs is None:
        ts = [torch.empty(max(A.shape[0] - 1, 0), dtype=torch.float64, device=dev) for A in As]
        pivs = [torch.empty(A.shape[0], dtype=torch.int32, device=dev) for A in As]
        Ls = [fortran_empty(A.shape[0], A.shape[0], dev) if want_L else None for A in As]
    else:
        ts, pivs, Ls = outs
    if table is None:
        table = problem_table(As, Ls, ts, pivs, dev)
    logabs = torch.empty(count, dtype=torch.float64, device=dev)
    sign = torch.empty(count, dtype=torch.int32, device=dev)
    info = torch.empty(count, dtype=torch.int32, device=dev)
    mx = max((A.shape[0] for A in As), default=0) if max_n is None else max_n
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    st = lib().skew_ltlt_batched(count, _ptr(table) if count else None, _ptr(logabs),
                                 _ptr(sign), _ptr(info), mx, ws, wsb, _stream_handle(stream))
    _check("skew_ltlt_batched", st)
    return logabs, sign, info, ts, pivs, Ls



def pfaffian_batched(As, stream=None, max_n: int | None = None, table=None, outs=None,
                     workspace=None, results=None):
    """Pfaffians of the column-major float64 CUDA tensors ``As`` (destroyed) by the
    two-step elimination, one launch (orders <= 512).  Returns ``(logabs, sign,
    info, as_, pivs)``: per-problem CUDA tensors and the lists of pivot-block entries
    (n/2 each) and even-step pivots.  ``table``/``outs`` as for :func:`ltlt_batched`
    (``outs = (as_, pivs)``)."""
    import torch
    count = len(As)
    dev = As[0].device if count else torch.device("cuda")
    if outs is None:
        as_ = [torch.empty(max(A.shape[0] // 2, 1), dtype=torch.float64, device=dev) for A in As]
        pivs = [torch.empty(max(A.shape[0], 1), dtype=torch.int32, device=dev) for A in As]
    else:
        as_, pivs = outs
    if table is None:
        table = problem_table(As, [None] * count, as_, pivs, dev)
    if results is None:
        logabs = torch.empty(count, dtype=torch.float64, device=dev)
        sign = torch.empty(count, dtype=torch.int32, device=dev)
        info = torch.empty(count, dtype=torch.int32, device=dev)
    else:
        logabs, sign, info = results
    mx = max((A.shape[0] for A in As), default=0) if max_n is None else max_n
    ws, wsb = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    st = lib().skew_pfaffian_batched(count, _ptr(table) if count else None, _ptr(logabs),
                                     _ptr(sign), _ptr(info), mx, ws, wsb, _stream_handle(stream))
    _check("skew_pfaffian_batched", st)
    return logabs, sign, info, as_, pivs


SERVE_FACTORS, SERVE_FACTORS_L, SERVE_PFAFFIAN = 0, 1, 2   # SKEW_SERVE_*


class Server:
    """Continuous-batching server (skew_server_*).  Requests are column-major float64
    CUDA tensors; keep each one unchanged until its result has been waited for."""

    def __init__(self, budget_bytes: int, n_streams: int = 4, small_n_max: int = 512):
        self._h = ctypes.c_void_p()
        _check("skew_server_create", lib().skew_server_create(int(budget_bytes), n_streams,
                                                              small_n_max, ctypes.byref(self._h)))
        self._keep = {}

    def submit(self, A, want_L: bool = False, pfaffian_only: bool = False) -> int:
        """Queue A; want_L keeps L with the factors, pfaffian_only asks for log|Pf|
        and sign alone (two-step elimination, no factors kept)."""
        if want_L and pfaffian_only:
            raise ValueError("a Pfaffian-only request keeps no L")
        n = A.shape[0]
        lda = _colmajor("A", A, n)
        tk = ctypes.c_uint64()
        mode = SERVE_PFAFFIAN if pfaffian_only else (SERVE_FACTORS_L if want_L else SERVE_FACTORS)
        _check("skew_server_submit", lib().skew_server_submit(
            self._h, n, _ptr(A) if n > 0 else None, lda, mode, ctypes.byref(tk)))
        self._keep[tk.value] = A
        return tk.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check("skew_server_poll", lib().skew_server_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """Returns dict(logabs, sign, info, t_ptr, piv_ptr, L_ptr, latency_s)."""
        la, sg, inf, lat = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        tp, pp, lp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        st = lib().skew_server_wait(self._h, ticket, float(timeout_s), ctypes.byref(la),
                                    ctypes.byref(sg), ctypes.byref(inf), ctypes.byref(tp),
                                    ctypes.byref(pp), ctypes.byref(lp), ctypes.byref(lat))
        _check("skew_server_wait", st)
        out = {"logabs": la.value, "sign": sg.value, "info": inf.value, "t_ptr": tp.value,
               "piv_ptr": pp.value, "L_ptr": lp.value, "latency_s": lat.value}
        q, w, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        if lib().skew_server_timing(self._h, ticket, ctypes.byref(q), ctypes.byref(w),
                                    ctypes.byref(r)) == 0:
            out.update(queued_s=q.value, waiting_s=w.value, running_s=r.value)
        return out

    def factors(self, ticket: int, n: int, want_L: bool = False):
        """Host copies (t, piv, L or None) of a completed request's factors."""
        t = np.zeros(max(n - 1, 1), dtype=np.float64)
        piv = np.zeros(max(n, 1), dtype=np.int32)
        L = np.zeros((n, n), dtype=np.float64, order="F") if want_L else None
        st = lib().skew_server_copy_factors(self._h, ticket, ctypes.c_void_p(t.ctypes.data),
                                            ctypes.c_void_p(piv.ctypes.data),
                                            None if L is None else ctypes.c_void_p(L.ctypes.data),
                                            max(n, 1))
        _check("skew_server_copy_factors", st)
        return t[: max(n - 1, 0)], piv[:n], L

    def release(self, ticket: int):
        _check("skew_server_release", lib().skew_server_release(self._h, ticket))
        self._keep.pop(ticket, None)

    def stats(self):
        used, q, f = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        _check("skew_server_stats", lib().skew_server_stats(self._h, ctypes.byref(used),
                                                            ctypes.byref(q), ctypes.byref(f)))
        return {"used_bytes": used.value, "queued": q.value, "in_flight": f.value}

    def close(self):
        if self._h:
            _check("skew_server_destroy", lib().skew_server_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
