"""GB300 (sm_103a) pivoted skew-symmetric LTL^T factorization and Pfaffian.

Python binding of the C ABI in ``include/skewltlt.h`` (library ``libskewltlt.so``
built in-tree by ``python -m paper_2411_09859_gb300.build``).  The functions here
only marshal arguments: every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or no sm_103 GPU is
current, calls raise.

Matrices are torch float64 CUDA tensors in column-major layout: shape (n, n) with
``stride(0) == 1`` (e.g. ``fortran_empty(n, n)``, or a Fortran-ordered numpy array
moved with ``torch.from_numpy(a).cuda()``).  Device work is enqueued on the current
torch CUDA stream unless another stream is given.
"""
from __future__ import annotations

from ._native import (SkewError, fortran_empty, kernel_launches, lib, ltlt, ltlt_host,
                      ltlt_host_timing,
                      pfaffian, pfaffian_twostep, pfaffian_from_factors, rank2k, tridiag_rankk,
                      default_nb, set_nb_table, set_batched_nb_table, batched_nb, batched_warp_tile, set_batched_threads, workspace_bytes, set_lookahead, set_cluster_panel, set_lookahead_switch, lookahead_used, trim_memory, pool_usage, STATUS, profile_enable,
                      profile_read, ltlt_batched, pfaffian_batched, batched_workspace_bytes, problem_table, BATCH_MAX_N, Server,
                      PRECISION_FP64, PRECISION_SPLIT_BF16)

__all__ = ["SkewError", "fortran_empty", "kernel_launches", "lib", "ltlt", "ltlt_host",
           "ltlt_host_timing",
           "pfaffian", "pfaffian_twostep", "pfaffian_from_factors", "rank2k", "tridiag_rankk", "default_nb", "set_nb_table", "set_batched_nb_table", "batched_nb", "batched_warp_tile", "set_batched_threads",
           "workspace_bytes", "set_lookahead", "set_cluster_panel", "set_lookahead_switch", "lookahead_used", "trim_memory", "pool_usage", "STATUS", "profile_enable", "profile_read",
           "ltlt_batched", "pfaffian_batched", "batched_workspace_bytes", "problem_table", "BATCH_MAX_N", "Server", "PRECISION_FP64",
           "PRECISION_SPLIT_BF16"]
