"""skew_pfaffian_noalloc, the entry point for callers that must not have the library
allocate device memory (their HBM belongs to another allocator, or an allocation on
their critical path is not acceptable), checked through the C ABI against the
ordinary skew_pfaffian entry point.

The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test before this one.  It also passes on its own in a
fresh process: the first call on the device performs the one-time address lookup.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _outputs():
    dev = "cuda"
    return (torch.empty(1, dtype=torch.float64, device=dev),
            torch.empty(1, dtype=torch.int32, device=dev),
            torch.empty(1, dtype=torch.int32, device=dev))


def call_noalloc(A_dev, n, nb, la, sg, info):
    stream = torch.cuda.current_stream().cuda_stream
    return skew.lib().skew_pfaffian_noalloc(
        n, ctypes.c_void_p(A_dev.data_ptr()), max(n, 1), ctypes.c_void_p(la.data_ptr()),
        ctypes.c_void_p(sg.data_ptr()), ctypes.c_void_p(info.data_ptr()), nb,
        ctypes.c_void_p(stream))


def test_noalloc_matches_pfaffian_on_two_calls_in_a_row():
    cases = [(1000, 21, 0), (778, 22, 32)]      # different orders: stale scratch content
    devA = [torch.from_numpy(inputs.skew_gaussian(n, s)).cuda() for n, s, _ in cases]
    refA = [a.clone() for a in devA]
    outs = [_outputs() for _ in cases]
    # expected values from the ordinary entry point
    expected = []
    for (n, _, nb), a in zip(cases, refA):
        la, sg, t, piv, info = skew.pfaffian(a, nb=nb)
        torch.cuda.synchronize()
        expected.append((float(la.item()), int(sg.item()), int(info.item())))
    # the two calls in a row
    for (n, _, nb), a, (la, sg, info) in zip(cases, devA, outs):
        assert call_noalloc(a, n, nb, la, sg, info) == 0
    torch.cuda.synchronize()
    for (la, sg, info), (la0, sg0, i0) in zip(outs, expected):
        assert int(info.item()) == i0 == 0
        assert int(sg.item()) == sg0 != 0
        assert abs(float(la.item()) - la0) <= 1e-10 * max(1.0, abs(la0))


def test_noalloc_allocates_no_device_memory():
    n = 600
    A1 = torch.from_numpy(inputs.skew_gaussian(n, 31)).cuda()
    A2 = A1.clone()
    A3 = A1.clone()
    la, sg, info = _outputs()
    assert call_noalloc(A1, n, 0, la, sg, info) == 0      # first call on the device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call_noalloc(A2, n, 0, la, sg, info) == 0
    assert call_noalloc(A3, n, 16, la, sg, info) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(info.item()) == 0 and int(sg.item()) != 0


def test_noalloc_rejects_problems_beyond_its_scratch():
    big = 40000                                 # needs more than the fixed 16 MiB at nb = 64
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    la, sg, info = _outputs()
    assert skew.lib().skew_workspace_bytes(big, 64, 0) > 16 << 20
    st = skew.lib().skew_pfaffian_noalloc(big, ctypes.c_void_p(A.data_ptr()), big,
                                          ctypes.c_void_p(la.data_ptr()),
                                          ctypes.c_void_p(sg.data_ptr()), None, 64, None)
    assert st == -105
    assert skew.STATUS[st] == "SKEW_ERR_SCRATCH_LIMIT"


def test_noalloc_trivial_orders():
    la, sg, info = _outputs()
    A0 = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    assert call_noalloc(A0, 0, 0, la, sg, info) == 0
    torch.cuda.synchronize()
    assert float(la.item()) == 0.0 and int(sg.item()) == 1
    assert call_noalloc(A0, 1, 0, la, sg, info) == 0
    torch.cuda.synchronize()
    assert int(sg.item()) == 0 and float(la.item()) == -math.inf
