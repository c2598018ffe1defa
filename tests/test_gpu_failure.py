"""Failure detection without a GPU fault: a device-side wait on something that never
happens ends by its time limit, the kernel returns a status the host reads, and the
context stays usable."""
import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    status = ctypes.c_int32(0)
    t0 = time.perf_counter()
    rc = skew.lib().skew_selftest_bounded_wait(0.25, ctypes.byref(status))
    el = time.perf_counter() - t0
    assert rc == 0
    assert status.value == -103                 # SKEW_ERR_TIMEOUT recorded on the device
    assert 0.2 <= el < 5.0
    # the context still works: a factorization afterwards
    A = torch.from_numpy(inputs.skew_gaussian(64, 1)).cuda()
    L, t, piv, info = skew.ltlt(A, nb=16)
    torch.cuda.synchronize()
    assert int(info.item()) == 0


def test_selftest_rejects_bad_limits():
    status = ctypes.c_int32(0)
    assert skew.lib().skew_selftest_bounded_wait(0.0, ctypes.byref(status)) == -1
    assert skew.lib().skew_selftest_bounded_wait(60.0, ctypes.byref(status)) == -1


def test_mbarrier_wait_times_out_and_split_path_still_works():
    """The bounded mbarrier wait of the tcgen05 kernels, on a barrier nothing arrives at,
    gives up after its limit with SKEW_ERR_TIMEOUT; the split-precision (tcgen05)
    factorization runs correctly afterwards on the same context."""
    import oracle
    status = ctypes.c_int32(0)
    t0 = time.perf_counter()
    rc = skew.lib().skew_selftest_mbarrier_wait(0.25, ctypes.byref(status))
    el = time.perf_counter() - t0
    assert rc == 0
    assert status.value == -103
    assert 0.2 <= el < 5.0
    A = inputs.skew_gaussian(300, 5)
    L, t, piv, info = skew.ltlt(torch.from_numpy(A).cuda(), nb=32,
                                precision=skew.PRECISION_SPLIT_BF16)
    torch.cuda.synchronize()
    L0, t0_, p0, i0 = oracle.ltlt(A)
    assert int(info.item()) == 0
    assert np.array_equal(piv.cpu().numpy(), p0)
    assert skew.lib().skew_selftest_mbarrier_wait(0.0, ctypes.byref(status)) == -1
