"""CUDA graph capture of the single-matrix calls: with a caller-supplied workspace,
skew_ltlt and skew_pfaffian_twostep enqueue only kernels, memsets and event
fork/joins (the side stream of the deferred row exchanges), so a whole factorization
-- every panel, update and exchange launch -- can be captured once and replayed.
Each replay on the restored input must give exactly the direct call's results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(A):
    return torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda()


@pytest.mark.parametrize("n,nb", [(1000, 64), (3001, 32)])
def test_ltlt_replays_from_a_cuda_graph(n, nb):
    pristine = dev(inputs.skew_gaussian(n, 31))
    work = skew.fortran_empty(n, n, "cuda")
    L = skew.fortran_empty(n, n, "cuda")
    t = torch.empty(n - 1, dtype=torch.float64, device="cuda")
    piv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(skew.workspace_bytes(n, nb, True), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()

    def call():
        work.copy_(pristine)
        skew.ltlt(work, nb=nb, stream=s, L=L, t=t, piv=piv, info=info, workspace=ws)

    with torch.cuda.stream(s):                    # warm up outside the capture
        call()
    torch.cuda.synchronize()
    direct = [x.clone() for x in (L, t, piv, info)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call()
    for _ in range(3):
        for x in (L, t, piv):
            x.zero_()
        g.replay()
        torch.cuda.synchronize()
        for x, d in zip((L, t, piv, info), direct):
            assert torch.equal(x, d)


def test_pfaffian_twostep_replays_from_a_cuda_graph():
    n, nb = 2000, 64
    pristine = dev(inputs.skew_gaussian(n, 32))
    work = skew.fortran_empty(n, n, "cuda")
    a = torch.empty(n // 2, dtype=torch.float64, device="cuda")
    piv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(skew.lib().skew_workspace_bytes_twostep(n, nb, 0), dtype=torch.uint8,
                     device="cuda")
    s = torch.cuda.Stream()
    out = {}

    def call():
        work.copy_(pristine)
        out["r"] = skew.pfaffian_twostep(work, nb=nb, stream=s, a=a, piv=piv, info=info,
                                         workspace=ws)

    with torch.cuda.stream(s):
        call()
    torch.cuda.synchronize()
    la, sg = out["r"][0].clone(), out["r"][1].clone()
    direct = (a.clone(), piv.clone())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call()
    la_g, sg_g = out["r"][0], out["r"][1]
    for _ in range(3):
        a.zero_()
        la_g.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(a, direct[0]) and torch.equal(piv, direct[1])
        assert torch.equal(la_g, la) and torch.equal(sg_g, sg)
