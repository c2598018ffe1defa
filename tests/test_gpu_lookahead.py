"""The look-ahead path of skew_ltlt / skew_pfaffian against the oracle and against the
plain path.

With the look-ahead (where it applies: FP64 update, panel width 2 .. 64, n - 1 <= 128 x
the multiprocessors; taken by default for the orders where it is faster, and here
forced with skew_set_lookahead(2)), the panel of each block runs beside the trailing
update of the block before it, reading the state before that update and deferring its
exchanges to the next (out-of-place) update.  Both paths factor the same matrix to the
oracle's factorization: pivots identical, factors within the parity bars of
test_gpu_parity.  Off (skew_set_lookahead(0)) or with a workspace of only
skew_workspace_bytes, the plain path runs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_2411_09859_gb300 as skew  # noqa: E402
from paper_2411_09859_gb300 import inputs  # noqa: E402
from skewcheck import EPS, backward_error, check_structure  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_C = 2000.0


def dev(A):
    return torch.from_numpy(np.asfortranarray(A, dtype=np.float64)).cuda()


def factor(A, nb, lookahead, workspace=None, with_L=True, switch=0):
    # 2: the look-ahead wherever it applies (the default, 1, takes it by order only);
    # switch 0: the look-ahead to the last block
    old = skew.set_lookahead(2 if lookahead else 0)
    old_sw = skew.set_lookahead_switch(switch)
    try:
        if with_L:
            L, t, piv, info = skew.ltlt(dev(A), nb=nb, workspace=workspace)
            torch.cuda.synchronize()
            return L.cpu().numpy(), t.cpu().numpy(), piv.cpu().numpy(), int(info.item())
        la, sg, t, piv, info = skew.pfaffian(dev(A), nb=nb, workspace=workspace)
        torch.cuda.synchronize()
        return (float(la.item()), int(sg.item())), t.cpu().numpy(), piv.cpu().numpy(), \
            int(info.item())
    finally:
        skew.set_lookahead(old)
        skew.set_lookahead_switch(old_sw)


def check(A, L, t, piv, info):
    n = A.shape[0]
    L0, t0, p0, i0 = oracle.ltlt(A)
    assert np.array_equal(piv, p0), np.nonzero(piv != p0)[0][:5]
    assert info == i0
    tol = TOL_C * n * EPS
    if n > 1:
        assert np.max(np.abs(t - t0)) <= tol * max(1.0, np.max(np.abs(t0)))
        if L is not None:
            assert np.max(np.abs(L - L0)) <= tol
    if L is not None:
        check_structure(L, t, piv, n)
        if n <= 1500:
            assert backward_error(A, L, t, piv) <= 10


@pytest.mark.parametrize("n,nb", [(4, 2), (9, 3), (33, 8), (100, 16), (129, 64), (300, 7),
                                  (513, 32), (1000, 64), (1031, 48), (2050, 64)])
def test_lookahead_and_plain_match_the_oracle(n, nb):
    A = inputs.skew_gaussian(n, 12000 + n)
    for lookahead in (True, False):
        check(A, *factor(A, nb, lookahead))


@pytest.mark.parametrize("n,nb", [(300, 32), (1001, 64)])
def test_lookahead_pfaffian_only(n, nb):
    """skew_pfaffian (no L: two panel buffers in the workspace) takes the look-ahead
    too; its pivots, t and log|Pf| equal the oracle's."""
    A = inputs.skew_gaussian(n, 12500 + n)
    (la, sg), t, piv, info = factor(A, nb, True, with_L=False)
    check(A, None, t, piv, info)
    L0, t0, p0, _ = oracle.ltlt(A)
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    assert sg == sg0
    if sg0 != 0:                              # odd n: Pf = 0, log|Pf| = -inf on both
        assert abs(la - la0) <= 1e-10 * max(1.0, abs(la0))


@pytest.mark.parametrize("n,nb,switch", [(1031, 48, 300), (1031, 48, 700), (1031, 48, -1),
                                         (2050, 32, 1000), (700, 16, 5000), (513, 32, 490)])
def test_lookahead_then_plain(n, nb, switch):
    """Look-ahead blocks until the trailing order falls below the switch order, the
    remaining blocks on the plain path in place (the last look-ahead panel's updated
    column copied into the state): the oracle's factorization, with and without L."""
    A = inputs.skew_gaussian(n, 13000 + n + switch)
    check(A, *factor(A, nb, True, switch=switch))
    (la, sg), t, piv, info = factor(A, nb, True, with_L=False, switch=switch)
    check(A, None, t, piv, info)
    L0, t0, p0, _ = oracle.ltlt(A)
    la0, sg0 = oracle.pfaffian_from_factors(n, t0, p0)
    assert sg == sg0
    if sg0 != 0:
        assert abs(la - la0) <= 1e-10 * max(1.0, abs(la0))


def test_switch_setting_round_trip():
    old = skew.set_lookahead_switch(1234)
    try:
        assert skew.set_lookahead_switch(-5) == 1234
        assert skew.set_lookahead_switch(0) == -1      # negative values mean the default
    finally:
        skew.set_lookahead_switch(old)


def test_default_path_choice():
    """Mode 1 (the default) takes the look-ahead by order: the panel-width table's
    choice, else the built-in rule (3072 <= n <= 5120 with cluster panels, 3072 <= n <=
    10240 with grid-wide panels); mode 0 never."""
    old = skew.set_lookahead(1)
    old_cl = skew.set_cluster_panel(True)
    try:
        skew.set_nb_table([])
        assert skew.lookahead_used(4096, 32) and not skew.lookahead_used(2000, 32)
        assert not skew.lookahead_used(8192, 32)
        skew.set_cluster_panel(False)
        assert not skew.lookahead_used(2000, 32) and skew.lookahead_used(4096, 64)
        assert skew.lookahead_used(8192, 32) and not skew.lookahead_used(16384, 64)
        skew.set_cluster_panel(True)
        skew.set_nb_table([(3000, 32, 1), (20000, 64, 0)])
        assert skew.lookahead_used(2000) and not skew.lookahead_used(4096)
        assert not skew.lookahead_used(4096, 128)             # wider than 64: plain
        skew.set_lookahead(0)
        assert not skew.lookahead_used(2000)
    finally:
        skew.set_lookahead(old)
        skew.set_cluster_panel(old_cl)
        from paper_2411_09859_gb300 import autotune
        if not autotune.load():
            skew.set_nb_table([])


def test_workspace_size_selects_the_path():
    """A caller's workspace of skew_workspace_bytes takes the plain path, one of
    skew_workspace_bytes_lookahead the look-ahead; both reach the oracle."""
    n, nb = 700, 32
    A = inputs.skew_gaussian(n, 12701)
    plain = skew.workspace_bytes(n, nb, True)
    la = skew.workspace_bytes(n, nb, True, lookahead=True)
    assert la >= plain + 8 * n * n
    for size in (plain, la):
        ws = torch.empty(size, dtype=torch.uint8, device="cuda")
        check(A, *factor(A, nb, True, workspace=ws))


def test_lookahead_block_diagonal_zero_pivots_and_ties():
    """Zero pivot columns (t = 0 at odd steps) and exact ties in the pivot search take
    the same path through the deferred exchanges as through the plain ones."""
    s = np.arange(1.0, 41.0)
    D = inputs.block_diag_skew(s)
    P = np.random.default_rng(3).permutation(80)
    A = np.asfortranarray(D[np.ix_(P, P)])
    for nb in (2, 8, 16):
        L, t, piv, info = factor(A, nb, True)
        check(A, L, t, piv, info)
    B = np.asfortranarray(np.tril(np.ones((90, 90)), -1) - np.triu(np.ones((90, 90)), 1))
    for nb in (4, 32):
        check(B, *factor(B, nb, True))


def test_lookahead_graph_capture_replays_equal():
    """A whole look-ahead factorization (its two extra streams forked from and joined
    to the capturing stream) captured in a CUDA graph and replayed gives the direct
    call's results bitwise."""
    n, nb = 600, 32
    A = inputs.skew_gaussian(n, 12801)
    Ad = dev(A)
    work = skew.fortran_empty(n, n, "cuda")
    L = skew.fortran_empty(n, n, "cuda")
    t = torch.empty(n - 1, dtype=torch.float64, device="cuda")
    piv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(skew.workspace_bytes(n, nb, True, lookahead=True), dtype=torch.uint8,
                     device="cuda")
    s = torch.cuda.Stream()
    old = skew.set_lookahead(2)
    old_sw = skew.set_lookahead_switch(300)      # look-ahead blocks, then plain ones
    try:
        run_graph_case(A, Ad, work, L, t, piv, info, ws, s, n, nb)
    finally:
        skew.set_lookahead(old)
        skew.set_lookahead_switch(old_sw)


def run_graph_case(A, Ad, work, L, t, piv, info, ws, s, n, nb):
    assert skew.lookahead_used(n, nb)
    work.copy_(Ad)
    torch.cuda.synchronize()
    skew.ltlt(work, nb=nb, stream=s, L=L, t=t, piv=piv, info=info, workspace=ws)
    torch.cuda.synchronize()
    ref = (L.clone(), t.clone(), piv.clone())
    g = torch.cuda.CUDAGraph()
    work.copy_(Ad)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        skew.ltlt(work, nb=nb, stream=s, L=L, t=t, piv=piv, info=info, workspace=ws)
    for _ in range(2):
        work.copy_(Ad)
        L.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            g.replay()
        torch.cuda.synchronize()
        assert torch.equal(L, ref[0]) and torch.equal(t, ref[1]) and torch.equal(piv, ref[2])
    check(A, ref[0].cpu().numpy(), ref[1].cpu().numpy(), ref[2].cpu().numpy(), int(info.item()))


def test_lookahead_at_its_largest_order_and_beyond():
    """n - 1 = 128 x (multiprocessors) is the largest order whose panel rows fit one per
    thread in 128-row CTAs: the look-ahead runs there and gives the plain path's pivots
    and Pfaffian; one order more falls back to the plain path."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    old = skew.set_lookahead(2)
    try:
        assert skew.lookahead_used(128 * sms + 1, 64)
        assert not skew.lookahead_used(128 * sms + 2, 64)
    finally:
        skew.set_lookahead(old)
    # an even order (an odd one has Pf = 0) whose first panel needs every multiprocessor
    n = 128 * sms
    A = inputs.skew_gaussian(n, 12901)
    res = {}
    for mode in (2, 0):
        old = skew.set_lookahead(mode)
        old_sw = skew.set_lookahead_switch(0)
        try:
            la, sg, t, piv, info = skew.pfaffian(dev(A), nb=64)
            torch.cuda.synchronize()
            res[mode] = (float(la.item()), int(sg.item()), t.cpu().numpy(), piv.cpu().numpy(),
                         int(info.item()))
        finally:
            skew.set_lookahead(old)
            skew.set_lookahead_switch(old_sw)
    (la2, sg2, t2, p2, i2), (la0, sg0, t0, p0, i0) = res[2], res[0]
    assert np.array_equal(p2, p0) and i2 == i0 == 0 and sg2 == sg0
    assert abs(la2 - la0) <= 1e-10 * abs(la0)
    assert np.max(np.abs(t2 - t0)) <= TOL_C * n * EPS * np.max(np.abs(t0))


@pytest.mark.parametrize("switch", [0, 500])
def test_lookahead_cluster_panel_nonfinite_leaves_together(switch):
    """A NaN in the input (flagged by the prologue) reaches every CTA of the cluster
    look-ahead panel through its first exchange; all leave together with a valid map,
    the call returns info = -100 on both schedules, and the context stays usable."""
    A = inputs.skew_gaussian(900, 16)
    A[700, 200] = np.nan
    A[200, 700] = np.nan
    for with_L in (True, False):
        res = factor(A, 32, True, with_L=with_L, switch=switch)
        assert res[3] == -100
    B = inputs.skew_gaussian(500, 17)
    check(B, *factor(B, 32, True, switch=switch))


@pytest.mark.parametrize("switch", [0, 500])
def test_lookahead_host_call_rows_during_factorization(switch):
    """skew_ltlt_host on the look-ahead path with a page-locked L (its rows sent back
    while later panels run, through the switch to the plain path): the same factors as
    the device call on the same path."""
    n, nb = 1000, 32
    A = inputs.skew_gaussian(n, 18)
    old = skew.set_lookahead(2)
    old_sw = skew.set_lookahead_switch(switch)
    try:
        assert skew.lookahead_used(n, nb)
        Lpin = torch.empty((n, n), dtype=torch.float64).pin_memory().t()
        Lpin.fill_(float("nan"))
        L, t, piv, la, sg, info = skew.ltlt_host(A, want_L=True, nb=nb, L_out=Lpin.numpy())
        L1, t1, p1, i1 = skew.ltlt(dev(A), nb=nb)
        torch.cuda.synchronize()
        assert info == 0 and np.array_equal(piv, p1.cpu().numpy())
        assert np.array_equal(t, t1.cpu().numpy()) and np.array_equal(L, L1.cpu().numpy())
    finally:
        skew.set_lookahead(old)
        skew.set_lookahead_switch(old_sw)
