"""The one-launch cluster form of SSYMV / SYPRD (small n) against the FP64 oracle,
on both sides of the size limit, with rows split between the cluster's CTAs,
out-of-range columns, graph capture and run-to-run SYPRD determinism."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu


def errors(sg, A, x, y, s):
    yr, ya = oracle.ssymv(A.n, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(A.n, A.rowptr, A.col, A.val, x.astype(np.float64))
    e_y = oracle.componentwise_error(host(y), yr, ya)
    e_s = abs(float(s.item()) - sr) / sa if sa > 0 else abs(float(s.item()))
    return e_y, e_s


def largest_single_launch_nnz(sg, n):
    lo, hi = 0, 1 << 22
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if sg.spmv_single_launch(n, mid):
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("n,nnz,seed,single", [
    (2000, 20000, 0, True),      # the 2,000 x 2,000, 1 % dense matrix
    (1, 1, 1, True), (7, 20, 2, True), (33, 300, 3, True), (1000, 100, 4, True),
    (4096, 30000, 5, True), (8192, 9000, 6, True),
    (8193, 9000, 7, False),     # just past the row limit: multi-block form
    (3000, 160000, 8, False),   # past the shared-memory limit
])
def test_cluster_form_matches_oracle(n, nnz, seed, single):
    sg = need_gpu()
    nnz = min(nnz, n * (n + 1) // 2)
    assert sg.spmv_single_launch(n, nnz) == single
    A = synth.upper_csr_uniform(n, nnz, seed)
    x = synth.vector_uniform(n, seed)
    y, s = sg.spmv(n, dev(A.rowptr), dev(A.col), dev(A.val), dev(x), syprd=True)
    e_y, e_s = errors(sg, A, x, y, s)
    assert e_y <= TOL_F32 and e_s <= TOL_F32, (e_y, e_s)
    y2 = sg.spmv(n, dev(A.rowptr), dev(A.col), dev(A.val), dev(x))
    yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    assert oracle.componentwise_error(host(y2), yr, ya) <= TOL_F32


@pytest.mark.parametrize("n", [257, 2000, 8192])
def test_cluster_form_at_its_size_limit(n):
    sg = need_gpu()
    nnz = min(largest_single_launch_nnz(sg, n), n * (n + 1) // 2)
    assert sg.spmv_single_launch(n, nnz)
    A = synth.upper_csr_uniform(n, nnz, 11)
    x = synth.vector_uniform(n, 12)
    y, s = sg.spmv(n, dev(A.rowptr), dev(A.col), dev(A.val), dev(x), syprd=True)
    e_y, e_s = errors(sg, A, x, y, s)
    assert e_y <= TOL_F32 and e_s <= TOL_F32, (e_y, e_s)


def test_cluster_form_rows_split_between_ctas():
    """Long rows: every CTA holds part of row 0 and of a middle row."""
    sg = need_gpu()
    n = 2048
    rows = [np.arange(0, n, dtype=np.int32), np.arange(1000, n, dtype=np.int32), np.array([2047], np.int32)]
    rowptr = np.zeros(n + 1, np.int32)
    rowptr[1] = len(rows[0])
    rowptr[2:1001] = rowptr[1]
    rowptr[1001] = rowptr[1000] + len(rows[1])
    rowptr[1001:2048] = rowptr[1001]
    rowptr[2048] = rowptr[2047] + 1
    col = np.concatenate(rows)
    # row 0: cols 0..n-1; row 1000: cols 1000..n-1; row 2047: the diagonal
    A = synth.UpperCSR(n, rowptr, col, synth.vector_uniform(len(col), 13))
    assert sg.spmv_single_launch(n, len(col))
    x = synth.vector_uniform(n, 14)
    y, s = sg.spmv(n, dev(A.rowptr), dev(A.col), dev(A.val), dev(x), syprd=True)
    e_y, e_s = errors(sg, A, x, y, s)
    assert e_y <= TOL_F32 and e_s <= TOL_F32, (e_y, e_s)


def test_cluster_form_skips_out_of_range_columns():
    sg = need_gpu()
    n = 500
    A = synth.upper_csr_uniform(n, 4000, 15)
    col = A.col.copy()
    bad = np.array([3, 777, 1500, 3999])
    col[bad[:2]] = n + 5
    col[bad[2:]] = -1
    assert sg.spmv_single_launch(n, len(col))
    x = synth.vector_uniform(n, 16)
    y, s = sg.spmv(n, dev(A.rowptr), dev(col), dev(A.val), dev(x), syprd=True)
    keep = np.ones(len(col), bool)
    keep[bad] = False
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))[keep]
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int32)
    B = synth.UpperCSR(n, rp, A.col[keep], A.val[keep])
    e_y, e_s = errors(sg, B, x, y, s)
    assert e_y <= TOL_F32 and e_s <= TOL_F32, (e_y, e_s)


def test_cluster_form_syprd_is_deterministic_and_graph_capturable():
    sg = need_gpu()
    n = 2000
    A = synth.upper_csr_uniform(n, 20000, 17)
    x = synth.vector_uniform(n, 17)
    rp, cl, vl, xd = dev(A.rowptr), dev(A.col), dev(A.val), dev(x)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    s_out = torch.empty(1, dtype=torch.float64, device="cuda")
    sg.spmv_noalloc(n, rp, cl, vl, xd, y, s_out)  # first call outside capture
    first = float(s_out.item())
    for _ in range(5):
        sg.spmv_noalloc(n, rp, cl, vl, xd, y, s_out)
        assert float(s_out.item()) == first
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    y.fill_(np.nan)
    with torch.cuda.graph(g, stream=side):
        sg.spmv_noalloc(n, rp, cl, vl, xd, y, s_out, stream=side)
    s_out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert float(s_out.item()) == first
    e_y, e_s = errors(sg, A, x, y, s_out)
    assert e_y <= TOL_F32 and e_s <= TOL_F32, (e_y, e_s)


def test_cluster_form_from_several_host_threads():
    """Calls with different shared-memory sizes from several host threads, each on its own stream:
    the kernel's shared-memory limit is only ever raised, so no launch is undercut by another."""
    import threading
    sg = need_gpu()
    cases = [(300, 3000, 21), (2000, 20000, 22), (6000, 60000, 23), (8000, 30000, 24)]
    data = []
    for n, nnz, seed in cases:
        assert sg.spmv_single_launch(n, nnz)
        A = synth.upper_csr_uniform(n, nnz, seed)
        x = synth.vector_uniform(n, seed)
        yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
        data.append((n, dev(A.rowptr), dev(A.col), dev(A.val), dev(x), yr, ya))
    errs = [[] for _ in cases]

    def work(k):
        n, rp, cl, vl, xd, yr, ya = data[k]
        st = torch.cuda.Stream()
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        for _ in range(20):
            sg.spmv(n, rp, cl, vl, xd, y=y, stream=st)
            st.synchronize()
            errs[k].append(oracle.componentwise_error(host(y), yr, ya))

    th = [threading.Thread(target=work, args=(k,)) for k in range(len(cases))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in range(len(cases)):
        assert len(errs[k]) == 20 and max(errs[k]) <= TOL_F32, (cases[k], errs[k][:3])


@pytest.mark.parametrize("skip_to", [3, 0])
def test_cluster_inbox_wait_runs_out_without_fault(skip_to):
    """The bounded inbox wait made to run out: no CTA pushes into CTA skip_to's inbox (nothing is left in
    flight towards it), the wait limit is 1 ms; that CTA's rows come back NaN (and SYPRD when it is CTA 0),
    every other row is exact, and the next normal call is clean."""
    sg = need_gpu()
    n, nnz = 2000, 20000
    A = synth.upper_csr_uniform(n, nnz, 41)
    x = synth.vector_uniform(n, 42)
    rp, cl, vl, xd = dev(A.rowptr), dev(A.col), dev(A.val), dev(x)
    y, s = sg.spmv_cluster_bounded(n, rp, cl, vl, xd, wait_limit_ns=1_000_000, skip_to=skip_to)
    torch.cuda.synchronize()
    yh = host(y)
    bad = np.isnan(yh)
    assert bad.any()
    rows = np.nonzero(bad)[0]
    assert rows.max() - rows.min() + 1 == len(rows)   # one contiguous slice: the skipped CTA's rows
    yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    ok = ~bad
    assert oracle.componentwise_error(yh[ok], yr[ok], ya[ok]) <= TOL_F32
    sr, sa = oracle.syprd(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    if skip_to == 0:
        assert rows.min() == 0 and np.isnan(float(s.item()))
    else:
        assert rows.min() > 0 and abs(float(s.item()) - sr) <= TOL_F32 * sa
    # a normal run afterwards, through the hook with no skip and through sym_spmv
    y2, s2 = sg.spmv_cluster_bounded(n, rp, cl, vl, xd)
    y3, s3 = sg.spmv(n, rp, cl, vl, xd, syprd=True)
    for yy, ss in ((y2, s2), (y3, s3)):
        assert oracle.componentwise_error(host(yy), yr, ya) <= TOL_F32
        assert abs(float(ss.item()) - sr) <= TOL_F32 * sa
