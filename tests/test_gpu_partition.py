"""Partition invariance of the natural multi-device shard, run as several launches on one GPU.

The symmetric MTTKRP shards by contiguous ranges of canonical entries (factor
replicated, partial outputs summed) and SSYMV / SYPRD by row ranges (partial y
and partial SYPRD summed).  Each part here is one sym_mttkrp_range /
sym_spmv_rows launch into its own output; the parts are summed on the host in
FP64 and the sum is checked against the FP64 oracle with the same
componentwise tolerance as the whole-tensor calls.  The all-reduce itself is
not run: every run of this build sees one GPU.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, factor, host, need_gpu

pytestmark = pytest.mark.gpu


def cuts(total, K, seed):
    """K contiguous parts of [0, total) with uneven, seeded sizes (empty parts allowed)."""
    if K == 1:
        return [0, total]
    inner = np.sort(synth.Stream(seed).randint(K - 1, total + 1))
    return [0] + [int(c) for c in inner] + [total]


@pytest.mark.parametrize("K", [2, 3, 7])
@pytest.mark.parametrize("case", ["zipf3_r32", "unif4_r16", "unif5_r8_diag", "unif2_r4"])
@pytest.mark.parametrize("kernel", ["plain", "lane"])
def test_mttkrp_entry_partition(K, case, kernel):
    sg = need_gpu()
    if case == "zipf3_r32":
        T, R = synth.tensor3_zipf(2000, 50000, 21), 32
    elif case == "unif4_r16":
        T, R = synth.tensor_uniform(4, 60, 20000, 22), 16
    elif case == "unif5_r8_diag":
        T, R = synth.tensor_uniform(5, 12, 3000, 23), 8    # many repeated indices: the cut crosses the diagonal stream
    else:
        T, R = synth.tensor_uniform(2, 500, 6000, 24), 4
    X = sg.SymTensor(dev(T.idx), dev(T.val), T.n)
    if kernel == "lane":
        X.set_config(strict_kernel=sg.MTTKRP_LANE, entries_per_warp=64, threads_per_cta=256, leaf_index=1,
                     vec_per_lane=4 if R >= 16 else 1)
    info = X.info()
    Bt, B32, _ = factor(T.n, R, 7)
    c = cuts(info["nnz"], K, 100 + K)
    total = np.zeros((T.n, R), np.float64)
    acc = None
    for a, b in zip(c[:-1], c[1:]):
        part = host(X.mttkrp_range(Bt, a, b - a))
        total += part.astype(np.float64)
        acc = X.mttkrp_range(Bt, a, b - a, M=acc, accumulate=acc is not None)
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
    ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, B32.astype(np.float64))
    assert oracle.componentwise_error(total, ref, ra) <= TOL_F32
    assert oracle.componentwise_error(host(acc), ref, ra) <= TOL_F32   # the same parts accumulated on the device


def test_mttkrp_range_rejects_bad_ranges():
    sg = need_gpu()
    T = synth.tensor_uniform(3, 40, 300, 3)
    X = sg.SymTensor(dev(T.idx), dev(T.val), T.n)
    Bt, _, _ = factor(T.n, 8, 1)
    nnz = X.info()["nnz"]
    for a, n in ((-1, 5), (0, nnz + 1), (nnz, 1), (5, -1)):
        with pytest.raises(sg.SymError):
            X.mttkrp_range(Bt, a, n)
    M = X.mttkrp_range(Bt, nnz, 0)     # an empty part: zeros
    assert float(M.abs().max()) == 0.0


@pytest.mark.parametrize("K", [2, 3, 7])
@pytest.mark.parametrize("n,nnz", [(2000, 20000), (40_000, 700_000), (300, 300)])
def test_spmv_row_partition(K, n, nnz):
    sg = need_gpu()
    A = synth.upper_csr_uniform(n, nnz, 30 + K)
    x = synth.vector_uniform(n, 31)
    rp, cl, vl, xd = dev(A.rowptr), dev(A.col), dev(A.val), dev(x)
    c = cuts(n, K, 200 + K)
    ysum = np.zeros(n, np.float64)
    ssum = 0.0
    yacc = None
    for a, b in zip(c[:-1], c[1:]):
        y, s = sg.spmv_rows(n, rp, cl, vl, xd, a, b, syprd=True)
        ysum += host(y).astype(np.float64)
        ssum += float(s.item())
        yacc = sg.spmv_rows(n, rp, cl, vl, xd, a, b, y=yacc, accumulate=yacc is not None)
    yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    assert oracle.componentwise_error(ysum, yr, ya) <= TOL_F32
    assert oracle.componentwise_error(host(yacc), yr, ya) <= TOL_F32
    assert abs(ssum - sr) <= TOL_F32 * sa
