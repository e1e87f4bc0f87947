"""Parity at the benchmark workloads' full sizes, in the configuration bench.py times.

The oracle computes sampled outputs one by one (rows selected by a mask: the
Zipf-hot rows, rows touched by repeated-index entries, and random rows); the
GPU result is the autotuned kernel's, as in the benchmark.  Counts are compared
exactly for the whole tensor.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_BF16, TOL_F32, dev, host, need_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WORKLOADS = [
    # order, n, nnz, rank, seed, recipe
    (3, 100_000, 20_000_000, 64, 1, "zipf"),
    (4, 20_000, 10_000_000, 32, 2, "uniform"),
    (5, 2_000, 5_000_000, 16, 2, "uniform"),
]


def sample_rows(n, cidx, seed, k=48):
    st = synth.Stream(seed, tag=5)
    rows = set(range(min(16, n)))
    rows |= set(st.randint(k, n).tolist())
    diag = np.nonzero((cidx[1:] == cidx[:-1]).any(axis=0))[0]
    if diag.size:
        rows |= set(cidx[0, diag[st.randint(8, diag.size)]].tolist())
    return np.array(sorted(rows))


@pytest.mark.parametrize("order,n,nnz,rank,seed,recipe", WORKLOADS)
def test_fullsize_mttkrp_sampled_rows(order, n, nnz, rank, seed, recipe):
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    T = synth.make_tensor(order, n, nnz, seed, recipe)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    # exact counts over the whole tensor
    cnt = oracle.counts(order, cidx, cval)
    info = X.info()
    assert info["nnz"] == nnz and info["counts_by_pattern"] == cnt["by_pattern"].tolist()
    assert info["expanded_nnz"] == cnt["expanded"]
    assert info["root_fibers"] == cnt["root_fibers"] and info["l2_fibers"] == cnt["l2_fibers"]
    B32 = synth.factor_normal(n, rank, seed)
    rows = sample_rows(n, cidx, seed)
    for bf16 in (False, True):
        if bf16:
            bits = synth.bf16_rne(B32)
            Bt = dev(bits.view(np.int16)).view(torch.bfloat16)
            Bused = synth.bf16_to_f32(bits)
        else:
            Bt, Bused = dev(B32), B32
        X.autotune(Bt)
        M = host(X.mttkrp(Bt))[rows]
        ref, ra = oracle.mttkrp_enum(order, n, cidx, cval, B32.astype(np.float64), rows=rows)
        e32 = oracle.componentwise_error(M, ref[rows], ra[rows])
        if bf16:
            refb, rab = oracle.mttkrp_enum(order, n, cidx, cval, Bused.astype(np.float64), rows=rows)
            assert e32 <= TOL_BF16, e32
            assert oracle.componentwise_error(M, refb[rows], rab[rows]) <= TOL_F32
        else:
            assert e32 <= TOL_F32, e32


def test_fullsize_ssymv_n2000():
    sg = need_gpu()
    A = synth.upper_csr_uniform(2000, 20000, 0)
    x = synth.vector_uniform(2000, 0)
    y, s = sg.spmv(2000, dev(A.rowptr), dev(A.col), dev(A.val), dev(x), syprd=True)
    yr, ya = oracle.ssymv(2000, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(2000, A.rowptr, A.col, A.val, x.astype(np.float64))
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    assert abs(float(s.item()) - sr) / sa <= TOL_F32


def test_fullsize_batch_sampled_instances():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    sizes = synth.batch_sizes(4096, 256, 65536, 3)
    batch = sg.make_batch(sizes, 16, 3)
    rows = int(batch.host_row_off[-1])
    x = synth.vector_uniform(rows, 3)
    xd = dev(x)
    y = torch.empty_like(xd)
    sy = torch.empty(4096, dtype=torch.float64, device="cuda")
    cfg, _ = sg.autotune_batch(batch, xd, y, sy)
    plan = sg.BatchPlan(batch, cfg)
    plan.capture(xd, y, sy)
    plan.launch()
    torch.cuda.synchronize()
    yh, sh = host(y), host(sy)
    ro = batch.host_row_off
    rp_all = host(batch.rowptr)
    for b in [0, 1, 17, 1024, 2047, 3000, 4095] + list(np.argsort(sizes)[-3:]):
        r0, r1 = int(ro[b]), int(ro[b + 1])
        p0, p1 = int(rp_all[r0]), int(rp_all[r1])
        rp = (rp_all[r0:r1 + 1] - p0).astype(np.int32)
        cl = (host(batch.col[p0:p1]) - r0).astype(np.int32)
        vl = host(batch.val[p0:p1])
        yr, ya = oracle.ssymv(r1 - r0, rp, cl, vl, x[r0:r1].astype(np.float64))
        sr, sa = oracle.syprd(r1 - r0, rp, cl, vl, x[r0:r1].astype(np.float64))
        assert oracle.componentwise_error(yh[r0:r1], yr, ya) <= TOL_F32, b
        assert abs(sh[b] - sr) / sa <= TOL_F32, b


def test_fullsize_ptensor_parts22():
    """The partially symmetric bench workload: parts (2, 2), n = 20,000 per part, 5M canonical entries, R = 32.
    Canonical form and counts exact; every row of both parts' MTTKRP within the FP32 tolerance."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    parts, dims, rank = (2, 2), (20_000, 20_000), 32
    T = synth.ptensor_uniform(parts, dims, 5_000_000, 4)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    gi, gv = X.export()
    assert np.array_equal(host(gi), cidx) and np.array_equal(host(gv), cval)
    cnt = oracle.pcounts(parts, cidx, cval)
    assert X.info()["expanded_nnz"] == cnt["expanded"]
    F = [synth.factor_normal(d, rank, 4 + p) for p, d in enumerate(dims)]
    Fd = [dev(f) for f in F]
    for out in range(2):
        M = host(X.mttkrp(Fd, out))
        ref, ref_abs = oracle.pmttkrp_enum(parts, dims, cidx, cval, [f.astype(np.float64) for f in F], out)
        assert oracle.componentwise_error(M, ref, ref_abs) <= TOL_F32, out
