"""SSYMV / SYPRD / Bellman-Ford / full-CSR baseline on the GPU vs the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, host, need_gpu

pytestmark = pytest.mark.gpu


def check_ssymv(sg, A, x):
    y, s = sg.spmv(A.n, dev(A.rowptr), dev(A.col), dev(A.val), dev(x), syprd=True)
    yr, ya = oracle.ssymv(A.n, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(A.n, A.rowptr, A.col, A.val, x.astype(np.float64))
    e_y = oracle.componentwise_error(host(y), yr, ya)
    e_s = abs(float(s.item()) - sr) / sa if sa > 0 else abs(float(s.item()))
    return e_y, e_s, host(y), float(s.item())


@pytest.mark.parametrize("n,nnz,seed", [(2000, 20000, 0), (2000, 20000, 1), (257, 4000, 2), (5000, 160000, 3),
                                        (64, 2080, 4)])
def test_ssymv_syprd(n, nnz, seed):
    sg = need_gpu()
    A = synth.upper_csr_uniform(n, nnz, seed)
    x = synth.vector_uniform(n, seed)
    e_y, e_s, y, s = check_ssymv(sg, A, x)
    assert e_y <= TOL_F32 and e_s <= TOL_F32, (e_y, e_s)
    # invariant x^T (A x) = SYPRD (within the FP32 tolerance of y)
    assert abs(float(x.astype(np.float64) @ y.astype(np.float64)) - s) <= 1e-4 * max(1.0, abs(s))


def test_ssymv_edge_cases():
    sg = need_gpu()
    # empty rows and a diagonal-only matrix
    rowptr = np.array([0, 0, 1, 1, 3, 3], np.int32)
    col = np.array([1, 3, 4], np.int32)
    val = np.array([2.0, -1.0, 0.5], np.float32)
    A = synth.UpperCSR(5, rowptr, col, val)
    x = synth.vector_uniform(5, 1)
    e_y, e_s, _, _ = check_ssymv(sg, A, x)
    assert e_y <= TOL_F32 and e_s <= TOL_F32
    n = 1000
    A = synth.UpperCSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                       synth.vector_uniform(n, 2))
    e_y, e_s, _, _ = check_ssymv(sg, A, synth.vector_uniform(n, 3))
    assert e_y <= TOL_F32 and e_s <= TOL_F32
    # one dense row (long fiber across many lanes)
    n = 3000
    A = synth.UpperCSR(n, np.array([0] + [n] * n, np.int32), np.arange(n, dtype=np.int32),
                       synth.vector_uniform(n, 4))
    e_y, e_s, _, _ = check_ssymv(sg, A, synth.vector_uniform(n, 5))
    assert e_y <= TOL_F32 and e_s <= TOL_F32


def test_csr_upper_check():
    sg = need_gpu()
    A = synth.upper_csr_uniform(300, 3000, 5)
    assert sg.csr_upper_check(300, dev(A.rowptr), dev(A.col), dev(A.val)) == 0
    bad_col = A.col.copy()
    r = 10
    p0 = A.rowptr[r]
    bad_col[p0] = r - 1 if r > 0 else 0       # below the diagonal
    assert sg.csr_upper_check(300, dev(A.rowptr), dev(bad_col), dev(A.val)) >= 1
    assert oracle.check_upper_csr(300, A.rowptr, bad_col) != 0


def test_bellman_exact():
    sg = need_gpu()
    A = synth.upper_csr_uniform(800, 6000, 6)
    w = np.abs(A.val) + np.float32(0.01)
    d = (synth.vector_uniform(800, 6) + 3).astype(np.float32)
    y = host(sg.bellman_step(800, dev(A.rowptr), dev(A.col), dev(w), dev(d)))
    want = oracle.bellman(800, A.rowptr, A.col, w, d.astype(np.float64)).astype(np.float32)
    assert np.array_equal(y, want)


def test_bellman_negative_weights_exact():
    sg = need_gpu()
    A = synth.upper_csr_uniform(400, 3000, 7)
    d = synth.vector_uniform(400, 8)
    y = host(sg.bellman_step(400, dev(A.rowptr), dev(A.col), dev(A.val), dev(d)))
    want = oracle.bellman(400, A.rowptr, A.col, A.val, d.astype(np.float64)).astype(np.float32)
    assert np.array_equal(y, want)


def test_full_csr_baseline():
    sg = need_gpu()
    A = synth.upper_csr_uniform(1500, 15000, 9)
    x = synth.vector_uniform(1500, 9)
    F = sg.FullCSR(1500, dev(A.rowptr), dev(A.col), dev(A.val))
    rp, col, val = (host(t) for t in F.arrays())
    D = np.zeros((1500, 1500), np.float32)
    rows = np.repeat(np.arange(1500), np.diff(A.rowptr))
    D[rows, A.col] = A.val
    D[A.col, rows] = A.val
    full_rows = np.repeat(np.arange(1500), np.diff(rp))
    assert rp[-1] == np.count_nonzero(D)
    assert np.array_equal(D[full_rows, col], val)
    assert all(np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0) for i in range(0, 1500, 7))
    y = host(F.spmv(dev(x)))
    yr, ya = oracle.ssymv(1500, A.rowptr, A.col, A.val, x.astype(np.float64))
    assert oracle.componentwise_error(y, yr, ya) <= TOL_F32
