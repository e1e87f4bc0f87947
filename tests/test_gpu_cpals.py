"""Symmetric CP-ALS update on the GPU vs the FP64 oracle.

Tolerance: the update multiplies the FP32 MTTKRP (componentwise error <= 1e-5)
by H^{-1} (formed in FP64, applied in FP32); with the well-conditioned H of
random factors the result agrees with the oracle to 1e-4 of its largest entry.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import dev, factor, host, need_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.mark.parametrize("order,n,nnz,rank", [(3, 400, 20000, 16), (3, 300, 8000, 64), (4, 60, 9000, 32),
                                              (5, 25, 6000, 8), (3, 2000, 30000, 128)])
@pytest.mark.parametrize("bf16", [False, True])
def test_cp_als_step(order, n, nnz, rank, bf16):
    sg = need_gpu()
    T = synth.tensor_uniform(order, n, nnz, 70 + order)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    Bt, B32, Bused = factor(n, rank, 4, bf16)
    Bn, info = X.cp_als_step(Bt, ridge=1e-3)
    assert int(info.item()) == 0
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    want, oinfo = oracle.cp_als_step(order, n, cidx, cval, Bused.astype(np.float64), ridge=1e-3)
    assert oinfo == 0
    got = host(Bn.float())
    scale = np.max(np.abs(want))
    tol = TOL if not bf16 else 2 ** -8   # the BF16 output is rounded once more
    assert np.max(np.abs(got - want)) <= tol * scale


def test_cp_als_fixed_point_on_gpu():
    sg = need_gpu()
    n, R = 12, 4
    Bs = synth.factor_normal(n, R, 5)
    rows = np.array(list(itertools.combinations_with_replacement(range(n), 3)), np.int32)
    vals = np.array([sum(np.prod(Bs[list(t), r].astype(np.float64)) for r in range(R)) for t in rows], np.float32)
    X = sg.SymTensor(dev(rows.T.copy()), dev(vals), n)
    Bn, info = X.cp_als_step(dev(Bs))
    assert int(info.item()) == 0
    assert np.allclose(host(Bn), Bs, rtol=1e-3, atol=1e-4)


def test_cp_als_reports_singular_H():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    T = synth.tensor_uniform(3, 50, 500, 9)
    X = sg.SymTensor(dev(T.idx), dev(T.val), 50)
    B = torch.zeros((50, 8), device="cuda")
    Bn, info = X.cp_als_step(B)
    assert int(info.item()) == 1
    assert float(Bn.abs().max()) == 0.0
