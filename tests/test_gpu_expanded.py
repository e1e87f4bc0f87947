"""The expanded (non-symmetric) baseline: expansion bit-exact vs the oracle, MTTKRP parity."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, host, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order,n,nnz", [(2, 100, 800), (3, 60, 4000), (4, 20, 3000), (5, 10, 1500)])
def test_expansion_bitexact(order, n, nnz):
    sg = need_gpu()
    T = synth.tensor_uniform(order, n, nnz, 50 + order)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    E = X.expanded()
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    ei, ev = oracle.expand(order, cidx, cval)
    gi, gv = E.export()
    assert E.nnz == ei.shape[1] == X.info()["expanded_nnz"]
    assert np.array_equal(host(gi), ei)
    assert np.array_equal(host(gv), ev)


@pytest.mark.parametrize("order,n,nnz,rank", [(3, 300, 20000, 64), (4, 40, 8000, 32), (5, 15, 3000, 16)])
def test_expanded_mttkrp(order, n, nnz, rank):
    sg = need_gpu()
    T = synth.tensor_uniform(order, n, nnz, 60 + order)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    E = X.expanded()
    B = synth.factor_normal(n, rank, 2)
    M = host(E.mttkrp(dev(B)))
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    ref, ra = oracle.mttkrp_enum(order, n, cidx, cval, B.astype(np.float64))
    assert oracle.componentwise_error(M, ref, ra) <= TOL_F32
