"""Serving: continuous batching results equal the alone results and the oracle; admission and errors."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_BF16, TOL_F32, dev, factor, host, need_gpu

pytestmark = pytest.mark.gpu


def pool(sg, specs, seed=0):
    out = []
    for k, (order, n, nnz) in enumerate(specs):
        T = synth.tensor_uniform(order, n, nnz, seed + k)
        out.append((T, sg.SymTensor(dev(T.idx), dev(T.val), n)))
    return out


SPECS = [(3, 400, 20000), (4, 60, 9000), (5, 20, 4000), (3, 2000, 100000), (4, 300, 50000), (3, 50, 3000)]


def test_mix_equals_alone_and_oracle():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    P = pool(sg, SPECS)
    S = sg.Server(max_slots=4, max_rank=64, small_nnz=10000)
    reqs = []
    ranks = [8, 16, 32, 64]
    for k in range(24):
        T, X = P[k % len(P)]
        R = ranks[k % 4]
        bf16 = (k % 3 == 0)
        Bt, B32, Bused = factor(T.n, R, 100 + k, bf16)
        M = torch.empty((T.n, R), device="cuda")
        t = S.submit(X, Bt, M, residual=True, tag=k)
        reqs.append((t, T, X, Bt, B32, Bused, M, bf16))
    for (t, T, X, Bt, B32, Bused, M, bf16) in reqs:
        r = S.wait(t, 60)
        assert r["status"] == 0
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
        alone, res_alone = X.mttkrp(Bt, residual=True)
        cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
        ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        # same result alone and in the mix, within the tolerance (atomic order differs)
        assert oracle.componentwise_error(host(M), host(alone).astype(np.float64), ra) <= 2 * TOL_F32
        assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
        want, ab, _ = oracle.cpfit(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert abs(r["residual"] - want) / ab <= TOL_F32
        assert abs(r["residual"] - float(res_alone.item())) / ab <= 2 * TOL_F32
    st = S.stats()
    assert st["completed"] == 24 and st["admitted"] == 24 and st["peak_inflight"] <= 4
    S.close()


def test_budget_admission_and_rejection():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    P = pool(sg, [(3, 2000, 100000)] * 3, seed=7)
    one = P[0][1].info()["arena_used"] + 2 * 2000 * 16 * 4
    S = sg.Server(max_slots=8, max_rank=16, hbm_budget_bytes=int(one * 1.5))   # room for one at a time
    tickets = []
    for k in range(6):
        T, X = P[k % 3]
        B = dev(synth.factor_normal(T.n, 16, k))
        M = torch.empty((T.n, 16), device="cuda")
        tickets.append((S.submit(X, B, M), X, B, M))
    for t, X, B, M in tickets:
        assert S.wait(t, 60)["status"] == 0
        ref = X.mttkrp(B)
        assert float((ref - M).abs().max()) <= 1e-4 * float(ref.abs().max())
    st = S.stats()
    assert st["peak_inflight"] == 1 and st["peak_bytes"] <= int(one * 1.5)
    # a request larger than the whole budget is refused at submission
    T, X = P[0]
    big = torch.empty((T.n, 16), device="cuda")
    with pytest.raises(sg.SymError) as e:
        S2 = sg.Server(max_slots=2, max_rank=16, hbm_budget_bytes=1024)
        S2.submit(X, dev(synth.factor_normal(T.n, 16, 1)), big)
    assert e.value.code == -6
    S2.close()
    S.close()


def test_bad_requests_and_unknown_tickets():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    (T, X), = pool(sg, [(3, 100, 2000)], seed=3)
    S = sg.Server(max_slots=2, max_rank=32)
    M = torch.empty((100, 64), device="cuda")
    with pytest.raises(sg.SymError) as e:      # rank above the server's max_rank
        S.submit(X, dev(synth.factor_normal(100, 64, 1)), M)
    assert e.value.code == -9
    with pytest.raises(sg.SymError) as e:      # rank not a multiple of 4
        S.submit(X, torch.zeros((100, 6), device="cuda"), torch.zeros((100, 6), device="cuda"))
    assert e.value.code == -9
    good = S.submit(X, dev(synth.factor_normal(100, 16, 2)), torch.empty((100, 16), device="cuda"))
    assert S.wait(good, 30)["status"] == 0
    with pytest.raises(sg.SymError) as e:
        S.poll(987654321)
    assert e.value.code == -11
    S.close()


def test_poll_until_done():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    (T, X), = pool(sg, [(4, 200, 40000)], seed=4)
    S = sg.Server(max_slots=2, max_rank=32)
    B = dev(synth.factor_normal(200, 32, 5))
    M = torch.empty((200, 32), device="cuda")
    t = S.submit(X, B, M)
    import time
    deadline = time.time() + 30
    r = None
    while r is None and time.time() < deadline:
        r = S.poll(t)
    assert r is not None and r["status"] == 0
    with pytest.raises(sg.SymError):
        S.poll(t)         # results are handed out once
    S.close()
