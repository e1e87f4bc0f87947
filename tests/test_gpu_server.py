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
    with pytest.raises(sg.SymError) as e:      # want_residual outside 0..2
        S.submit(X, dev(synth.factor_normal(100, 16, 2)), torch.empty((100, 16), device="cuda"), residual=3)
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


def test_registered_tensors_evicted_and_reloaded():
    """Registered tensors live in a pool smaller than all of them together: requests cycling through them
    force loads and least-recently-used evictions; every result equals the tensor's own MTTKRP and the oracle."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    P = pool(sg, [(3, 500, 30000), (4, 80, 20000), (5, 25, 8000), (3, 900, 40000), (4, 120, 25000)], seed=31)
    images = [X.save_image() for _, X in P]
    sizes = [X.info()["arena_used"] for _, X in P]
    pool_bytes = int(max(sizes) * 2.2)          # room for about two tensors at once
    S = sg.Server(max_slots=4, max_rank=32, hbm_budget_bytes=pool_bytes + (64 << 20), pool_bytes=pool_bytes)
    ids = [S.register(img) for img in images]
    reqs = []
    for k in range(20):
        j = (k * 3) % len(P)            # revisits tensors after others pushed them out
        T, X = P[j]
        R = (8, 16, 32)[k % 3]
        Bt, B32, Bused = factor(T.n, R, 200 + k, bf16=(k % 4 == 1))
        M = torch.empty((T.n, R), device="cuda")
        reqs.append((S.submit_registered(ids[j], Bt, M, residual=True, tag=k), T, X, Bt, Bused, M))
    for t, T, X, Bt, Bused, M in reqs:
        r = S.wait(t, 60)
        assert r["status"] == 0
        cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
        ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
        want, ab, _ = oracle.cpfit(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert abs(r["residual"] - want) / ab <= TOL_F32
    st = S.stats()
    assert st["completed"] == 20 and st["loads"] >= len(P) and st["evictions"] >= len(P) - 2
    assert st["peak_resident_bytes"] <= pool_bytes and st["peak_bytes"] <= pool_bytes + (64 << 20)
    # a tensor larger than the whole pool is refused at registration
    big_pool = sg.Server(max_slots=2, max_rank=16, hbm_budget_bytes=1 << 30, pool_bytes=4096)
    with pytest.raises(sg.SymError) as e:
        big_pool.register(images[0])
    assert e.value.code == -6
    big_pool.close()
    with pytest.raises(sg.SymError) as e:
        S.submit_registered(999, Bt, M)
    assert e.value.code == -11
    S.close()


def test_registered_requests_share_loads():
    """A pool with room for one of two registered tensors and a burst of requests alternating between them:
    admission takes the requests for the resident tensor first, so the queued requests for the other share
    one load instead of one load each (first-come order would load for every request)."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    P = pool(sg, [(3, 600, 40000), (4, 90, 30000)], seed=51)
    images = [X.save_image() for _, X in P]
    sizes = [X.info()["arena_used"] for _, X in P]
    pool_bytes = int(max(sizes) * 1.5)
    S = sg.Server(max_slots=1, max_rank=16, hbm_budget_bytes=pool_bytes + (64 << 20), pool_bytes=pool_bytes)
    ids = [S.register(img) for img in images]
    made = []
    for k in range(16):
        T, X = P[k % 2]
        Bt, B32, Bused = factor(T.n, 16, 500 + k)
        made.append((k % 2, T, Bt, Bused, torch.empty((T.n, 16), device="cuda")))
    torch.cuda.synchronize()
    reqs = [(S.submit_registered(ids[j], Bt, M, residual=True, tag=k), T, Bused, M)
            for k, (j, T, Bt, Bused, M) in enumerate(made)]
    for t, T, Bused, M in reqs:
        r = S.wait(t, 60)
        assert r["status"] == 0
        cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
        ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
        want, ab, _ = oracle.cpfit(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert abs(r["residual"] - want) / ab <= TOL_F32
    st = S.stats()
    assert st["completed"] == 16 and 2 <= st["loads"] <= 6, st
    assert st["peak_resident_bytes"] <= pool_bytes
    S.close()


def test_cached_gram_reused_and_refreshed():
    """residual=2 declares the factor unchanged since an earlier request: the residual reuses the Gram matrix
    cached then (gram_hits counts it) and still equals the oracle's.  Overwriting the factor in place and
    submitting with residual=True recomputes it; later residual=2 requests see the new factor."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    P = pool(sg, [(3, 400, 20000), (4, 60, 9000)], seed=71)
    S = sg.Server(max_slots=3, max_rank=32)
    facs = []
    for k, (T, X) in enumerate(P):
        Bt, B32, Bused = factor(T.n, 16, 700 + k, bf16=(k == 1))
        facs.append([T, X, Bt, Bused])

    def run(flags):
        outs = []
        for j, flag in flags:
            T, X, Bt, Bused = facs[j]
            M = torch.empty((T.n, 16), device="cuda")
            outs.append((S.submit(X, Bt, M, residual=flag), j, M, Bused.copy()))
        for t, j, M, Bused in outs:
            r = S.wait(t, 60)
            assert r["status"] == 0
            T = facs[j][0]
            cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
            ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, Bused.astype(np.float64))
            assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
            want, ab, _ = oracle.cpfit(T.order, T.n, cidx, cval, Bused.astype(np.float64))
            assert abs(r["residual"] - want) / ab <= TOL_F32

    run([(0, True), (1, True)])
    run([(0, 2), (1, 2), (0, 2), (1, 2)])
    hits = S.stats()["gram_hits"]
    assert hits == 4
    # the factor changes in place: the caller says so (residual=True), the cache is refreshed
    T, X, Bt, _ = facs[0]
    torch.manual_seed(5)
    newB = torch.randn(Bt.shape, device="cuda") / 4.0
    Bt.copy_(newB.to(Bt.dtype))
    torch.cuda.synchronize()
    facs[0][3] = host(Bt.float()).astype(np.float32)
    run([(0, True)])
    run([(0, 2), (0, 2)])
    assert S.stats()["gram_hits"] == hits + 2
    S.close()


def test_small_requests_grouped_launches():
    """coalesce_small: small requests admitted together share one slot (grouped launch); results unchanged."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    P = pool(sg, [(3, 200, 3000), (4, 40, 2000), (5, 15, 1500)], seed=41)
    # one slot and a burst of submissions: requests queue while the slot is busy, and the backlog is admitted
    # as groups
    S = sg.Server(max_slots=1, max_rank=16, small_nnz=100_000, coalesce_small=True)
    made = []
    for k in range(40):
        T, X = P[k % 3]
        Bt, B32, Bused = factor(T.n, 16, 300 + k)
        made.append((T, X, Bt, Bused, torch.empty((T.n, 16), device="cuda")))
    torch.cuda.synchronize()
    reqs = [(S.submit(X, Bt, M, residual=True, tag=k), T, Bused, M) for k, (T, X, Bt, Bused, M) in enumerate(made)]
    for t, T, Bused, M in reqs:
        r = S.wait(t, 60)
        assert r["status"] == 0
        cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
        ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
        want, ab, _ = oracle.cpfit(T.order, T.n, cidx, cval, Bused.astype(np.float64))
        assert abs(r["residual"] - want) / ab <= TOL_F32
    st = S.stats()
    assert st["completed"] == 40 and st["launches"] < 40 and st["grouped_launches"] >= 1
    S.close()


def test_destroy_timeout_keeps_buffers_valid():
    """A drain limit that runs out: destroy returns SYM_E_TIMEOUT while work is in flight; the caller keeps the
    buffers until the device is done, and the results are still right."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    T = synth.tensor_uniform(3, 3000, 400_000, 51)
    X = sg.SymTensor(dev(T.idx), dev(T.val), T.n)
    S = sg.Server(max_slots=2, max_rank=64, wait_limit_s=1e-9)
    B = dev(synth.factor_normal(T.n, 64, 51))
    Ms = [torch.empty((T.n, 64), device="cuda") for _ in range(6)]
    for M in Ms:
        S.submit(X, B, M)
    import time
    t0 = time.time()
    while S.stats()["admitted"] < 1 and time.time() - t0 < 10:
        time.sleep(1e-4)
    code = sg.lib().sym_server_destroy(S.handle)
    S.handle = None
    assert code in (0, -7)     # -7 when work was still in flight at the limit
    torch.cuda.synchronize()
    time.sleep(0.2)            # the scheduler thread finishes and releases the server's own resources
    ref = X.mttkrp(B)
    torch.cuda.synchronize()
    # requests that were admitted before the limit ran to completion; queued ones were dropped
    assert any(float((M - ref).abs().max()) <= 1e-4 * float(ref.abs().max()) for M in Ms)
