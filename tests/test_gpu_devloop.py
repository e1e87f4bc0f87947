"""Device-resident request loop (sym_devloop_*): MTTKRP and SSYMV / SYPRD requests of mixed orders, ranks,
factor types and sizes served by one persistent kernel, checked against the FP64 oracle; ring wrap-around,
host-side queueing, idle exit and relaunch, the HBM budget, bad requests, empty inputs and factors rewritten
between requests."""
import time

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, factor, host, need_gpu, tol_bf16

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def mttkrp_ref(T, Bused):
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
    return oracle.mttkrp_enum(T.order, T.n, cidx, cval, Bused.astype(np.float64))


def ssymv_ref(A, x):
    yr, ya = oracle.ssymv(A.n, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(A.n, A.rowptr, A.col, A.val, x.astype(np.float64))
    return yr, ya, sr, sa


# (order, n, nnz): orders 2..5; two-word keys for order 4 with n > 65,536 and order 5 with n > 4,096
TENSORS = [(3, 400, 20000), (4, 60, 9000), (5, 20, 4000), (2, 3000, 30000), (4, 70000, 30000), (5, 5000, 20000),
           (3, 50, 3000)]
CSRS = [(500, 4000), (3000, 40000), (40000, 200000), (1, 1)]   # n = 40,000: two zero chunks of y


def test_devloop_mix_matches_oracle_and_single_calls():
    sg = need_gpu()
    pool = []
    for k, (order, n, nnz) in enumerate(TENSORS):
        T = synth.tensor_uniform(order, n, nnz, 40 + k)
        pool.append((T, sg.SymTensor(dev(T.idx), dev(T.val), n)))
    mats = []
    for k, (n, nnz) in enumerate(CSRS):
        A = synth.upper_csr_uniform(n, nnz, 60 + k)
        x = synth.vector_uniform(n, 60 + k)
        mats.append((A, x, dev(A.rowptr), dev(A.col), dev(A.val), dev(x)))
    # every buffer first, then all requests in one burst (the loop kernel runs while they are submitted)
    plan = []
    ranks = [4, 8, 16, 64, 128, 12]
    for k in range(2 * len(pool)):
        T, X = pool[k % len(pool)]
        R = ranks[k % len(ranks)]
        bf16 = k % 3 == 1
        Bt, B32, Bused = factor(T.n, R, 200 + k, bf16)
        # output with a row stride wider than the rank, filled with NaN: the loop clears the rank columns
        Mbig = torch.full((T.n, R + 4), float("nan"), device="cuda")
        plan.append(("m", T, X, Bt, B32, Bused, Mbig[:, :R], Mbig, bf16))
        if k % 2 == 0:
            A, x, rp, cl, vl, xd = mats[(k // 2) % len(mats)]
            y = torch.full((A.n,), float("nan"), device="cuda")
            s = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            plan.append(("s", A, x, rp, cl, vl, xd, y, s))
    torch.cuda.synchronize()
    L = sg.DevLoop(ring_slots=64, idle_exit_s=0.005)
    reqs = []
    for k, p in enumerate(plan):
        if p[0] == "m":
            reqs.append((p[0], L.submit_mttkrp(p[2], p[3], p[6], tag=k)) + p[1:])
        else:
            A, x, rp, cl, vl, xd, y, s = p[1:]
            reqs.append((p[0], L.submit_ssymv(A.n, rp, cl, vl, xd, y, s, tag=k)) + p[1:])
    for k, q in enumerate(reqs):
        r = L.wait(q[1], 120)
        assert r["status"] == 0 and r["tag"] == k
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
        if q[0] == "m":
            _, t, T, X, Bt, B32, Bused, M, Mbig, bf16 = q
            ref, ra = mttkrp_ref(T, Bused)
            got = host(M)
            assert oracle.componentwise_error(got, ref, ra) <= TOL_F32
            if bf16:
                ref32, ra32 = mttkrp_ref(T, B32)
                assert oracle.componentwise_error(got, ref32, ra32) <= tol_bf16(T.order)
            assert np.isnan(host(Mbig)[:, M.shape[1]:]).all()   # columns past the rank untouched
            alone = host(X.mttkrp(Bt)).astype(np.float64)
            assert oracle.componentwise_error(got, alone, ra) <= 2 * TOL_F32
        else:
            _, t, A, x, rp, cl, vl, xd, y, s = q
            yr, ya, sr, sa = ssymv_ref(A, x)
            assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
            got_s = float(s.item())
            assert (abs(got_s - sr) / sa if sa > 0 else abs(got_s)) <= TOL_F32
    st = L.stats()
    assert st["completed"] == len(reqs) and st["published"] == len(reqs) and st["launches"] >= 1
    L.close()
    for _, X in pool:
        X.close()


def test_devloop_ring_wrap_queue_and_relaunch():
    sg = need_gpu()
    T = synth.tensor_uniform(3, 100, 2000, 7)
    X = sg.SymTensor(dev(T.idx), dev(T.val), T.n)
    A = synth.upper_csr_uniform(300, 2000, 8)
    x = synth.vector_uniform(300, 8)
    rp, cl, vl, xd = dev(A.rowptr), dev(A.col), dev(A.val), dev(x)
    Bs = [factor(T.n, 8, 300 + k) for k in range(4)]
    refs = [mttkrp_ref(T, b[2]) for b in Bs]
    yr, ya, sr, sa = ssymv_ref(A, x)
    torch.cuda.synchronize()
    # 16 ring slots, 200 requests submitted at once: most wait on the host until a slot frees
    L = sg.DevLoop(ring_slots=16, ctas=8, idle_exit_s=0.001)
    outs = []
    for k in range(200):
        if k % 4 == 3:
            y = torch.empty(300, device="cuda")
            s = torch.empty(1, dtype=torch.float64, device="cuda")
            outs.append(("s", L.submit_ssymv(300, rp, cl, vl, xd, y, s), y, s))
        else:
            M = torch.empty((T.n, 8), device="cuda")
            outs.append(("m", L.submit_mttkrp(X, Bs[k % 4][0], M), M, k % 4))
    for o in outs:
        assert L.wait(o[1], 120)["status"] == 0
    for o in outs:
        if o[0] == "m":
            ref, ra = refs[o[3]]
            assert oracle.componentwise_error(host(o[2]), ref, ra) <= TOL_F32
        else:
            assert oracle.componentwise_error(host(o[2]), yr, ya) <= TOL_F32
            assert abs(float(o[3].item()) - sr) / sa <= TOL_F32
    st = L.stats()
    assert st["completed"] == 200 and st["peak_inflight"] <= 16
    # the loop kernel leaves once idle; the next submission launches it again
    time.sleep(0.05)
    launches = st["launches"]
    M = torch.empty((T.n, 8), device="cuda")
    assert L.wait(L.submit_mttkrp(X, Bs[0][0], M), 60)["status"] == 0
    assert oracle.componentwise_error(host(M), *refs[0]) <= TOL_F32
    assert L.stats()["launches"] > launches
    L.close()
    X.close()


def test_devloop_factor_rewritten_between_requests():
    sg = need_gpu()
    T = synth.tensor_uniform(4, 80, 6000, 9)
    X = sg.SymTensor(dev(T.idx), dev(T.val), T.n)
    B1, B2 = synth.factor_normal(T.n, 16, 1), synth.factor_normal(T.n, 16, 2)
    Bd, B2d = dev(B1), dev(B2)
    M1 = torch.empty((T.n, 16), device="cuda")
    M2 = torch.empty((T.n, 16), device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    L = sg.DevLoop(ring_slots=16, idle_exit_s=1.0)   # the kernel stays resident across both requests
    assert L.wait(L.submit_mttkrp(X, Bd, M1), 60)["status"] == 0
    # same buffer, new contents, copied on a stream of its own while the loop kernel keeps running
    with torch.cuda.stream(s):
        Bd.copy_(B2d)
    s.synchronize()
    assert L.wait(L.submit_mttkrp(X, Bd, M2), 60)["status"] == 0
    for M, B in ((M1, B1), (M2, B2)):
        ref, ra = mttkrp_ref(T, B)
        assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
    assert L.stats()["launches"] == 1
    L.close()
    X.close()


def test_devloop_budget_admission_empty_inputs_and_bad_requests():
    sg = need_gpu()
    T = synth.tensor_uniform(3, 2000, 50000, 10)
    X = sg.SymTensor(dev(T.idx), dev(T.val), T.n)
    one = X.info()["arena_used"] + 2 * T.n * 16 * 4
    torch.cuda.synchronize()
    L = sg.DevLoop(ring_slots=16, hbm_budget_bytes=int(one * 1.5))   # room for one MTTKRP at a time
    work = []
    for k in range(5):
        Bt, B32, Bused = factor(T.n, 16, 500 + k)
        M = torch.empty((T.n, 16), device="cuda")
        work.append((L.submit_mttkrp(X, Bt, M), Bused, M))
    for t, Bused, M in work:
        assert L.wait(t, 60)["status"] == 0
        ref, ra = mttkrp_ref(T, Bused)
        assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
    st = L.stats()
    assert st["peak_inflight"] == 1 and st["peak_bytes"] <= int(one * 1.5)
    # empty CSRs: y cleared, SYPRD 0
    for n in (0, 7):
        rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
        cl = torch.zeros(0, dtype=torch.int32, device="cuda")
        vl = torch.zeros(0, dtype=torch.float32, device="cuda")
        x = torch.ones(n, device="cuda")
        y = torch.full((n,), 5.0, device="cuda")
        s = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert L.wait(L.submit_ssymv(n, rp, cl, vl, x, y, s), 60)["status"] == 0
        assert (host(y) == 0).all() and float(s.item()) == 0.0
    # refused on the host: over the whole budget, residual asked for, rank not a multiple of 4, bad ring size
    big = torch.empty((T.n, 16), device="cuda")
    L2 = sg.DevLoop(ring_slots=16, hbm_budget_bytes=1024)
    with pytest.raises(sg.SymError) as e:
        L2.submit_mttkrp(X, dev(synth.factor_normal(T.n, 16, 1)), big)
    assert e.value.code == -6
    L2.close()
    req = sg.Request(X.handle.value, big.data_ptr(), 0, 16, 16, big.data_ptr(), 16, 1, 0)
    t = sg.C.c_uint64(0)
    assert sg.lib().sym_devloop_submit_mttkrp(L.handle, sg.C.byref(req), sg.C.byref(t)) == -9
    B6 = torch.empty((T.n, 6), device="cuda")
    M6 = torch.empty((T.n, 8), device="cuda")
    req = sg.Request(X.handle.value, B6.data_ptr(), 0, 6, 6, M6.data_ptr(), 8, 0, 0)
    assert sg.lib().sym_devloop_submit_mttkrp(L.handle, sg.C.byref(req), sg.C.byref(t)) == -9
    r = sg.Result()
    assert sg.lib().sym_devloop_poll(L.handle, 10**9, sg.C.byref(r)) == -11
    bad = sg.DevLoopCfg(24, 0, 1 << 30, 1000000, 1000000000)
    h = sg.C.c_void_p()
    assert sg.lib().sym_devloop_create(sg.C.byref(bad), torch.cuda.current_device(), sg.C.byref(h)) == -1
    assert L.stats()["rejected"] == 0
    L.close()
    X.close()


def test_devloop_zero_wait_runs_out_and_loop_goes_on():
    """The compute chunks' bounded wait for the zero chunks, made to run out without any fault: the test hook
    leaves one request's zero chunks uncounted; that request completes with SYM_E_TIMEOUT and NaN SYPRD, the
    loop kernel keeps running, and the next request is exact."""
    sg = need_gpu()
    A = synth.upper_csr_uniform(2000, 30000, 11)
    x = synth.vector_uniform(2000, 11)
    rp, cl, vl, xd = dev(A.rowptr), dev(A.col), dev(A.val), dev(x)
    y1, y2 = torch.empty(2000, device="cuda"), torch.empty(2000, device="cuda")
    s1 = torch.empty(1, dtype=torch.float64, device="cuda")
    s2 = torch.empty(1, dtype=torch.float64, device="cuda")
    yr, ya, sr, sa = ssymv_ref(A, x)
    torch.cuda.synchronize()
    L = sg.DevLoop(ring_slots=16, ctas=4, idle_exit_s=2.0, wait_limit_s=0.005)
    sg.check(sg.lib().sym_devloop_set_test_hook(L.handle, 1), "sym_devloop_set_test_hook")
    t1 = L.submit_ssymv(2000, rp, cl, vl, xd, y1, s1)
    sg.check(sg.lib().sym_devloop_set_test_hook(L.handle, 0), "sym_devloop_set_test_hook")
    r1 = L.wait(t1, 60)
    assert r1["status"] == -7
    assert np.isnan(float(s1.item()))
    r2 = L.wait(L.submit_ssymv(2000, rp, cl, vl, xd, y2, s2), 60)
    assert r2["status"] == 0
    assert oracle.componentwise_error(host(y2), yr, ya) <= TOL_F32
    assert abs(float(s2.item()) - sr) / sa <= TOL_F32
    assert L.stats()["launches"] == 1
    L.close()
