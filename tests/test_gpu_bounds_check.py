"""The bounds-checked build (libsymgpu_bc.so, compiled with -DSYM_BOUNDS_CHECK) on in-range inputs.

Every gathered or scattered index of the hot-path kernels is checked against its array's extent there; a
violation is counted in a caller-given device word and the access skipped.  On valid inputs the counter must stay
zero and every result must match the FP64 oracle exactly as the normal build's do.  One out-of-range case is run:
columns past n in the one-launch SSYMV form, which the normal build already skips by construction, so the
checked build must count them without touching memory outside the arrays.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu


def bc_lib(sg):
    from paper_2406_09266_gb300 import build
    path = build.build(bounds_check=True)
    L = C.CDLL(path)
    for name, (args, res) in sg._SIGS.items():
        f = getattr(L, name, None)
        if f is not None:
            f.argtypes, f.restype = args, res
    assert L.sym_bounds_check_enabled() == 1
    return L


def test_normal_build_is_not_bounds_checked():
    sg = need_gpu()
    assert sg.lib().sym_bounds_check_enabled() == 0
    assert sg.lib().sym_bounds_check_attach(None) == -10   # SYM_E_UNSUPPORTED


@pytest.mark.parametrize("case", ["zipf3_plain", "unif4_lane_two_pass", "unif5_lane_one_pass", "diag_only"])
def test_bounds_checked_mttkrp_in_range(case):
    sg = need_gpu()
    L = bc_lib(sg)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert L.sym_bounds_check_attach(C.c_void_p(counter.data_ptr())) == 0
    if case == "zipf3_plain":
        T, R, cfg = synth.tensor3_zipf(2000, 40000, 61), 32, dict(strict_kernel=0, entries_per_warp=256, leaf_index=0)
    elif case == "unif4_lane_two_pass":
        T, R, cfg = synth.tensor_uniform(4, 60, 12001, 62), 16, dict(strict_kernel=4, entries_per_warp=128,
                                                                      leaf_index=1)
    elif case == "unif5_lane_one_pass":
        T, R, cfg = synth.tensor_uniform(5, 20, 6003, 63), 16, dict(strict_kernel=4, entries_per_warp=64, leaf_index=0)
    else:
        T0 = synth.tensor_small_all_patterns(4, 8, 3, density=1.0)
        keep = np.array([len(set(T0.idx[:, e])) < 4 for e in range(T0.nnz)])
        T, R, cfg = synth.SymCOO(4, 8, np.ascontiguousarray(T0.idx[:, keep]), T0.val[keep]), 8, dict(
            strict_kernel=0, entries_per_warp=128, leaf_index=0)
    idx, val = dev(T.idx), dev(T.val)
    ab, wb = C.c_size_t(0), C.c_size_t(0)
    assert L.sym_tensor_create_bytes(T.order, T.n, T.nnz, C.byref(ab), C.byref(wb)) == 0
    arena = torch.empty(ab.value, dtype=torch.uint8, device="cuda")
    ws = torch.empty(max(wb.value, 256), dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.sym_tensor_create(T.order, T.n, T.nnz, C.c_void_p(idx.data_ptr()), T.nnz, C.c_void_p(val.data_ptr()), 0,
                               C.c_void_p(arena.data_ptr()), arena.numel(), C.c_void_p(ws.data_ptr()), ws.numel(),
                               stream, C.byref(h)) == 0
    if cfg.get("leaf_index"):
        la, lw = C.c_size_t(0), C.c_size_t(0)
        assert L.sym_tensor_leaf_index_bytes(h, C.byref(la), C.byref(lw)) == 0
        larena = torch.empty(max(la.value, 256), dtype=torch.uint8, device="cuda")
        lws = torch.empty(max(lw.value, 256), dtype=torch.uint8, device="cuda")
        assert L.sym_tensor_add_leaf_index(h, C.c_void_p(larena.data_ptr()), larena.numel(),
                                           C.c_void_p(lws.data_ptr()), lws.numel(), stream) == 0
    c = sg.MttkrpCfg(cfg["strict_kernel"], cfg["entries_per_warp"], 256, 2, 0, 96, 0, cfg["leaf_index"], 1, 1, 0)
    assert L.sym_mttkrp_set_config(h, C.byref(c)) == 0
    B = synth.factor_normal(T.n, R, 64)
    Bd = dev(B)
    M = torch.empty((T.n, R), device="cuda")
    assert L.sym_mttkrp(h, C.c_void_p(Bd.data_ptr()), 0, R, R, C.c_void_p(M.data_ptr()), R, None, None, 0,
                        stream) == 0
    torch.cuda.synchronize()
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx, T.val)
    ref, ra = oracle.mttkrp_enum(T.order, T.n, cidx, cval, B.astype(np.float64))
    assert oracle.componentwise_error(host(M), ref, ra) <= TOL_F32
    assert int(counter.item()) == 0
    L.sym_tensor_destroy(h)
    assert L.sym_bounds_check_attach(None) == 0


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


@pytest.mark.parametrize("n,nnz", [(2000, 20000), (40000, 500000)])
def test_bounds_checked_ssymv_in_range(n, nnz):
    """Both forms (one launch for n = 2,000, multi-block for n = 40,000) on valid matrices: counter stays 0."""
    sg = need_gpu()
    L = bc_lib(sg)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert L.sym_bounds_check_attach(C.c_void_p(counter.data_ptr())) == 0
    A = synth.upper_csr_uniform(n, nnz, 70)
    x = synth.vector_uniform(n, 71)
    rp, cl, vl, xd = dev(A.rowptr), dev(A.col), dev(A.val), dev(x)
    desc = Csr(n, A.nnz, rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
    ws = torch.empty(max(L.sym_spmv_workspace_bytes(C.byref(desc)), 256), dtype=torch.uint8, device="cuda")
    y = torch.empty(n, device="cuda")
    s = torch.empty(1, dtype=torch.float64, device="cuda")
    assert L.sym_spmv(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y.data_ptr()), C.c_void_p(s.data_ptr()),
                      C.c_void_p(ws.data_ptr()), ws.numel(), None) == 0
    torch.cuda.synchronize()
    yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    assert abs(float(s.item()) - sr) <= TOL_F32 * sa
    assert int(counter.item()) == 0
    assert L.sym_bounds_check_attach(None) == 0


def test_bounds_checked_counts_out_of_range_columns():
    """Columns at or past n in the one-launch form (skipped by every build) are counted by the checked build."""
    sg = need_gpu()
    L = bc_lib(sg)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert L.sym_bounds_check_attach(C.c_void_p(counter.data_ptr())) == 0
    n = 500
    A = synth.upper_csr_uniform(n, 3000, 72)
    col = A.col.copy()
    bad = np.arange(5, len(col), 97)[:20]
    col[bad] = n + 3                                  # 20 entries point past the matrix
    x = synth.vector_uniform(n, 73)
    rp, cl, vl, xd = dev(A.rowptr), dev(col), dev(A.val), dev(x)
    desc = Csr(n, A.nnz, rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
    assert L.sym_spmv_single_launch(C.byref(desc)) == 1
    y = torch.empty(n, device="cuda")
    assert L.sym_spmv(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y.data_ptr()), None, None, 0, None) == 0
    torch.cuda.synchronize()
    assert int(counter.item()) == len(bad)
    # the result is the product of the remaining entries
    keep = np.ones(len(col), bool)
    keep[bad] = False
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    rp2 = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=n))]).astype(np.int32)
    yr, ya = oracle.ssymv(n, rp2, A.col[keep], A.val[keep], x.astype(np.float64))
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    assert L.sym_bounds_check_attach(None) == 0
