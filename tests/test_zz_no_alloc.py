"""The allocation-free SSYMV + SYPRD entry point (sym_spmv_noalloc).

sym_spmv_noalloc serves callers that cannot give the library device memory
(a host pool allocator that owns the whole device, code that must keep running
once memory is exhausted, loops that must not call cudaMalloc because it can
synchronise the device).  Its SYPRD partials live in a fixed array inside the
library that every call shares, so each case calls it twice in a row (the
second call starts from the first call's leftovers) and checks both results
against the FP64 oracle and against sym_spmv, all through the C ABI with
ctypes.  One case fills every slot of the array (n = 262,144 rows, about 17
upper entries per row).  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

TOL = 1e-5   # componentwise tolerance of the FP32 tests


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09266_gb300 import build
    L = C.CDLL(build.build())
    L.sym_spmv.argtypes = [C.c_void_p] * 5 + [C.c_size_t, C.c_void_p]
    L.sym_spmv_workspace_bytes.argtypes = [C.c_void_p]
    L.sym_spmv_workspace_bytes.restype = C.c_size_t
    L.sym_spmv_noalloc.argtypes = [C.c_void_p] * 5
    return torch, L


def _cases():
    yield "n2000_cluster_form", synth.upper_csr_uniform(2000, 20000, 0)
    yield "n50k_multiblock", synth.upper_csr_uniform(50_000, 600_000, 1)
    # every one of the 32,768 partial slots written and read: 8 rows per slot at >16 entries per row
    yield "n262144_every_slot", synth.upper_csr_rowdegree(262_144, 17.5, 2)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["n2000_cluster_form", "n50k_multiblock", "n262144_every_slot"])
def test_noalloc_matches_oracle_and_spmv_twice(name):
    torch, L = _lib()
    dev = torch.device("cuda")
    A = dict(_cases())[name]
    n, nnz = int(A.n), int(A.nnz)
    x = synth.vector_uniform(n, 3)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, cl, vl, xd = t(A.rowptr), t(A.col), t(A.val), t(x)
    desc = Csr(n, nnz, rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
    if name == "n262144_every_slot":
        assert L.sym_spmv_workspace_bytes(C.byref(desc)) == 32768 * 8   # the array's full size
    yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    sr, sa = oracle.syprd(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    # the existing entry point, with its workspace
    ws = torch.empty(max(L.sym_spmv_workspace_bytes(C.byref(desc)), 256), dtype=torch.uint8, device=dev)
    y_ref = torch.empty(n, device=dev)
    s_ref = torch.empty(1, dtype=torch.float64, device=dev)
    assert L.sym_spmv(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y_ref.data_ptr()),
                      C.c_void_p(s_ref.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), None) == 0
    torch.cuda.synchronize()
    y_ref_h = y_ref.cpu().numpy()
    for _call in range(2):   # the second call starts from the first call's leftovers
        y = torch.full((n,), 7.0, device=dev)
        s = torch.full((1,), 7.0, dtype=torch.float64, device=dev)
        rc = L.sym_spmv_noalloc(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y.data_ptr()),
                                C.c_void_p(s.data_ptr()), None)
        assert rc == 0
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        assert oracle.componentwise_error(yh, yr, ya) <= TOL
        assert abs(float(s.item()) - sr) <= TOL * sa
        # and the same results as sym_spmv, within the same tolerance
        assert oracle.componentwise_error(yh, y_ref_h.astype(np.float64), ya) <= TOL
        assert abs(float(s.item()) - float(s_ref.item())) <= TOL * sa


@pytest.mark.gpu
def test_noalloc_y_only_has_no_size_limit():
    torch, L = _lib()
    dev = torch.device("cuda")
    A = synth.upper_csr_rowdegree(300_000, 17.5, 4)   # 37,500 slots: more than the array holds
    n, nnz = int(A.n), int(A.nnz)
    x = synth.vector_uniform(n, 5)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, cl, vl, xd = t(A.rowptr), t(A.col), t(A.val), t(x)
    desc = Csr(n, nnz, rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
    y = torch.full((n,), 7.0, device=dev)
    assert L.sym_spmv_noalloc(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y.data_ptr()), None, None) == 0
    torch.cuda.synchronize()
    yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
    assert oracle.componentwise_error(y.cpu().numpy(), yr, ya) <= TOL


@pytest.mark.gpu
def test_noalloc_rejects_oversize_syprd_without_touching_the_device():
    torch, L = _lib()
    n = 262_152            # 32,769 slots at more than 16 entries per row: one past the array
    y = torch.empty(1, dtype=torch.float64, device="cuda")
    p = y.data_ptr()
    desc = Csr(n, 17 * n, p, p, p)     # valid pointers, never read: the size check comes first
    rc = L.sym_spmv_noalloc(C.byref(desc), C.c_void_p(p), C.c_void_p(p), C.c_void_p(p), None)
    assert rc == -10   # SYM_E_UNSUPPORTED
