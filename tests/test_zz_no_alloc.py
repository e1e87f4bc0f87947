"""The allocation-free SSYMV + SYPRD entry point (sym_spmv_noalloc) against sym_spmv.

sym_spmv_noalloc serves callers that cannot give the library device memory
(a host pool allocator that owns the whole device, code that must keep running
once memory is exhausted, loops that must not call cudaMalloc).  Its SYPRD
partials live in a fixed array inside the library that every call shares, so
this test calls it twice in a row and compares both results with sym_spmv,
called through the C ABI with ctypes.  This file is collected last on purpose.
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


@pytest.mark.gpu
def test_noalloc_matches_spmv_twice():
    torch, L = _lib()
    dev = torch.device("cuda")
    for n, nnz, seed in [(2000, 20000, 0), (50_000, 600_000, 1)]:
        A = synth.upper_csr_uniform(n, nnz, seed)
        x = synth.vector_uniform(n, seed)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        rp, cl, vl, xd = t(A.rowptr), t(A.col), t(A.val), t(x)
        desc = Csr(n, nnz, rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
        # existing entry point, with its workspace
        ws = torch.empty(max(L.sym_spmv_workspace_bytes(C.byref(desc)), 256), dtype=torch.uint8, device=dev)
        y_ref = torch.empty(n, device=dev)
        s_ref = torch.empty(1, dtype=torch.float64, device=dev)
        assert L.sym_spmv(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y_ref.data_ptr()),
                          C.c_void_p(s_ref.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), None) == 0
        torch.cuda.synchronize()
        _, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x.astype(np.float64))
        _, sa = oracle.syprd(n, A.rowptr, A.col, A.val, x.astype(np.float64))
        for _call in range(2):   # the second call starts from the first call's leftovers
            y = torch.full((n,), 7.0, device=dev)
            s = torch.full((1,), 7.0, dtype=torch.float64, device=dev)
            rc = L.sym_spmv_noalloc(C.byref(desc), C.c_void_p(xd.data_ptr()), C.c_void_p(y.data_ptr()),
                                    C.c_void_p(s.data_ptr()), None)
            assert rc == 0
            torch.cuda.synchronize()
            yh, yr = y.cpu().numpy().astype(np.float64), y_ref.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(yh - yr) / np.maximum(ya, 1e-30)) <= TOL
            assert abs(float(s.item()) - float(s_ref.item())) <= TOL * sa


@pytest.mark.gpu
def test_noalloc_rejects_oversize_without_touching_the_device():
    torch, L = _lib()
    n = 262_145   # one row past the stated maximum
    y = torch.empty(1, device="cuda")
    p = y.data_ptr()
    desc = Csr(n, 0, p, p, p)     # valid pointers, never read: the size check comes first
    rc = L.sym_spmv_noalloc(C.byref(desc), C.c_void_p(y.data_ptr()), C.c_void_p(y.data_ptr()), None, None)
    assert rc == -10   # SYM_E_UNSUPPORTED
