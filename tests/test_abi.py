"""The C-ABI library loads and exports every entry point include/symgpu.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "symgpu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sym_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_09266_gb300 import build
    return build.build()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("sym_spmv", "sym_mttkrp", "sym_batch_submit", "sym_batch_poll", "sym_tensor_create"):
        assert core in names
    assert len(names) >= 40


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wires_every_declared_symbol(libpath):
    import paper_2406_09266_gb300 as sg
    assert sorted(declared_functions()) == sg.exported_symbols()
    sg.load(libpath)


def test_host_side_calls_without_gpu(libpath):
    """Calls that touch no device: status strings and size queries."""
    import paper_2406_09266_gb300 as sg
    L = sg.load(libpath)
    assert L.sym_status_string(-4) == b"duplicate entry"
    assert L.sym_version() == 1
    ab, wb = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert L.sym_tensor_create_bytes(3, 100_000, 20_000_000, ctypes.byref(ab), ctypes.byref(wb)) == 0
    assert ab.value >= 20_000_000 * 12 and wb.value > ab.value
    assert L.sym_tensor_create_bytes(6, 10, 10, ctypes.byref(ab), ctypes.byref(wb)) == -1
    assert L.sym_tensor_create_bytes(5, 1 << 30, 10, ctypes.byref(ab), ctypes.byref(wb)) == -10
    assert L.sym_mttkrp(None, None, 0, 64, 64, None, 64, None, None, 0, None) == -1


def test_spmv_path_choice(libpath):
    """The one-launch cluster form is chosen on the host from n and nnz alone:
    n <= 8192 and x, a partial y, rowptr, 1/8 of the entries and the exchange
    inbox within 160 KiB."""
    import paper_2406_09266_gb300 as sg
    sg.load(libpath)

    def smem(n, nnz):
        r4 = lambda v: (v + 3) // 4 * 4
        S = r4((n + 7) // 8)
        return 4 * (r4(n) + 8 * S + r4(n + 1) + 2 * r4((nnz + 7) // 8) + 7 * S + 32 + 32 + 4)

    assert sg.spmv_single_launch(2000, 20000)
    assert sg.spmv_single_launch(1, 0) and sg.spmv_single_launch(1, 1)
    assert not sg.spmv_single_launch(0, 0)
    assert not sg.spmv_single_launch(8193, 10)
    assert not sg.spmv_single_launch(5000, 160000)
    for n in (1, 64, 257, 2000, 4096, 8192):
        lo, hi = 0, 1 << 22
        while lo < hi:  # largest nnz the library accepts
            mid = (lo + hi + 1) // 2
            if sg.spmv_single_launch(n, mid):
                lo = mid
            else:
                hi = mid - 1
        assert 0 < lo and smem(n, lo) <= 160 * 1024 < smem(n, lo + 1), (n, lo)


def test_missing_library_fails_loudly(tmp_path):
    import paper_2406_09266_gb300 as sg
    with pytest.raises(RuntimeError):
        sg.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(sg.load, "__wrapped__") else \
            _fresh_load(sg, str(tmp_path / "nope.so"))


def _fresh_load(sg, path):
    saved = sg._lib
    sg._lib = None
    try:
        sg.load(path)
    finally:
        sg._lib = saved
