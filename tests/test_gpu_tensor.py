"""GPU canonicalisation (sorting, dedupe, classification, counts) vs the oracle: bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import canonical_split, dev, host, need_gpu

pytestmark = pytest.mark.gpu

CASES = [
    (2, 50, 600, "uniform"), (3, 40, 3000, "uniform"), (3, 2000, 50000, "zipf"), (4, 30, 5000, "uniform"),
    (5, 12, 3000, "uniform"), (5, 200_000, 20000, "uniform"),  # 5 x 18 bits: two-word keys
    (4, 70_000, 20000, "uniform"),                             # 4 x 17 bits: two-word keys
]


@pytest.mark.parametrize("order,n,nnz,recipe", CASES)
def test_canonical_bitexact(order, n, nnz, recipe):
    sg = need_gpu()
    T = synth.tensor3_zipf(n, nnz, 3) if recipe == "zipf" else synth.tensor_uniform(order, n, nnz, 3)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    want_idx, want_val, n_strict = canonical_split(order, cidx, cval)
    gi, gv = X.export()
    assert np.array_equal(host(gi), want_idx)
    assert np.array_equal(host(gv).view(np.uint32), want_val.view(np.uint32))
    info = X.info()
    cnt = oracle.counts(order, cidx, cval)
    assert info["nnz"] == cval.shape[0] and info["nnz_strict"] == n_strict
    assert info["counts_by_pattern"] == cnt["by_pattern"].tolist()
    assert info["expanded_nnz"] == cnt["expanded"]
    assert info["root_fibers"] == cnt["root_fibers"]
    assert info["l2_fibers"] == cnt["l2_fibers"]
    assert abs(info["normsq"] - cnt["normsq"]) <= 1e-12 * cnt["normsq"]
    assert info["key_bits"] * order > 64 or n < 70_000


@pytest.mark.parametrize("order,n,nnz,recipe", [CASES[2], CASES[5]])
def test_canonical_from_pinned_host_coordinates(order, n, nnz, recipe):
    """The coordinate list (and the values) may stay in page-locked host memory (the coordinates read in place
    by the packing kernel, the values copied during the sort): the canonical form and the counts equal the
    oracle's bit for bit; pageable host memory is refused."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    T = synth.tensor3_zipf(n, nnz, 3) if recipe == "zipf" else synth.tensor_uniform(order, n, nnz, 3)
    idx_h = torch.from_numpy(np.ascontiguousarray(T.idx)).pin_memory()
    val_h = torch.from_numpy(np.ascontiguousarray(T.val)).pin_memory()
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    want_idx, want_val, n_strict = canonical_split(order, cidx, cval)
    # host coordinates with device values, then host coordinates and host values (copied during the sort)
    for X in (sg.SymTensor(idx_h, dev(T.val), n), sg.SymTensor(idx_h, val_h, n)):
        gi, gv = X.export()
        assert np.array_equal(host(gi), want_idx)
        assert np.array_equal(host(gv).view(np.uint32), want_val.view(np.uint32))
        info = X.info()
        assert info["nnz"] == cval.shape[0] and info["nnz_strict"] == n_strict
        assert info["expanded_nnz"] == oracle.counts(order, cidx, cval)["expanded"]
    # pageable host memory cannot be read by the device: refused before any launch
    C = sg.C
    idx_p = torch.from_numpy(np.ascontiguousarray(T.idx))
    ab, wb = C.c_size_t(0), C.c_size_t(0)
    assert sg.lib().sym_tensor_create_bytes(order, n, nnz, C.byref(ab), C.byref(wb)) == 0
    arena = torch.empty(ab.value, dtype=torch.uint8, device="cuda")
    ws = torch.empty(wb.value, dtype=torch.uint8, device="cuda")
    val_d = dev(T.val)
    out = C.c_void_p()
    rc = sg.lib().sym_tensor_create(order, n, nnz, C.c_void_p(idx_p.data_ptr()), nnz, C.c_void_p(val_d.data_ptr()),
                                    0, C.c_void_p(arena.data_ptr()), arena.numel(), C.c_void_p(ws.data_ptr()),
                                    ws.numel(), None, C.byref(out))
    assert rc == -1 and not out.value   # SYM_E_INVALID, no tensor


def test_ragged_tail_and_tiles():
    """Sizes around the radix-sort tile (2048) and scan tile (4096) boundaries."""
    sg = need_gpu()
    for nnz in (1, 2, 31, 2047, 2048, 2049, 4095, 4096, 4097, 10_001):
        T = synth.tensor_uniform(3, 60, nnz, nnz)
        X = sg.SymTensor(dev(T.idx), dev(T.val), 60)
        cidx, cval = oracle.canonicalize(3, 60, T.idx, T.val)
        wi, wv, _ = canonical_split(3, cidx, cval)
        gi, gv = X.export()
        assert np.array_equal(host(gi), wi), nnz
        assert np.array_equal(host(gv), wv), nnz


def test_empty_tensor():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    X = sg.SymTensor(torch.zeros((3, 0), dtype=torch.int32, device="cuda"),
                     torch.zeros(0, dtype=torch.float32, device="cuda"), 10)
    assert X.info()["nnz"] == 0
    B = torch.randn(10, 8, device="cuda")
    M = X.mttkrp(B)
    assert float(M.abs().max()) == 0.0


def test_duplicate_policies_and_range():
    sg = need_gpu()
    idx = np.array([[0, 2, 1, 3], [2, 0, 1, 3], [1, 1, 3, 3]], dtype=np.int32)  # (0,2,1)~(2,0,1)
    val = np.array([1.5, 1.5, 2.0, -1.0], np.float32)
    with pytest.raises(sg.SymError) as e:
        sg.SymTensor(dev(idx), dev(val), 4, dup=sg.DUP_ERROR)
    assert e.value.code == -4
    X = sg.SymTensor(dev(idx), dev(val), 4, dup=sg.DUP_KEEP_EQUAL)
    c, v = oracle.canonicalize(3, 4, idx, val, dup_policy=1)
    wi, wv, _ = canonical_split(3, c, v)
    gi, gv = X.export()
    assert np.array_equal(host(gi), wi) and np.array_equal(host(gv), wv)
    assert X.info()["duplicates_dropped"] == 1
    val2 = val.copy()
    val2[1] = -1.5
    with pytest.raises(sg.SymError):
        sg.SymTensor(dev(idx), dev(val2), 4, dup=sg.DUP_KEEP_EQUAL)
    with pytest.raises(sg.SymError) as e:
        sg.SymTensor(dev(idx), dev(val), 3, dup=sg.DUP_KEEP_EQUAL)
    assert e.value.code == -3


def test_device_generator_matches_host_definition():
    sg = need_gpu()
    for order, n, count, seed in [(3, 1000, 5000, 7), (5, 200_000, 3000, 11), (4, 20, 999, 3)]:
        gi, gv = sg.gen_coords(order, n, count, seed)
        hi, hv = synth.coord_pool(order, n, count, seed)
        assert np.array_equal(host(gi), hi)
        assert np.array_equal(host(gv).view(np.uint32), hv.view(np.uint32))


def test_generated_pool_keep_equal_dedupes():
    sg = need_gpu()
    gi, gv = sg.gen_coords(3, 40, 20000, 5)   # many repeated multisets, equal values
    X = sg.SymTensor(gi, gv, 40, dup=sg.DUP_KEEP_EQUAL)
    hi, hv = synth.coord_pool(3, 40, 20000, 5)
    c, v = oracle.canonicalize(3, 40, hi, hv, dup_policy=1)
    wi, wv, _ = canonical_split(3, c, v)
    ei, ev = X.export()
    assert np.array_equal(host(ei), wi) and np.array_equal(host(ev), wv)
