"""Symmetric mode-1 TTM (order 3, visible output symmetry) on the GPU vs the FP64 oracle.

The oracle computes the full output C[j, l, :] by enumerating the distinct
permutations of every canonical entry; the packed GPU output is compared with
its canonical triangle j <= l, the full GPU output (canonical triangle plus the
replication pass) with all of it.  Componentwise error, gates as for MTTKRP.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_BF16, TOL_F32, dev, factor, host, need_gpu

pytestmark = pytest.mark.gpu


def packed_of(full):
    """Canonical triangle j <= l of an (n, n, R) array in the packed order."""
    n = full.shape[0]
    j, l = np.triu_indices(n)
    return full[j, l]


def check(C, ref, ra, tol):
    e = oracle.componentwise_error(C, ref, ra)
    assert e <= tol, e
    return e


CASES = [
    # n, nnz, rank, recipe
    (40, 3000, 4, "uniform"),      # many diagonal entries, ragged last warp
    (64, 9000, 16, "uniform"),
    (257, 20000, 32, "uniform"),   # n not a power of two
    (300, 30000, 64, "uniform"),
    (90, 12000, 128, "uniform"),
    (120, 5000, 12, "uniform"),    # rank not a power of two
    (9, 0, 8, "patterns"),         # every equality pattern, tiny
]


def make(n, nnz, recipe, seed):
    if recipe == "patterns":
        return synth.tensor_small_all_patterns(3, n, seed, density=0.6)
    return synth.tensor_uniform(3, n, nnz, seed)


@pytest.mark.parametrize("n,nnz,rank,recipe", CASES)
@pytest.mark.parametrize("bf16", [False, True])
def test_ttm_packed_and_full(n, nnz, rank, recipe, bf16):
    sg = need_gpu()
    T = make(n, nnz, recipe, 11 + rank)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    Bt, B32, Bused = factor(n, rank, 5, bf16)
    cidx, cval = oracle.canonicalize(3, n, T.idx, T.val)
    ref, ra = oracle.ttm_enum(3, n, cidx, cval, B32.astype(np.float64))
    Cp = host(X.ttm(Bt, "packed"))
    Cf = host(X.ttm(Bt, "full"))
    assert Cp.shape == (n * (n + 1) // 2, rank) and Cf.shape == (n, n, rank)
    # the replication pass copies exactly: the full output is symmetric bit for bit
    assert np.array_equal(Cf, Cf.transpose(1, 0, 2))
    if bf16:
        check(Cp, packed_of(ref), packed_of(ra), TOL_BF16)
        check(Cf, ref, ra, TOL_BF16)
        refb, rab = oracle.ttm_enum(3, n, cidx, cval, Bused.astype(np.float64))
        check(Cp, packed_of(refb), packed_of(rab), TOL_F32)
        check(Cf, refb, rab, TOL_F32)
    else:
        check(Cp, packed_of(ref), packed_of(ra), TOL_F32)
        check(Cf, ref, ra, TOL_F32)


def test_ttm_single_entries_every_pattern():
    """One stored entry per call: B = I makes every update land in its own cell, so the GPU's
    nonzero cells must be exactly the oracle's (3 / 2 / 2 / 1 canonical updates)."""
    sg = need_gpu()
    n = 8
    B = np.zeros((n, 8), np.float32)
    B[np.arange(n), np.arange(n)] = 1.0
    for tup in [(1, 3, 5), (2, 2, 6), (0, 4, 4), (3, 3, 3), (7, 0, 2)]:
        idx = np.array(tup, np.int32).reshape(3, 1)
        X = sg.SymTensor(dev(idx), dev(np.array([1.5], np.float32)), n)
        Cf = host(X.ttm(dev(B), "full"))
        cidx, cval = oracle.canonicalize(3, n, idx, np.array([1.5], np.float32))
        ref = oracle.ttm_enum(3, n, cidx, cval, B.astype(np.float64), want_abs=False)
        assert np.array_equal(Cf, ref.astype(np.float32)), tup
        nz = np.count_nonzero(packed_of(Cf))
        assert nz == len(set(tup)), (tup, nz)


def test_ttm_empty_tensor_and_errors():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    X = sg.SymTensor(torch.zeros((3, 0), dtype=torch.int32, device="cuda"),
                     torch.zeros(0, dtype=torch.float32, device="cuda"), 50)
    B = dev(synth.factor_normal(50, 16, 1))
    C = X.ttm(B, "full", C_out=torch.full((50, 50, 16), 7.0, device="cuda"))
    assert float(C.abs().max()) == 0.0
    # order 4 is not a TTM of this form
    T4 = synth.tensor_uniform(4, 20, 100, 1)
    X4 = sg.SymTensor(dev(T4.idx), dev(T4.val), 20)
    with pytest.raises(sg.SymError) as ei:
        X4.ttm(dev(synth.factor_normal(20, 8, 1)))
    assert ei.value.code == -10
    with pytest.raises(sg.SymError):
        X.ttm(dev(synth.factor_normal(50, 6, 1)))      # rank not a multiple of 4


@pytest.mark.parametrize("bf16", [False, True])
def test_ttm_expanded_baseline(bf16):
    sg = need_gpu()
    n, rank = 70, 16
    T = synth.tensor_uniform(3, n, 6000, 21)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    Bt, B32, Bused = factor(n, rank, 6, bf16)
    E = X.expanded()
    Ce = host(E.ttm(Bt))
    cidx, cval = oracle.canonicalize(3, n, T.idx, T.val)
    ref, ra = oracle.ttm_enum(3, n, cidx, cval, Bused.astype(np.float64))
    check(Ce, ref, ra, TOL_F32)
    # the symmetric kernel and the baseline agree
    Cf = host(X.ttm(Bt, "full"))
    check(Cf, ref, ra, TOL_F32)


@pytest.mark.slow
def test_ttm_fullsize_sampled_rows():
    """The benchmark's TTM workload (n = 2,000, 5M canonical entries, R = 32), sampled output rows."""
    sg = need_gpu()
    n, nnz, rank = 2000, 5_000_000, 32
    T = synth.make_tensor(3, n, nnz, 3, "uniform")
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    Bt, B32, _ = factor(n, rank, 3)
    cidx, cval = oracle.canonicalize(3, n, T.idx, T.val)
    st = synth.Stream(3, tag=9)
    rows = np.unique(np.concatenate([[0, 1, n - 1], st.randint(13, n)]))
    ref, ra = oracle.ttm_enum(3, n, cidx, cval, B32.astype(np.float64), rows=rows)
    Cf = host(X.ttm(Bt, "full"))[rows]
    check(Cf, ref, ra, TOL_F32)
    Cp = X.ttm(Bt, "packed")
    # packed rows: positions (j, l >= j) of row j start at j n - j (j - 1) / 2
    Cp = host(Cp)
    for s, j in enumerate(rows):
        p0 = j * n - j * (j - 1) // 2
        check(Cp[p0:p0 + n - j], ref[s, j:], ra[s, j:], TOL_F32)


TTM_CFGS = [
    dict(entries_per_warp=32),
    dict(ctas_per_sm=2, entries_per_warp=64),
    dict(leaf_index=1),
    dict(leaf_index=1, ctas_per_sm=1, entries_per_warp=32),
    dict(leaf_index=0, ctas_per_sm=8, entries_per_warp=96),
]


@pytest.mark.parametrize("cfg", TTM_CFGS, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
@pytest.mark.parametrize("n,nnz,rank,bf16", [(257, 20000, 32, False), (64, 9000, 16, True), (30, 2500, 128, False)])
def test_ttm_schedules(cfg, n, nnz, rank, bf16):
    """Every schedule (chunk size, persistent grid, leaf-index second pass) gives the oracle's result."""
    sg = need_gpu()
    T = synth.tensor_uniform(3, n, nnz, 31 + n)
    X = sg.SymTensor(dev(T.idx), dev(T.val), n)
    if cfg.get("leaf_index", -1) == 1:
        X.add_leaf_index()
    Bt, B32, Bused = factor(n, rank, 7, bf16)
    cidx, cval = oracle.canonicalize(3, n, T.idx, T.val)
    ref, ra = oracle.ttm_enum(3, n, cidx, cval, Bused.astype(np.float64))
    check(host(X.ttm(Bt, "packed", cfg=cfg)), packed_of(ref), packed_of(ra), TOL_F32)
    check(host(X.ttm(Bt, "full", cfg=cfg)), ref, ra, TOL_F32)


def test_ttm_leaf_index_required_but_absent():
    sg = need_gpu()
    T = synth.tensor_uniform(3, 20, 300, 2)
    X = sg.SymTensor(dev(T.idx), dev(T.val), 20)
    with pytest.raises(sg.SymError):
        X.ttm(dev(synth.factor_normal(20, 8, 1)), cfg=dict(leaf_index=1))
