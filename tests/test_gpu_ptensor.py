"""Partially symmetric tensors on the GPU (sym_ptensor_*, sym_pmttkrp) against the FP64 oracle.

Canonical entries, arrangement counts and duplicate handling must be bit-exact;
the MTTKRP for every part's factor must meet the componentwise tolerance
(FP32 1e-5; BF16 factors 1e-2 against the oracle on the FP32 factors and 1e-5
against the oracle on the BF16-rounded factors)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_BF16, TOL_F32, dev, host, need_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARTITIONS = [((2, 1), (5, 4)), ((1, 2), (4, 5)), ((2, 2), (4, 3)), ((3, 1), (4, 3)), ((1, 1, 1), (3, 4, 5)),
              ((2, 1, 2), (3, 2, 3)), ((1, 3), (3, 4)), ((5,), (4,)), ((2, 3), (3, 3))]


def factors(dims, rank, seed, bf16=False):
    F = [synth.factor_normal(d, rank, seed + p) for p, d in enumerate(dims)]
    if not bf16:
        return [dev(f) for f in F], [f.astype(np.float64) for f in F], None
    bits = [synth.bf16_rne(f) for f in F]
    Fd = [dev(b.view(np.int16)).view(torch.bfloat16) for b in bits]
    return Fd, [f.astype(np.float64) for f in F], [synth.bf16_to_f32(b).astype(np.float64) for b in bits]


@pytest.mark.parametrize("parts,dims", PARTITIONS)
def test_pcanonical_bit_exact_and_counts(parts, dims):
    sg = need_gpu()
    T = synth.ptensor_small_all_patterns(parts, dims, 3, density=0.7)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    gi, gv = X.export()
    assert np.array_equal(host(gi), cidx)
    assert np.array_equal(host(gv).view(np.uint32), cval.view(np.uint32))
    inf = X.info()
    cnt = oracle.pcounts(parts, cidx, cval)
    assert inf["nnz"] == cidx.shape[1] and inf["expanded_nnz"] == cnt["expanded"]
    assert abs(inf["normsq"] - cnt["normsq"]) <= 1e-12 * cnt["normsq"]


@pytest.mark.parametrize("parts,dims", PARTITIONS)
@pytest.mark.parametrize("rank", [4, 12, 32])
def test_pmttkrp_every_part_vs_oracle(parts, dims, rank):
    sg = need_gpu()
    T = synth.ptensor_small_all_patterns(parts, dims, 5, density=0.8)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    Fd, F64, _ = factors(dims, rank, 20)
    for out in range(len(parts)):
        M = X.mttkrp(Fd, out)
        torch.cuda.synchronize()
        ref, ref_abs = oracle.pmttkrp_enum(parts, dims, cidx, cval, F64, out)
        assert oracle.componentwise_error(host(M), ref, ref_abs) <= TOL_F32, out


@pytest.mark.parametrize("parts,dims,nnz", [((2, 2), (3000, 800), 200_000), ((2, 1), (20000, 300), 300_000),
                                            ((1, 3), (500, 2000), 150_000), ((2, 1, 2), (900, 40, 700), 100_000)])
@pytest.mark.parametrize("rank", [16, 64, 128])
def test_pmttkrp_larger_uniform(parts, dims, nnz, rank):
    sg = need_gpu()
    T = synth.ptensor_uniform(parts, dims, nnz, 7)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    gi, gv = X.export()
    assert np.array_equal(host(gi), cidx) and np.array_equal(host(gv), cval)
    Fd, F64, _ = factors(dims, rank, 30)
    for out in range(len(parts)):
        M = X.mttkrp(Fd, out)
        torch.cuda.synchronize()
        ref, ref_abs = oracle.pmttkrp_enum(parts, dims, cidx, cval, F64, out)
        assert oracle.componentwise_error(host(M), ref, ref_abs) <= TOL_F32, out


@pytest.mark.parametrize("parts,dims", [((2, 2), (300, 200)), ((3, 1), (120, 50))])
def test_pmttkrp_bf16_factors(parts, dims):
    sg = need_gpu()
    T = synth.ptensor_uniform(parts, dims, 40_000, 9)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    Fd, F64, F16 = factors(dims, 32, 40, bf16=True)
    for out in range(len(parts)):
        M = host(X.mttkrp(Fd, out))
        ref, ref_abs = oracle.pmttkrp_enum(parts, dims, cidx, cval, F64, out)
        assert oracle.componentwise_error(M, ref, ref_abs) <= TOL_BF16
        ref16, abs16 = oracle.pmttkrp_enum(parts, dims, cidx, cval, F16, out)
        assert oracle.componentwise_error(M, ref16, abs16) <= TOL_F32


@pytest.mark.parametrize("order,n", [(3, 40), (4, 25), (5, 12)])
def test_one_part_matches_symmetric_mttkrp(order, n):
    """A single part is full symmetry: the partial path and the symmetric MTTKRP agree."""
    sg = need_gpu()
    T = synth.tensor_small_all_patterns(order, n, 11, density=0.3)
    X = sg.PTensor(dev(T.idx), dev(T.val), (order,), (n,))
    Y = sg.SymTensor(dev(T.idx), dev(T.val), n)
    B = dev(synth.factor_normal(n, 16, 11))
    Mp = X.mttkrp([B], 0)
    Ms = Y.mttkrp(B)
    torch.cuda.synchronize()
    scale = float(Ms.abs().max())
    assert float((Mp - Ms).abs().max()) <= 1e-5 * scale
    assert X.info()["expanded_nnz"] == Y.info()["expanded_nnz"]


def test_ptensor_errors_and_empty():
    sg = need_gpu()
    parts, dims = (2, 1), (10, 3)
    idx = np.array([[1, 2], [4, 2], [0, 1]], np.int32)    # tuples (1,4,0) and (2,2,1)
    val = np.array([1.0, 2.0], np.float32)
    X = sg.PTensor(dev(idx), dev(val), parts, dims)
    assert X.nnz == 2 and X.info()["expanded_nnz"] == 2 + 1
    bad = idx.copy()
    bad[2, 0] = 3                                         # mode 3 belongs to the part of size 3
    with pytest.raises(sg.SymError) as ei:
        sg.PTensor(dev(bad), dev(val), parts, dims)
    assert ei.value.code == -3
    dup = np.array([[1, 4], [4, 1], [0, 0]], np.int32)   # one tuple twice, permuted inside part 0
    with pytest.raises(sg.SymError) as ei:
        sg.PTensor(dev(dup), dev(np.array([1.0, 1.0], np.float32)), parts, dims)
    assert ei.value.code == -4
    Xk = sg.PTensor(dev(dup), dev(np.array([1.0, 1.0], np.float32)), parts, dims, dup=sg.DUP_KEEP_EQUAL)
    assert Xk.nnz == 1 and Xk.info()["duplicates_dropped"] == 1
    with pytest.raises(sg.SymError):
        sg.PTensor(dev(dup), dev(np.array([1.0, 2.0], np.float32)), parts, dims, dup=sg.DUP_KEEP_EQUAL)
    across = np.array([[0], [4], [1]], np.int32)
    swapped = across[[2, 1, 0]]                           # permuting across parts is another tensor
    a = sg.PTensor(dev(across), dev(np.array([1.0], np.float32)), parts, dims).export()[0]
    b = sg.PTensor(dev(swapped), dev(np.array([1.0], np.float32)), (2, 1), (10, 3)).export()[0]
    assert not np.array_equal(host(a), host(b))
    E = sg.PTensor(torch.zeros((3, 0), dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"), parts, dims)
    assert E.nnz == 0
    Fd, _, _ = factors(dims, 8, 1)
    M = E.mttkrp(Fd, 0)
    assert float(M.abs().max()) == 0.0


@pytest.mark.parametrize("parts,dims", [((2, 1), (5, 4)), ((2, 2), (4, 3)), ((1, 3), (3, 4)), ((2, 1, 2), (3, 2, 3)),
                                        ((5,), (4,))])
def test_expand_baseline_matches_oracle(parts, dims):
    """The device expansion stores exactly the oracle's arrangements; the MTTKRP on it (no symmetry left)
    equals the symmetric one for every part."""
    sg = need_gpu()
    T = synth.ptensor_small_all_patterns(parts, dims, 6, density=0.7)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    E = X.expand()
    ei, ev = E.export()
    oi, ov = oracle.pexpand(parts, cidx, cval)
    assert np.array_equal(host(ei), oi) and np.array_equal(host(ev).view(np.uint32), ov.view(np.uint32))
    assert E.info()["expanded_nnz"] == X.info()["expanded_nnz"] == oi.shape[1]
    rank = 8
    Fd, F64, _ = factors(dims, rank, 50)
    per_mode = [Fd[p] for p, s in enumerate(parts) for _ in range(s)]
    first = np.cumsum([0] + list(parts))[:-1]
    for out in range(len(parts)):
        Ms = X.mttkrp(Fd, out)
        Me = E.mttkrp(per_mode, int(first[out]))
        torch.cuda.synchronize()
        ref, ref_abs = oracle.pmttkrp_enum(parts, dims, cidx, cval, F64, out)
        assert oracle.componentwise_error(host(Ms), ref, ref_abs) <= TOL_F32
        assert oracle.componentwise_error(host(Me), ref, ref_abs) <= TOL_F32


PARTITIONS3 = [((1, 2), (40, 50)), ((2, 1), (50, 40)), ((1, 1, 1), (30, 40, 50)), ((3,), (45,))]


@pytest.mark.parametrize("parts,dims", PARTITIONS3)
@pytest.mark.parametrize("rank", [4, 12, 32, 128])
@pytest.mark.parametrize("bf16", [False, True])
def test_pttm_matches_oracle(parts, dims, rank, bf16):
    """Mode-1 TTM of a partially symmetric order-3 tensor, full layout (and packed where modes 2, 3 share a
    part), every equality pattern inside every part, ragged entry counts."""
    sg = need_gpu()
    T = synth.ptensor_small_all_patterns(parts, dims, 11, density=0.15)
    X = sg.PTensor(dev(T.idx), dev(T.val), parts, dims)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    Fd, F64, Fb = factors(dims[:1], rank, 9, bf16)
    used = Fb[0] if bf16 else F64[0]
    want, wabs = oracle.pttm_enum(parts, dims, cidx, cval, used)
    got = host(X.ttm(Fd[0], "full")).reshape(want.shape)
    assert oracle.componentwise_error(got, want, wabs) <= TOL_F32
    if bf16:
        w32, a32 = oracle.pttm_enum(parts, dims, cidx, cval, F64[0])
        assert oracle.componentwise_error(got, w32, a32) <= TOL_BF16
    if parts in ((1, 2), (3,)):
        d = dims[-1]
        pk = host(X.ttm(Fd[0], "packed"))
        j, l = np.triu_indices(d)
        ref = want[j, l].reshape(-1)
        assert oracle.componentwise_error(pk, ref, wabs[j, l].reshape(-1)) <= TOL_F32
    else:
        with pytest.raises(sg.SymError):
            X.ttm(Fd[0], "packed")
    X.close()


def test_pttm_one_part_matches_symmetric_ttm():
    """One part of three modes is full symmetry: the same output as sym_ttm on the symmetric tensor."""
    sg = need_gpu()
    T = synth.tensor_uniform(3, 60, 4000, 12)
    Xp = sg.PTensor(dev(T.idx), dev(T.val), (3,), (60,))
    Xs = sg.SymTensor(dev(T.idx), dev(T.val), 60)
    B = dev(synth.factor_normal(60, 16, 12))
    a = host(Xp.ttm(B, "packed"))
    b = host(Xs.ttm(B, "packed"))
    cidx, cval = oracle.canonicalize(3, 60, T.idx, T.val)
    want, wabs = oracle.ttm_enum(3, 60, cidx, cval, synth.factor_normal(60, 16, 12).astype(np.float64))
    j, l = np.triu_indices(60)
    assert oracle.componentwise_error(a, want[j, l].reshape(-1), wabs[j, l].reshape(-1)) <= TOL_F32
    assert oracle.componentwise_error(b.reshape(-1), want[j, l].reshape(-1), wabs[j, l].reshape(-1)) <= TOL_F32
