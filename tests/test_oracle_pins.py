"""Pins for the FP64 oracle: what the paper and plain mathematics fix, independent of the oracle.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/), closed forms, dense brute force on tiny tensors
(the canonical triangle expanded over all N! position permutations, then a
dense contraction), invariants, and textbook special cases.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- brute force

def dense_full(order, n, cidx, cval):
    """Full symmetric dense tensor: every position permutation of every stored tuple."""
    X = np.zeros((n,) * order, dtype=np.float64)
    for e in range(cidx.shape[1]):
        c = tuple(int(x) for x in cidx[:, e])
        for p in itertools.permutations(range(order)):
            X[tuple(c[q] for q in p)] = float(cval[e])
    return X


def dense_mttkrp(X, B):
    order = X.ndim
    n, R = B.shape
    M = np.zeros((n, R))
    for r in range(R):
        T = X
        for _ in range(order - 1):
            T = T @ B[:, r]
        M[:, r] = T
    return M


def dense_mttkrp_abs(X, B):
    return dense_mttkrp(np.abs(X), np.abs(B))


def canon(T):
    return oracle.canonicalize(T.order, T.n, T.idx, T.val)


# ----------------------------------------------------------------------------- multiplicities

def compositions(order):
    """All run-length structures (m_1..m_d) of a canonical tuple of the given order."""
    for d in range(1, order + 1):
        for cut in itertools.combinations(range(1, order), d - 1):
            b = (0,) + cut + (order,)
            yield tuple(b[t + 1] - b[t] for t in range(d))


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_distinct_perms_closed_form_and_bruteforce(order):
    for ms in compositions(order):
        tup = []
        for t, m in enumerate(ms):
            tup += [10 * t + 3] * m
        closed = math.factorial(order) // math.prod(math.factorial(m) for m in ms)
        brute = len(set(itertools.permutations(tup)))
        assert oracle.distinct_perms(np.array(tup)) == closed == brute


def test_paper_3way_unique_symmetry_groups():
    g = golden("paper_mttkrp3_multiplicities.json")
    cases = {"i<k<l": [0, 1, 2], "i=k<l": [0, 0, 2], "i<k=l": [0, 2, 2], "i=k=l": [1, 1, 1]}
    for name, tup in cases.items():
        assert oracle.distinct_perms(np.array(tup)) == g["unique_symmetry_groups"][name]
    # The listed members of S_P|E for i=k<l, applied to (i, k, l), are the distinct arrangements.
    i, k, l = 0, 0, 2
    got = {tuple((i, k, l)[s - 1] for s in sig) for sig in g["unique_symmetry_group_members_i=k<l"]}
    assert got == set(itertools.permutations((i, k, l)))


def _one_entry_counts(tup, form):
    """Row sums of the oracle's MTTKRP for a single entry with v=1 and B=1 (update counts)."""
    order = len(tup)
    n = 16
    cidx = np.array(tup, dtype=np.int32).reshape(order, 1)
    cval = np.ones(1, dtype=np.float32)
    B = np.ones((n, 1))
    if form == "enum":
        M = oracle.mttkrp_enum(order, n, cidx, cval, B, want_abs=False)
    else:
        M = oracle.mttkrp_runs(order, n, cidx, cval, B)
    return M[:, 0]


@pytest.mark.parametrize("form", ["enum", "runs"])
def test_paper_normalized_update_counts(form):
    g = golden("paper_mttkrp3_multiplicities.json")["normalized_update_counts"]
    i, k, l = 1, 4, 7
    cases = {"i<k<l": (i, k, l), "i=k<l": (i, i, l), "i<k=l": (i, k, k), "i=k=l": (i, i, i)}
    for name, tup in cases.items():
        M = _one_entry_counts(tup, form)
        names = {"i": tup[0], "k": tup[1], "l": tup[2]}
        want = np.zeros_like(M)
        for lab, cnt in g[name].items():
            want[names[lab]] = cnt
        assert np.array_equal(M, want), name


@pytest.mark.parametrize("form", ["enum", "runs"])
def test_paper_lookup_table(form):
    g = golden("paper_mttkrp3_multiplicities.json")
    lut = g["lookup_table"]
    for tup in [(1, 4, 7), (1, 1, 7), (1, 4, 4), (1, 1, 1)]:
        i, k, l = tup
        # printed index, with the all-equal case read as entry 7 (see the fixture)
        idx = 2 * (i == k) + 3 * (k == l) + 1 + (i == k and k == l)
        name = {1: "i<k<l", 3: "i=k<l", 4: "i<k=l", 7: "i=k=l"}[idx]
        assert g["lookup_index_used"][name] == idx
        factor = lut[idx - 1]
        # The table factor applies once per position; positions sharing a row add up.
        want = np.zeros(16)
        for pos in tup:
            want[pos] += factor
        M = _one_entry_counts(tup, form)
        assert np.allclose(M, want, rtol=0, atol=1e-15), tup


def test_paper_split_loop_weights():
    g = golden("paper_mttkrp3_multiplicities.json")["split_loop_weights"]
    assert np.array_equal(_one_entry_counts((0, 3, 5), "runs")[[0, 3, 5]],
                          [g["strict_weight_per_position"]] * 3)
    m = _one_entry_counts((2, 2, 5), "runs")
    assert m[2] == 2 * g["mixed_diagonal_weight_per_position"] and m[5] == 1
    assert _one_entry_counts((4, 4, 4), "runs")[4] == g["all_equal_updates"]


def test_paper_savings_ratios():
    """Sec. 5.2.6: reads shrink by N!, operations by (N-1)! for the 3/4/5-way MTTKRP."""
    g = golden("paper_mttkrp3_multiplicities.json")["savings_Sec_5_2_6"]
    for order in (3, 4, 5):
        strict = np.arange(order, dtype=np.int32) * 3 + 1
        assert oracle.distinct_perms(strict) == g[str(order)]["reads"]
        # Updates per canonical read equal N! (one per permutation), grouped into N rows.
        M = _one_entry_counts(tuple(strict), "enum")
        assert M.sum() == g[str(order)]["reads"]
        assert set(M[strict]) == {g[str(order)]["ops"]}


def test_paper_ssymv_syprd_assignments():
    g = golden("paper_ssymv_syprd.json")
    rowptr = np.array([0, 2, 2, 2], np.int32)
    col = np.array([0, 2], np.int32)
    val = np.array([1.0, 1.0], np.float32)
    y, _ = oracle.ssymv(3, rowptr, col, val, np.ones(3))
    # (0,0) diagonal: one assignment to y[0]; (0,2): one to y[0], one to y[2].
    assert y.tolist() == [g["ssymv_assignments"]["i=j"] + 1, 0.0, 1.0]
    s, _ = oracle.syprd(3, rowptr, col, val, np.ones(3))
    assert s == g["syprd_factor"]["i=j"] + g["syprd_factor"]["i<j"]


# ----------------------------------------------------------------------------- brute force vs oracle

@pytest.mark.parametrize("order,n", [(2, 6), (3, 6), (4, 5), (5, 4)])
@pytest.mark.parametrize("seed", [0, 1])
def test_mttkrp_vs_dense_bruteforce(order, n, seed):
    T = synth.tensor_small_all_patterns(order, n, seed)
    cidx, cval = canon(T)
    B = synth.factor_normal(n, 5, seed).astype(np.float64)
    X = dense_full(order, n, cidx, cval)
    want = dense_mttkrp(X, B)
    M, Ma = oracle.mttkrp_enum(order, n, cidx, cval, B)
    Mr = oracle.mttkrp_runs(order, n, cidx, cval, B)
    assert np.allclose(M, want, rtol=1e-12, atol=1e-12)
    assert np.allclose(Mr, want, rtol=1e-12, atol=1e-12)
    assert np.allclose(Ma, dense_mttkrp_abs(X, B), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("order,n", [(3, 6), (4, 5), (5, 4)])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_mttkrp_threads_vs_dense_bruteforce(order, n, threads):
    """The multi-threaded timing form equals the dense brute force (and so the definitional form)."""
    T = synth.tensor_small_all_patterns(order, n, 5)
    cidx, cval = canon(T)
    B = synth.factor_normal(n, 5, 5).astype(np.float64)
    want = dense_mttkrp(dense_full(order, n, cidx, cval), B)
    Mt = oracle.mttkrp_enum_threads(order, n, cidx, cval, B, threads)
    assert np.allclose(Mt, want, rtol=1e-12, atol=1e-12)


def test_mttkrp_row_mask_matches_full():
    T = synth.tensor_small_all_patterns(4, 6, 3)
    cidx, cval = canon(T)
    B = synth.factor_normal(6, 4, 3).astype(np.float64)
    M, _ = oracle.mttkrp_enum(4, 6, cidx, cval, B)
    rows = [0, 3, 5]
    Ms, _ = oracle.mttkrp_enum(4, 6, cidx, cval, B, rows=rows)
    assert np.array_equal(Ms[rows], M[rows])
    assert not Ms[[1, 2, 4]].any()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ssymv_syprd_vs_dense(seed):
    A = synth.upper_csr_uniform(40, 300, seed)
    x = synth.vector_uniform(40, seed).astype(np.float64)
    D = np.zeros((40, 40))
    rows = np.repeat(np.arange(40), np.diff(A.rowptr))
    D[rows, A.col] = A.val
    full = D + D.T - np.diag(np.diag(D))     # textbook (U + U^T - diag U)
    y, ya = oracle.ssymv(40, A.rowptr, A.col, A.val, x)
    assert np.allclose(y, full @ x, rtol=1e-13, atol=1e-13)
    assert np.allclose(ya, np.abs(full) @ np.abs(x), rtol=1e-13, atol=1e-13)
    s, sa = oracle.syprd(40, A.rowptr, A.col, A.val, x)
    assert np.isclose(s, x @ full @ x, rtol=1e-12, atol=1e-12)
    # invariant: x^T (A x) = SYPRD
    assert np.isclose(x @ y, s, rtol=1e-12, atol=1e-12)


def test_bellman_vs_dense():
    A = synth.upper_csr_uniform(30, 120, 5)
    d = synth.vector_uniform(30, 5).astype(np.float64) + 2.0
    val = np.abs(A.val)
    D = np.full((30, 30), np.inf)
    rows = np.repeat(np.arange(30), np.diff(A.rowptr))
    D[rows, A.col] = val
    D[A.col, rows] = val
    want = np.minimum(d, (D + d[None, :]).min(axis=1))
    got = oracle.bellman(30, A.rowptr, A.col, val, d)
    assert np.allclose(got, want, rtol=0, atol=1e-6)


@pytest.mark.parametrize("order,n", [(3, 5), (4, 4), (5, 3)])
def test_cpfit_vs_dense(order, n):
    T = synth.tensor_small_all_patterns(order, n, 7)
    cidx, cval = canon(T)
    B = synth.factor_normal(n, 3, 7).astype(np.float64)
    X = dense_full(order, n, cidx, cval)
    Mcp = np.zeros_like(X)
    for r in range(B.shape[1]):
        t = B[:, r]
        for _ in range(order - 1):
            t = np.multiply.outer(t, B[:, r])
        Mcp += t
    want = float(((X - Mcp) ** 2).sum())
    res, ab, parts = oracle.cpfit(order, n, cidx, cval, B)
    assert np.isclose(res, want, rtol=1e-11, atol=1e-11)
    assert np.isclose(parts[0], (X ** 2).sum(), rtol=1e-12)
    assert ab >= abs(res)


# ----------------------------------------------------------------------------- canonical form / counts

def test_canonicalize_properties():
    T = synth.tensor_uniform(4, 30, 3000, 9)
    cidx, cval = canon(T)
    assert cidx.shape == (4, 3000)
    assert oracle.check_canonical(4, 30, cidx) == oracle.OK
    # same multisets as the input (independent check with numpy sorting)
    a = np.sort(T.idx.T, axis=1)
    o = np.lexsort(a.T[::-1])
    assert np.array_equal(a[o].T, cidx)
    assert np.array_equal(T.val[o], cval)


def test_canonicalize_input_permutation_invariance():
    T = synth.tensor_uniform(5, 12, 800, 4)
    c1, v1 = canon(T)
    st = synth.Stream(99)
    perm = np.argsort(st.uniform(5 * 800).reshape(800, 5), axis=1)
    idx2 = np.take_along_axis(T.idx.T, perm, axis=1).T
    shuf = np.argsort(st.u64(800))
    c2, v2 = oracle.canonicalize(5, 12, idx2[:, shuf], T.val[shuf])
    assert np.array_equal(c1, c2) and np.array_equal(v1, v2)


def test_canonicalize_duplicates_and_range():
    idx = np.array([[0, 2, 1], [2, 0, 1], [1, 1, 3]], dtype=np.int32)  # (0,2,1) and (2,0,1) same multiset
    val = np.array([1.5, 1.5, 2.0], np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.canonicalize(3, 4, idx, val, dup_policy=0)
    assert e.value.code == oracle.DUPLICATE
    c, v = oracle.canonicalize(3, 4, idx, val, dup_policy=1)
    assert c.T.tolist() == [[0, 1, 2], [1, 1, 3]] and v.tolist() == [1.5, 2.0]
    val2 = np.array([1.5, -1.5, 2.0], np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.canonicalize(3, 4, idx, val2, dup_policy=1)
    with pytest.raises(oracle.OracleError) as e:
        oracle.canonicalize(3, 3, idx, val, dup_policy=1)
    assert e.value.code == oracle.RANGE


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_counts_closed_forms(order):
    T = synth.tensor_small_all_patterns(order, 7, 11, density=0.7)
    cidx, cval = canon(T)
    cnt = oracle.counts(order, cidx, cval)
    rows = cidx.T
    eq = rows[:, 1:] == rows[:, :-1]
    pat = (eq * (1 << np.arange(order - 1))).sum(axis=1)
    assert np.array_equal(cnt["by_pattern"][: 1 << (order - 1)], np.bincount(pat, minlength=1 << (order - 1)))
    closed = 0
    nsq = 0.0
    for e, row in enumerate(rows):
        _, m = np.unique(row, return_counts=True)
        k = math.factorial(order) // math.prod(math.factorial(int(x)) for x in m)
        closed += k
        nsq += k * float(cval[e]) ** 2
    assert cnt["expanded"] == closed
    X = dense_full(order, 7, cidx, cval)
    assert cnt["expanded"] == int(np.count_nonzero(X))
    assert np.isclose(cnt["normsq"], (X ** 2).sum(), rtol=1e-12)
    assert cnt["root_fibers"] == len(np.unique(rows[:, 0]))
    assert cnt["l2_fibers"] == len({(a, b) for a, b in rows[:, :2]})


@pytest.mark.parametrize("order", [3, 4])
def test_expand_matches_dense(order):
    T = synth.tensor_small_all_patterns(order, 5, 13)
    cidx, cval = canon(T)
    eidx, ev = oracle.expand(order, cidx, cval)
    X = dense_full(order, 5, cidx, cval)
    nz = np.argwhere(X != 0)               # lexicographic order from argwhere
    assert np.array_equal(eidx.T, nz)
    assert np.array_equal(ev.astype(np.float64), X[tuple(nz.T)])


# ----------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("order", [3, 4, 5])
def test_mttkrp_relabel_invariance(order):
    n = 12
    T = synth.tensor_uniform(order, n, 150, 21)
    cidx, cval = canon(T)
    B = synth.factor_normal(n, 4, 21).astype(np.float64)
    M, _ = oracle.mttkrp_enum(order, n, cidx, cval, B)
    pi = np.argsort(synth.Stream(5).uniform(n))     # new label of old index a is pi[a]
    c2, v2 = oracle.canonicalize(order, n, pi[cidx], cval)
    B2 = np.empty_like(B)
    B2[pi] = B
    M2, _ = oracle.mttkrp_enum(order, n, c2, v2, B2)
    assert np.allclose(M2[pi], M, rtol=1e-12, atol=1e-12)


def test_enum_equals_runs_on_zipf():
    T = synth.tensor3_zipf(500, 20000, 3)
    cidx, cval = canon(T)
    B = synth.factor_normal(500, 8, 3).astype(np.float64)
    M, Ma = oracle.mttkrp_enum(3, 500, cidx, cval, B)
    Mr = oracle.mttkrp_runs(3, 500, cidx, cval, B)
    assert oracle.componentwise_error(Mr, M, Ma) < 1e-14
    cnt = oracle.counts(3, cidx, cval)
    assert cnt["by_pattern"][0] == T.meta["strict"]
    assert cnt["by_pattern"][1] == T.meta["i=j<k"]
    assert cnt["by_pattern"][2] == T.meta["i<j=k"]
    assert cnt["by_pattern"][3] == T.meta["i=j=k"]


# ----------------------------------------------------------------------------- symmetric CP-ALS step

@pytest.mark.parametrize("order,n,R", [(3, 6, 2), (4, 5, 3), (5, 4, 2)])
def test_cp_als_step_vs_dense(order, n, R):
    """Independent path: dense MTTKRP by einsum, H by numpy, rows solved with numpy.linalg.solve."""
    T = synth.tensor_small_all_patterns(order, n, 31, density=0.8)
    cidx, cval = canon(T)
    B = synth.factor_normal(n, R, 31).astype(np.float64)
    X = dense_full(order, n, cidx, cval)
    M = dense_mttkrp(X, B)
    H = (B.T @ B) ** (order - 1) + 0.1 * np.eye(R)
    want = np.linalg.solve(H, M.T).T
    got, info = oracle.cp_als_step(order, n, cidx, cval, B, ridge=0.1)
    assert info == 0
    assert np.allclose(got, want, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("order", [3, 4])
def test_cp_als_fixed_point(order):
    """An exact symmetric CP tensor sum_r b_r^(x)N is a fixed point of the update (ridge 0)."""
    n, R = 6, 2
    Bs = synth.factor_normal(n, R, 77).astype(np.float64)
    rows = np.array(list(itertools.combinations_with_replacement(range(n), order)), np.int32)
    vals = np.array([sum(np.prod(Bs[list(t), r]) for r in range(R)) for t in rows])
    # values in float32 carry the rounding; the update returns Bs up to that rounding
    got, info = oracle.cp_als_step(order, n, rows.T.copy(), vals.astype(np.float32), Bs)
    assert info == 0
    assert np.allclose(got, Bs, rtol=1e-5, atol=1e-5)


def test_cp_als_reports_singular_H():
    n, R = 5, 3
    T = synth.tensor_small_all_patterns(3, n, 3)
    cidx, cval = canon(T)
    B = np.zeros((n, R))          # B^T B = 0: the first pivot is not positive
    got, info = oracle.cp_als_step(3, n, cidx, cval, B)
    assert info == 1 and not got.any()


# ----------------------------------------------------------------------------- TTM

@pytest.mark.parametrize("order,n,seed", [(2, 6, 0), (3, 6, 1), (3, 5, 2), (4, 4, 3)])
def test_ttm_vs_dense_bruteforce(order, n, seed):
    """Independent path: the dense full tensor contracted over its first axis with B."""
    T = synth.tensor_small_all_patterns(order, n, seed, density=0.7)
    cidx, cval = canon(T)
    R = 3
    B = synth.factor_normal(n, R, seed + 10).astype(np.float64)
    X = dense_full(order, n, cidx, cval)
    want = np.tensordot(X, B, axes=([0], [0]))
    got, gabs = oracle.ttm_enum(order, n, cidx, cval, B)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-13)
    assert np.allclose(gabs, np.tensordot(np.abs(X), np.abs(B), axes=([0], [0])), rtol=1e-12, atol=1e-13)


def _ttm_cells(C):
    """Nonzero (out1, out2, B-row) cells of an order-3 TTM output taken with B = I."""
    return {tuple(int(x) for x in t) for t in zip(*np.nonzero(C))}


def test_paper_ttm_listing_assignments():
    """With B = I (R = n), each assignment C[i,p,q] += A * B[s,i] lands in its own cell (p, q, s): the
    oracle's nonzero cells for one stored entry are exactly the listing's assignments, and its
    canonical-output cells (p <= q) are the three kept by the output-symmetry listing."""
    gold = json.load(open(os.path.join(GOLD, "paper_ttm_assignments.json")))
    n = 7
    B = np.eye(n)
    cases = {"j<k<l": (1, 3, 5), "j=k<l": (2, 2, 6), "j<k=l": (0, 4, 4), "j=k=l": (3, 3, 3)}
    for pat, (j, k, l) in cases.items():
        env = {"j": j, "k": k, "l": l}
        # the stored permutation of the entry is irrelevant: give it reversed
        C = oracle.ttm_enum(3, n, np.array([[l], [k], [j]], np.int32), np.array([1.0], np.float32), B,
                            want_abs=False)
        want = {tuple(env[s] for s in a) for a in gold["assignments"][pat]}
        assert _ttm_cells(C) == want, pat
        assert len(want) == len(gold["assignments"][pat])       # no two assignments share a cell
        assert np.all(C[np.nonzero(C)] == 1.0)                    # each applied exactly once
        if pat == "j<k<l":
            canon_cells = {c for c in _ttm_cells(C) if c[0] <= c[1]}
            kept = {tuple(env[s] for s in a) for a in gold["canonical_output_assignments_strict"]}
            assert canon_cells == kept
            assert len(_ttm_cells(C)) / len(canon_cells) == gold["savings_Sec_5_2_5"]["computations"]


@pytest.mark.parametrize("seed", [4, 5])
def test_ttm_output_symmetry_and_mttkrp_relation(seed):
    """C[j,l,:] = C[l,j,:] (visible output symmetry), and contracting C with B once more gives the
    MTTKRP: M[j,r] = sum_l C[j,l,r] B[l,r] (two oracle functions with no shared arithmetic)."""
    T = synth.tensor_small_all_patterns(3, 9, seed, density=0.5)
    cidx, cval = canon(T)
    B = synth.factor_normal(9, 4, seed).astype(np.float64)
    C = oracle.ttm_enum(3, 9, cidx, cval, B, want_abs=False)
    assert np.array_equal(C, C.transpose(1, 0, 2))
    M = oracle.mttkrp_enum(3, 9, cidx, cval, B, want_abs=False)
    assert np.allclose(np.einsum("jlr,lr->jr", C, B), M, rtol=1e-12, atol=1e-13)


def test_ttm_row_restriction_is_a_slice():
    T = synth.tensor_small_all_patterns(3, 8, 6, density=0.6)
    cidx, cval = canon(T)
    B = synth.factor_normal(8, 4, 6).astype(np.float64)
    full, fa = oracle.ttm_enum(3, 8, cidx, cval, B)
    rows = np.array([5, 0, 7])
    part, pa = oracle.ttm_enum(3, 8, cidx, cval, B, rows=rows)
    assert np.array_equal(part, full[rows]) and np.array_equal(pa, fa[rows])


# ----------------------------------------------------------------------------- partial symmetry

def dense_partial(parts, dims, cidx, cval):
    """Dense tensor with every stored tuple written at all its inside-part arrangements."""
    mdims = [d for s, d in zip(parts, dims) for _ in range(s)]
    X = np.zeros(mdims, dtype=np.float64)
    starts = np.cumsum([0] + list(parts))[:-1]
    for e in range(cidx.shape[1]):
        c = [int(x) for x in cidx[:, e]]
        segs = [list(itertools.permutations(c[s0:s0 + s])) for s0, s in zip(starts, parts)]
        for combo in itertools.product(*segs):
            X[tuple(x for seg in combo for x in seg)] = float(cval[e])
    return X


def dense_pmttkrp(X, parts, factors, out_part):
    """Contract every mode but the first of out_part with its part's factor (einsum, column r shared)."""
    letters = "abcde"
    order = X.ndim
    owner = [p for p, s in enumerate(parts) for _ in range(s)]
    f = int(np.cumsum([0] + list(parts))[out_part])
    ins = [letters[:order]]
    ops = [X]
    for q in range(order):
        if q != f:
            ins.append(letters[q] + "r")
            ops.append(np.asarray(factors[owner[q]], dtype=np.float64))
    return np.einsum(",".join(ins) + "->" + letters[f] + "r", *ops)


PARTITIONS = [((2, 1), (5, 4)), ((1, 2), (4, 5)), ((2, 2), (4, 3)), ((3, 1), (4, 3)), ((1, 1, 1), (3, 4, 5)),
              ((2, 1, 2), (3, 2, 3)), ((1, 3), (3, 4))]


@pytest.mark.parametrize("parts,dims", PARTITIONS)
def test_pmttkrp_vs_dense_bruteforce(parts, dims):
    T = synth.ptensor_small_all_patterns(parts, dims, 3, density=0.6)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    R = 3
    F = [synth.factor_normal(d, R, 10 + p).astype(np.float64) for p, d in enumerate(dims)]
    X = dense_partial(parts, dims, cidx, cval)
    for out in range(len(parts)):
        M, Ma = oracle.pmttkrp_enum(parts, dims, cidx, cval, F, out)
        assert np.allclose(M, dense_pmttkrp(X, parts, F, out), rtol=1e-12, atol=1e-13), out
        assert np.allclose(Ma, dense_pmttkrp(np.abs(X), parts, [np.abs(f) for f in F], out), rtol=1e-12,
                           atol=1e-13), out


PARTITIONS3 = [((1, 2), (4, 5)), ((2, 1), (5, 4)), ((1, 1, 1), (3, 4, 5)), ((3,), (5,))]


@pytest.mark.parametrize("parts,dims", PARTITIONS3)
def test_pttm_vs_dense_bruteforce(parts, dims):
    """Mode-1 TTM of a partially symmetric order-3 tensor against the dense contraction of the tensor
    expanded over every inside-part arrangement."""
    T = synth.ptensor_small_all_patterns(parts, dims, 7, density=0.6)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    B = synth.factor_normal(dims[0], 3, 21).astype(np.float64)
    X = dense_partial(parts, dims, cidx, cval)
    Cm, Ca = oracle.pttm_enum(parts, dims, cidx, cval, B)
    assert np.allclose(Cm, np.einsum("kjl,kr->jlr", X, B), rtol=1e-12, atol=1e-13)
    assert np.allclose(Ca, np.einsum("kjl,kr->jlr", np.abs(X), np.abs(B)), rtol=1e-12, atol=1e-13)
    if parts in ((1, 2), (3,)):   # modes 2 and 3 in one part: the output is symmetric
        assert np.array_equal(Cm, Cm.transpose(1, 0, 2))


@pytest.mark.parametrize("parts,dims", PARTITIONS3)
def test_pttm_contracted_again_is_pmttkrp(parts, dims):
    """Contracting the TTM output with the factors of modes 2 and 3 gives B^T weighted MTTKRP rows of part 0:
    sum_{j,l} C[j,l,r] F2[j,r] F3[l,r] = sum_k B[k,r] M0[k,r]."""
    T = synth.ptensor_small_all_patterns(parts, dims, 8, density=0.7)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    R = 4
    F = [synth.factor_normal(d, R, 30 + p).astype(np.float64) for p, d in enumerate(dims)]
    owner = [p for p, sz in enumerate(parts) for _ in range(sz)]
    Cm = oracle.pttm_enum(parts, dims, cidx, cval, F[owner[0]], want_abs=False)
    M0 = oracle.pmttkrp_enum(parts, dims, cidx, cval, F, 0, want_abs=False)
    lhs = np.einsum("jlr,jr,lr->r", Cm, F[owner[1]], F[owner[2]])
    rhs = np.einsum("kr,kr->r", F[owner[0]], M0)
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-12)


def test_pttm_one_part_is_full_symmetry_ttm():
    T = synth.tensor_small_all_patterns(3, 7, 19, density=0.6)
    cidx, cval = oracle.canonicalize(3, 7, T.idx, T.val)
    B = synth.factor_normal(7, 3, 19).astype(np.float64)
    got = oracle.pttm_enum((3,), (7,), cidx, cval, B, want_abs=False)
    want = oracle.ttm_enum(3, 7, cidx, cval, B, want_abs=False)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("order,n", [(2, 6), (3, 6), (4, 5), (5, 4)])
def test_pmttkrp_one_part_is_full_symmetry(order, n):
    """A partition with a single part is full symmetry: equals the symmetric MTTKRP's own enumeration."""
    T = synth.tensor_small_all_patterns(order, n, 17, density=0.6)
    cidx, cval = oracle.canonicalize(order, n, T.idx, T.val)
    B = synth.factor_normal(n, 3, 17).astype(np.float64)
    got = oracle.pmttkrp_enum((order,), (n,), cidx, cval, [B], 0, want_abs=False)
    want = oracle.mttkrp_enum(order, n, cidx, cval, B, want_abs=False)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("parts,dims", PARTITIONS)
def test_pcounts_closed_form_and_expansion(parts, dims):
    T = synth.ptensor_small_all_patterns(parts, dims, 5, density=0.5)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    starts = np.cumsum([0] + list(parts))[:-1]
    closed = 0
    for e in range(cidx.shape[1]):
        k = 1
        for s0, s in zip(starts, parts):
            seg = cidx[s0:s0 + s, e].tolist()
            k *= math.factorial(s) // math.prod(math.factorial(seg.count(v)) for v in set(seg))
        closed += k
    cnt = oracle.pcounts(parts, cidx, cval)
    assert cnt["expanded"] == closed
    X = dense_partial(parts, dims, cidx, cval)
    assert np.count_nonzero(X) == closed          # values are nonzero normal draws
    assert math.isclose(cnt["normsq"], float((X ** 2).sum()), rel_tol=1e-12)
    eidx, ev = oracle.pexpand(parts, cidx, cval)
    assert eidx.shape[1] == closed
    rows = [tuple(r) for r in eidx.T.tolist()]
    assert rows == sorted(rows) and len(set(rows)) == closed
    assert all(X[r] == v for r, v in zip(rows, ev.astype(np.float64)))


def test_pcanonicalize_properties():
    parts, dims = (2, 1, 2), (6, 3, 5)
    T = synth.ptensor_uniform(parts, dims, 400, 8)
    cidx, cval = oracle.pcanonicalize(parts, dims, T.idx, T.val)
    # non-decreasing inside parts only; across parts any order
    assert np.all(cidx[0] <= cidx[1]) and np.all(cidx[3] <= cidx[4])
    assert np.any(cidx[1] > cidx[2]) or np.any(cidx[2] > cidx[3])
    rows = [tuple(r) for r in cidx.T.tolist()]
    assert rows == sorted(rows) and len(set(rows)) == len(rows)
    # any inside-part permutation of the stored tuples gives the same canonical form
    perm = T.idx[[1, 0, 2, 4, 3]]
    c2, v2 = oracle.pcanonicalize(parts, dims, perm, T.val)
    assert np.array_equal(c2, cidx) and np.array_equal(v2, cval)
    # a permutation across parts is a different tensor (here: out of range for part 2's dimension)
    swapped = T.idx[[2, 1, 0, 3, 4]]
    bad = swapped[2] >= 3
    if bad.any():
        with pytest.raises(oracle.OracleError) as ei:
            oracle.pcanonicalize(parts, dims, swapped, T.val)
        assert ei.value.code == oracle.RANGE
    # a 2-mode non-symmetric tensor keeps (3, 1) as (3, 1)
    c3, _ = oracle.pcanonicalize((1, 1), (5, 5), np.array([[3], [1]]), np.array([1.0], np.float32))
    assert c3[:, 0].tolist() == [3, 1]
