"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and bench.py.

This module only draws random numbers and lays them out as user-level inputs
(coordinate lists, upper-triangle CSR matrices, dense factors).  It holds none of
the symmetric-kernel arithmetic: no multiplicities, no permutation enumeration,
no kernel math.  Both the oracle and the GPU path consume exactly the arrays
produced here.

Random source: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  The generator is counter based: draw k of a
stream with seed s is mix(s + (k+1) * 0x9E3779B97F4A7C15), where mix is the
published SplitMix64 finaliser.  `sym_gen_*` on the device implements the same
definition for large on-device tensor pools; `coord_value` below is the one
value rule both sides share for those pools.

Workload recipes (the paper's workloads are real matrices and Erdos-Renyi
random symmetric tensors; these seeded generators stand in for them):
  * upper-triangle CSR matrices with uniformly placed distinct positions
    (stands in for the symmetrised Vuduc matrix suite of the SSYMV evaluation);
  * 3-way tensors with Zipf(1.2) indices and an exact 1% share of repeated
    indices, built by construction;
  * 4-/5-way tensors with uniform indices (the paper's Erdos-Renyi tensors),
    where repeated indices occur naturally;
  * dense factors B ~ N(0, 1/R), optionally rounded to bfloat16 (RNE).
Every coordinate list is emitted with each tuple's positions shuffled and the
entries in random order, so canonicalisation is exercised on both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31 = np.uint64(30), np.uint64(27), np.uint64(31)


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser applied elementwise to a uint64 array."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
        return z ^ (z >> _S31)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream with the given seed."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
    return splitmix64_mix(z)


class Stream:
    """A sequential view of one SplitMix64 stream (deterministic draw order)."""

    def __init__(self, seed: int, tag: int = 0):
        # Distinct tags give unrelated streams from one user seed.
        base = splitmix64_mix(np.array([(seed * 1_000_003 + tag) & 0xFFFFFFFFFFFFFFFF],
                                       dtype=np.uint64))[0]
        self.seed = int(base)
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        out = splitmix64(self.seed, self.pos, count)
        self.pos += count
        return out

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_open0(self, count: int) -> np.ndarray:
        """Doubles in (0, 1]."""
        return ((self.u64(count) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)

    def randint(self, count: int, n: int) -> np.ndarray:
        """Integers uniform on [0, n) (multiply-high of a 53-bit fraction)."""
        r = np.floor(self.uniform(count) * n).astype(np.int64)
        return np.minimum(r, n - 1)

    def normal(self, count: int) -> np.ndarray:
        """Standard normal doubles by the Box-Muller transform (cosine branch)."""
        u1 = self.uniform_open0(count)
        u2 = self.uniform(count)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def zipf_cdf(n: int, s: float) -> np.ndarray:
    """Cumulative distribution of P(k) proportional to k^-s on k = 1..n (FP64)."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_draw(st: Stream, count: int, cdf: np.ndarray) -> np.ndarray:
    """Inverse-CDF Zipf sample; returns 0-based indices k-1."""
    u = st.uniform(count)
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, len(cdf) - 1).astype(np.int64)


def bf16_rne(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even); returns uint16 bits."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    out = r.astype(np.uint16)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = 0x7FC0
    return out


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)


# ----------------------------------------------------------------------------
# Symmetric tensors (coordinate lists)
# ----------------------------------------------------------------------------

@dataclass
class SymCOO:
    """A fully symmetric tensor given by one stored coordinate per distinct index multiset.

    idx has shape (order, nnz), int32, each tuple in arbitrary position order;
    val has shape (nnz,), float32.
    """
    order: int
    n: int
    idx: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])


def _row_keys(rows_sorted: np.ndarray, n: int) -> np.ndarray:
    """Injective key of each ascending row, used only for generator-side dedupe."""
    order = rows_sorted.shape[1]
    bits = max(1, int(n - 1).bit_length())
    if bits * order <= 64:
        key = np.zeros(rows_sorted.shape[0], dtype=np.uint64)
        for q in range(order):
            key = (key << np.uint64(bits)) | rows_sorted[:, q].astype(np.uint64)
        return key
    # Wide keys: a void view of the row bytes is unique per row.
    r = np.ascontiguousarray(rows_sorted.astype(np.int64))
    return r.view(np.dtype((np.void, 8 * order))).ravel()


def _draw_distinct(maker, need: int, n: int) -> np.ndarray:
    """Draw rows with maker(m) until `need` distinct multisets exist; keep them in draw order.

    Every round re-deduplicates everything drawn so far (first occurrence wins),
    so the result depends only on the draw sequence.
    """
    if need <= 0:
        return np.zeros((0, 1), dtype=np.int64)
    drawn = []
    factor = 1.2
    have = 0
    while True:
        m = int((need - have) * factor) + 256
        drawn.append(np.sort(maker(m), axis=1))
        rows = np.concatenate(drawn)
        keys = _row_keys(rows, n)
        _, first = np.unique(keys, return_index=True)
        if first.shape[0] >= need:
            first.sort()
            return rows[first[:need]]
        got = first.shape[0] - have
        have = first.shape[0]
        # next round: oversample by the observed yield of fresh multisets
        factor = min(8.0, max(1.2, 1.3 * m / max(got, 1)))


def _scramble(st: Stream, rows: np.ndarray) -> np.ndarray:
    """Shuffle the positions inside every tuple (uniform random permutation)."""
    nnz, order = rows.shape
    keys = st.uniform(nnz * order).reshape(nnz, order)
    perm = np.argsort(keys, axis=1, kind="stable")
    return np.take_along_axis(rows, perm, axis=1)


def _finish(st: Stream, order: int, n: int, rows: np.ndarray, val: np.ndarray, meta: dict,
            scramble: bool) -> SymCOO:
    nnz = rows.shape[0]
    if scramble:
        rows = _scramble(st, rows)
        shuffle = np.argsort(st.u64(nnz), kind="stable")
        rows, val = rows[shuffle], val[shuffle]
    idx = np.ascontiguousarray(rows.T.astype(np.int32))
    return SymCOO(order, n, idx, np.ascontiguousarray(val.astype(np.float32)), meta)


def tensor_uniform(order: int, n: int, nnz: int, seed: int, scramble: bool = True,
                   values: str = "normal") -> SymCOO:
    """nnz distinct index multisets with indices uniform on [0, n) (Erdos-Renyi style)."""
    if order < 2 or order > 5:
        raise ValueError("order must be 2..5")
    total = math.comb(n + order - 1, order)
    if nnz > total:
        raise ValueError("more nonzeros than canonical positions")
    st = Stream(seed, tag=order)
    rows = _draw_distinct(lambda m: st.randint(m * order, n).reshape(m, order), nnz, n)
    val = st.normal(nnz) if values == "normal" else st.uniform(nnz) * 2.0 - 1.0
    return _finish(st, order, n, rows, val, {"recipe": "uniform", "seed": seed}, scramble)


def tensor3_zipf(n: int, nnz: int, seed: int, s: float = 1.2, repeat_frac: float = 0.01,
                 scramble: bool = True) -> SymCOO:
    """3-way tensor: Zipf(s) indices, exactly repeat_frac of entries with a repeated index.

    Strict triples: three Zipf draws, rejected when any two are equal or the
    multiset already exists.  Repeated-index entries: half i=j<k, half i<j=k
    (minus the all-equal ones, which are 0.01 of the repeated share), drawn the
    same way with the equality forced.
    """
    st = Stream(seed, tag=3)
    cdf = zipf_cdf(n, s)
    n_rep = int(round(nnz * repeat_frac))
    n_all = max(1, n_rep // 100) if n_rep else 0
    n_ijk = (n_rep - n_all) // 2
    n_ikk = n_rep - n_all - n_ijk
    n_strict = nnz - n_rep

    def draw_until(need, maker):
        return _draw_distinct(maker, need, n)

    def strict(m):
        a = zipf_draw(st, m, cdf); b = zipf_draw(st, m, cdf); c = zipf_draw(st, m, cdf)
        ok = (a != b) & (b != c) & (a != c)
        return np.stack([a[ok], b[ok], c[ok]], axis=1)

    def pair(m, low_repeated):
        a = zipf_draw(st, m, cdf); b = zipf_draw(st, m, cdf)
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        return np.stack([lo, lo, hi] if low_repeated else [lo, hi, hi], axis=1)

    def triple(m):
        a = zipf_draw(st, m, cdf)
        return np.stack([a, a, a], axis=1)

    parts = [draw_until(n_strict, strict)]
    if n_ijk:
        parts.append(draw_until(n_ijk, lambda m: pair(m, True)))
    if n_ikk:
        parts.append(draw_until(n_ikk, lambda m: pair(m, False)))
    if n_all:
        parts.append(draw_until(n_all, triple))
    rows = np.concatenate(parts)
    val = st.normal(rows.shape[0])
    meta = {"recipe": "zipf", "s": s, "seed": seed, "strict": n_strict, "i=j<k": n_ijk,
            "i<j=k": n_ikk, "i=j=k": n_all}
    return _finish(st, 3, n, rows, val, meta, scramble)


def tensor_small_all_patterns(order: int, n: int, seed: int, density: float = 0.5) -> SymCOO:
    """Tiny tensor with every equality pattern present (for brute-force checks, n small)."""
    st = Stream(seed, tag=100 + order)
    import itertools
    rows = np.array(list(itertools.combinations_with_replacement(range(n), order)), dtype=np.int64)
    keep = st.uniform(rows.shape[0]) < density
    # Always keep one example of each equality pattern so no case is missing.
    pat = np.zeros(rows.shape[0], dtype=np.int64)
    for q in range(order - 1):
        pat |= (rows[:, q] == rows[:, q + 1]).astype(np.int64) << q
    for p in np.unique(pat):
        keep[np.nonzero(pat == p)[0][0]] = True
    rows = rows[keep]
    val = st.normal(rows.shape[0])
    return _finish(st, order, n, rows, val, {"recipe": "all-patterns", "seed": seed}, True)


# ----------------------------------------------------------------------------
# Partially symmetric tensors (symmetric within consecutive groups of modes)
# ----------------------------------------------------------------------------

@dataclass
class PartCOO:
    """A tensor symmetric within each part of a partition of its modes into
    consecutive groups (`parts` = group sizes, `dims` = one dimension per part),
    given by one stored coordinate per distinct tuple of per-part multisets.

    idx has shape (order, nnz), int32, positions permuted arbitrarily inside each
    part; val has shape (nnz,), float32.
    """
    parts: tuple
    dims: tuple
    idx: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def order(self) -> int:
        return int(sum(self.parts))

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])

    def mode_dims(self) -> list:
        return [d for s, d in zip(self.parts, self.dims) for _ in range(s)]


def _part_sort(rows: np.ndarray, parts) -> np.ndarray:
    out = rows.copy()
    q = 0
    for s in parts:
        out[:, q:q + s] = np.sort(out[:, q:q + s], axis=1)
        q += s
    return out


def _draw_distinct_rows(maker, need: int, parts) -> np.ndarray:
    """Like _draw_distinct, for tuples sorted within parts (first occurrence in draw order wins)."""
    if need <= 0:
        return np.zeros((0, int(sum(parts))), dtype=np.int64)
    drawn, have, factor = [], 0, 1.2
    while True:
        m = int((need - have) * factor) + 256
        drawn.append(_part_sort(maker(m), parts))
        rows = np.ascontiguousarray(np.concatenate(drawn).astype(np.int64))
        keys = rows.view(np.dtype((np.void, 8 * rows.shape[1]))).ravel()
        _, first = np.unique(keys, return_index=True)
        if first.shape[0] >= need:
            first.sort()
            return rows[first[:need]]
        got = first.shape[0] - have
        have = first.shape[0]
        factor = min(8.0, max(1.2, 1.3 * m / max(got, 1)))


def _finish_parts(st: Stream, parts, dims, rows: np.ndarray, val: np.ndarray, meta: dict,
                  scramble: bool) -> PartCOO:
    nnz = rows.shape[0]
    if scramble:
        q = 0
        for s in parts:
            if s > 1:
                keys = st.uniform(nnz * s).reshape(nnz, s)
                perm = np.argsort(keys, axis=1, kind="stable")
                rows[:, q:q + s] = np.take_along_axis(rows[:, q:q + s], perm, axis=1)
            q += s
        shuffle = np.argsort(st.u64(nnz), kind="stable")
        rows, val = rows[shuffle], val[shuffle]
    idx = np.ascontiguousarray(rows.T.astype(np.int32))
    return PartCOO(tuple(parts), tuple(dims), idx, np.ascontiguousarray(val.astype(np.float32)), meta)


def ptensor_uniform(parts, dims, nnz: int, seed: int, scramble: bool = True) -> PartCOO:
    """nnz distinct canonical tuples, every index uniform on its part's range."""
    parts, dims = tuple(int(s) for s in parts), tuple(int(d) for d in dims)
    order = sum(parts)
    total = 1
    for s, d in zip(parts, dims):
        total *= math.comb(d + s - 1, s)
    if nnz > total:
        raise ValueError("more nonzeros than canonical positions")
    st = Stream(seed, tag=300 + 16 * order + len(parts))
    mdims = [d for s, d in zip(parts, dims) for _ in range(s)]

    def maker(m):
        return np.stack([st.randint(m, d) for d in mdims], axis=1)

    rows = _draw_distinct_rows(maker, nnz, parts)
    val = st.normal(nnz)
    return _finish_parts(st, parts, dims, rows, val, {"recipe": "partial-uniform", "seed": seed}, scramble)


def ptensor_small_all_patterns(parts, dims, seed: int, density: float = 0.5) -> PartCOO:
    """Every canonical tuple of a tiny partially symmetric tensor, kept with probability
    `density`, plus at least one tuple of every combination of per-part equality patterns."""
    import itertools
    parts, dims = tuple(int(s) for s in parts), tuple(int(d) for d in dims)
    st = Stream(seed, tag=400 + 16 * sum(parts) + len(parts))
    per_part = [list(itertools.combinations_with_replacement(range(d), s)) for s, d in zip(parts, dims)]
    rows = np.array([sum(combo, ()) for combo in itertools.product(*per_part)], dtype=np.int64)
    keep = st.uniform(rows.shape[0]) < density
    pat = np.zeros(rows.shape[0], dtype=np.int64)
    bit, q = 0, 0
    for s in parts:
        for t in range(s - 1):
            pat |= (rows[:, q + t] == rows[:, q + t + 1]).astype(np.int64) << bit
            bit += 1
        q += s
    for p in np.unique(pat):
        keep[np.nonzero(pat == p)[0][0]] = True
    rows = rows[keep]
    val = st.normal(rows.shape[0])
    return _finish_parts(st, parts, dims, rows, val, {"recipe": "partial-all-patterns", "seed": seed}, True)


# ----------------------------------------------------------------------------
# Counter-based coordinate pools (shared definition with the device generator)
# ----------------------------------------------------------------------------

def coord_pool(order: int, n: int, count: int, seed: int):
    """Raw (not deduplicated) uniform coordinates, draw q of entry e = stream[e*order+q].

    The value of an entry depends only on its index multiset (`coord_value`), so
    repeated multisets carry bit-identical values and can be merged by the
    keep-equal duplicate policy.  The device generator implements the same rule.
    """
    z = splitmix64(seed, 0, count * order).reshape(count, order)
    idx = ((z >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    idx = idx.astype(np.int64)
    val = coord_value(idx, seed)
    return np.ascontiguousarray(idx.T.astype(np.int32)), val


def coord_value(rows: np.ndarray, seed: int) -> np.ndarray:
    """Value of an entry from its index multiset: a 24-bit uniform in [-1, 1).

    The multiset is summarised order-independently by a sum and a sum of mixed
    indices (both wrap modulo 2^64), so no position order is involved.
    """
    r = rows.astype(np.uint64)
    with np.errstate(over="ignore"):
        s1 = r.sum(axis=1, dtype=np.uint64)
        s2 = splitmix64_mix(r + np.uint64(seed & 0xFFFFFFFFFFFFFFFF)).sum(axis=1, dtype=np.uint64)
        h = splitmix64_mix(s1 * GOLDEN + s2)
    m = (h >> np.uint64(40)).astype(np.int64)          # 24 random bits
    return ((m.astype(np.float64) * (2.0 ** -23)) - 1.0).astype(np.float32)


def batch_coords(row_off: np.ndarray, draw_off: np.ndarray, seed: int):
    """Counter-based draws for batched symmetric matrices (same definition as sym_gen_batch_coords).

    Instance b owns global rows [row_off[b], row_off[b+1]) and draws
    [draw_off[b], draw_off[b+1]).  Draw d: u = (word_d >> 11) * 2^-53 of the
    SplitMix64 stream, slot s = floor(u * n_b (n_b + 1) / 2) of the row-major
    upper triangle, mapped to (i, j) with i <= j; returned as global indices,
    value from the pair's multiset (`coord_value`).
    """
    row_off = np.asarray(row_off, dtype=np.int64)
    draw_off = np.asarray(draw_off, dtype=np.int64)
    total = int(draw_off[-1])
    d = np.arange(total, dtype=np.int64)
    b = np.searchsorted(draw_off, d, side="right") - 1
    n = row_off[b + 1] - row_off[b]
    slots = n * (n + 1) // 2
    z = splitmix64(seed, 0, total)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    sl = np.floor(u * slots.astype(np.float64)).astype(np.int64)
    sl = np.minimum(sl, slots - 1)
    t = (2 * n + 1).astype(np.float64)
    i = np.floor((t - np.sqrt(t * t - 8.0 * sl.astype(np.float64))) * 0.5).astype(np.int64)
    i = np.clip(i, 0, n - 1)
    start = lambda r: r * (2 * n - r + 1) // 2
    for _ in range(4):  # integer fix-up of the floating-point row estimate
        down = (i > 0) & (start(i) > sl)
        i = i - down
        up = (i + 1 < n) & (start(i + 1) <= sl)
        i = i + up
    j = i + (sl - start(i))
    gi, gj = row_off[b] + i, row_off[b] + j
    idx = np.stack([gi, gj]).astype(np.int32)
    return idx, coord_value(np.stack([gi, gj], axis=1), seed)


def batch_upper_csr_host(row_off, idx, val):
    """Upper CSR (global rows and columns) of deduplicated draws; host-side, for small batches."""
    total_rows = int(row_off[-1])
    key = idx[0].astype(np.int64) * total_rows + idx[1]
    _, first = np.unique(key, return_index=True)
    i, j, v = idx[0][first], idx[1][first], val[first]
    o = np.lexsort((j, i))
    i, j, v = i[o], j[o], v[o]
    rowptr = np.zeros(total_rows + 1, dtype=np.int64)
    np.add.at(rowptr, i.astype(np.int64) + 1, 1)
    return np.cumsum(rowptr), j.astype(np.int32), v.astype(np.float32)


# ----------------------------------------------------------------------------
# Symmetric matrices (upper-triangle CSR) and dense operands
# ----------------------------------------------------------------------------

@dataclass
class UpperCSR:
    """Upper triangle (col >= row) of a symmetric n x n matrix, cols ascending per row."""
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def upper_csr_uniform(n: int, nnz: int, seed: int) -> UpperCSR:
    """nnz distinct upper positions (diagonal included) uniform over the n(n+1)/2 slots."""
    slots = n * (n + 1) // 2
    if nnz > slots:
        raise ValueError("too many nonzeros")
    st = Stream(seed, tag=2)
    chosen = np.empty(0, dtype=np.int64)
    while chosen.shape[0] < nnz:
        need = nnz - chosen.shape[0]
        d = st.randint(int(need * 1.1) + 32, slots)
        _, first = np.unique(d, return_index=True)
        first.sort()
        d = d[first]
        d = d[~np.isin(d, chosen)]
        chosen = np.concatenate([chosen, d[:need]])
    # slot -> (i, j): slots are laid out row by row, row i holding n - i slots.
    start = np.concatenate([[0], np.cumsum(np.arange(n, 0, -1, dtype=np.int64))])
    i = np.searchsorted(start, chosen, side="right") - 1
    j = i + (chosen - start[i])
    val = (st.uniform(nnz) * 2.0 - 1.0).astype(np.float32)
    o = np.lexsort((j, i))
    i, j, val = i[o], j[o], val[o]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, i + 1, 1)
    rowptr = np.cumsum(rowptr)
    return UpperCSR(n, rowptr.astype(np.int32), j.astype(np.int32), val)


def upper_csr_rowdegree(n: int, per_row: float, seed: int) -> UpperCSR:
    """Batched-instance recipe: exactly round(per_row * n) distinct uniform upper positions."""
    return upper_csr_uniform(n, min(int(round(per_row * n)), n * (n + 1) // 2), seed)


def vector_uniform(n: int, seed: int, tag: int = 7) -> np.ndarray:
    st = Stream(seed, tag=tag)
    return (st.uniform(n) * 2.0 - 1.0).astype(np.float32)


def factor_normal(n: int, rank: int, seed: int, tag: int = 11) -> np.ndarray:
    """Dense factor B (n x rank, row-major float32) with entries N(0, 1/rank)."""
    st = Stream(seed, tag=tag)
    return (st.normal(n * rank) / math.sqrt(rank)).astype(np.float32).reshape(n, rank)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Instance dimensions log-uniform on [lo, hi], rounded to integers."""
    st = Stream(seed, tag=31)
    u = st.uniform(count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    "ssymv_n2000": dict(kind="ssymv", n=2000, nnz=20000, seed=0),
    "mttkrp3_zipf_n100k_nnz20M_r64": dict(kind="mttkrp", order=3, n=100_000, nnz=20_000_000,
                                          rank=64, seed=1, recipe="zipf"),
    "mttkrp4_unif_n20k_nnz10M_r32": dict(kind="mttkrp", order=4, n=20_000, nnz=10_000_000,
                                         rank=32, seed=2, recipe="uniform"),
    "mttkrp5_unif_n2k_nnz5M_r16": dict(kind="mttkrp", order=5, n=2_000, nnz=5_000_000,
                                       rank=16, seed=2, recipe="uniform"),
}


CACHE_VERSION = 1


def _cache_dir() -> str:
    import os
    import tempfile
    d = os.environ.get("SYMGPU_SYNTH_CACHE") or os.path.join(tempfile.gettempdir(), "symgpu_synth_cache")
    os.makedirs(d, exist_ok=True)
    return d


def make_tensor(order: int, n: int, nnz: int, seed: int, recipe: str, cache: bool = True) -> SymCOO:
    """Named-recipe tensor; large ones are cached on local disk (same bytes every time)."""
    import os
    path = os.path.join(_cache_dir(), f"t{CACHE_VERSION}_{recipe}_{order}_{n}_{nnz}_{seed}.npz")
    if cache and nnz >= 1_000_000 and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        meta = {k[5:]: (z[k].item() if z[k].ndim == 0 else z[k]) for k in z.files if k.startswith("meta_")}
        return SymCOO(order, n, z["idx"], z["val"], meta)
    if recipe == "zipf":
        if order != 3:
            raise ValueError("the Zipf recipe is 3-way")
        T = tensor3_zipf(n, nnz, seed)
    else:
        T = tensor_uniform(order, n, nnz, seed)
    if cache and nnz >= 1_000_000:
        tmp = path + f".{os.getpid()}.npz"
        np.savez(tmp, idx=T.idx, val=T.val, **{"meta_" + k: np.asarray(v) for k, v in T.meta.items()})
        os.replace(tmp, path)
    return T
