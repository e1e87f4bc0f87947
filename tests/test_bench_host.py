"""Host-side logic of the benchmark (no GPU): the CSF fiber counts behind the roofline, the roofline arithmetic,
the kernel labels and the DRAM-traffic records it looks up."""
import itertools

import numpy as np
import pytest

import bench
import synth


def brute_fibers(order, idx):
    tuples = {tuple(sorted(int(idx[q, e]) for q in range(order))) for e in range(idx.shape[1])}
    strict = [t for t in tuples if len(set(t)) == order]
    return len(strict), [len({t[:q + 1] for t in strict}) for q in range(order - 1)]


@pytest.mark.parametrize("order,n,nnz,seed", [(3, 30, 2000, 1), (4, 14, 1500, 2), (5, 9, 800, 3), (3, 500, 40, 4)])
def test_strict_fiber_counts_match_brute_force(order, n, nnz, seed):
    T = synth.tensor_uniform(order, n, nnz, seed)
    assert bench.strict_fiber_counts(order, T.idx) == brute_fibers(order, np.asarray(T.idx))


def test_strict_fiber_counts_ignores_repeated_and_permuted_tuples():
    idx = np.array([[0, 2, 1, 1, 3], [1, 1, 2, 0, 3], [2, 0, 0, 2, 4]], dtype=np.int32)
    # (0,1,2) three times in different orders, (1,1,2) diagonal, (3,3,4) diagonal
    assert bench.strict_fiber_counts(3, idx) == (1, [1, 1])


def test_l2_roof_arithmetic():
    ceil = {"row_gather_rows_per_s_t": 4e10, "row_red_rows_per_s_t": 2e10, "gather_red_rows_per_s_t": 1e10}
    r = bench.l2_roof(1_000_000, 1_000_000, 64, ceil, "t", kernel_ms=0.2)
    assert r["bound"] == "l2" and r["frac"] == pytest.approx((1e6 / 1e10) / 2e-4)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    assert r["achieved"] == pytest.approx(2e6 * 64 * 4 / 2e-4 / 1e9)
    # gathers beyond the pairs run at the gather-only rate
    r2 = bench.l2_roof(3_000_000, 1_000_000, 64, ceil, "t", kernel_ms=0.2)
    assert r2["frac"] == pytest.approx((1e6 / 1e10 + 2e6 / 4e10) / 2e-4)


def test_strict_variant_labels_and_keys():
    base = dict(strict_kernel=0, entries_per_warp=128, leaf_index=0, vec_per_lane=1, root_combine=1)
    name, key, plain = bench.strict_variant(base, 64, 3)
    assert key == "plain_m0_c128_r1" and plain and name.startswith("k_mttkrp_strict<3,1,16,f32,MODE0>")
    lane = dict(base, strict_kernel=4, entries_per_warp=256, vec_per_lane=4)
    name, key, plain = bench.strict_variant(lane, 64, 3)
    assert key == "lane_m0_d4_v1_c256_r1" and not plain and "D4,V1" in name
    name, key, _ = bench.strict_variant(dict(lane, vec_per_lane=2, leaf_index=1, root_combine=0), 64, 3)
    assert key == "lane_m1_d1_v2_c256_r0" and "<3,1,8,f32,MODE1" in name
    name, key, _ = bench.strict_variant(dict(base, strict_kernel=3), 32, 4)
    assert key == "k3_c128" and name.startswith("k_mttkrp_strict_staged<4,1,8,f32>")


def test_traffic_records_parse_and_match_the_current_source():
    lines = [ln.split() for ln in open(bench.os.path.join(bench.ROOT, "profiles", "traffic.txt"))
             if ln.strip() and not ln.startswith("#")]
    assert lines and all(len(f) == 4 and f[2].startswith("src=") and f[3].startswith("dram_bytes_per_launch=")
                         for f in lines)
    for f in lines:
        plain = f[0].startswith("mttkrp_strict:plain")
        current = f[2] == "src=" + bench.kernel_source_hash(plain)
        v = bench.recorded_traffic(f[0], f[1], plain_only=plain)
        # a record of the current source is returned; a stale one reads as None (the bench then reports null)
        assert (v == int(f[3].split("=")[1])) if current else (v is None)
    assert bench.kernel_source_hash(True) != bench.kernel_source_hash(False)
