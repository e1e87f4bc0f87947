"""Benchmark of the symmetric sparse kernels on one GB300 (or N replicas under torchrun).

Headline workload: 3-way symmetric sparse MTTKRP, n = 100,000, 20,000,000
canonical nonzeros (i <= j <= k), Zipf(1.2) indices with an exact 1% share of
repeated indices, values N(0,1), shared factor B of 100,000 x 64 FP32, N(0,1/64).
A step is one sym_mttkrp call (strict stream + diagonal stream) on the resident
canonicalised tensor; the metric is canonical nonzeros per second.  L2 is
flushed (256 MB write) between timed steps and each step is timed with its own
CUDA event pair on the launching stream.

Also reported: the dominant kernel's roofline fraction from live per-kernel CUDA
events, an end-to-end figure through the public API with host buffers
(copies of the coordinate list and factor in, the result out, canonicalisation
included), the FP64 CPU oracle on a bounded sample, the expanded non-symmetric
baseline, the CP-fit residual cost, the 4-/5-way, SSYMV, TTM, partial-symmetry and
batched workloads (each with its error against the FP64 oracle), two serving traces
(host-scheduled continuous batching at 2,000 req/s; the device-resident request loop
at 20,000 req/s of small MTTKRP and SSYMV requests), and the SM clocks sampled
during the timed region.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference] [--rows main|all]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MAIN = dict(order=3, n=100_000, nnz=20_000_000, rank=64, seed=1, recipe="zipf")
WORKLOAD_NAME = "sym_mttkrp3_zipf1.2_n100k_nnz20M_r64_f32"
L2_FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons (every 20 ms) while running.

    Started before the warm-up; `window(t0, t1)` marks the timed region (host
    perf_counter times) so the summary uses the samples read inside it, and
    falls back to all samples taken under load when the region was shorter than
    the sampling period (said in the summary)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []   # (host time, csv line)
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.perf_counter() + 5.0
            while not self.lines and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def window(self, t0: float, t1: float):
        self.t0, self.t1 = t0, t1

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _parse(lines):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return sm, mx, reasons

    def summary(self):
        inside = [ln for t, ln in self.lines if self.t0 is not None and self.t0 <= t <= self.t1 + 0.02]
        sm, mx, reasons = self._parse(inside)
        scope = "timed region"
        if not sm:
            sm, mx, reasons = self._parse([ln for _, ln in self.lines])
            scope = "warm-up and timed region (timed region shorter than the 20 ms sampling period)"
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "scope": scope}


# ---------------------------------------------------------------------------- helpers

def kernel_source_hash(plain_only=True):
    """Hash of a strict-stream kernel's source.  plain_only: mttkrp.cuh up to the end of k_mttkrp_strict (its
    helpers and body; the other kernels follow it), else all of mttkrp.cuh; plus the headers it includes."""
    h = hashlib.sha256()
    for f in ("mttkrp.cuh", "common.cuh", "tensor.cuh"):
        with open(os.path.join(ROOT, "paper_2406_09266_gb300", "csrc", f), "rb") as fh:
            text = fh.read()
        if f == "mttkrp.cuh" and plain_only:
            cut = text.find(b"// The plain kernel with VPL float4 column groups per lane")
            text = text[:cut] if cut > 0 else text
        h.update(text)
    return h.hexdigest()[:16]


def strict_variant(cfg, rank=64, order=3):
    """(kernel name for the bench line, key of its DRAM-traffic record, whether the plain-kernel source hash
    applies) of the strict-stream kernel a configuration runs (one-word keys, FP32 factor)."""
    k, epw, leaf, shape = cfg["strict_kernel"], cfg["entries_per_warp"], cfg["leaf_index"], cfg["vec_per_lane"]
    rc = cfg.get("root_combine", 1)
    lanes = max(1, rank // 4)
    if k == 0:
        mode = 1 if leaf else 0
        if shape == 2 and not leaf:
            return (f"k_mttkrp_strict_wide<{order},1,{lanes // 2},2,f32> ({epw} entries/warp)", f"plain_wide_c{epw}",
                    False)
        return (f"k_mttkrp_strict<{order},1,{lanes},f32,MODE{mode}> ({epw} entries/warp, root combine {rc})",
                f"plain_m{mode}_c{epw}_r{rc}", True)
    if k == 4:
        mode = 1 if leaf else 0
        d, v = (4, 1) if shape == 4 else (1, shape)
        return (f"k_mttkrp_lane<{order},1,{lanes // v},f32,MODE{mode},D{d},V{v}> ({epw} entries/warp, root combine "
                f"{rc})", f"lane_m{mode}_d{d}_v{v}_c{epw}_r{rc}", False)
    name = {1: "k_mttkrp_strict_pipe", 2: "k_mttkrp_entries", 3: "k_mttkrp_strict_staged"}.get(k, "?")
    return f"{name}<{order},1,{lanes},f32> ({epw} entries/warp)", f"k{k}_c{epw}", False


def recorded_traffic(kernel: str, workload: str, plain_only=True):
    """DRAM bytes per launch recorded in profiles/ for this kernel source, else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    want = kernel_source_hash(plain_only)
    with open(p) as f:
        for ln in f:
            m = re.match(r"\s*(\S+)\s+(\S+)\s+src=(\w+)\s+dram_bytes_per_launch=(\d+)", ln)
            if m and m.group(1) == kernel and m.group(2) == workload and m.group(3) == want:
                return int(m.group(4))
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as td
            td.init_process_group("gloo")
            self.td = td

    def barrier(self):
        if self.ws > 1:
            self.td.barrier()

    def max(self, v: float) -> float:
        if self.ws == 1:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64)
        self.td.all_reduce(t, op=self.td.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.ws > 1:
            self.td.destroy_process_group()


def make_main_tensor():
    return synth.make_tensor(MAIN["order"], MAIN["n"], MAIN["nnz"], MAIN["seed"], MAIN["recipe"])


# ---------------------------------------------------------------------------- CPU oracle

def oracle_sample_rate(T, rank, target_s=12.0):
    """Times the FP64 oracle MTTKRP (definitional form) on a bounded sample of the workload."""
    import oracle
    B = synth.factor_normal(T.n, rank, MAIN["seed"]).astype(np.float64)
    # the coordinate list is in random order, so a prefix is a uniform sample
    probe = min(T.nnz, 100_000)
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx[:, :probe], T.val[:probe])
    t0 = time.perf_counter()
    oracle.mttkrp_enum(T.order, T.n, cidx, cval, B, want_abs=False)
    rate = probe / max(time.perf_counter() - t0, 1e-9)
    size = int(min(T.nnz, max(probe, rate * target_s)))
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx[:, :size], T.val[:size])
    t0 = time.perf_counter()
    oracle.mttkrp_enum(T.order, T.n, cidx, cval, B, want_abs=False)
    dt = time.perf_counter() - t0
    return cidx.shape[1] / dt, {"kind": "oracle", "cores": 1,
                                "sample": f"first {size} of {T.nnz} entries of the shuffled coordinate list "
                                          f"({cidx.shape[1]} canonical), FP64 definitional MTTKRP, "
                                          f"rank {rank}, {dt:.1f} s"}


def oracle_threads_rate(T, rank, target_s=8.0):
    """The FP64 oracle's threaded definitional MTTKRP on every core this process may run on
    (len(os.sched_getaffinity(0))), on a bounded sample of the workload."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    B = synth.factor_normal(T.n, rank, MAIN["seed"]).astype(np.float64)
    probe = min(T.nnz, 400_000)
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx[:, :probe], T.val[:probe])
    t0 = time.perf_counter()
    oracle.mttkrp_enum_threads(T.order, T.n, cidx, cval, B, cores)
    rate = probe / max(time.perf_counter() - t0, 1e-9)
    size = int(min(T.nnz, max(probe, rate * target_s)))
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx[:, :size], T.val[:size])
    t0 = time.perf_counter()
    oracle.mttkrp_enum_threads(T.order, T.n, cidx, cval, B, cores)
    dt = time.perf_counter() - t0
    return cidx.shape[1] / dt, {"kind": "oracle", "cores": cores,
                                "sample": f"first {size} of {T.nnz} entries of the shuffled coordinate list "
                                          f"({cidx.shape[1]} canonical), FP64 definitional MTTKRP on {cores} host "
                                          f"threads (contiguous entry ranges, private outputs summed in order), "
                                          f"rank {rank}, {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    T = make_main_tensor()
    import oracle
    B = synth.factor_normal(T.n, MAIN["rank"], MAIN["seed"]).astype(np.float64)
    # about 8M canonical entries over the whole timed run (a few seconds per million on one core)
    default_sample = max(20_000, min(400_000, 8_000_000 // max(args.steps, 1)))
    sample = min(T.nnz, int(os.environ.get("SYMGPU_REF_SAMPLE", str(default_sample))))
    cidx, cval = oracle.canonicalize(T.order, T.n, T.idx[:, :sample], T.val[:sample])
    for _ in range(args.warmup):
        oracle.mttkrp_enum(T.order, T.n, cidx, cval, B, want_abs=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.mttkrp_enum(T.order, T.n, cidx, cval, B, want_abs=False)
    dt = (time.perf_counter() - t0) / args.steps
    v = cidx.shape[1] / dt
    out = {"impl": "reference", "metric": "canonical_nnz_per_s", "value": v, "unit": "canonical nnz/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "sample_canonical_nnz": int(cidx.shape[1]), "same_config": False,
                      "note": "the oracle arm times a bounded sample of the workload's entries each step (a full "
                              "20M-entry step takes about 10 s on one core); the metric is per canonical entry"},
           "cpu_baseline": {"value": v, "unit": "canonical nnz/s", "cores": 1, "kind": "oracle",
                            "sample": f"first {sample} entries of the shuffled coordinate list, FP64 definitional "
                                      f"MTTKRP per step"},
           "e2e": {"value": v, "unit": "canonical nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------- GPU arm

def timed_steps(torch, step, K, flush_buf, stream):
    """Runs K steps, each between its own CUDA events; L2 flushed before each step (flush_buf None: warm L2)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        if flush_buf is not None:
            flush_buf.fill_(k & 0xff)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def measure_ceilings(sg):
    """Measured ceilings of the primitive operations (sym_ceiling_run), each timed alone on this GPU:
    FP32 FMA issue, random L2 row gathers / vector row reductions / both at the three MTTKRP row shapes,
    and a streaming copy of our own.  The denominators of the per-kernel roofline fractions."""
    c = {"fp32_fma_flop_per_s": sg.ceiling("fma", ops=1 << 28, reps=5)[0]}
    for n, R in ((100_000, 64), (20_000, 32), (2_000, 16)):
        for k in ("row_gather", "row_red", "gather_red"):
            c[f"{k}_rows_per_s_n{n}_r{R}"] = sg.ceiling(k, rows=n, rank=R, ops=1 << 25, reps=5)[0]
    c["hbm_copy_bytes_per_s"] = sg.ceiling("hbm_copy", rows=1 << 27, ops=0, reps=10)[0]
    return c


def l2_roof(gathers, reds, R, ceil, n_tag, kernel_ms):
    """Roofline of an L2-bound MTTKRP pass: it moves `gathers` random factor rows and `reds` random vector row
    reductions of R floats through L2.  The ceiling time for that mix is taken from the measured primitives:
    min(gathers, reds) pairs at the gather+reduction rate, the rest at the gather-only or reduction-only rate."""
    g_rate = ceil[f"row_gather_rows_per_s_{n_tag}"]
    r_rate = ceil[f"row_red_rows_per_s_{n_tag}"]
    gr_rate = ceil[f"gather_red_rows_per_s_{n_tag}"]
    pairs = min(gathers, reds)
    t_ceil = pairs / gr_rate + (gathers - pairs) / g_rate + (reds - pairs) / r_rate
    row_bytes = (gathers + reds) * R * 4
    t = kernel_ms * 1e-3
    return {"bound": "l2", "achieved": row_bytes / t / 1e9, "peak": row_bytes / t_ceil / 1e9, "unit": "GB/s",
            "frac": t_ceil / t, "row_gathers": int(gathers), "row_reductions": int(reds),
            "peak_source": "measured (sym_ceiling_run: random row gathers / vector row reductions in L2, this run)"}


def strict_fiber_counts(order, idx):
    """Strict canonical entries and their distinct prefixes (c1..cq) for q = 1..N-1 (host, numpy): the fiber
    counts of the CSF traversal, from which the algorithmic row operations of an MTTKRP pass follow."""
    rows = np.sort(np.asarray(idx).T, axis=1)
    rows = rows[np.all(rows[:, 1:] != rows[:, :-1], axis=1)]
    rows = rows[np.lexsort(rows.T[::-1])]
    if len(rows) > 1:  # repeated tuples (any stored permutation of one entry) count once
        rows = rows[np.concatenate(([True], np.any(rows[1:] != rows[:-1], axis=1)))]
    change = np.zeros(len(rows), bool)
    if len(rows):
        change[0] = True
    counts = []
    for q in range(order - 1):
        change[1:] |= rows[1:, q] != rows[:-1, q]
        counts.append(int(change.sum()))
    return len(rows), counts


def sampled_row_errors(order, n, idx, val, B32, M, Mb=None, Bb=None, rows=64, seed=0):
    """Componentwise error of the GPU result on a sample of output rows, against the FP64 oracle (the
    definitional enumeration restricted to those rows).  BF16: against the oracle on the FP32 factor (gate
    1e-2) and on the BF16-rounded factor (expected <= 1e-5)."""
    import oracle
    sel = np.unique(np.concatenate([np.arange(min(8, n)),
                                    synth.Stream(seed, tag=91).randint(rows, n)]))
    cidx, cval = oracle.canonicalize(order, n, idx, val)
    ref, ra = oracle.mttkrp_enum(order, n, cidx, cval, B32.astype(np.float64), rows=sel)
    out = {"rows_sampled": int(len(sel)),
           "f32_componentwise": oracle.componentwise_error(M[sel], ref[sel], ra[sel])}
    if Mb is not None:
        out["bf16_vs_f32_factor_componentwise"] = oracle.componentwise_error(Mb[sel], ref[sel], ra[sel])
        rb, rba = oracle.mttkrp_enum(order, n, cidx, cval, Bb.astype(np.float64), rows=sel)
        out["bf16_vs_bf16_factor_componentwise"] = oracle.componentwise_error(Mb[sel], rb[sel], rba[sel])
    return out


def run_ours(args):
    import torch

    import paper_2406_09266_gb300 as sg

    D = Dist()
    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    sg.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    hbm_peak, peak_kind = peaks()

    # ---- workload (host), resident copy (device), canonicalisation
    T = make_main_tensor()
    Bh = synth.factor_normal(T.n, MAIN["rank"], MAIN["seed"])
    idx_d = torch.from_numpy(T.idx).to(dev)
    val_d = torch.from_numpy(T.val).to(dev)
    B = torch.from_numpy(Bh).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = sg.SymTensor(idx_d, val_d, T.n)
    torch.cuda.synchronize()
    create_ms = (time.perf_counter() - t0) * 1e3
    info = X.info()
    M = torch.empty((T.n, MAIN["rank"]), dtype=torch.float32, device=dev)
    ws_res = X.mttkrp_workspace(MAIN["rank"])
    import tempfile
    t0 = time.perf_counter()
    if args.kernel_only:
        # profiling mode: a fixed configuration (by default the one the autotuner picks for this workload)
        fields = dict(strict_kernel=0, entries_per_warp=512, diag_smem_kb=48, leaf_index=0)
        for kv in filter(None, args.mttkrp_cfg.split(",")):
            k, v = kv.split("=")
            fields[k.strip()] = int(v)
        if fields.get("leaf_index"):
            X.add_leaf_index()
        X.set_config(**fields)
        tuned_cfg, tuned_ms = X.get_config(), 0.0
    else:
        # configurations compared with L2 flushed before each timed run, as the timed steps are
        tuned_cfg, tuned_ms = X.autotune(B, M=M, cache_path=os.path.join(tempfile.gettempdir(), "symgpu_tune.txt"),
                                         flush=flush)
    tune_s = time.perf_counter() - t0

    step = lambda: X.mttkrp(B, M=M)
    with ClockSampler(D.local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()

        # ---- timed region (device value)
        sg.profile_reset()
        sg.profile_enable(True)
        D.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        times = timed_steps(torch, step, args.steps, flush, stream)
        t_end = time.perf_counter()
        clk.window(t_wall, t_end)
        t_wall = t_end - t_wall
    D.barrier()
    sg.profile_enable(False)
    prof = sg.profile_read()
    ms = D.max(float(np.mean(times)))
    value = info["nnz"] * D.ws / (ms * 1e-3)
    launches = sum(v[0] for v in prof.values())

    # ---- roofline of the dominant kernel (strict stream)
    strict_launches, strict_ms = prof.get("mttkrp_strict", (0, 0.0))
    per_launch_ms = strict_ms / max(strict_launches, 1)
    kw_bytes = 8 * (2 if info["key_bits"] * 3 > 64 else 1)
    alg_bytes = info["nnz_strict"] * (kw_bytes + 4) + T.n * MAIN["rank"] * 4 * 3   # stream + B read + M rmw
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    # The kernel's binding roof is L2, not HBM: per strict entry it gathers the leaf's factor row and reduces
    # into the leaf's output row (R floats each), and per (c1, c2) fiber and per c1 fiber one more of each.
    # Those algorithmic row operations, at the measured random-row ceilings of this GPU, give the ceiling time.
    # With the leaf index (two passes) this launch is the first pass: no leaf reductions.
    ceil = measure_ceilings(sg) if D.rank == 0 and not args.kernel_only else None
    kname, tkey, plain_src = strict_variant(tuned_cfg, MAIN["rank"])
    if ceil is not None:
        rows_ops = info["nnz_strict"] + info["l2_fibers"] + info["root_fibers"]
        reds = rows_ops - (info["nnz_strict"] if tuned_cfg["leaf_index"] else 0)
        roof = l2_roof(rows_ops, reds, MAIN["rank"], ceil, "n100000_r64", per_launch_ms)
    else:
        roof = {"bound": "l2", "achieved": None, "peak": None, "unit": "GB/s", "frac": None}
    roof.update({"kernel": kname, "traffic": recorded_traffic("mttkrp_strict:" + tkey, WORKLOAD_NAME, plain_src),
                 "launch_ms": per_launch_ms,
                 # (the diagonal stream's kernel runs beside it on a second stream: share of the step's time)
                 "share_of_step": per_launch_ms / max(ms, 1e-12),
                 "hbm": {"algorithmic_bytes_per_launch": alg_bytes, "achieved_gbs": achieved, "peak_gbs": hbm_peak,
                         "frac": achieved / hbm_peak, "peak_source": peak_kind},
                 "fp32_issue": {"flop_per_launch": info["nnz_strict"] * 3 * 3 * MAIN["rank"],
                                "frac": (info["nnz_strict"] * 9 * MAIN["rank"] / (per_launch_ms * 1e-3)
                                         / ceil["fp32_fma_flop_per_s"]) if ceil else None}})

    if args.kernel_only:
        if D.rank == 0:
            print(json.dumps({"metric": "canonical_nnz_per_s", "value": value, "ms_per_step": ms,
                              "mode": "kernel-only (profiling)", "canonicalise_ms": create_ms, "per_kernel": prof}))
        D.close()
        return

    # the same step with L2 left warm between steps (inputs stay L2-resident: B, M and part of the stream)
    warm = timed_steps(torch, step, max(5, min(args.steps, 20)), None, stream)
    extras = {"per_kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()},
              "warm_l2_ms_per_step": float(np.mean(warm)),
              "step_ms": {"mean": float(np.mean(times)), "p50": float(np.median(times)), "min": float(np.min(times)),
                          "max": float(np.max(times))},
              "inputs_sha256": {"idx": hashlib.sha256(np.ascontiguousarray(T.idx).tobytes()).hexdigest()[:16],
                                "val": hashlib.sha256(np.ascontiguousarray(T.val).tobytes()).hexdigest()[:16],
                                "B": hashlib.sha256(np.ascontiguousarray(Bh).tobytes()).hexdigest()[:16]},
              "mttkrp_config": tuned_cfg, "autotune_s": tune_s,
              "canonicalise_ms": create_ms, "tensor": {k: info[k] for k in (
                  "nnz", "nnz_strict", "nnz_diag", "expanded_nnz", "root_fibers", "l2_fibers")}}

    # ---- error of the timed result on sampled rows, against the FP64 oracle
    if D.rank == 0:
        try:
            Mh = M.cpu().numpy()
            extras["error"] = sampled_row_errors(3, T.n, T.idx, T.val, Bh, Mh)
            extras["error"]["gate"] = "f32 <= 1e-5 componentwise (FP64 oracle, sampled output rows)"
        except Exception as e:
            extras["error"] = {"error": repr(e)}
        extras["ceilings"] = ceil

    # ---- CP-fit residual cost (FP64), same tensor
    Mr, res = X.mttkrp(B, residual=True, ws=ws_res)
    torch.cuda.synchronize()
    rt = timed_steps(torch, lambda: X.mttkrp(B, M=M, residual=True, ws=ws_res), 5, flush, stream)
    extras["mttkrp_plus_residual_ms"] = float(np.mean(rt))
    extras["residual"] = float(res.item())

    # ---- one symmetric CP-ALS update (MTTKRP, FP64 Gram, Cholesky inverse, apply), same tensor
    try:
        Bn = torch.empty_like(B)
        ws_als = torch.empty(sg.lib().sym_cp_als_workspace_bytes(X.handle, MAIN["rank"]), dtype=torch.uint8,
                             device=dev)
        als = lambda: X.cp_als_step(B, B_out=Bn, ridge=1e-6, ws=ws_als)
        als()
        torch.cuda.synchronize()
        sg.profile_reset()
        sg.profile_enable(True)
        at = timed_steps(torch, als, 5, flush, stream)
        sg.profile_enable(False)
        ap = sg.profile_read()
        extras["cp_als_step"] = {"ms": float(np.mean(at)), "rank": MAIN["rank"],
                                 "per_kernel_ms": {k: v[1] / max(v[0], 1) for k, v in ap.items()}}
        del ws_als, Bn
    except Exception as e:
        extras["cp_als_step"] = {"error": repr(e)}

    # ---- expanded non-symmetric baseline on the same tensor
    if args.rows == "all" and D.rank == 0:
        try:
            E = X.expanded()
            Me = torch.empty_like(M)
            for _ in range(2):
                E.mttkrp(B, M=Me)
            et = timed_steps(torch, lambda: E.mttkrp(B, M=Me), 5, flush, stream)
            extras["expanded_baseline"] = {"expanded_nnz": E.nnz, "ms": float(np.mean(et)),
                                           "speedup_sym_over_expanded": float(np.mean(et)) / ms,
                                           "read_reduction": E.nnz / info["nnz"],
                                           "max_abs_diff_vs_sym": float((Me - M).abs().max())}
            E.close()
            del Me
        except Exception as e:  # report, do not hide
            extras["expanded_baseline"] = {"error": str(e)}

    # ---- end to end through the public API with host buffers
    idx_h = torch.from_numpy(np.ascontiguousarray(T.idx)).pin_memory()
    val_h = torch.from_numpy(T.val).pin_memory()
    B_h = torch.from_numpy(Bh).pin_memory()
    M_h = torch.empty((T.n, MAIN["rank"]), dtype=torch.float32).pin_memory()
    ws_create = torch.empty(sg.SymTensor.create_ws_bytes(3, T.n, T.nnz), dtype=torch.uint8, device=dev)
    del X
    torch.cuda.empty_cache()

    # The coordinate list and the values stay in pinned host memory: sym_tensor_create reads the coordinates
    # in place (packing kernel) and copies the values on a stream of its own while the keys are sorted; the
    # factor's copy runs on a side stream meanwhile.
    side = torch.cuda.Stream()

    def e2e_step():
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            b_d = B_h.to(dev, non_blocking=True)
        Xe = sg.SymTensor(idx_h, val_h, T.n, ws=ws_create)
        torch.cuda.current_stream().wait_stream(side)
        Xe.mttkrp(b_d, M=M)
        M_h.copy_(M, non_blocking=True)
        torch.cuda.synchronize()
        Xe.close()

    e2e_step()
    # one more step with events between its phases (where the end-to-end time goes)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_host = time.perf_counter()
    ev[0].record()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b_d = B_h.to(dev, non_blocking=True)
    Xe = sg.SymTensor(idx_h, val_h, T.n, ws=ws_create)
    ev[1].record()
    torch.cuda.current_stream().wait_stream(side)
    Xe.mttkrp(b_d, M=M)
    ev[2].record()
    M_h.copy_(M, non_blocking=True)
    ev[3].record()
    torch.cuda.synchronize()
    e2e_parts = {"create_from_host_ms": ev[0].elapsed_time(ev[1]),
                 "mttkrp_ms": ev[1].elapsed_time(ev[2]), "d2h_ms": ev[2].elapsed_time(ev[3]),
                 "host_wall_ms": (time.perf_counter() - t_host) * 1e3,
                 "note": "create_from_host: coordinates read in place, values copied during the sort, the "
                         "factor's copy overlapped on a side stream"}
    Xe.close()
    e2e_k = max(5, min(args.steps, 20))
    D.barrier()
    t0 = time.perf_counter()
    e2e_steps = []
    for _ in range(e2e_k):
        t1 = time.perf_counter()
        e2e_step()
        e2e_steps.append((time.perf_counter() - t1) * 1e3)
    e2e_s = D.max((time.perf_counter() - t0) / e2e_k)
    h2d = idx_h.numel() * 4 + val_h.numel() * 4 + B_h.numel() * 4
    d2h = M_h.numel() * 4

    # ---- secondary rows
    if args.rows == "all" and D.rank == 0:
        extras["rows"] = secondary_rows(torch, sg, dev, flush, stream, hbm_peak, ceil)
        try:
            extras["rows"]["batched_ssymv_syprd_4096"] = batch_row(torch, sg, dev, flush, stream, hbm_peak)
        except Exception as e:
            extras["rows"]["batched_ssymv_syprd_4096"] = {"error": repr(e)}
        try:
            extras["rows"]["serving_poisson_2000rps"] = serving_row(torch, sg, dev)
        except Exception as e:
            extras["rows"]["serving_poisson_2000rps"] = {"error": repr(e)}
        try:
            extras["rows"]["serving_device_loop_20000rps"] = devloop_row(torch, sg, dev)
        except Exception as e:
            extras["rows"]["serving_device_loop_20000rps"] = {"error": repr(e)}

    out = {"metric": "canonical_nnz_per_s", "value": value, "unit": "canonical nnz/s", "n_gpus": D.ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "order": 3, "n": T.n, "canonical_nnz": info["nnz"],
                      "rank": MAIN["rank"], "factor_dtype": "f32", "indices": "zipf(1.2), 1% repeated",
                      "l2": "flushed between steps (256 MB write); each step timed by its own event pair",
                      "parallelism": f"replicas{D.ws}"},
           "effective_gbs": alg_bytes / (ms * 1e-3) / 1e9,
           "roofline": roof,
           "e2e": {"value": info["nnz"] * D.ws / e2e_s, "unit": "canonical nnz/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
                   "includes": "coordinate list read from pinned host memory by the packing kernel, H2D of "
                               "values (during the sort) and factor (side stream), canonicalisation, MTTKRP, "
                               "D2H of M",
                   "one_step_breakdown": e2e_parts, "steps": e2e_k,
                   "step_ms": {"p50": float(np.median(e2e_steps)), "min": float(min(e2e_steps)),
                               "max": float(max(e2e_steps))}},
           "gpu_launches": launches, "clocks": clk.summary(), "wall_s_timed": t_wall, "extras": extras}
    if D.rank == 0 and not args.no_cpu:
        rate, meta = oracle_sample_rate(T, MAIN["rank"])
        meta["value"] = rate
        meta["unit"] = "canonical nnz/s"
        out["cpu_baseline"] = meta
        try:
            rate_t, meta_t = oracle_threads_rate(T, MAIN["rank"])
            meta_t["value"] = rate_t
            meta_t["unit"] = "canonical nnz/s"
            out["cpu_baseline_all_cores"] = meta_t
        except Exception as e:
            out["cpu_baseline_all_cores"] = {"error": repr(e)}
    if D.rank == 0:
        print(json.dumps(out))
    D.close()


def secondary_rows(torch, sg, dev, flush, stream, hbm_peak, ceil=None):
    rows = {}
    # 4-way and 5-way symmetric MTTKRP, FP32 and BF16 factors
    for name, order, n, nnz, rank in [("mttkrp4_unif_n20k_nnz10M_r32", 4, 20_000, 10_000_000, 32),
                                      ("mttkrp5_unif_n2k_nnz5M_r16", 5, 2_000, 5_000_000, 16)]:
        T = synth.make_tensor(order, n, nnz, 2, "uniform")
        X = sg.SymTensor(torch.from_numpy(T.idx).to(dev), torch.from_numpy(T.val).to(dev), n)
        info = X.info()
        B32 = synth.factor_normal(n, rank, 2)
        r = {"canonical_nnz": info["nnz"], "nnz_diag": info["nnz_diag"]}
        res = {}
        X.add_leaf_index()
        tune_cache = os.path.join(__import__("tempfile").gettempdir(), "symgpu_tune.txt")
        for tag, Bt in (("f32", torch.from_numpy(B32).to(dev)),
                        ("bf16", torch.from_numpy(synth.bf16_rne(B32).view(np.int16)).to(dev).view(torch.bfloat16))):
            M = torch.empty((n, rank), dtype=torch.float32, device=dev)
            cfg, tune_ms = X.autotune(Bt, M=M, cache_path=tune_cache, flush=flush)
            # the tuner's pick against the plain kernel (128 entries per warp), both timed as the row is
            plain = dict(strict_kernel=0, entries_per_warp=128, leaf_index=0, l1_pref=1, stream_hint=1,
                         root_combine=1, diag_smem_kb=cfg["diag_smem_kb"])
            X.set_config(**plain)
            t_plain = float(np.mean(timed_steps(torch, lambda: X.mttkrp(Bt, M=M), 5, flush, stream)))
            X.set_config(**cfg)
            t_tuned = float(np.mean(timed_steps(torch, lambda: X.mttkrp(Bt, M=M), 5, flush, stream)))
            if t_plain < t_tuned:
                X.set_config(**plain)
                cfg = X.get_config()
            for _ in range(3):
                X.mttkrp(Bt, M=M)
            sg.profile_reset()
            sg.profile_enable(True)
            t = timed_steps(torch, lambda: X.mttkrp(Bt, M=M), 10, flush, stream)
            sg.profile_enable(False)
            prof = sg.profile_read()
            ms = float(np.mean(t))
            r[tag] = {"ms": ms, "canonical_nnz_per_s": info["nnz"] / (ms * 1e-3), "mttkrp_config": cfg,
                      "per_kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()},
                      "selection": {"autotune_ms": tune_ms, "tuned_ms": t_tuned, "plain_128_ms": t_plain}}
            X.mttkrp(Bt, M=M)
            res[tag] = M.cpu().numpy()
        try:
            r["error"] = sampled_row_errors(order, n, T.idx, T.val, B32, res["f32"], res["bf16"],
                                            synth.bf16_to_f32(synth.bf16_rne(B32)))
            r["error"]["gate"] = "f32 <= 1e-5, bf16 vs f32 factor <= 1e-2 (componentwise, FP64 oracle)"
        except Exception as e:
            r["error"] = {"error": repr(e)}
        try:
            E = X.expanded()
            Me = torch.empty((n, rank), dtype=torch.float32, device=dev)
            Bt = torch.from_numpy(B32).to(dev)
            E.mttkrp(Bt, M=Me)
            t = timed_steps(torch, lambda: E.mttkrp(Bt, M=Me), 5, flush, stream)
            r["expanded_ms"] = float(np.mean(t))
            r["speedup_sym_over_expanded"] = r["expanded_ms"] / r["f32"]["ms"]
            r["read_reduction"] = E.nnz / info["nnz"]
            E.close()
        except Exception as e:
            r["expanded_error"] = str(e)
        if ceil:
            # one factor-row gather and one row reduction per strict entry (leaf) and per fiber of every level
            ns, fib = strict_fiber_counts(order, T.idx)
            ops = ns + sum(fib)
            strict_ms = sum(v for k, v in r["f32"]["per_kernel_ms"].items() if k.startswith("mttkrp_strict"))
            r["roofline"] = l2_roof(ops, ops, rank, ceil, f"n{n}_r{rank}", strict_ms)
            r["roofline"]["fibers_per_level"] = fib
            r["roofline"]["kernel"] = strict_variant(r["f32"]["mttkrp_config"], rank, order)[0]
            r["roofline"]["model"] = ("one-pass row operations (a gather and a reduction per strict entry and per "
                                      "fiber) against the strict-stream time of the tuned configuration")
        rows[name] = r
        X.close()
    rows["ssymv_n2000_nnz20k"] = small_ssymv_row(torch, sg, dev, flush, stream)
    try:
        rows["ssymv_bellman_n2M_16perrow"] = large_ssymv_row(torch, sg, dev, flush, stream, hbm_peak)
    except Exception as e:
        rows["ssymv_bellman_n2M_16perrow"] = {"error": repr(e)}
    try:
        rows["ttm3_unif_n2k_nnz5M_r32"] = ttm_row(torch, sg, dev, flush, stream, hbm_peak)
    except Exception as e:
        rows["ttm3_unif_n2k_nnz5M_r32"] = {"error": repr(e)}
    try:
        rows["pmttkrp_parts22_n20k_nnz5M_r32"] = ptensor_row(torch, sg, dev, flush, stream, hbm_peak)
    except Exception as e:
        rows["pmttkrp_parts22_n20k_nnz5M_r32"] = {"error": repr(e)}
    return rows


def small_ssymv_row(torch, sg, dev, flush, stream, n=2000, nnz=20000, seed=0, K=50):
    """SSYMV + SYPRD on the 2,000 x 2,000, 1 % dense matrix: launch-latency bound.
    `ms`: each call between its own events (L2 flushed before each); `graph_ms`:
    the same call captured once in a CUDA graph and replayed (no host work
    inside the timed window)."""
    A = synth.upper_csr_uniform(n, nnz, seed)
    x = synth.vector_uniform(n, seed)
    t_ = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, cl, vl, xd = t_(A.rowptr), t_(A.col), t_(A.val), t_(x)
    y = torch.empty(n, dtype=torch.float32, device=dev)
    ws = sg.spmv_workspace(n, rp, cl, vl)
    for _ in range(5):
        sg.spmv(n, rp, cl, vl, xd, y=y, syprd=True, ws=ws)
    t = timed_steps(torch, lambda: sg.spmv(n, rp, cl, vl, xd, y=y, syprd=True, ws=ws), K, flush, stream)
    ms = float(np.mean(t))
    row = {"ms": ms, "p50_ms": float(np.median(t)), "canonical_nnz_per_s": A.nnz / (ms * 1e-3),
           "path": "cluster_1launch" if sg.spmv_single_launch(n, A.nnz) else "multi_block"}
    s_out = torch.empty(1, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        sg.spmv_noalloc(n, rp, cl, vl, xd, y, s_out, stream=side)
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        sg.spmv_noalloc(n, rp, cl, vl, xd, y, s_out, stream=side)
    for _ in range(5):
        g.replay()
    torch.cuda.synchronize()
    t = timed_steps(torch, g.replay, K, flush, stream)
    row["graph_ms"] = float(np.mean(t))
    row["graph_p50_ms"] = float(np.median(t))
    dd = torch.abs(xd)
    yb = torch.empty_like(dd)
    for _ in range(5):
        sg.bellman_step(n, rp, cl, vl, dd, y=yb)
    t = timed_steps(torch, lambda: sg.bellman_step(n, rp, cl, vl, dd, y=yb), K, flush, stream)
    row["bellman_ford_step_ms"] = float(np.mean(t))
    try:
        import oracle
        x64 = x.astype(np.float64)
        yr, ya = oracle.ssymv(n, A.rowptr, A.col, A.val, x64)
        sr, sa = oracle.syprd(n, A.rowptr, A.col, A.val, x64)
        y1, s1 = sg.spmv(n, rp, cl, vl, xd, syprd=True, ws=ws)
        torch.cuda.synchronize()
        bref = oracle.bellman(n, A.rowptr, A.col, A.val, np.abs(x).astype(np.float64))
        row["error"] = {"ssymv_componentwise": oracle.componentwise_error(y1.cpu().numpy(), yr, ya),
                        "syprd_relative": abs(float(s1.item()) - sr) / sa,
                        "noalloc_graph_ssymv_componentwise": oracle.componentwise_error(y.cpu().numpy(), yr, ya),
                        "noalloc_graph_syprd_relative": abs(float(s_out.item()) - sr) / sa,
                        "bellman_ford_max_abs_diff": float(np.max(np.abs(yb.cpu().numpy().astype(np.float64) - bref))),
                        "gate": "SSYMV / SYPRD <= 1e-5 (componentwise / relative to the sum of |terms|, FP64 oracle)"}
    except Exception as e:
        row["error"] = {"error": repr(e)}
    return row


def ptensor_row(torch, sg, dev, flush, stream, hbm_peak, parts=(2, 2), dims=(20_000, 20_000), nnz=5_000_000,
                rank=32, seed=4):
    """Partially symmetric 4-way tensor (symmetric inside modes {1,2} and inside {3,4}), uniform indices:
    the MTTKRP for each part's factor, against the same kernel on the tensor with its symmetry expanded."""
    T = synth.ptensor_uniform(parts, dims, nnz, seed)
    X = sg.PTensor(torch.from_numpy(T.idx).to(dev), torch.from_numpy(T.val).to(dev), parts, dims)
    info = X.info()
    F = [torch.from_numpy(synth.factor_normal(d, rank, seed + p)).to(dev) for p, d in enumerate(dims)]
    out = {"parts": list(parts), "dims": list(dims), "canonical_nnz": info["nnz"], "rank": rank,
           "expanded_nnz": info["expanded_nnz"], "read_reduction": info["expanded_nnz"] / max(info["nnz"], 1)}
    Ms = [torch.empty((d, rank), dtype=torch.float32, device=dev) for d in dims]
    per_mode = [F[p] for p, s_ in enumerate(parts) for _ in range(s_)]
    first = np.cumsum([0] + list(parts))[:-1]
    E = X.expand()
    for o in range(len(parts)):
        for _ in range(3):
            X.mttkrp(F, o, M=Ms[o])
        ms = float(np.mean(timed_steps(torch, lambda: X.mttkrp(F, o, M=Ms[o]), 10, flush, stream)))
        ref = X.mttkrp(F, o)
        Me = E.mttkrp(per_mode, int(first[o]))
        ems = float(np.mean(timed_steps(torch, lambda: E.mttkrp(per_mode, int(first[o]), M=Me), 5, flush, stream)))
        torch.cuda.synchronize()
        # bytes: canonical entries (4 int32 + value), the factor rows read once, M zeroed and reduced
        alg = info["nnz"] * (4 * len(T.idx) + 4) + sum(d * rank * 4 for d in dims) + 2 * dims[o] * rank * 4
        out[f"part{o}"] = {"ms": ms, "canonical_nnz_per_s": info["nnz"] / (ms * 1e-3),
                           "effective_gbs": alg / (ms * 1e-3) / 1e9, "hbm_frac": alg / (ms * 1e-3) / 1e9 / hbm_peak,
                           "expanded_ms": ems, "speedup_sym_over_expanded": ems / ms,
                           "max_abs_diff_vs_expanded": float((Me - ref).abs().max())}
    E.close()
    X.close()
    try:
        import oracle
        pc, pv = oracle.pcanonicalize(parts, dims, T.idx, T.val)
        F64 = [f.cpu().numpy().astype(np.float64) for f in F]
        for o in range(len(parts)):
            rf, ra = oracle.pmttkrp_enum(parts, dims, pc, pv, F64, o)
            out[f"part{o}"]["error"] = {"componentwise": oracle.componentwise_error(Ms[o].cpu().numpy(), rf, ra),
                                        "gate": "<= 1e-5 componentwise (FP64 oracle, every row)"}
    except Exception as e:
        out["error"] = {"error": repr(e)}
    return out


def large_ssymv_row(torch, sg, dev, flush, stream, hbm_peak, n=1 << 21, per_row=16, seed=5):
    """One symmetric matrix, n = 2^21, 16 upper draws per row (device-generated): SSYMV + SYPRD,
    the full-CSR baseline and one Bellman-Ford min-plus step, all HBM-sized (~0.3 GB per operand)."""
    batch = sg.make_batch(np.array([n]), per_row, seed)
    rp = batch.rowptr.to(torch.int32)
    cl, vl = batch.col, batch.val
    nnz = int(cl.numel())
    x = torch.from_numpy(synth.vector_uniform(n, seed)).to(dev)
    y = torch.empty_like(x)
    ws = sg.spmv_workspace(n, rp, cl, vl)
    for _ in range(3):
        sg.spmv(n, rp, cl, vl, x, y=y, syprd=True, ws=ws)
    t = timed_steps(torch, lambda: sg.spmv(n, rp, cl, vl, x, y=y, syprd=True, ws=ws), 10, flush, stream)
    ms = float(np.mean(t))
    alg = nnz * 8 + (n + 1) * 4 + n * 4 * 3          # col + val, rowptr, x read, y read + write
    out = {"n": n, "upper_nnz": nnz, "ssymv_syprd_ms": ms, "canonical_nnz_per_s": nnz / (ms * 1e-3),
           "effective_gbs": alg / (ms * 1e-3) / 1e9, "hbm_frac": alg / (ms * 1e-3) / 1e9 / hbm_peak}
    F = sg.FullCSR(n, rp, cl, vl)
    yf = torch.empty_like(x)
    for _ in range(3):
        F.spmv(x, y=yf)
    tf = timed_steps(torch, lambda: F.spmv(x, y=yf), 10, flush, stream)
    out["full_csr_ms"] = float(np.mean(tf))
    out["speedup_over_full_csr"] = out["full_csr_ms"] / ms
    d = torch.abs(x)
    yb = torch.empty_like(d)
    for _ in range(3):
        sg.bellman_step(n, rp, cl, vl, d, y=yb)
    tb = timed_steps(torch, lambda: sg.bellman_step(n, rp, cl, vl, d, y=yb), 10, flush, stream)
    out["bellman_ford_step_ms"] = float(np.mean(tb))
    out["bellman_ford_effective_gbs"] = alg / (out["bellman_ford_step_ms"] * 1e-3) / 1e9
    try:
        import oracle
        y1, s1 = sg.spmv(n, rp, cl, vl, x, syprd=True, ws=ws)
        torch.cuda.synchronize()
        rp_h = rp.cpu().numpy().astype(np.int32)
        cl_h = cl.cpu().numpy().astype(np.int32)
        vl_h = vl.cpu().numpy().astype(np.float32)
        x64 = x.cpu().numpy().astype(np.float64)
        yr, ya = oracle.ssymv(n, rp_h, cl_h, vl_h, x64)
        sr, sa = oracle.syprd(n, rp_h, cl_h, vl_h, x64)
        out["error"] = {"ssymv_componentwise": oracle.componentwise_error(y1.cpu().numpy(), yr, ya),
                        "syprd_relative": abs(float(s1.item()) - sr) / sa,
                        "full_csr_componentwise": oracle.componentwise_error(yf.cpu().numpy(), yr, ya),
                        "gate": "<= 1e-5 (componentwise / relative to the sum of |terms|, FP64 oracle, every row)"}
    except Exception as e:
        out["error"] = {"error": repr(e)}
    return out


def ttm_row(torch, sg, dev, flush, stream, hbm_peak, n=2000, nnz=5_000_000, rank=32, seed=3):
    """Symmetric mode-1 TTM (3-way, uniform): canonical-triangle output (packed), full output
    (canonical + replication), and the expanded non-symmetric baseline."""
    T = synth.make_tensor(3, n, nnz, seed, "uniform")
    X = sg.SymTensor(torch.from_numpy(T.idx).to(dev), torch.from_numpy(T.val).to(dev), n)
    X.add_leaf_index()
    info = X.info()
    B = torch.from_numpy(synth.factor_normal(n, rank, seed)).to(dev)
    Cp = torch.empty((n * (n + 1) // 2, rank), dtype=torch.float32, device=dev)
    Cf = torch.empty((n, n, rank), dtype=torch.float32, device=dev)
    for _ in range(3):
        X.ttm(B, "packed", C_out=Cp)
    sg.profile_reset()
    sg.profile_enable(True)
    tp = timed_steps(torch, lambda: X.ttm(B, "packed", C_out=Cp), 10, flush, stream)
    sg.profile_enable(False)
    prof = sg.profile_read()
    for _ in range(2):
        X.ttm(B, "full", C_out=Cf)
    tf = timed_steps(torch, lambda: X.ttm(B, "full", C_out=Cf), 10, flush, stream)
    ms_p, ms_f = float(np.mean(tp)), float(np.mean(tf))
    # stream (+ leaf index) read once, B read once, packed output written once
    alg = info["nnz"] * 12 + info["nnz_strict"] * 12 + n * rank * 4 + n * (n + 1) // 2 * rank * 4
    kl, kms = prof.get("ttm", (1, ms_p))
    out = {"canonical_nnz": info["nnz"], "rank": rank, "packed_ms": ms_p, "full_ms": ms_f,
           "canonical_nnz_per_s": info["nnz"] / (ms_p * 1e-3),
           "effective_gbs": alg / (ms_p * 1e-3) / 1e9, "hbm_frac": alg / (ms_p * 1e-3) / 1e9 / hbm_peak,
           "per_kernel_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()}}
    E = X.expanded()
    Ce = torch.empty((n, n, rank), dtype=torch.float32, device=dev)
    for _ in range(2):
        E.ttm(B, C_out=Ce)
    te = timed_steps(torch, lambda: E.ttm(B, C_out=Ce), 10, flush, stream)
    out["expanded_ms"] = float(np.mean(te))
    out["expanded_nnz"] = E.nnz
    out["speedup_packed_over_expanded"] = out["expanded_ms"] / ms_p
    out["speedup_full_over_expanded"] = out["expanded_ms"] / ms_f
    X.ttm(B, "full", C_out=Cf)
    torch.cuda.synchronize()
    out["max_abs_diff_full_vs_expanded"] = float((Cf - Ce).abs().max())
    E.close()
    X.close()
    try:
        # sampled output rows j against the FP64 oracle: C[j, :, :] of the full output and the packed
        # positions j <= l of row j (at j n - j (j - 1) / 2 + (l - j))
        import oracle
        sel = np.unique(np.concatenate([[0, 1, n - 1], synth.Stream(seed, tag=93).randint(13, n)]))
        cidx, cval = oracle.canonicalize(3, n, T.idx, T.val)
        ref, ra = oracle.ttm_enum(3, n, cidx, cval, synth.factor_normal(n, rank, seed).astype(np.float64), rows=sel)
        full = Cf[torch.from_numpy(sel).to(dev)].cpu().numpy()
        Cph = Cp.cpu().numpy()
        packed = np.concatenate([Cph[int(j) * n - int(j) * (int(j) - 1) // 2:][:n - int(j)] for j in sel])
        out["error"] = {"rows_sampled": int(sel.size),
                        "full_componentwise": oracle.componentwise_error(full, ref, ra),
                        "packed_componentwise": oracle.componentwise_error(
                            packed, np.concatenate([ref[s_, int(j):] for s_, j in enumerate(sel)]),
                            np.concatenate([ra[s_, int(j):] for s_, j in enumerate(sel)])),
                        "gate": "<= 1e-5 componentwise (FP64 oracle)"}
    except Exception as e:
        out["error"] = {"error": repr(e)}
    return out


def batch_row(torch, sg, dev, flush, stream, hbm_peak, count=4096, per_row=16, seed=3):
    """4,096 independent symmetric matrices, n log-uniform on [256, 65536], 16 draws per row."""
    import tempfile
    sizes = synth.batch_sizes(count, 256, 65536, seed)
    t0 = time.perf_counter()
    batch = sg.make_batch(sizes, per_row, seed)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    rows = int(batch.host_row_off[-1])
    nnz = int(batch.col.numel())
    x = torch.from_numpy(synth.vector_uniform(rows, seed)).to(dev)
    y = torch.empty_like(x)
    sy = torch.empty(count, dtype=torch.float64, device=dev)
    cache = os.path.join(tempfile.gettempdir(), "symgpu_tune.txt")
    t0 = time.perf_counter()
    cfg, tuned_ms = sg.autotune_batch(batch, x, y, sy, cache_path=cache)
    tune_s = time.perf_counter() - t0
    plan = sg.BatchPlan(batch, cfg)
    plan.capture(x, y, sy)
    for _ in range(3):
        plan.launch()
    t = timed_steps(torch, plan.launch, 10, flush, stream)
    ms = float(np.mean(t))
    banded = cfg.band_rows > 0
    kname = "ssymv_band" if banded else "ssymv_batch"
    # the kernel alone: plain (non-graph) runs with per-launch events, L2 flushed before each
    sg.profile_reset()
    sg.profile_enable(True)
    timed_steps(torch, lambda: plan.run(x, y, sy), 5, flush, stream)
    sg.profile_enable(False)
    kern = sg.profile_read().get(kname, (1, 0.0))
    # algorithmic bytes of what the timed kernels read and write: tile path: col + val, rowptr, x, y zeroed
    # then reduced, SYPRD; banded path: the packed (row, col) + value copy, x, y zeroed then written / reduced
    if banded:
        alg = nnz * 8 + rows * 4 * 3 + count * 8
    else:
        alg = nnz * 8 + (rows + count) * 8 + rows * 4 * 3 + count * 8
    kern_ms = kern[1] / max(kern[0], 1)
    out = {"instances": count, "rows": rows, "upper_nnz": nnz, "generate_s": gen_s, "autotune_s": tune_s,
           "tile_cfg": cfg.as_dict(), "path": "banded" if banded else "tiles", "graph_ms": ms,
           "canonical_nnz_per_s": nnz / (ms * 1e-3), "algorithmic_bytes": alg,
           "effective_gbs": alg / (ms * 1e-3) / 1e9, "hbm_frac": alg / (ms * 1e-3) / 1e9 / hbm_peak,
           "kernel": kname, "kernel_ms": kern_ms}
    # plain form: one sym_spmv launch per instance (each with its own upper CSR, local indices)
    ro = batch.host_row_off
    rp_h = batch.rowptr.cpu()
    views = []
    for b in range(count):
        r0, r1 = int(ro[b]), int(ro[b + 1])
        p0, p1 = int(rp_h[r0]), int(rp_h[r1])
        rp = (batch.rowptr[r0:r1 + 1] - p0).to(torch.int32)
        cl = batch.col[p0:p1] - r0
        views.append((r1 - r0, rp, cl, batch.val[p0:p1], x[r0:r1], y[r0:r1]))
    sy2 = torch.empty(count, dtype=torch.float64, device=dev)
    wss = [sg.spmv_workspace(v[0], v[1], v[2], v[3]) for v in views]

    def plain():
        for b, (n_b, rp, cl, vl, xb, yb) in enumerate(views):
            sg.spmv(n_b, rp, cl, vl, xb, y=yb, syprd=False, ws=wss[b])
    plain()
    tp = timed_steps(torch, plain, 3, flush, stream)
    out["one_launch_per_instance_ms"] = float(np.mean(tp))
    out["speedup_over_one_launch_per_instance"] = float(np.mean(tp)) / ms
    # full-size parity on sampled instances (the oracle computes them one by one)
    import oracle
    plan.launch()
    torch.cuda.synchronize()
    yh, sh = y.cpu().numpy(), sy.cpu().numpy()
    xh = x.cpu().numpy()
    worst_y, worst_s = 0.0, 0.0
    for b in list(range(0, count, max(1, count // 12)))[:12]:
        r0, r1 = int(ro[b]), int(ro[b + 1])
        p0, p1 = int(rp_h[r0]), int(rp_h[r1])
        rp = (rp_h[r0:r1 + 1] - p0).numpy().astype(np.int32)
        cl = (batch.col[p0:p1] - r0).cpu().numpy().astype(np.int32)
        vl = batch.val[p0:p1].cpu().numpy()
        yr, ya = oracle.ssymv(r1 - r0, rp, cl, vl, xh[r0:r1].astype(np.float64))
        sr, sa = oracle.syprd(r1 - r0, rp, cl, vl, xh[r0:r1].astype(np.float64))
        worst_y = max(worst_y, oracle.componentwise_error(yh[r0:r1], yr, ya))
        worst_s = max(worst_s, abs(sh[b] - sr) / sa if sa > 0 else 0.0)
    out["sampled_parity"] = {"instances": 12, "ssymv_componentwise": worst_y, "syprd_componentwise": worst_s}
    plan.close()
    return out


def serving_row(torch, sg, dev, requests=20000, rate=2000.0, pool_size=32, seed=4, affinity_s=1.0, pool_frac=0.6):
    """Poisson arrivals of MTTKRP requests; continuous batching vs one launch per request (FP32).

    Run 1: the tensors are resident (created by the caller) under the 120 GB budget; small requests are
    grouped.  Run 2: the same trace over registered tensor images with a device pool smaller than the set, so
    the server loads tensors on demand and evicts the least recently used ones (host images are the master
    copy); requests for resident tensors go first, a request needing a load waits up to `affinity_s`.  A
    request whose factor an earlier request used declares it unchanged (residual=2): the server reuses that
    factor's cached Gram matrix for the residual.  Latency is t_done - t_arrival (host steady clock); 'steady' statistics use the second half of the
    trace only."""
    import threading
    st = synth.Stream(seed, tag=77)
    orders = np.where(st.uniform(pool_size) < 0.6, 3, np.where(st.uniform(pool_size) < 0.75, 4, 5))
    ns = np.rint(np.exp(math.log(1e3) + st.uniform(pool_size) * math.log(200.0))).astype(np.int64)
    nnzs = np.rint(np.exp(math.log(1e4) + st.uniform(pool_size) * math.log(5000.0))).astype(np.int64)
    pool = []
    t0 = time.perf_counter()
    for k in range(pool_size):
        idx, val = sg.gen_coords(int(orders[k]), int(ns[k]), int(nnzs[k]), seed * 1000 + k)
        X = sg.SymTensor(idx, val, int(ns[k]), dup=sg.DUP_KEEP_EQUAL)
        del idx, val
        pool.append(X)
    torch.cuda.synchronize()
    pool_s = time.perf_counter() - t0
    ranks = [8, 16, 32, 64]
    facs = {}
    for k, X in enumerate(pool):
        for R in ranks:
            B = torch.randn((X.n, R), device=dev, generator=torch.Generator(device=dev).manual_seed(k * 7 + R))
            B /= math.sqrt(R)
            facs[(k, R, "f32")] = B
            facs[(k, R, "bf16")] = B.to(torch.bfloat16)
    # trace
    gaps = -np.log(st.uniform_open0(requests)) / rate
    arrive = np.cumsum(gaps)
    which = (st.uniform(requests) * pool_size).astype(np.int64)
    rsel = np.array(ranks)[(st.uniform(requests) * 4).astype(np.int64)]
    dts = np.where(st.uniform(requests) < 0.5, "bf16", "f32")
    work_nnz = float(sum(pool[w].nnz for w in which))
    # residual=2 once a factor has been used by an earlier request of the trace (its Gram matrix may be reused)
    seen, res_flag = set(), []
    for i in range(requests):
        key = (int(which[i]), int(rsel[i]), str(dts[i]))
        res_flag.append(2 if key in seen else True)
        seen.add(key)
    # one output buffer per (tensor, rank), shared by that pair's requests: the trace is timed, not checked (the
    # results of the serving paths are checked in the tests)
    outs = {(k, R): torch.empty((pool[k].n, R), device=dev) for k in range(pool_size) for R in ranks}
    half = requests // 2

    def summarize(lat, span, done_pc):
        lat = np.asarray(lat)
        srt = np.sort(lat)
        tail = np.sort(lat[half:])
        # steady state: throughput over the second half of the trace (arrivals and completions both inside it)
        span2 = max(done_pc[half:]) - (arrive[half] + base_ref[0])
        return {"p50_ms": float(np.percentile(srt, 50) * 1e3), "p99_ms": float(np.percentile(srt, 99) * 1e3),
                "throughput_req_per_s": requests / span, "canonical_nnz_per_s": work_nnz / span,
                "steady_second_half": {"p50_ms": float(np.percentile(tail, 50) * 1e3),
                                       "p99_ms": float(np.percentile(tail, 99) * 1e3),
                                       "throughput_req_per_s": (requests - half) / max(span2, 1e-9)}}

    base_ref = [0.0]
    t_ref_ns = time.monotonic_ns()
    t_ref_pc = time.perf_counter()
    to_pc = lambda ns_: t_ref_pc + (ns_ - t_ref_ns) * 1e-9

    def serve(S, submit):
        tickets = [None] * requests
        base = time.perf_counter() + 0.05
        base_ref[0] = base

        def submitter():
            for i in range(requests):
                while time.perf_counter() < base + arrive[i]:
                    pass
                tickets[i] = submit(S, i)
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        done_ns = []
        for i in range(requests):
            r = S.wait(tickets[i], 300.0)
            assert r["status"] == 0
            done_ns.append(r["t_done_ns"])
        done_pc = [to_pc(d) for d in done_ns]
        lat = [done_pc[i] - (base + arrive[i]) for i in range(requests)]
        span = max(done_pc) - base
        return summarize(lat, span, done_pc)

    # run 1: resident tensors, 120 GB budget, small requests grouped
    S = sg.Server(max_slots=8, max_rank=64, hbm_budget_bytes=120 << 30, small_nnz=1_000_000, coalesce_small=True)
    cb = serve(S, lambda S_, i: S_.submit(pool[which[i]], facs[(int(which[i]), int(rsel[i]), dts[i])],
                                          outs[(int(which[i]), int(rsel[i]))], residual=res_flag[i], tag=i))
    cb["server_stats"] = S.stats()
    S.close()
    # run 2: registered images, device pool at 60 % of the images' total: loads and LRU evictions
    images = [X.save_image() for X in pool]
    image_bytes = sum(int(sg.lib().sym_tensor_load_bytes(sg.C.c_void_p(im.data_ptr()))) for im in images)
    pool_bytes = int(image_bytes * pool_frac)
    S = sg.Server(max_slots=8, max_rank=64, hbm_budget_bytes=pool_bytes + (16 << 30), small_nnz=1_000_000,
                  coalesce_small=True, pool_bytes=pool_bytes, affinity_wait_s=affinity_s)
    ids = [S.register(im) for im in images]
    ev = serve(S, lambda S_, i: S_.submit_registered(ids[which[i]], facs[(int(which[i]), int(rsel[i]), dts[i])],
                                                    outs[(int(which[i]), int(rsel[i]))], residual=res_flag[i], tag=i))
    ev["server_stats"] = S.stats()
    ev["pool_bytes"] = pool_bytes
    ev["registered_image_bytes"] = image_bytes
    ev["hbm_budget_bytes"] = pool_bytes + (16 << 30)
    ev["affinity_wait_ms"] = affinity_s * 1e3
    S.close()
    del images
    # plain: one launch per request on one stream, FP32 factors, in arrival order (first 4,000 requests)
    n_plain = min(requests, 4000)
    torch.cuda.synchronize()
    base = time.perf_counter() + 0.05
    lat2 = []
    for i in range(n_plain):
        while time.perf_counter() < base + arrive[i]:
            pass
        X = pool[which[i]]
        X.mttkrp(facs[(int(which[i]), int(rsel[i]), "f32")], M=outs[(int(which[i]), int(rsel[i]))], residual=True)
        torch.cuda.synchronize()
        lat2.append(time.perf_counter() - (base + arrive[i]))
    span2 = time.perf_counter() - base
    lat2 = np.sort(np.asarray(lat2))
    plain_nnz = float(sum(pool[w].nnz for w in which[:n_plain]))
    plain = {"requests": n_plain, "p50_ms": float(np.percentile(lat2, 50) * 1e3),
             "p99_ms": float(np.percentile(lat2, 99) * 1e3), "throughput_req_per_s": n_plain / span2,
             "canonical_nnz_per_s": plain_nnz / span2}
    pool_nnz = int(sum(X_.nnz for X_ in pool))
    for X in pool:
        X.close()
    return {"requests": requests, "rate_req_per_s": rate, "pool": {"tensors": pool_size, "build_s": pool_s,
            "canonical_nnz": pool_nnz, "orders": [int(o) for o in orders]},
            "offered_canonical_nnz_per_s": work_nnz / arrive[-1],
            "continuous_batching": cb, "registered_pool_with_eviction": ev, "one_launch_per_request_f32": plain}


def devloop_row(torch, sg, dev, requests=20000, rate=20000.0, seed=5):
    """Poisson arrivals of small requests (70 % MTTKRP of orders 3/4/5 with ranks 8-64, half BF16 factors;
    30 % SSYMV + SYPRD) served three ways on the same trace: the device-resident loop (one persistent kernel,
    requests published into mapped memory), one launch per request (synchronised before the next), and, for
    the MTTKRP requests of the trace alone, the host-scheduled continuous-batching server next to the device
    loop.  Latency is completion - arrival on the host steady clock (the loop's completion time is its
    kernel's %globaltimer stamp, calibrated against that clock); 'steady' statistics use the second half."""
    import threading
    st = synth.Stream(seed, tag=91)
    n_t, n_m = 12, 8
    orders = np.where(st.uniform(n_t) < 0.5, 3, np.where(st.uniform(n_t) < 0.7, 4, 5))
    ns = np.rint(np.exp(math.log(500.0) + st.uniform(n_t) * math.log(40.0))).astype(np.int64)
    nnzs = np.rint(np.exp(math.log(2e3) + st.uniform(n_t) * math.log(50.0))).astype(np.int64)
    tensors = []
    for k in range(n_t):
        idx, val = sg.gen_coords(int(orders[k]), int(ns[k]), int(nnzs[k]), seed * 100 + k)
        tensors.append(sg.SymTensor(idx, val, int(ns[k]), dup=sg.DUP_KEEP_EQUAL))
    mats = []
    for k in range(n_m):
        n = int(round(math.exp(math.log(1e3) + float(st.uniform(1)[0]) * math.log(100.0))))
        A = synth.upper_csr_rowdegree(n, 8.0 + 24.0 * float(st.uniform(1)[0]), seed * 100 + 50 + k)
        x = synth.vector_uniform(n, seed * 100 + 50 + k)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        mats.append((n, t(A.rowptr), t(A.col), t(A.val), t(x), int(A.col.shape[0])))
    ranks = [8, 16, 32, 64]
    facs = {}
    for k, X in enumerate(tensors):
        for R in ranks:
            B = torch.randn((X.n, R), device=dev, generator=torch.Generator(device=dev).manual_seed(k * 7 + R))
            B /= math.sqrt(R)
            facs[(k, R, "f32")] = B
            facs[(k, R, "bf16")] = B.to(torch.bfloat16)
    outs = {(k, R): torch.empty((tensors[k].n, R), device=dev) for k in range(n_t) for R in ranks}
    youts = [(torch.empty(m[0], device=dev), torch.empty(1, dtype=torch.float64, device=dev)) for m in mats]
    gaps = -np.log(st.uniform_open0(requests)) / rate
    arrive = np.cumsum(gaps)
    is_mt = st.uniform(requests) < 0.7
    which_t = (st.uniform(requests) * n_t).astype(np.int64)
    which_m = (st.uniform(requests) * n_m).astype(np.int64)
    rsel = np.array(ranks)[(st.uniform(requests) * 4).astype(np.int64)]
    dts = np.where(st.uniform(requests) < 0.5, "bf16", "f32")
    torch.cuda.synchronize()
    t_ref_ns, t_ref_pc = time.monotonic_ns(), time.perf_counter()
    to_pc = lambda ns_: t_ref_pc + (ns_ - t_ref_ns) * 1e-9

    def summarize(lat, span, done_pc, base, arr):
        lat = np.asarray(lat)
        m = len(lat)
        h = m // 2
        span2 = max(done_pc[h:]) - (arr[h] + base)
        return {"requests": m, "p50_us": float(np.percentile(lat, 50) * 1e6),
                "p99_us": float(np.percentile(lat, 99) * 1e6), "throughput_req_per_s": m / span,
                "steady_second_half": {"p50_us": float(np.percentile(lat[h:], 50) * 1e6),
                                       "p99_us": float(np.percentile(lat[h:], 99) * 1e6),
                                       "throughput_req_per_s": (m - h) / max(span2, 1e-9)}}

    def submit_dl(L, i):
        if is_mt[i]:
            k, R = int(which_t[i]), int(rsel[i])
            return L.submit_mttkrp(tensors[k], facs[(k, R, str(dts[i]))], outs[(k, R)], tag=i)
        m = mats[which_m[i]]
        y, s = youts[which_m[i]]
        return L.submit_ssymv(m[0], m[1], m[2], m[3], m[4], y, s, tag=i)

    def serve(obj, submit, sel):
        arr = arrive[sel]
        tickets = [None] * len(sel)
        base = time.perf_counter() + 0.05

        def submitter():
            for j, i in enumerate(sel):
                while time.perf_counter() < base + arr[j]:
                    pass
                tickets[j] = submit(obj, i)
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        done_pc = []
        for tk in tickets:
            r = obj.wait(tk, 300.0)
            assert r["status"] == 0
            done_pc.append(to_pc(r["t_done_ns"]))
        lat = [done_pc[j] - (base + arr[j]) for j in range(len(sel))]
        return summarize(lat, max(done_pc) - base, done_pc, base, arr)

    everything = np.arange(requests)
    only_mt = np.nonzero(is_mt)[0]
    L = sg.DevLoop(ring_slots=1024, idle_exit_s=0.002)
    dl = serve(L, submit_dl, everything)
    dl["loop_stats"] = L.stats()
    L.close()
    # one launch per request, synchronised before the next, in arrival order (FP32 and BF16 as in the trace)
    torch.cuda.synchronize()
    base = time.perf_counter() + 0.05
    lat, done = [], []
    ws = {}
    for i in everything:
        while time.perf_counter() < base + arrive[i]:
            pass
        if is_mt[i]:
            k, R = int(which_t[i]), int(rsel[i])
            tensors[k].mttkrp(facs[(k, R, str(dts[i]))], M=outs[(k, R)])
        else:
            j = int(which_m[i])
            m = mats[j]
            if j not in ws:
                ws[j] = sg.spmv_workspace(m[0], m[1], m[2], m[3])
            sg.spmv(m[0], m[1], m[2], m[3], m[4], y=youts[j][0], syprd=True, ws=ws[j])
        torch.cuda.synchronize()
        done.append(time.perf_counter())
        lat.append(done[-1] - (base + arrive[i]))
    plain = summarize(lat, max(done) - base, done, base, arrive)
    # the MTTKRP requests alone: host-scheduled server (grouped small requests) and the device loop
    S = sg.Server(max_slots=8, max_rank=64, hbm_budget_bytes=120 << 30, small_nnz=1_000_000, coalesce_small=True)
    srv = serve(S, lambda S_, i: S_.submit(tensors[which_t[i]], facs[(int(which_t[i]), int(rsel[i]), str(dts[i]))],
                                           outs[(int(which_t[i]), int(rsel[i]))], residual=False, tag=i), only_mt)
    srv["server_stats"] = S.stats()
    S.close()
    L = sg.DevLoop(ring_slots=1024, idle_exit_s=0.002)
    dl_mt = serve(L, submit_dl, only_mt)
    L.close()
    work = {"tensors": n_t, "orders": [int(o) for o in orders], "tensor_canonical_nnz": [X.nnz for X in tensors],
            "matrices": n_m, "matrix_n": [m[0] for m in mats], "matrix_nnz": [m[5] for m in mats]}
    for X in tensors:
        X.close()
    return {"requests": requests, "rate_req_per_s": rate, "mttkrp_share": float(is_mt.mean()), "pool": work,
            "device_loop": dl, "one_launch_per_request": plain,
            "mttkrp_only": {"requests": int(only_mt.size), "device_loop": dl_mt, "host_scheduled_server": srv}}


def run_devloop_only(args):
    """The device-resident serving row alone."""
    import torch

    import paper_2406_09266_gb300 as sg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sg.load()
    print(json.dumps({"mode": "devloop-only", "serving_device_loop_20000rps": devloop_row(torch, sg, dev)}))


def run_batch_only(args):
    """Profiling mode for the batched SSYMV: one fixed shape (--batch-cfg), plain runs (no graph)."""
    import torch

    import paper_2406_09266_gb300 as sg
    sg.load()
    dev = torch.device("cuda")
    sizes = synth.batch_sizes(args.batch_only, 256, 65536, 3)
    batch = sg.make_batch(sizes, 16, 3)
    x = torch.from_numpy(synth.vector_uniform(int(batch.host_row_off[-1]), 3)).to(dev)
    y = torch.empty_like(x)
    sy = torch.empty(len(sizes), dtype=torch.float64, device=dev)
    cfg = [int(v) for v in args.batch_cfg.split(",")] if args.batch_cfg else [256, 8, 256, 8, 0, 0, 0]
    plan = sg.BatchPlan(batch, sg.TileCfg(*cfg))
    for _ in range(args.warmup + args.steps):
        plan.run(x, y, sy)
    torch.cuda.synchronize()
    plan.check()
    print(json.dumps({"mode": "batch-only (profiling)", "instances": len(sizes), "upper_nnz": int(batch.col.numel()),
                      "tile_cfg": cfg}))


def run_ttm_only(args):
    """Profiling mode for the symmetric TTM row (3-way uniform, n = 2,000, 5M entries, R = 32): the packed
    and full layouts with the default schedule (leaf-index second pass), `--steps` times each."""
    import torch

    import paper_2406_09266_gb300 as sg
    sg.load()
    dev = torch.device("cuda")
    n, rank = 2000, 32
    T = synth.make_tensor(3, n, 5_000_000, 3, "uniform")
    X = sg.SymTensor(torch.from_numpy(T.idx).to(dev), torch.from_numpy(T.val).to(dev), n)
    X.add_leaf_index()
    B = torch.from_numpy(synth.factor_normal(n, rank, 3)).to(dev)
    Cp = torch.empty((n * (n + 1) // 2, rank), dtype=torch.float32, device=dev)
    Cf = torch.empty((n, n, rank), dtype=torch.float32, device=dev)
    for _ in range(args.warmup + args.steps):
        X.ttm(B, "packed", C_out=Cp)
        X.ttm(B, "full", C_out=Cf)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "ttm-only (profiling)", "canonical_nnz": X.info()["nnz"], "rank": rank}))


def run_ptensor_only(args):
    """The partially symmetric MTTKRP row alone (also the profiling entry for its kernel)."""
    import torch

    import paper_2406_09266_gb300 as sg
    sg.load()
    dev = torch.device("cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    hbm_peak, _ = peaks()
    out = ptensor_row(torch, sg, dev, flush, torch.cuda.current_stream(), hbm_peak)
    print(json.dumps({"mode": "ptensor-only", "pmttkrp_parts22_n20k_nnz5M_r32": out}))


def run_small_only(args):
    import torch

    import paper_2406_09266_gb300 as sg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sg.load()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = small_ssymv_row(torch, sg, dev, flush, torch.cuda.current_stream(), K=args.steps)
    print(json.dumps({"mode": "small-only", "ssymv_n2000_nnz20k": out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", default="all", choices=["main", "all"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--kernel-only", action="store_true",
                    help="profiling mode: setup, warm-up and the timed steps only (no e2e or extra rows), with "
                         "the MTTKRP configuration fixed instead of autotuned")
    ap.add_argument("--mttkrp-cfg", default="", metavar="FIELDS",
                    help="kernel-only mode: comma-separated name=value sym_mttkrp_cfg fields that replace the "
                         "default fixed configuration (leaf_index=1 also builds the leaf index)")
    ap.add_argument("--ttm-only", action="store_true",
                    help="profiling mode: the symmetric TTM kernels on the TTM row's tensor, nothing else")
    ap.add_argument("--ptensor-only", action="store_true",
                    help="profiling mode: the partially symmetric MTTKRP row alone")
    ap.add_argument("--small-only", action="store_true",
                    help="profiling mode: the 2,000 x 2,000 SSYMV + SYPRD row alone")
    ap.add_argument("--devloop-only", action="store_true",
                    help="the device-resident serving row alone")
    ap.add_argument("--batch-only", type=int, default=0, metavar="INSTANCES",
                    help="profiling mode: build a batch of this many instances and run the batched SSYMV a few times")
    ap.add_argument("--batch-cfg", default="", metavar="FIELDS",
                    help="batch-only mode: comma-separated sym_tile_cfg fields (default: the tile kernel, 256 rows)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.batch_only:
        run_batch_only(args)
    elif args.ttm_only:
        run_ttm_only(args)
    elif args.ptensor_only:
        run_ptensor_only(args)
    elif args.small_only:
        run_small_only(args)
    elif args.devloop_only:
        run_devloop_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
