"""Benchmark of the GB300 adaptive 2-D FMM (complex-log potential).

One step = one pass of the whole hot path on one batch of synthetic input:
fmm_build_tree (tree + interaction lists) followed by fmm_evaluate (P2M,
M2M, M2L, L2L, L2P, P2P), inputs already resident in HBM.  The workload is
the 1e6-point cluster mixture (16 Gaussian clusters, sigma log-uniform in
[1e-3, 1e-1], 10 % uniform background, complex strengths), p = 24,
theta = 0.5, at most 64 particles per leaf.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (rank 0 only).  Multi-GPU runs are independent replicas (one per
rank, weak scaling); the method has no data exchange between ranks here.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "FMM particles/s at N=1e6, rel err <=1e-10: mixed/batched vs FP64 GPU path"
UNIT = "particles/s"
WORKLOAD = "clusters_1e6"
WORKLOAD_DESCS = {
    "clusters_1e6": ("cluster mixture: N=1e6 sources evaluated at the sources, 16 Gaussian "
                     "clusters (centres U[0,1]^2, sigma log-uniform [1e-3,1e-1]) + 10% uniform "
                     "background, complex q (re, im U[-1,1]), p=24, theta=0.5, leaf<=64"),
    "curve_4e6": ("curve: N=4e6 sources evaluated at the sources on the curve "
                  "r(t)=0.4+0.1 cos 7t about (0.5,0.5), jitter N(0,1e-4), real q ~ N(0,1), "
                  "theta=0.5, leaf<=64"),
    "clusters_1p6e7_targets": ("separate targets: N=1.6e7 cluster-mixture sources, M=1.6e7 "
                               "uniform evaluation points, complex q, p=30, theta=0.5, leaf<=64"),
    "uniform_45x2p16": ("the paper's time-breakdown case (Sec. 5.1): N=45*2^16 uniform points, "
                        "complex q, p=17, theta=0.5, leaf<=45 (run with --kernel harmonic for "
                        "the paper's kernel)"),
}
WORKLOAD_DESC = WORKLOAD_DESCS[WORKLOAD]

# Measured on a GB300 (FMA-chain probe, 152 SMs at ~2.0 GHz).
FP64_PEAK_GFLOPS = 1190.0
FP32_PEAK_GFLOPS = 69600.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ CPU oracle arm

def cpu_info():
    """Host CPU model and core counts (recorded beside every CPU timing)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"model": model or platform.machine(), "nproc": os.cpu_count(), "usable": usable}


def oracle_sample_run(src, q, p, leaf, n_sample, seed=0, shortcut=False, box_fit=False,
                      threads=1):
    """The oracle on a bounded sample of the workload: the full tree, lists and
    expansion phases, then L2P + P2P at n_sample random evaluation points.
    `threads` spreads the oracle's independent per-target loops (M2L per
    target box, L2P + P2P per point) over that many threads; the tree, the
    lists, P2M, M2M, L2L and P2L stay serial.  Returns (extrapolated seconds
    for all N points, details, phi_sample, sample, tree, lists, shortcut lists
    or None)."""
    import oracle as O
    O.set_threads(threads)
    n = len(src)
    sample = np.sort(np.random.default_rng(seed).choice(n, n_sample, replace=False))
    t0 = time.perf_counter()
    L = O.levels_cap(n, leaf)
    tree = O.build_tree(src, L)
    if box_fit:
        tree = O.shrink(tree, src)
    t1 = time.perf_counter()
    lists = O.connect(tree)
    sc = O.leaf_shortcut(tree, lists) if shortcut else None
    t2 = time.perf_counter()
    secs = np.zeros(2)
    phi = O.evaluate(tree, lists, src, q, p, sample=sample, seconds=secs, shortcut=sc)
    t3 = time.perf_counter()
    per_point = secs[1] / n_sample
    total = (t1 - t0) + (t2 - t1) + secs[0] + per_point * n
    O.set_threads(1)
    det = dict(tree_s=t1 - t0, connect_s=t2 - t1, expansions_s=float(secs[0]),
               points_s=float(secs[1]), wall_s=t3 - t0, threads=threads,
               full_n_s=total)
    return total, det, phi, sample, tree, lists, sc


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    src, q, _ = W.make(WORKLOAD)
    n = len(src)
    p, leaf = args.p, args.leaf
    cpu = cpu_info()
    threads = cpu["usable"]
    n_sample = args.ref_arm_sample
    for _ in range(args.warmup):
        oracle_sample_run(src, q, p, leaf, n_sample, shortcut=bool(args.p2l_m2p),
                          box_fit=bool(args.box_fit), threads=threads)
    times, walls = [], []
    for k in range(args.steps):
        tot, det = oracle_sample_run(src, q, p, leaf, n_sample, seed=k,
                                     shortcut=bool(args.p2l_m2p),
                                     box_fit=bool(args.box_fit), threads=threads)[:2]
        times.append(tot)
        walls.append(det["wall_s"])
    mean = sum(times) / len(times)
    value = n / mean
    sample_desc = (f"per step: full tree, lists and expansion phases of the N=1e6 workload, then "
                   f"L2P+P2P at {n_sample} random points; the rate is N over the step's time "
                   f"with the per-point time scaled to all N points; {threads} threads "
                   f"(OpenMP over M2L target boxes and evaluation points), {cpu['model']}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # the wall time of the sampled steps that ran; the full-N time is extrapolated
        "ms_per_step": statistics.mean(walls) * 1e3,
        "ms_per_step_full_n_extrapolated": mean * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "precision": "fp64", "p": args.p,
                   "leaf_shortcut": bool(args.p2l_m2p),
                   "box_geometry": ("bounding rectangles of the points" if args.box_fit
                                    else "split rectangles")},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample_desc, "cpu": cpu},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s_timed": sum(walls),
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def pair_count(ex, sc=None):
    """Near-field pair evaluations per evaluate (from the exported topology;
    with the leaf shortcut, from its near lists)."""
    nb = ex["n_boxes"]
    L = ex["levels"]
    base = (4 ** L - 1) // 3
    cnt_s = ex["box_src"][:, 1]
    cnt_t = ex["box_tgt"][:, 1]
    so = ex["strong_off"] if sc is None else sc["near_off"]
    st = ex["strong"] if sc is None else sc["near"]
    near = np.add.reduceat(cnt_s[st], so[base:nb]) if len(st) else np.zeros(nb - base)
    empty = so[base + 1:nb + 1] == so[base:nb]
    near = np.where(empty, 0, near)
    return int(np.sum(cnt_t[base:nb] * near))


def self_pair_count(ex):
    """Pair evaluations inside the leaves (a leaf with n points: n (n - 1))."""
    L = ex["levels"]
    base = (4 ** L - 1) // 3
    n = ex["box_src"][base:, 1].astype(np.int64)
    return int(np.sum(n * (n - 1)))


# FP32-pipe operations per near-field pair of the mixed P2P kernel, counted from
# its source (df32 difference 22, |D|^2 and checks 14, log 44, atan2 59,
# corrections 16, complex multiply-accumulate 50, loop and loads 10)
MIXED_OPS_PER_PAIR = 215
# FP64 flops per pair of the FP64 P2P by convention: difference 2, |d|^2 3,
# log 20, atan2 24, complex multiply-accumulate 8
FP64_FLOPS_PER_PAIR = 57
FP32_PEAK_TOPS = FP32_PEAK_GFLOPS / 2e3   # one FMA = one FP32-pipe operation
# The FP64 symmetric kernel's reverse term: one more complex multiply-accumulate
# (8 flops) and the i pi shift (1 add) per unordered pair (pairs of distinct
# leaves and, by the cyclic schedule, pairs within one leaf).
FP64_SYM_EXTRA_FLOPS = 9
# The symmetric kernel (self-evaluation) evaluates each unordered pair of
# points once (pairs of distinct leaves, and within a leaf by a cyclic
# schedule) and adds the reverse term: a second complex multiply-accumulate
# (50 ops) and the i pi shift with its sign (10 ops: three comparisons, two
# selects, a Fast2Sum and two additions).
SYM_EXTRA_OPS_PER_PAIR = 60
# Harmonic kernel, per pair, counted from the source in the same way: df32
# difference 22, |D|^2 and checks 14, df32 complex reciprocal 36, sign 4,
# complex multiply-accumulate 46, loop and loads 10; the reverse term adds a
# second multiply-accumulate and the shared-memory round trip (48).
HARM_OPS_PER_PAIR = 132
HARM_SYM_EXTRA_OPS_PER_PAIR = 48
# DRAM bytes (read + write) of one k_p2p_sym<0> launch per source point, from
# an ncu capture of the cluster workload scaled to N = 2.5e5 (8,520,704 B read
# + 6,912 B written).  The kernel reads
# each point's df32 offsets and strengths (32 B) once from DRAM; its partial
# sums stay in L2.  Scaled by N for the full launch; valid while the kernel is
# unchanged since that capture, and for the cluster workload it was taken on.
P2P_SYM_DRAM_BYTES_PER_POINT = (8_520_704 + 6_912) / 250_000


def roofline(prec_mixed, pairs, p2p_ms, self_pairs=None, harmonic=False, n_points=None,
             clusters=False):
    per_pair = HARM_OPS_PER_PAIR if harmonic else MIXED_OPS_PER_PAIR
    extra = HARM_SYM_EXTRA_OPS_PER_PAIR if harmonic else SYM_EXTRA_OPS_PER_PAIR
    if prec_mixed and self_pairs is not None:
        # every unordered pair once: the pairs of distinct leaves' points and,
        # by the cyclic schedule, the pairs within one leaf
        cross = (pairs - self_pairs) // 2
        unordered = cross + self_pairs // 2
        ops = unordered * (per_pair + extra)
        achieved = ops / (p2p_ms * 1e-3) / 1e12
        traffic = (round(P2P_SYM_DRAM_BYTES_PER_POINT * n_points)
                   if n_points and clusters and not harmonic else None)
        return {"kernel": "k_p2p_sym (df32 P2P, each unordered pair of points once)",
                "bound": "alu", "achieved": achieved,
                "peak": FP32_PEAK_TOPS, "unit": "TOP/s (FP32-pipe operations)",
                "frac": achieved / FP32_PEAK_TOPS, "traffic": traffic,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                   "launch at N = 2.5e5 (same workload), scaled by N; "
                                   "algorithmic bytes 32 per point" if traffic else None),
                "ops_per_unordered_pair": per_pair + extra,
                "pairs_per_launch": pairs, "unordered_pairs": unordered,
                "unordered_pairs_within_leaves": self_pairs // 2,
                "gpairs_per_s": pairs / (p2p_ms * 1e-3) / 1e9, "launch_ms": p2p_ms,
                "peak_source": "measured FP32 FMA-chain probe on a GB300 "
                               "(69.6 TFLOP/s = 34.8 T FMA/s); not in MEASURED_PEAKS.json"}
    if prec_mixed:
        achieved = pairs * per_pair / (p2p_ms * 1e-3) / 1e12
        return {"kernel": "k_p2p_mixed (df32 P2P)", "bound": "alu", "achieved": achieved,
                "peak": FP32_PEAK_TOPS, "unit": "TOP/s (FP32-pipe operations)",
                "frac": achieved / FP32_PEAK_TOPS, "traffic": None,
                "ops_per_pair": per_pair, "pairs_per_launch": pairs,
                "gpairs_per_s": pairs / (p2p_ms * 1e-3) / 1e9, "launch_ms": p2p_ms,
                "peak_source": "measured FP32 FMA-chain probe on a GB300 "
                               "(69.6 TFLOP/s = 34.8 T FMA/s); not in MEASURED_PEAKS.json"}
    peak = FP64_PEAK_GFLOPS / 1e3
    if self_pairs is not None:
        unordered = (pairs - self_pairs) // 2 + self_pairs // 2
        flops = unordered * (FP64_FLOPS_PER_PAIR + FP64_SYM_EXTRA_FLOPS)
        achieved = flops / (p2p_ms * 1e-3) / 1e12
        return {"kernel": "k_p2p_sym64 (FP64 P2P, each unordered pair of points once)",
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s (FP64)",
                "frac": achieved / peak, "traffic": None,
                "flops_per_unordered_pair": FP64_FLOPS_PER_PAIR + FP64_SYM_EXTRA_FLOPS,
                "pairs_per_launch": pairs, "unordered_pairs": unordered,
                "unordered_pairs_within_leaves": self_pairs // 2,
                "gpairs_per_s": pairs / (p2p_ms * 1e-3) / 1e9, "launch_ms": p2p_ms,
                "peak_source": "measured FP64 FMA-chain probe on a GB300"}
    achieved = pairs * FP64_FLOPS_PER_PAIR / (p2p_ms * 1e-3) / 1e12
    return {"kernel": "k_p2p64 (FP64 P2P)", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s (FP64)", "frac": achieved / peak, "traffic": None,
            "flops_per_pair": FP64_FLOPS_PER_PAIR, "pairs_per_launch": pairs,
            "gpairs_per_s": pairs / (p2p_ms * 1e-3) / 1e9, "launch_ms": p2p_ms,
            "peak_source": "measured FP64 FMA-chain probe on a GB300"}


# Tensor-core M2L: per item of 128 weak pairs and per component (re, im), the
# MMA chains of the 5 fp16 digit slices A_j against the operator slices
# B_0 .. B_{5-j} (N = 32 (6 - j); the j = 0 chain includes the zero sixth
# slice): 6 + 5 + 4 + 3 + 2 = 20 products of 128 x 32 x 32 MACs.
M2L_TC_ITEM = 128
M2L_TC_PRODUCTS = 20


def m2l_roofline(mixed, tensor, n_weak, p, m2l_ms, peaks):
    """Useful work of M2L: the complex contraction with the binomial
    operator, 4 p (p + 1) real flops per weak pair (plus the scalings, not
    counted).  Mixed tensor path: also the executed tensor flops of the digit
    slices, against the measured bf16/fp16 dense peak; FP64 path: the FP64
    peak."""
    useful = n_weak * 4.0 * p * (p + 1)
    if mixed and tensor:
        items = -(-n_weak // M2L_TC_ITEM)
        executed = items * 2 * M2L_TC_PRODUCTS * 2.0 * 128 * 32 * 32
        peak = peaks.get("bf16_tflops")
        src = "MEASURED_PEAKS.json bf16_tflops (burst; fp16 runs at the bf16 rate)"
        if not peak:
            peak, src = 1900.0, "fallback 1.9 PFLOP/s bf16"
        return {"kernel": "k_m2l_tc (fp16 digit slices on tcgen05)", "bound": "tensor",
                "launch_ms": m2l_ms, "weak_pairs": n_weak,
                "useful_tflops": useful / (m2l_ms * 1e-3) / 1e12,
                "executed_tflops": executed / (m2l_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": src,
                "useful_frac": useful / (m2l_ms * 1e-3) / 1e12 / peak,
                "executed_frac": executed / (m2l_ms * 1e-3) / 1e12 / peak,
                "useful_flops_per_pair": 4 * p * (p + 1),
                "executed_flops_per_item": executed / max(items, 1)}
    peak = FP64_PEAK_GFLOPS / 1e3
    return {"kernel": "k_m2l (FP64)" if not mixed else "k_m2l_mixed (df32 sweeps)",
            "bound": "alu", "launch_ms": m2l_ms, "weak_pairs": n_weak,
            "useful_tflops": useful / (m2l_ms * 1e-3) / 1e12,
            "peak": peak if not mixed else FP32_PEAK_TOPS * 2,
            "unit": "TFLOP/s", "useful_frac": useful / (m2l_ms * 1e-3) / 1e12
            / (peak if not mixed else FP32_PEAK_TOPS * 2),
            "peak_source": "measured FP64 FMA-chain probe" if not mixed
            else "measured FP32 FMA-chain probe", "useful_flops_per_pair": 4 * p * (p + 1)}


def phase_bandwidth(ex, n, m, p, phases, peaks):
    """Achieved HBM bandwidth of the tree build and the translations from
    algorithmic bytes.  Tree: the bounding box reads 16 B per point, each of
    the 2L median-split rounds reads a key and an index (12 B) and writes an
    index (4 B) per point, and the final gather reads and writes the
    coordinates and writes the permutation (36 B).  P2M reads 32 B per point
    (coordinates, strengths) and writes each leaf's (p + 1) coefficients;
    M2M and L2L read and write (p + 1) complex coefficients per box."""
    L = ex["levels"]
    nb = ex["n_boxes"]
    nleaf = 4 ** L
    hbm = peaks.get("hbm_gbs") or 6800.0
    tree_bytes = n * (16 + 2 * L * 16 + 36) + (m - n if m != n else 0) * (16 + 36)
    coef = 16 * (p + 1)
    p2m_bytes = 32 * n + nleaf * coef
    m2m_bytes = 2 * nb * coef
    l2l_bytes = 2 * nb * coef
    out = {"hbm_peak_gbs": hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks.get(
        "hbm_gbs") else "fallback 6.8 TB/s"}
    for name, b, ms in (("tree", tree_bytes, phases["tree"]), ("p2m", p2m_bytes, phases["p2m"]),
                        ("m2m", m2m_bytes, phases["m2m"]), ("l2l", l2l_bytes, phases["l2l"])):
        gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else None
        out[name] = {"bytes": int(b), "ms": ms, "gbs": gbs,
                     "frac": gbs / hbm if gbs else None}
    return out


def max_over_ranks(total_ms, ws, device):
    """The slowest rank's timed total (every rank times the same amount of
    work); all ranks receive it."""
    if ws <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(points_per_rank, ws, ms_per_step):
    """Whole-job throughput: the points of all ranks over the slowest rank's
    step time."""
    return points_per_rank * ws / (ms_per_step * 1e-3)


def run_gpu(args, ws, rank, local):
    import torch

    import paper_1205_4611_gb300 as G

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    G.load()
    wl = args.workload
    full_n = W.WORKLOADS[wl]["n"]
    src_np, q_np, tgt_np = W.make(wl, scale=args.n / full_n if args.n else 1.0)
    n = len(src_np)
    m = len(tgt_np) if tgt_np is not None else n  # evaluation points
    src = torch.from_numpy(src_np).to(dev)
    q = torch.from_numpy(q_np).to(dev)
    tgt = torch.from_numpy(tgt_np).to(dev) if tgt_np is not None else None
    phi = torch.empty((m, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def options(precision):
        return G.fmm_default_options(
            p=args.p, leaf_size=args.leaf, level_shift=args.level_shift,
            precision=G.FMM_PREC_MIXED if precision == "mixed" else G.FMM_PREC_FP64,
            m2l_slices=args.m2l_slices if precision == "mixed" else 0,
            p2l_m2p=args.p2l_m2p, box_fit=args.box_fit,
            kernel=G.FMM_KERNEL_HARMONIC if args.kernel == "harmonic" else G.FMM_KERNEL_LOG)

    def measure(precision, steps, warmup, clocks=False, barrier=False):
        opt = options(precision)

        def step(timing=False):
            tree = G.fmm_build_tree(src, tgt, opt)
            if timing:
                G.fmm_set_timing(tree, True)
            G.fmm_evaluate(tree, q, phi)
            return tree

        for _ in range(warmup):
            t = step()
            G.fmm_tree_sync(t)
            t.free()
        t = step()  # topology facts for the roofline (untimed)
        G.fmm_tree_sync(t)
        ex = G.fmm_tree_export(t)
        sc = G.fmm_tree_export_shortcut(t) if args.p2l_m2p else None
        pairs = pair_count(ex, sc)
        # the library takes the symmetric near field in self-evaluation (both
        # precisions) when every leaf holds <= 64 points (ceil(N / 4^L) <= 64)
        sym = tgt is None and -(-n // 4 ** ex["levels"]) <= 64
        selfp = self_pair_count(ex) if sym else None
        if sc is not None:
            ex["n_near"], ex["n_p2l"], ex["n_m2p"] = len(sc["near"]), len(sc["p2l"]), len(sc["m2p"])
        t.free()
        sampler = ClockSampler(local) if clocks else None
        if barrier and ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        launches0 = G.fmm_launch_count()
        G.fmm_memory_info(reset_peak=True)
        step_ms = []
        for _ in range(steps):
            flush.zero_()  # L2 flush outside the timed events (inputs are 32 MB < L2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree = step()
            e1.record(stream)
            G.fmm_tree_sync(tree)
            step_ms.append(e0.elapsed_time(e1))
            tree.free()
        torch.cuda.synchronize()
        clk = sampler.stop() if sampler else None
        launches = G.fmm_launch_count() - launches0
        mem = G.fmm_memory_info()
        total_ms = sum(step_ms)
        if barrier:
            total_ms = max_over_ranks(total_ms, ws, dev)
        # the phase spans come from further steps with phase timing on, outside
        # the timed region: the library then runs the phases one after another
        # (in the timed steps the far field overlaps the near field), so that
        # each span measures its own kernels
        eval_ms = []
        for _ in range(max(1, min(steps, 5))):
            flush.zero_()
            tree = step(timing=True)
            G.fmm_tree_sync(tree)
            eval_ms.append(G.fmm_get_timings(tree))
            tree.free()
        phases = {k: statistics.mean(d[k] for d in eval_ms) for k in eval_ms[0].keys()}
        return dict(ms_per_step=total_ms / steps, phases=phases, pairs=pairs, ex=ex, selfp=selfp,
                    launches=launches, clocks=clk, opt=opt, mem_peak=mem["peak"])

    head = measure(args.precision, args.steps, args.warmup, clocks=True, barrier=True)
    phi_head = phi.cpu().numpy() if rank == 0 else None
    phi_real = None
    if rank == 0 and not args.no_cpu_baseline:
        # untimed: the same path with real strengths (Re q), whose real part
        # has no branch ambiguity and is checked against the plain direct sum
        q_re = q.clone()
        q_re[:, 1] = 0.0
        t = G.fmm_build_tree(src, tgt, head["opt"])
        G.fmm_evaluate(t, q_re, phi)
        G.fmm_tree_sync(t)
        t.free()
        phi_real = phi.cpu().numpy()
    value = job_value(m, ws, head["ms_per_step"])
    other = "fp64" if args.precision == "mixed" else "mixed"
    comp = None
    if not args.no_compare:
        comp = measure(other, min(args.steps, 3), 2)

    # e2e through the C ABI with host buffers (copies inside the timed region)
    src_h = torch.from_numpy(src_np).pin_memory().numpy()
    q_h = torch.from_numpy(q_np).pin_memory().numpy()
    tgt_h = torch.from_numpy(tgt_np).pin_memory().numpy() if tgt_np is not None else None
    out_h = torch.empty((m, 2), dtype=torch.float64).pin_memory().numpy()
    G.fmm_solve_host(src_h, q_h, tgt_h, head["opt"], out=out_h)
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.fmm_solve_host(src_h, q_h, tgt_h, head["opt"], out=out_h)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_times)

    batched = None
    if not args.no_batched and not args.n and wl == WORKLOAD:
        batched = run_batched_section(args, G, torch, dev, stream)
    configs = None
    if not args.no_configs and not args.n and wl == WORKLOAD and ws == 1:
        configs = run_configs_section(G, torch, dev, stream, flush)

    line = None
    if rank == 0:
        peaks = load_peaks()
        ex = head["ex"]
        mixed = args.precision == "mixed"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2 (double-float pairs) + f64" if mixed else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESCS[wl], "precision": args.precision, "p": args.p,
                       "kernel": ("harmonic: u(y) = sum q_j / (x_j - y)" if args.kernel == "harmonic"
                                  else "log: Phi(y) = sum q_j Log(y - x_j)"),
                       "m2l": ("tcgen05 fp16 digits x%d, one GEMM row per weak pair"
                               % (args.m2l_slices or 5)
                               if mixed and args.m2l_slices >= 0 else
                               ("df32 sweeps" if mixed else "fp64")),
                       "leaf": args.leaf, "level_shift": args.level_shift,
                       "levels": ex["levels"], "n_weak": ex["n_weak"], "n_strong": ex["n_strong"],
                       "p2p_pairs": head["pairs"],
                       "p2p": (("symmetric df32" if mixed else "symmetric fp64")
                               + ": each unordered pair of points once"
                               if head["selfp"] is not None else
                               ("df32 per evaluation point" if mixed else "fp64")),
                       "box_geometry": ("bounding rectangles of the points" if args.box_fit
                                        else "split rectangles"),
                       "leaf_shortcut": (
                           {"p2l_pairs": ex["n_p2l"], "m2p_pairs": ex["n_m2p"],
                            "near_pairs": ex["n_near"]} if args.p2l_m2p else "off"),
                       "l2": "256 MB buffer written between steps, outside the timed events",
                       "far_field": "own stream, overlapping the near field (timed steps)",
                       "parallelism": f"replicas x{ws}"},
            "phases_ms": head["phases"],
            "phases_source": ("separate untimed steps with phase timing on: the phases then "
                              "run one after another, each span timing its own kernels"),
            "roofline": roofline(mixed, head["pairs"], head["phases"]["p2p"], head["selfp"],
                                 args.kernel == "harmonic", n_points=n,
                                 clusters=wl.startswith("clusters_1e6")),
            "m2l_roofline": m2l_roofline(mixed, mixed and args.m2l_slices >= 0 and args.p <= 31,
                                         ex["n_weak"], args.p, head["phases"]["m2l"], peaks),
            "phase_bandwidth": phase_bandwidth(ex, n, m, args.p, head["phases"], peaks),
            "e2e": {"value": m / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 32 * n + (16 * m if tgt_np is not None else 0),
                    "d2h_bytes_per_step": 16 * m,
                    "api": "fmm_solve_host (pinned host buffers, copies + build + evaluate)"},
            "clocks": head["clocks"],
            "gpu_launches": head["launches"],
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            "hbm_footprint": {
                "library_peak_bytes": head["mem_peak"],
                "caller_buffers_bytes": 32 * n + (32 * m if tgt_np is not None else 16 * m),
                "total_bytes": head["mem_peak"] + 32 * n + (32 * m if tgt_np is not None
                                                          else 16 * m),
                "source": ("fmm_memory_info: the largest device memory the library held (tree, "
                           "lists, expansions, work items, scratch) during the timed steps; "
                           "plus the caller's points, strengths and potentials")},
        }
        if comp is not None:
            line[f"{other}_path"] = {
                "value": n / (comp["ms_per_step"] * 1e-3), "unit": UNIT,
                "ms_per_step": comp["ms_per_step"], "steps": min(args.steps, 3), "warmup": 2,
                "phases_ms": comp["phases"],
                "roofline": roofline(other == "mixed", comp["pairs"],
                                     comp["phases"]["p2p"], comp["selfp"],
                                     args.kernel == "harmonic"),
                "m2l_roofline": m2l_roofline(other == "mixed", other == "mixed" and args.p <= 31,
                                             comp["ex"]["n_weak"], args.p,
                                             comp["phases"]["m2l"], peaks)}
            line["speedup_mixed_vs_fp64"] = (
                comp["ms_per_step"] / head["ms_per_step"] if mixed
                else head["ms_per_step"] / comp["ms_per_step"])
        if batched is not None:
            line["batched"] = batched
        if configs is not None:
            line["configs"] = configs
        if args.n:
            line["config"]["workload"] += f" [scaled to N={n} for profiling]"
        if (not args.no_cpu_baseline and ws == 1 and not args.n and wl == WORKLOAD
                and args.kernel == "log"):
            line["cpu_baseline"], line["error"] = cpu_baseline(args, src_np, q_np, phi_head,
                                                               phi_real)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


def levels_cap(n, leaf):
    """The level rule of the library's default options: the least L with
    ceil(n / 4^L) <= leaf (instances with the same L share one tree)."""
    L = 0
    while -(-n // 4 ** L) > leaf:
        L += 1
    return L


# The other configurations of the method's scope, timed in the default run so
# that the line carries them: (workload, p).
OTHER_CONFIGS = [("curve_4e6", 24), ("curve_4e6", 12), ("clusters_1p6e7_targets", 30)]


def run_configs_section(G, torch, dev, stream, flush, warmup=2, steps=3):
    """Build + evaluate per step (mixed precision, tensor M2L, leaf shortcut,
    shrink-wrapped boxes: the headline's options) on each of OTHER_CONFIGS at
    full size, inputs resident, CUDA events, the L2 flush between steps; one
    further step with phase timing gives the tree, connectivity, M2L and P2P
    spans; the library's device-memory peak plus the caller's buffers give
    the HBM footprint."""
    out = []
    for wl, p in OTHER_CONFIGS:
        src_np, q_np, tgt_np = W.make(wl)
        n = len(src_np)
        m = len(tgt_np) if tgt_np is not None else n
        src = torch.from_numpy(src_np).to(dev)
        q = torch.from_numpy(q_np).to(dev)
        tgt = torch.from_numpy(tgt_np).to(dev) if tgt_np is not None else None
        phi = torch.empty((m, 2), dtype=torch.float64, device=dev)
        opt = G.fmm_default_options(p=p, leaf_size=W.WORKLOADS[wl]["leaf"],
                                    precision=G.FMM_PREC_MIXED, p2l_m2p=1, box_fit=1)

        def step(timing=False):
            tree = G.fmm_build_tree(src, tgt, opt)
            if timing:
                G.fmm_set_timing(tree, True)
            G.fmm_evaluate(tree, q, phi)
            return tree

        for _ in range(warmup):
            tree = step()
            G.fmm_tree_sync(tree)
            tree.free()
        torch.cuda.synchronize()
        G.fmm_memory_info(reset_peak=True)
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree = step()
            e1.record(stream)
            G.fmm_tree_sync(tree)
            ms.append(e0.elapsed_time(e1))
            tree.free()
        peak = G.fmm_memory_info()["peak"]
        flush.zero_()
        tree = step(timing=True)
        G.fmm_tree_sync(tree)
        ph = G.fmm_get_timings(tree)
        info = G.fmm_tree_info(tree)
        tree.free()
        ms_step = statistics.mean(ms)
        caller = 32 * n + (32 * m if tgt_np is not None else 16 * m)
        out.append({
            "workload": WORKLOAD_DESCS[wl] + f" (p={p})", "p": p,
            "value": m / (ms_step * 1e-3), "unit": UNIT, "ms_per_step": ms_step,
            "steps": steps, "warmup": warmup,
            "phases_ms": {k: ph[k] for k in ("tree", "connect", "m2l", "p2p")},
            "levels": info["levels"], "n_weak": info["n_weak"],
            "hbm_footprint": {"library_peak_bytes": peak, "caller_buffers_bytes": caller,
                              "total_bytes": peak + caller}})
        del src, q, tgt, phi
        torch.cuda.empty_cache()
    return out


def run_batched_section(args, G, torch, dev, stream):
    """512 independent instances (N_i log-uniform in [1e3, 1e5], distribution
    per instance, complex q, p = 20): forest build once, then evaluation passes
    replayed as one CUDA graph; both precisions."""
    inst = W.batched_instances(args.batch_inst)
    sizes = np.array([len(s) for _, s, _ in inst], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    src = torch.from_numpy(np.concatenate([s for _, s, _ in inst])).to(dev)
    q = torch.from_numpy(np.concatenate([x for _, _, x in inst])).to(dev)
    phi = torch.empty((int(off[-1]), 2), dtype=torch.float64, device=dev)
    out = {"workload": f"{args.batch_inst} instances, N_i = floor(10^U[3,5]) "
                       f"(total {int(off[-1])}), uniform/clusters/curve per instance, "
                       f"complex q, p=20, theta=0.5, leaf and near-field item size autotuned",
           "n_points": int(off[-1])}
    tuned_leaf, tuned_items = 64, 0
    for prec in ("mixed", "fp64"):
        opt = G.fmm_default_options(p=20, leaf_size=64,
                                    precision=G.FMM_PREC_MIXED if prec == "mixed"
                                    else G.FMM_PREC_FP64, p2l_m2p=args.p2l_m2p,
                                    box_fit=args.box_fit)
        if prec == "mixed":
            # leaf size and near-field item size by the library's autotuner
            # (one build + 4 evaluations per trial)
            t0 = time.perf_counter()
            tuned, trials = G.fmm_autotune(src, q, opt, [24, 32, 48, 64, 96], [512, 2048, 8192],
                                           src_off=off, repeats=1, evaluations=4)
            out["autotune"] = {"leaf": tuned.leaf_size, "p2p_item_sources": tuned.p2p_item_sources,
                               "trial_ms": {f"{a}x{b}": v for (a, b), v in trials.items()},
                               "tuning_s": time.perf_counter() - t0,
                               "objective": "build + 4 evaluations"}
            tuned_leaf = tuned.leaf_size
            tuned_items = tuned.p2p_item_sources
        opt.leaf_size = tuned_leaf
        opt.p2p_item_sources = tuned_items
        torch.cuda.synchronize()
        l0 = G.fmm_launch_count()
        t0 = time.perf_counter()
        tree = G.fmm_build_batched(off, src, opt)
        build_s = time.perf_counter() - t0
        build_launches = G.fmm_launch_count() - l0
        G.fmm_set_graph(tree, True)
        for _ in range(2):
            G.fmm_evaluate(tree, q, phi)
        torch.cuda.synchronize()
        steps = 5 if prec == "mixed" else 2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            G.fmm_evaluate(tree, q, phi)
        e1.record(stream)
        G.fmm_tree_sync(tree)
        ms = e0.elapsed_time(e1) / steps
        info = G.fmm_tree_info(tree)
        tree.free()
        n_groups = len({levels_cap(int(n), tuned_leaf) for n in sizes})
        out[prec] = {"evaluate_ms": ms, "evaluate_particles_per_s": off[-1] / (ms * 1e-3),
                     "build_s": build_s, "build_launches": build_launches,
                     "build_trees": n_groups,
                     "build_plus_evaluate_particles_per_s": off[-1] / (build_s + ms * 1e-3),
                     "boxes": info["n_boxes"], "weak_pairs": info["n_weak"],
                     "steps": steps, "graph": True}
    out["evaluate_speedup_mixed_vs_fp64"] = out["fp64"]["evaluate_ms"] / out["mixed"]["evaluate_ms"]
    return out


def cpu_baseline(args, src, q, phi_gpu, phi_gpu_real):
    """The oracle timed on the host cores on a bounded sample (one thread, the
    paper's style, then every usable core), and the error of the GPU
    potentials: against the oracle FMM on that sample, against the
    branch-consistent direct sum on `args.gate_points` seeded points of it, and
    (real strengths, Re q) the real part against the plain direct sum there,
    which has no branch."""
    import oracle as O
    cpu = cpu_info()
    tot, det, phi_o, sample, tree, lists, sc = oracle_sample_run(
        src, q, args.p, args.leaf, args.ref_sample, shortcut=bool(args.p2l_m2p),
        box_fit=bool(args.box_fit), threads=1)
    tot_mt, det_mt, phi_mt = oracle_sample_run(
        src, q, args.p, args.leaf, args.ref_sample, shortcut=bool(args.p2l_m2p),
        box_fit=bool(args.box_fit), threads=cpu["usable"])[:3]
    g = phi_gpu[sample, 0] + 1j * phi_gpu[sample, 1]
    err_oracle = O.normwise_error(g, phi_o)
    ns = min(len(sample), args.gate_points)
    sub = np.sort(np.random.default_rng(W.BASE_SEED + 4096).choice(len(sample), ns,
                                                                  replace=False))
    pts = sample[sub]
    t0 = time.perf_counter()
    ref = O.direct_branch(tree, lists, src, q, sample=pts, shortcut=sc)
    t1 = time.perf_counter()
    err_direct = O.normwise_error(g[sub], ref)
    q_re = np.zeros_like(q)
    q_re[:, 0] = q[:, 0]
    plain = O.direct_sample(src, q_re, None, pts)
    t2 = time.perf_counter()
    re_gpu = phi_gpu_real[pts, 0]
    err_re = float(np.max(np.abs(re_gpu - plain.real)) / np.max(np.abs(plain.real)))
    desc = (f"full tree, lists and expansion phases of the N=1e6 workload, then L2P+P2P at "
            f"{args.ref_sample} random points; per-point time scaled to N points")
    base = {"value": len(src) / tot, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{desc} ({det['wall_s']:.1f} s of CPU work, 1 thread)",
            "phases_s": det, "cpu": cpu,
            "openmp": {"value": len(src) / tot_mt, "unit": UNIT, "cores": cpu["usable"],
                       "phases_s": det_mt,
                       "note": ("the same oracle with its independent per-target loops (M2L "
                                "per target box, L2P + P2P per point) on every usable core; "
                                "tree, lists, P2M, M2M, L2L and P2L serial"),
                       "identical_to_1_thread": bool(np.array_equal(phi_mt, phi_o))}}
    err = {"vs_oracle_fmm": err_oracle, "vs_direct_branch": err_direct,
           "re_vs_plain_direct_real_q": err_re,
           "n_points_oracle": int(len(sample)), "n_points_direct": int(ns),
           "gate": 1e-10, "gate_met": bool(err_direct <= 1e-10 and err_re <= 1e-10),
           "direct_sums_s": {"branch": t1 - t0, "plain": t2 - t1},
           "measure": ("max|d phi| / max|phi_ref| over the sampled points; the branch-"
                       "consistent direct sum evaluates every pair on the branch its FMM "
                       "path converges to; the real-strength check compares Re(phi) (Re q "
                       "only) with the plain FP64 direct sum")}
    return base, err


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the measurement of the other precision")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched section")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the section timing the other configurations")
    ap.add_argument("--batch-inst", type=int, default=512)
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_DESCS),
                    help="clusters_1e6 (the headline); curve_4e6 and clusters_1p6e7_targets "
                         "time the other configurations")
    ap.add_argument("--p", type=int, default=0, help="expansion order (0: the workload's)")
    ap.add_argument("--leaf", type=int, default=0, help="particles per leaf (0: the workload's)")
    ap.add_argument("--level-shift", type=int, default=0)
    ap.add_argument("--m2l-slices", type=int, default=0,
                    help="mixed path: 0 = tensor-core M2L with 5 digit slices, 1..5 = that many "
                         "slices, -1 = double-float sweeps")
    ap.add_argument("--ref-sample", type=int, default=98304,
                    help="evaluation points of the oracle sample in the GPU arm's CPU leg")
    ap.add_argument("--ref-arm-sample", type=int, default=16384,
                    help="evaluation points per step of the reference (oracle) arm")
    ap.add_argument("--gate-points", type=int, default=4096,
                    help="seeded points of the direct-sum error gate")
    ap.add_argument("--kernel", default="log", choices=["log", "harmonic"])
    ap.add_argument("--box-fit", type=int, default=1, choices=[0, 1],
                    help="shrink-wrapped box geometry (bounding rectangles of the points)")
    ap.add_argument("--p2l-m2p", type=int, default=1, choices=[0, 1],
                    help="leaf P2L/M2P shortcut of Sec. 2 (1 = on)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0,
                    help="scale the workload to N points (profiling runs only; default 1e6)")
    args = ap.parse_args()
    if not args.p:
        args.p = W.WORKLOADS[args.workload]["p"]
    if not args.leaf:
        args.leaf = W.WORKLOADS[args.workload]["leaf"]
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
