#!/usr/bin/env python3
"""Benchmark of the exact #DNN-Verification counter (SLR + bisection) on GB300.

One step is one whole count, Alg. 1 level by level (Sec. 3), of the
ACAS-shaped workload: a 5 -> 6x50 -> 5 ReLU network, a random sub-box of
[-0.5, 0.5]^5, the unsafe set "output 0 is not minimal", depth 20 (a frontier of
up to 2^20 boxes).  The metric is SLR subdomain bounds per second: boxes bounded
over all levels divided by the device time of the count; the time-to-count is
ms_per_step.

Prints one JSON line.  Besides the contract keys it carries
  roofline      the FP32 evaluation kernel's algorithmic FLOP rate (centre/radius
                form: 4 n_{k+1} n_k (d+1) per box and affine layer) against the
                FP32 CUDA-core peak 152 SMs x 128 lanes x 2 x the sampled SM clock,
  cpu_baseline  the FP64 oracle on the host cores over a bounded sample of the
                same count (one process per core, levels in order, ~15 s),
  e2e           the same metric through the C ABI with host buffers: network,
                box and property uploaded and the result read back every step,
  clocks        nvidia-smi samples taken during the timed region.
`--impl reference` times the oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SMS = 152
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 512 << 20          # written between timed steps (> 129 MB L2)
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense TF32 / BF16 tensor rates of GB300

# DRAM bytes per box of the FP32 evaluation kernel from one ncu capture of the
# kernel source hashed below (profiles/slr_eval_f32_acas_D20.md: levels 18 and
# 19, 8.56 and 8.29 B per box); reported as roofline.traffic only while the
# kernel source is unchanged.
TRAFFIC = {"source_sha": "45590470a99640c4", "bytes_per_box": 8.4}
KERNEL_SOURCES = ["paper_2312_05890_gb300/csrc/slr_eval.cuh", "paper_2312_05890_gb300/csrc/slr_eval_f32.cu",
                  "paper_2312_05890_gb300/csrc/slr_device.cuh"]


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def algorithmic_flops_per_box(widths, R):
    """4 n_{k+1} n_k (d+1) per affine layer after the first (W C and |W| R), last layer with R rows."""
    d = widths[0]
    n = list(widths[:-1]) + [R]
    return sum(4 * n[k + 1] * n[k] * (d + 1) for k in range(1, len(n) - 1))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline, parity, stated error; reference arm)
# ---------------------------------------------------------------------------

def oracle_count(p, D, budget_s, procs, leaves=False):
    """The oracle's level-by-level count of p on `procs` host processes, stopped at
    a level boundary after `budget_s` seconds (None: every level)."""
    from oracle import pool
    return pool.count_levels(p, D, procs=procs, budget_s=budget_s, leaves=leaves)


def parity_of(gpu, ref, D):
    """The GPU count against the oracle's, level by level over the levels the oracle finished
    (boxes, safe, unsafe, undecided), and the bracket when it finished all of them."""
    n = len(ref["levels"])
    keys = ("boxes", "safe", "unsafe", "undecided")
    first_bad = None
    for t, lv in enumerate(ref["levels"]):
        got = {k: gpu["level_" + k][t] for k in keys}
        if got != {k: lv[k] for k in keys}:
            first_bad = t
            break
    out = {"levels_compared": n, "oracle_complete": ref["complete"], "levels_equal": first_bad is None,
           "gpu_lo": gpu["unsafe_lo"], "gpu_hi": gpu["unsafe_hi"]}
    if first_bad is not None:
        out["first_differing_level"] = first_bad
    if ref["complete"]:
        out["oracle_lo"], out["oracle_hi"] = ref["unsafe_lo"], ref["unsafe_hi"]
        out["bracket_equal"] = (ref["unsafe_lo"], ref["unsafe_hi"]) == (gpu["unsafe_lo"], gpu["unsafe_hi"])
    out["equal"] = out["levels_equal"] and out.get("bracket_equal", True)
    return out


STATED_ERROR_BOXES = {"tiny": 1024, "acas": 1024, "nav": 512, "mnist": 32}


def stated_error(pkg, names=("tiny", "acas", "nav", "mnist"), seed=0):
    """Per configuration and path: the largest deviation of the GPU row bounds from the
    FP64 oracle's over random sub-boxes, relative to the row scale max(|lo|, |hi|) + (hi - lo).
    'raw' is the FP32 SLR bound (sound bound with its widening removed), 'sound' the
    widened bound the counter decides on, 'widening' the widening itself."""
    import numpy as np

    import oracle
    from workloads import generators as gen
    out = {}
    for name in names:
        p = gen.make(name)
        n = STATED_ERROR_BOXES[name]
        rng = np.random.default_rng(seed + 77)
        u = np.sort(rng.random((2, n, p.d)), axis=0)
        lo = (p.lo + (p.hi - p.lo) * u[0]).astype(np.float32)
        hi = (p.lo + (p.hi - p.lo) * u[1]).astype(np.float32)
        olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
        scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo) + 1e-30
        paths = {"fp32_tile": {}, "tf32_tile": {"precision": pkg.PREC_TC_TF32}, "wide_tf32": {"wide": 1}}
        if name == "mnist":
            paths = {"wide_tf32": {}}
        out[name] = {"boxes": n}
        for path, opt in paths.items():
            with pkg.Counter(0) as c:
                c.set_problem(p)
                if opt:
                    c.set_options(**opt)
                try:
                    rl, rh, _, err = c.bounds(lo, hi, want_err=True)
                except pkg.SlrError as e:      # e.g. a shape the tensor-core tile does not take
                    out[name][path] = {"unavailable": str(e)}
                    continue
            rl = rl.astype(np.float64)
            rh = rh.astype(np.float64)
            raw = max(np.max(np.abs(rl + err - olo) / scale), np.max(np.abs(rh - err - ohi) / scale))
            snd = max(np.max(np.abs(rl - olo) / scale), np.max(np.abs(rh - ohi) / scale))
            sound = bool(np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale))
            out[name][path] = {"raw": float(raw), "sound": float(snd), "widening": float(np.max(err / scale)),
                               "contains_oracle": sound}
    return out


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="acas")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--depth", type=int, default=0, help="depth cap (default: the workload's)")
    ap.add_argument("--cpu-budget", type=float, default=40.0,
                    help="the oracle leg stops at the first level boundary after this many seconds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=L2_FLUSH_BYTES >> 20,
                    help="L2 flush buffer written between timed steps (MB)")
    ap.add_argument("--alpha-steps", type=int, default=0,
                    help="projected-Adam steps on the lower ReLU slopes of each level's undecided boxes")
    ap.add_argument("--alpha-lr", type=float, default=0.1)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32"],
                    help="contraction of the fused kernel: FP32 CUDA cores or split-TF32 tensor cores")
    ap.add_argument("--tile", default="",
                    help="boxes x threads per CTA of the FP32 evaluation kernel, e.g. 16x256 (default: timed choice)")
    ap.add_argument("--alpha-cap", type=int, default=1 << 20,
                    help="most undecided boxes per level whose slopes are optimised")
    ap.add_argument("--alpha-margin", type=float, default=0.2,
                    help="optimise only boxes whose decision gap is within this fraction of their bound width "
                         "(0: every undecided box)")
    ap.add_argument("--shard-level", type=int, default=-1,
                    help="strong scaling: the ranks share one count, rank r taking every N-th subtree below this "
                         "level (default: weak scaling, a problem per rank)")
    ap.add_argument("--recheck-cluster", action="store_true",
                    help="FP64 re-check with each tile on a cluster of 4 CTAs instead of one CTA")
    ap.add_argument("--batch-widths", default="tile", choices=["full", "tile"],
                    help="batched workload: only the hidden widths a tile holds (32-128, default) or 32-512 as "
                         "stated (256- and 512-wide members on the wide path; one step takes minutes)")
    ap.add_argument("--no-forms", action="store_true", help="skip the short legs of the chosen forms")
    ap.add_argument("--no-batch-form", action="store_true", help="skip the batched leg among the forms")
    ap.add_argument("--form-steps", type=int, default=3, help="timed counts per form leg")
    ap.add_argument("--form-alpha-steps", type=int, default=20, help="Adam steps of the slope-optimised form")
    ap.add_argument("--no-stated-error", action="store_true",
                    help="skip the per-configuration bound error against the oracle")
    ap.add_argument("--split", default="widest", choices=["widest", "gradient"],
                    help="bisect the widest side, or per box the dimension of the 16-dimension split set "
                         "with the largest |dM/dr| r (adjoint gradient of the decision loss)")
    args = ap.parse_args()

    from paper_2312_05890_gb300 import multirank
    world, rank, local_rank = multirank.rank_env()
    procs = os.cpu_count() or 1

    from workloads import generators as gen
    if args.workload == "batch":
        return bench_batch(args, world, rank, local_rank)
    # weak scaling: rank r counts its own problem of the same shape (seed + r);
    # strong scaling (--shard-level): every rank takes a shard of one count
    strong = args.shard_level >= 0
    p = gen.make(args.workload, args.seed if strong else multirank.weak_seed(args.seed, rank))
    D = args.depth or p.depth
    # the seed filter maps the requested base seed to the first accepted one
    workload = f"{p.name} D={D} seed={p.seed}"
    config = {"workload": workload, "widths": p.net.widths, "depth": D, "rows": p.prop.R,
              "l2": f"flushed between steps ({args.flush_mb} MB write)", "parallelism": f"weak x{world}"}
    if args.alpha_steps:
        config["slopes"] = f"{args.alpha_steps} projected-Adam steps (lr {args.alpha_lr}) per undecided box"
    if args.split == "gradient":
        config["split"] = "per box: largest |dM/dr_i| r_i over the 16 dimensions of largest |dM/dr_i| w_i at the root"
    if strong:
        config["parallelism"] = f"strong x{world}: shard r of {world} = every {world}-th subtree below level {args.shard_level}"

    if args.impl == "reference":
        if rank != 0:
            return
        budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
        for _ in range(args.warmup):
            oracle_count(p, D, budget, procs)
        tot_boxes, tot_s, reached = 0, 0.0, []
        for _ in range(args.steps):
            r = oracle_count(p, D, budget, procs)
            tot_boxes += r["boxes"]
            tot_s += r["seconds"]
            reached.append(len(r["levels"]))
        v = tot_boxes / tot_s
        depths = f"{min(reached) - 1}" if min(reached) == max(reached) else f"{min(reached) - 1}-{max(reached) - 1}"
        sample = (f"levels 0..{depths} of the count: each step stops at the first level boundary after "
                  f"{budget:.1f} s (steps reached mixed depths when a range is given), "
                  f"{tot_boxes // max(1, args.steps)} boxes per step on average")
        print(json.dumps({
            "impl": "reference", "metric": "slr_subdomain_bounds_per_sec", "value": v, "unit": "boxes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": "boxes/s", "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    import torch
    torch.cuda.set_device(local_rank)
    dist = multirank.init(world)
    import paper_2312_05890_gb300 as pkg
    pkg.load_library()

    def barrier():
        multirank.barrier(dist)

    flush = torch.empty(max(1, args.flush_mb << 18), dtype=torch.float32, device="cuda")
    c = pkg.Counter(local_rank)
    c.set_problem(p)
    tile = {}
    if args.tile:
        tb, tt = (int(x) for x in args.tile.lower().split("x"))
        tile = {"tile_boxes": tb, "tile_threads": tt}
    if strong:
        tile.update(shard_count=world, shard_index=rank, shard_level=args.shard_level)
    if args.recheck_cluster:
        tile["recheck_cluster"] = 1
        config["recheck"] = "each FP64 tile on a cluster of 4 CTAs"
    if args.precision == "tf32":
        tile["precision"] = pkg.PREC_TC_TF32
        config["precision"] = "split-TF32 tensor-core contraction (tcgen05), FP32 re-bound and FP64 re-check"
    fixed = fixed_split = None
    if args.alpha_steps or args.split == "gradient":
        # the plain path (fixed slopes, widest side), for the comparison below
        c.set_options(**tile)
        fixed = c.count(D)
    if args.split == "gradient":
        tile["split_rule"] = pkg.SPLIT_GRADIENT
        if args.alpha_steps:
            c.set_options(alpha_cap=args.alpha_cap, **tile)
            fixed_split = c.count(D)     # fixed slopes, gradient split
    if args.alpha_steps:
        c.set_options(profile=1, alpha_steps=args.alpha_steps, alpha_lr=args.alpha_lr, alpha_cap=args.alpha_cap,
                      alpha_margin=args.alpha_margin, **tile)
    else:
        c.set_options(profile=1, alpha_cap=args.alpha_cap, **tile)
    for _ in range(args.warmup):
        c.count(D)

    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    t_wall = time.perf_counter()
    dev_ms, boxes, kern = [], 0, [0.0, 0.0, 0.0]
    launches = 0
    alpha_ms = 0.0
    gemm_ms, gemm_flop, gemm_launches = 0.0, 0.0, 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        r = c.count(D)
        dev_ms.append(r["device_ms"])
        boxes += r["boxes"]
        launches += r["launches"]
        for i in range(3):
            kern[i] += r["kernel_ms"][i]
        alpha_ms += r["alpha_ms"]
        gemm_ms += r["gemm_ms"]
        gemm_flop += r["gemm_flop"]
        gemm_launches += r["gemm_launches"]
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    # the FP32 FMA rate under the same clocks: the roofline denominator of the tile kernel
    fp32_peak = pkg.slr_measure_fp32_peak(local_rank)
    clocks = sampler.stop()
    last = r

    max_ms, _, value = multirank.job_rate(sum(dev_ms), boxes, dist)
    job_lo, job_hi = multirank.sum_counts(last["unsafe_lo"], last["unsafe_hi"], dist) if strong else (None, None)

    # ---- e2e: upload network, box and property from host memory every step ------
    e2e_s = []
    h2d = d2h = 0
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.set_problem(p)
        r = c.count(D)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_s.append(dt)
            h2d, d2h = r["h2d_bytes"], r["d2h_bytes"]
    e2e_value = last["boxes"] / statistics.mean(e2e_s)

    # ---- roofline of the FP32 evaluation kernel ---------------------------------
    fpb = algorithmic_flops_per_box(p.net.widths, p.prop.R)
    eval_s = kern[0] / 1e3
    achieved = fpb * boxes / eval_s / 1e12
    clk = clocks.get("sm_mhz") or 2070.0
    nominal = SMS * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
    peak = fp32_peak["tflops"]
    eval_launches = args.steps * (D + 1)
    traffic = None
    if TRAFFIC["source_sha"] == kernel_sha() and TRAFFIC["bytes_per_box"]:
        traffic = TRAFFIC["bytes_per_box"] * boxes / eval_launches
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "slr_eval_kernel<float>",
                "peak_basis": (f"measured: FFMA-throughput kernel in this process ({fp32_peak['ms']:.1f} ms, 16 "
                               f"independent chains per thread, 2048 threads per SM); nominal at the sampled "
                               f"{clk:.0f} MHz: {SMS} x {FP32_LANES_PER_SM} lanes x 2 = {nominal:.1f} TFLOP/s"),
                "frac_of_nominal": achieved / nominal,
                "flop_per_box": fpb, "kernel_share": kern[0] / max(1e-9, sum(dev_ms)),
                "avg_launch_ms": kern[0] / eval_launches}
    if gemm_launches:
        # wide path: the per-layer products on the tensor cores dominate
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        tf32_peak = peaks["bf16_tflops"] * TF32_PER_BF16
        ach = gemm_flop / (gemm_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s",
                    "frac": ach / tf32_peak, "traffic": None, "kernel": "wide_gemm_kernel (tcgen05 kind::tf32)",
                    "peak_basis": f"measured bf16 burst {peaks['bf16_tflops']} TFLOP/s x nominal TF32/BF16 "
                                  f"ratio {TF32_PER_BF16:.3f}",
                    "flop_basis": "2 M K (2d + 1) per box and layer (W C on d columns, |W| R on d + 1); "
                                  "the kernel issues 3 split products for each",
                    "executed_tflops": 3 * ach, "kernel_share": gemm_ms / max(1e-9, sum(dev_ms)),
                    "avg_launch_ms": gemm_ms / gemm_launches, "launches": gemm_launches}

    # ---- chosen forms against the plain FP32 path (short legs, same problem) ----
    forms = None
    if not args.no_forms and not strong and args.alpha_steps == 0 and args.precision == "fp32" \
            and args.split == "widest":
        forms = run_forms(pkg, p, D, args, last, flush)

    # ---- the oracle on the host cores: CPU baseline, parity of the count, stated error ----
    cpu = parity = serr = None
    if rank == 0 and not args.no_cpu_baseline:
        ref = oracle_count(p, D, args.cpu_budget, procs)
        lv = len(ref["levels"])
        cpu = {"value": ref["boxes"] / ref["seconds"], "unit": "boxes/s", "cores": ref["procs"], "kind": "oracle",
               "sample": (f"levels 0..{lv - 1} of the same count" + (" (the whole count)" if ref["complete"] else "")
                          + f", {ref['boxes']} boxes, {ref['seconds']:.1f} s, one process per core")}
        if not strong and args.alpha_steps == 0 and args.split == "widest":
            parity = parity_of(last, ref, D)
        if not args.no_stated_error and args.workload in STATED_ERROR_BOXES:
            serr = stated_error(pkg)

    if rank == 0:
        line = {
            "metric": "slr_subdomain_bounds_per_sec", "value": value, "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if strong else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config,
            "count": {"unsafe_lo": job_lo if strong else last["unsafe_lo"],
                      "unsafe_hi": job_hi if strong else last["unsafe_hi"], "boxes": last["boxes"],
                      "rechecked": last["rechecked"], "rechecked_fp64": last["rechecked_fp64"],
                      "tie_leaves": last["tie_leaves"],
                      "tile_boxes_threads": last["tile"]},
            "kernel_ms_per_step": {"eval_f32": kern[0] / args.steps, "recheck_f64": kern[1] / args.steps,
                                   "compact": kern[2] / args.steps},
            "wall_s": wall,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "boxes/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clocks,
        }
        if parity is not None:
            line["parity"] = parity
        if forms is not None:
            line["forms"] = forms
        if serr is not None:
            line["stated_error"] = serr
        def summary(x):
            return {"unsafe_lo": x["unsafe_lo"], "unsafe_hi": x["unsafe_hi"], "boxes": x["boxes"],
                    "device_ms": x["device_ms"], "boxes_per_s": x["boxes"] / (x["device_ms"] / 1e3)}
        if fixed is not None:
            line["slope_opt"] = {
                "alpha_boxes": last["alpha_boxes"], "alpha_decided": last["alpha_decided"],
                "alpha_ms_per_step": alpha_ms / args.steps,
                "fixed_slopes": summary(fixed)}
            if fixed_split is not None:
                line["slope_opt"]["fixed_slopes_gradient_split"] = summary(fixed_split)
        print(json.dumps(line))
        if parity is not None and not parity["equal"]:
            sys.stderr.write("bench: the GPU count differs from the oracle's: %s\n" % json.dumps(parity))
            c.close()
            multirank.finish(dist)
            sys.exit(3)
    c.close()
    multirank.finish(dist)


def run_forms(pkg, p, D, args, fp32, flush):
    """Short legs of the chosen forms on the same problem: the split-TF32 tensor-core
    contraction, slope-optimised counting (projected Adam on the lower slopes) and,
    as its own workload, the batched persistent count; each against the plain FP32
    path (the timed leg) at equal counts."""
    import torch

    def leg(opts, steps, warm):
        with pkg.Counter(torch.cuda.current_device()) as c:
            c.set_problem(p)
            c.set_options(**opts)
            for _ in range(warm):
                c.count(D)
            ms, boxes = [], 0
            for _ in range(steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                r = c.count(D)
                ms.append(r["device_ms"])
                boxes += r["boxes"]
        out = {"boxes_per_s": boxes / (sum(ms) / 1e3), "ms_per_count": sum(ms) / len(ms),
               "unsafe_lo": r["unsafe_lo"], "unsafe_hi": r["unsafe_hi"], "boxes": r["boxes"], "steps": steps}
        return out, r

    forms = {"fp32": {"boxes_per_s": fp32["boxes"] / (fp32["device_ms"] / 1e3), "ms_per_count": fp32["device_ms"],
                      "unsafe_lo": fp32["unsafe_lo"], "unsafe_hi": fp32["unsafe_hi"], "boxes": fp32["boxes"],
                      "note": "the timed leg above"}}
    try:
        f, r = leg({"precision": pkg.PREC_TC_TF32}, args.form_steps, 1)
        f["same_count_as_fp32"] = (r["unsafe_lo"], r["unsafe_hi"]) == (fp32["unsafe_lo"], fp32["unsafe_hi"])
        f["rechecked_fp32"] = r["rechecked_fp32"]
        forms["split_tf32"] = f
    except pkg.SlrError as e:
        forms["split_tf32"] = {"unavailable": str(e)}
    steps = args.form_alpha_steps
    f, r = leg({"alpha_steps": steps, "alpha_lr": 0.1, "alpha_margin": args.alpha_margin}, args.form_steps, 1)
    f["alpha_steps"] = steps
    f["alpha_margin"] = args.alpha_margin
    f["alpha_boxes"] = r["alpha_boxes"]
    f["alpha_decided"] = r["alpha_decided"]
    f["nested_in_fp32"] = fp32["unsafe_lo"] <= r["unsafe_lo"] <= r["unsafe_hi"] <= fp32["unsafe_hi"]
    f["boxes_saved_vs_fp32"] = fp32["boxes"] - r["boxes"]
    forms["slope_optimised"] = f
    if not args.no_batch_form:
        forms["batched"] = batch_form(pkg, args, flush)
    return forms


def batch_form(pkg, args, flush):
    """One short leg of the batched workload (256 problems of uneven size per step)."""
    import torch

    from workloads import generators as gen
    probs = gen.batched_uneven(args.seed)
    with pkg.Counter(torch.cuda.current_device()) as c:
        c.count_batch(probs)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        res = c.count_batch(probs)
    boxes = sum(r["boxes"] for r in res)
    ms = res[0]["device_ms"]
    return {"boxes_per_s": boxes / (ms / 1e3), "ms_per_step": ms, "problems": len(probs), "boxes": boxes,
            "workload": "batched: 256 problems over 16 networks, depth caps 12-22 (its own workload; "
                        "--workload batch times it in full)"}


BATCH_WIDTHS = {"full": {"widths": (32, 64, 128, 256, 512), "tile_only": False},
                "tile": {"widths": (32, 64, 128), "tile_only": True}}


def bench_batch(args, world, rank, local_rank):
    """The batched workload: 256 (network, property) problems counted together per step."""
    import torch

    import paper_2312_05890_gb300 as pkg
    from paper_2312_05890_gb300 import multirank
    from workloads import generators as gen
    torch.cuda.set_device(local_rank)
    dist = multirank.init(world)
    full = args.batch_widths == "full"
    probs = gen.batched_uneven(multirank.weak_seed(args.seed, rank), **BATCH_WIDTHS[args.batch_widths])
    flush = torch.empty(max(1, args.flush_mb << 18), dtype=torch.float32, device="cuda")
    c = pkg.Counter(local_rank)
    for _ in range(args.warmup):
        c.count_batch(probs)
    torch.cuda.synchronize()
    multirank.barrier(dist)
    sampler = ClockSampler(local_rank)
    sampler.start()
    ms, boxes, e2e = [], 0, []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = c.count_batch(probs)          # uploads every problem from host memory, reads back all counts
        e2e.append(time.perf_counter() - t0)
        ms.append(res[0]["device_ms"])
        boxes += sum(r["boxes"] for r in res)
    torch.cuda.synchronize()
    multirank.barrier(dist)
    clocks = sampler.stop()
    per_boxes = sorted(r["boxes"] for r in res)
    levels = sorted(r["levels"] for r in res)
    done = sorted(r["completion_ms"] for r in res)
    wide = [i for i, p in enumerate(probs) if max(p.net.widths[1:-1]) >= 256]
    max_ms, tot_boxes, value = multirank.job_rate(sum(ms), boxes, dist)
    tot_s = max_ms / 1e3
    _, _, e2e_value = multirank.job_rate(1e3 * sum(e2e), boxes, dist)
    # roofline: the algorithmic FLOPs of every problem's boxes over the whole
    # step's device time (evaluation, re-check and compaction together)
    flops = sum(algorithmic_flops_per_box(p.net.widths, p.prop.R) * r["boxes"] for p, r in zip(probs, res))
    clk = clocks.get("sm_mhz") or 2070.0
    fp32_peak = pkg.slr_measure_fp32_peak(local_rank)
    peak = fp32_peak["tflops"]
    achieved = flops * args.steps / (sum(ms) / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "slr_eval_batch_kernel<float>",
                "peak_basis": (f"measured: FFMA-throughput kernel in this process ({fp32_peak['ms']:.1f} ms); "
                               f"nominal at {clk:.0f} MHz: "
                               f"{SMS * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12:.1f} TFLOP/s"),
                "time_basis": "whole step (all kernels), so a lower bound on the kernel's own rate"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        cb = 0
        for p in probs:
            cb += oracle.count(p.net, p.lo, p.hi, p.prop, p.depth, max_boxes=4096).boxes
            if time.perf_counter() - t0 > min(args.cpu_budget, 20.0):
                break
        cs = time.perf_counter() - t0
        cpu = {"value": cb / cs, "unit": "boxes/s", "cores": 1, "kind": "oracle",
               "sample": f"the first levels (at most 4096 boxes) of the batch's problems in order, {cb} boxes, "
                         f"{cs:.1f} s, one process"}
    if rank == 0:
        print(json.dumps({
            "metric": "slr_subdomain_bounds_per_sec", "value": value, "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched: {len(probs)} problems over 16 networks (d 5-32, widths "
                                   f"{'32-512' if full else '32-128'}, 2-8 hidden layers), depth caps 12-22, "
                                   f"seed {args.seed}",
                       "wide_members": len(wide),
                       "l2": f"flushed between steps ({args.flush_mb} MB write)", "parallelism": f"weak x{world}",
                       "tile_boxes": res[0]["tile"][0], "launches_per_step": res[0]["launches"]},
            "per_problem": {"boxes_min_median_max": [per_boxes[0], per_boxes[len(per_boxes) // 2], per_boxes[-1]],
                            "levels_min_max": [levels[0], levels[-1]],
                            "completion_ms_min_median_max": [done[0], done[len(done) // 2], done[-1]],
                            "wide_members_boxes": sum(res[i]["boxes"] for i in wide),
                            # wide members run after the tiled ones: their share of the step
                            "wide_members_ms": (max(res[i]["completion_ms"] for i in wide) - max(
                                (r["completion_ms"] for j, r in enumerate(res) if j not in wide), default=0.0))
                            if wide else 0.0},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "boxes/s", "h2d_bytes_per_step": res[0]["h2d_bytes"],
                    "d2h_bytes_per_step": res[0]["d2h_bytes"]},
            "gpu_launches": res[0]["launches"] * args.steps, "clocks": clocks,
        }))
    c.close()
    multirank.finish(dist)


if __name__ == "__main__":
    main()
