#!/usr/bin/env python3
"""Benchmark of NSW fair ranking by gradient ascent over batched Sinkhorn solves (one JSON line).

Workload (default `plain2000x1000`): 2000 consumers x 1000 items, K = 10 real slots plus the dummy
slot (11 columns), relevance sigmoid(p_u . q_i + b_i) with p, q ~ N(0, 1/32) of dimension 32 and
b_i ~ N(-1, 1), exposure 1/log2(k+1), free cost tensor C, Adam (lr 0.1), 50 Sinkhorn iterations per
consumer per step, 500 ascent steps. One benchmark step is one whole solve: reset to C = 0, the
initial Sinkhorn solve and 500 ascent steps, i.e. 501 x 50 Sinkhorn iterations over every cell.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --compare batch|unrolled|bf16|paper-shapes [--steps K]

--compare runs one of the layered forms against the plain FP32 method on the same GPU and prints
one JSON line: 256 markets batched vs solved one after another (|U| ~ U[100, 4000], |I| ~
U[100, 2000], K in {5, 10, 20}); the unrolled adjoint gradient vs the implicit gradient (|U| =
20000, |I| = 2000, K = 20, L = 100, checkpoints every 10); BF16 vs FP32 relevance storage (|U| =
200000, |I| = 10^4, K = 20, rank-32 sigmoid relevance with 5% boosted items); paper-shapes times
the free-cost method on the shapes of the paper's timing figure (|U|, |I| around 250, K = 10)
next to the FP64 oracle on the host cores.

Under torchrun (N > 1) every rank solves its own independent market (seed = rank): weak scaling
with no collective on the data path; the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-NSW (rel err≤1e-5 vs FP64) & Sinkhorn cell-updates/s vs roofline"
UNIT = "cell-updates/s"
NSW_TOL = 1e-5
SMS_NOMINAL, SM_MAX_MHZ = 152, 2070.0
# The Sinkhorn sweep's on-chip bound: each cell-update reads one 4-byte entry of the shared tile
# (the exponential form's E_ik, or the log form's c~_ik), at the shared-memory load bandwidth that
# fr_measure_peaks measures with the sweep's 8-byte conflict-free loads (nominally 128 B/clk/SM,
# 32 cell-updates per clock per SM). The bound the method's statement names -- the slower of the
# HBM bytes at the measured copy bandwidth and the MUFU operations (one ex2 per cell-update plus
# one rcp per row and one lg2 per column, (1 + 2/m) per cell-update) at the measured ex2 rate --
# is reported beside it.
CELL_BYTES_SMEM = 4
HBM_FALLBACK_GBS = 6800.0


def hbm_peak_gbs():
    """Measured copy bandwidth (MEASURED_PEAKS.json), else the fallback figure; and its source."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def p1_kernel_name(g):
    """Name of the fused free-cost kernel serving FairRank context g (its compiled variant)."""
    v = g.kernel_variant()
    tile = f",tile{v['tile_stride']}" if v["tile_stride"] else ""
    return (f"p1_kernel<{v['n_cols_kernel']},{v['rows_per_thread']},"
            f"{'exact' if v['exact'] else 'padded'},update+sweep{tile}>")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="plain2000x1000")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the short measurements of the layered forms in the JSON line")
    ap.add_argument("--full-oracle", action="store_true",
                    help="with --compare precision: also one FP64 oracle forward over all consumers")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiling driver: set up the workload, run this many ascent steps, exit")
    ap.add_argument("--compare", choices=["batch", "unrolled", "bf16", "paper-shapes", "p1-scale",
                                          "precision", "p1-batch"],
                    default=None,
                    help="compare a layered form against the plain FP32 method (one JSON line)")
    ap.add_argument("--profile-item", choices=["implicit", "unrolled", "bf16", "batch", "metrics"],
                    default=None,
                    help="profiling driver for the per-item forms: set up the workload, run "
                         "--profile-steps ascent steps (metrics: then one fr_metrics call), exit")
    ap.add_argument("--profile-users", type=int, default=0,
                    help="with --profile-item: override the number of consumers (small captures)")
    ap.add_argument("--profile-items", type=int, default=0,
                    help="with --profile-item metrics: override the number of items")
    return ap.parse_args()


def workload(name):
    from paper_2406_10262_gb300 import synth
    w = dict(synth.WORKLOADS[name])
    w["n_cols"] = w["n_slots"] + 1 if w["n_items"] > w["n_slots"] else w["n_slots"]
    return w


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the kernel
    sources changed since that capture (their SHA-256 no longer matches). A source "file#Name"
    hashes only struct Name of that file."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec:
        return None
    h = hashlib.sha256()
    for src in rec["sources"]:
        path, _, block = src.partition("#")
        text = open(os.path.join(ROOT, path), "rb").read()
        if block:  # only the named struct of a shared header (the kernel's argument / state layout)
            start = text.index(("struct " + block + " {").encode())
            text = text[start:text.index(b"};", start) + 2]
        h.update(text)
    return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["sources_sha256"] else None


def golden_F_ref(name):
    p = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if not os.path.exists(p):
        return None
    return float(json.load(open(p))["F"][-1])


# ---- clocks during the timed region -------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device_index),
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- the oracle (CPU baseline and reference arm) --------------------------------------------
def oracle_sample(w, seed, budget_s, min_steps=1, threads=None, n_sub=200):
    """Times the FP64 oracle on a sub-market of the workload (first n_sub consumers, all items)
    until `budget_s` of CPU time: initial solve plus ascent steps, on `threads` host threads (all
    cores by default). Returns (cell-updates/s, info, seconds)."""
    import oracle
    from paper_2406_10262_gb300 import synth
    n_sub = max(1, min(w["n_users"], n_sub))
    r = synth.relevance_lowrank(w["n_users"], w["n_items"], seed=seed, rows=n_sub)
    cores = threads or os.cpu_count() or 1
    o = oracle.Oracle(n_sub, w["n_items"], w["n_slots"], iters=w["iters"], lr=0.1, threads=cores)
    o.set_relevance(r.astype(np.float32).astype(np.float64))
    o.set_exposure(synth.dcg_exposure(w["n_slots"]))
    cells = n_sub * w["n_items"] * w["n_cols"]
    t0 = time.perf_counter()
    o.impacts()  # initial Sinkhorn solve
    sweeps, steps = 1, 0
    while steps < min_steps or time.perf_counter() - t0 < budget_s:
        o.step(1)
        steps += 1
        sweeps += 1
    dt = time.perf_counter() - t0
    rate = cells * w["iters"] * sweeps / dt
    info = {"kind": "oracle", "cores": cores,
            "sample": f"first {n_sub} of {w['n_users']} consumers x {w['n_items']} items x "
                      f"{w['n_cols']} columns, initial solve + {steps} ascent steps "
                      f"({sweeps} x {w['iters']} Sinkhorn iterations), {dt:.1f} s, FP64"}
    return rate, info, dt


def workload_config(args, w, world):
    """The JSON line's config: the workload and its sizes (shared by both arms)."""
    U, I, K, L, S = w["n_users"], w["n_items"], w["n_slots"], w["iters"], w["steps"]
    state_mb = 3 * U * w["n_cols"] * ((I + 7) // 8 * 8) * 4 / 1e6
    l2 = (f"state larger than L2 (C, m1, m2: {state_mb:.0f} MB read and written per ascent step)"
          if state_mb > 129 else f"state {state_mb:.1f} MB, L2-resident (not flushed)")
    return {"workload": args.workload, "n_users": U, "n_items": I, "n_slots": K,
            "n_cols": w["n_cols"], "sinkhorn_iters": L, "ascent_steps": S, "param": "full_cost",
            "optimizer": "adam lr 0.1", "step": f"reset + initial solve + {S} ascent steps",
            "l2": l2,
            "parallelism": f"independent markets x{world}" if world > 1 else "single market"}


def run_reference(args, w, budget_s=8.0):
    """The reference arm: the FP64 oracle on the host cores, each step a sample of `budget_s`
    seconds of the workload; rank 0 prints the line, other ranks return without work."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rates = []
    for j in range(args.warmup + args.steps):
        rate, info, dt = oracle_sample(w, seed=0, budget_s=budget_s)
        if j >= args.warmup:
            rates.append((rate, dt, info))
    value = statistics.median([x[0] for x in rates])
    ms = statistics.median([x[1] for x in rates]) * 1e3
    info = dict(rates[-1][2])
    info["value"] = value
    info["unit"] = UNIT
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args, w, 1), sample=info["sample"]),
            "impl": "reference", "cpu_baseline": info,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- multi-rank host logic (independent markets per rank, weak scaling) -----------------------
def rank_relevance(w, rank):
    """Rank `rank`'s market: the workload's relevance generator with seed = rank."""
    from paper_2406_10262_gb300 import synth
    return synth.relevance_lowrank(w["n_users"], w["n_items"], seed=rank).astype(np.float32)


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the whole job ends when the last rank does."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units all ranks processed per second (every rank does the same work)."""
    return world * units_per_rank / (ms * 1e-3)


# ---- our arm ------------------------------------------------------------------------------
def run_ours(args, w):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2406_10262_gb300 import build as frbuild
    frbuild.build()
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth

    U, I, K, L, S = w["n_users"], w["n_items"], w["n_slots"], w["iters"], w["steps"]
    nc = w["n_cols"]
    r = rank_relevance(w, rank)
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, sinkhorn_iters=L, lr=0.1)
    g.set_relevance(r)
    g.set_exposure(e)
    cells = U * I * nc
    cu_per_solve = cells * L * (S + 1)

    def solve():
        g.reset()
        g.step(S, trace=False)

    if args.profile_steps:
        g.step(args.profile_steps, trace=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_steps": args.profile_steps, "launches": g.launch_count()}))
        return

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        solve()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    barrier()
    l0 = g.launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        solve()
    ev1.record(stream)
    barrier()
    launches = g.launch_count() - l0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
    value = whole_job_rate(cu_per_solve, world, ms)

    # ---- time to NSW within 1e-5 of the FP64 oracle's F after the full step budget ----------
    F_ref = golden_F_ref(args.workload) if rank == 0 else None
    g.reset()
    trace = g.step(S, trace=True)
    ttn = None
    first = None
    if F_ref is not None:
        ok = np.nonzero(np.abs(trace - F_ref) <= NSW_TOL * abs(F_ref))[0]
        if ok.size:
            first = int(ok[0]) + 1
            g.reset()
            torch.cuda.synchronize()
            ev0.record(stream)
            g.step(first, trace=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            ttn = ev0.elapsed_time(ev1) * 1e-3

    # ---- end to end through the C-ABI with host buffers ------------------------------------
    r_pinned = torch.from_numpy(r).pin_memory()
    imp_host = None
    e2e_ms = []
    for j in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_relevance(r_pinned.numpy())       # H2D of the step's input from pinned memory
        g.reset()
        tr = g.step(S, trace=True)              # D2H of the NSW trace
        imp_host = g.impacts()[0]               # D2H of the impacts
        torch.cuda.synchronize()
        if j > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.median(e2e_ms)
    h2d = r.nbytes + e.nbytes
    d2h = S * 8 + I * 8 + 64

    # ---- roofline of the dominant kernel (fused gradient + Adam + Sinkhorn) ---------------
    g.reset()
    g.step(1, trace=False)
    kms = g.time_kernels(20)
    cu_alg = float(cells) * L  # one cell-update per cell per Sinkhorn iteration
    achieved = cu_alg / (kms[0] * 1e-3)
    peaks = fr.measure_peaks()
    peak_smem = peaks["smem_bytes_per_s_8B"] / CELL_BYTES_SMEM  # cell-updates/s
    bytes_alg = cells * 4 * 6 + U * I * 4  # read C, m, v + write C, m, v; read r
    hbm_gbs, hbm_src = hbm_peak_gbs()
    t_hbm = bytes_alg / (hbm_gbs * 1e9)
    t_mufu = cu_alg * (1.0 + 2.0 / nc) / peaks["ex2_per_s"]
    t_roof = max(t_hbm, t_mufu)
    roof = {"bound": "alu", "unit": "Gcell-updates/s", "achieved": achieved / 1e9,
            "peak": peak_smem / 1e9, "frac": achieved / peak_smem,
            "traffic": recorded_traffic(p1_kernel_name(g)),
            "kernel": p1_kernel_name(g), "kernel_ms": kms[0], "reduce_ms": kms[1],
            "sweep_only_ms": kms[2], "sweep_only_frac": cu_alg / (kms[2] * 1e-3) / peak_smem,
            "cell_updates_per_launch": cu_alg,
            "peak_source": "measured shared-memory load bandwidth (fr_measure_peaks, 8-byte "
            f"conflict-free loads: {peaks['smem_bytes_per_s_8B'] / 1e12:.2f} TB/s at "
            f"{peaks['sm_mhz']:.0f} MHz) / 4 B per cell-update",
            "method_bound": {
                "what": "slower of HBM bytes at the measured copy bandwidth and (1 + 2/m) MUFU "
                        "operations per cell-update at the measured ex2 rate",
                "bound": "mufu" if t_mufu >= t_hbm else "hbm", "t_roof_ms": t_roof * 1e3,
                "t_mufu_ms": t_mufu * 1e3, "t_hbm_ms": t_hbm * 1e3, "hbm_peak_gbs": hbm_gbs,
                "hbm_peak_source": hbm_src, "frac": t_roof / (kms[0] * 1e-3),
                "sweep_only_frac": t_mufu / (kms[2] * 1e-3)},
            "measured_peaks": {"ex2_per_s": peaks["ex2_per_s"],
                               "smem_bytes_per_s_8B": peaks["smem_bytes_per_s_8B"],
                               "smem_bytes_per_s_16B": peaks["smem_bytes_per_s_16B"],
                               "ffma_per_s": peaks["ffma_per_s"],
                               "ffma2_fmas_per_s": peaks["ffma2_fmas_per_s"],
                               "sm_mhz": peaks["sm_mhz"]},
            "log_form_solves": g.log_form_solves(),
            "hbm_bytes_per_launch": bytes_alg, "hbm_gbs": bytes_alg / (kms[0] * 1e-3) / 1e9}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, w, world),
            "time_to_nsw_s": ttn, "time_to_nsw_step": first, "nsw_final": float(trace[-1]),
            "nsw_ref_fp64": F_ref,
            "nsw_rel_err_final": None if F_ref is None else abs(float(trace[-1]) - F_ref) / abs(F_ref),
            "e2e": {"value": whole_job_rate(cu_per_solve, world, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": launches, "roofline": roof, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, info, _ = oracle_sample(w, seed=0, budget_s=12.0)
        info["value"] = rate
        info["unit"] = UNIT
        rate1, info1, _ = oracle_sample(w, seed=0, budget_s=6.0, threads=1, n_sub=40)
        info["single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": info1["sample"]}
        line["cpu_baseline"] = info
    if rank == 0 and world == 1 and not args.no_forms:
        g.close()  # frees the headline context's device state before the other workloads
        line["forms"] = measure_forms(peaks["ex2_per_s"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def mufu_frac(cell_updates, m, ms, ex2_per_s):
    """Fraction of the log-form Sinkhorn bound ((1 + 2/m) MUFU operations per cell-update at the
    measured ex2 rate) reached by a sweep of `cell_updates` that took `ms` milliseconds."""
    return cell_updates * (1.0 + 2.0 / m) / ex2_per_s / (ms * 1e-3)


def measure_forms(ex2_per_s):
    """Short measurements of the layered forms, recorded beside the headline (each in its own
    try block, so a failure is reported instead of losing the line):
    per_item: |U| = 20000, |I| = 2000, K = 20, L = 100 -- Sinkhorn sweep, implicit gradient and
    unrolled adjoint (checkpoints every 10, and every iteration) kernel times;
    free_cost_gradients: 2000 x 1000 x 11, L = 50 -- the fused implicit step and the unrolled
    gradient's kernels (checkpoints every 10, and every iteration); batch: the 256-market workload, 8 ascent steps batched against 256 contexts run one
    after another;
    metrics: fr_metrics (the envy contraction) at 20000 consumers x 10^4 items;
    precision: the precision workload (200000 x 10^4, K = 20, L = 50) with BF16 against FP32
    relevance storage, one ascent step from theta = 0 each: Sinkhorn kernel times, bytes of
    relevance and the relative difference of F.
    Sinkhorn kernels carry "sweep_mufu_frac": the log-form bound of (1 + 2/m) MUFU operations per
    cell-update at the measured ex2 rate over the kernel's time (the headline's method bound)."""
    import torch
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    out = {}
    try:
        U, I, K, L = 20000, 2000, 20, 100
        r = synth.relevance_lowrank_fast(U, I, seed=7)
        res = {"n_users": U, "n_items": I, "n_slots": K, "sinkhorn_iters": L, "ckpt_every": 10}
        cu = U * I * fr.num_cols(I, K) * L
        for name, mode in (("implicit", fr.GRAD_IMPLICIT), ("unrolled", fr.GRAD_UNROLLED)):
            g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, grad_mode=mode,
                            ckpt_every=10)
            g.set_relevance(r)
            g.set_exposure(synth.dcg_exposure(K))
            g.step(2, trace=False)
            ms = g.time_kernels(3)
            res[name] = {"sweep_ms": ms[0], "grad_ms": ms[2]}
            g.close()
        # a checkpoint every iteration: the sweep also keeps the column sums, no forward re-runs
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, grad_mode=fr.GRAD_UNROLLED,
                        ckpt_every=1)
        g.set_relevance(r)
        g.set_exposure(synth.dcg_exposure(K))
        g.step(2, trace=False)
        ms = g.time_kernels(3)
        res["unrolled_ckpt_every_1"] = {"sweep_ms": ms[0], "grad_ms": ms[2]}
        g.close()
        res["sweep_cell_updates_per_s"] = cu / (res["implicit"]["sweep_ms"] * 1e-3)
        res["sweep_mufu_frac"] = mufu_frac(cu, fr.num_cols(I, K), res["implicit"]["sweep_ms"], ex2_per_s)
        res["adjoint_over_sweep"] = res["unrolled"]["grad_ms"] / res["unrolled"]["sweep_ms"]
        res["adjoint_over_sweep_ckpt_every_1"] = (res["unrolled_ckpt_every_1"]["grad_ms"] /
                                                  res["unrolled_ckpt_every_1"]["sweep_ms"])
        out["per_item"] = res
    except Exception as ex:  # noqa: BLE001 -- reported in the line
        out["per_item"] = {"error": repr(ex)}
    try:
        U, I, K, L = 2000, 1000, 10, 50
        r = synth.workload_relevance("plain2000x1000").astype(np.float32)
        res = {"n_users": U, "n_items": I, "n_slots": K, "sinkhorn_iters": L}
        for name, mode, ce in (("implicit", fr.GRAD_IMPLICIT, 10), ("unrolled", fr.GRAD_UNROLLED, 10),
                               ("unrolled_ckpt_every_1", fr.GRAD_UNROLLED, 1)):
            g = fr.FairRank(U, I, K, sinkhorn_iters=L, grad_mode=mode, ckpt_every=ce)
            g.set_relevance(r)
            g.set_exposure(synth.dcg_exposure(K))
            g.step(3, trace=False)
            ms = g.time_kernels(5)
            keys = (("fused_step_ms", "reduce_ms", "sweep_only_ms") if mode == fr.GRAD_IMPLICIT
                    else ("sweep_ms", "reduce_ms", "adjoint_adam_ms"))
            res[name] = dict(zip(keys, (float(x) for x in ms)))
            g.close()
        out["free_cost_gradients"] = res
    except Exception as ex:  # noqa: BLE001
        out["free_cost_gradients"] = {"error": repr(ex)}
    try:
        c = compare_batch(argparse.Namespace(steps=1))
        out["batch"] = {k: c[k] for k in ("markets", "ascent_steps", "sinkhorn_iters", "cells",
                                          "batched_s", "sequential_s", "speedup",
                                          "batched_cell_updates_per_s", "max_rel_F_diff_final",
                                          "launches_per_run")}
    except Exception as ex:  # noqa: BLE001
        out["batch"] = {"error": repr(ex)}
    try:
        U, I, K = 20000, 10000, 20
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=20)
        g.set_relevance(synth.relevance_lowrank_fast(U, I, seed=3))
        g.set_exposure(synth.dcg_exposure(K))
        g.step(1, trace=False)
        g.metrics()
        ts = [_timed(g.metrics)[1] * 1e3 for _ in range(3)]
        out["metrics"] = {"n_users": U, "n_items": I, "n_slots": K, "fr_metrics_ms": statistics.median(ts),
                          "envy_tf32_products": 3 * U * I * I}
        g.close()
    except Exception as ex:  # noqa: BLE001
        out["metrics"] = {"error": repr(ex)}
    try:
        c = compare_bf16(argparse.Namespace(steps=1))
        res = {k: c[k] for k in ("n_users", "n_items", "n_slots", "sinkhorn_iters", "ascent_steps",
                                 "rel_F_diff_final", "sweep_speedup")}
        cu = c["n_users"] * c["n_items"] * fr.num_cols(c["n_items"], c["n_slots"]) * c["sinkhorn_iters"]
        for name in ("fp32", "bf16"):
            res[name] = {k: c[name][k] for k in ("sweep_ms", "grad_ms", "sweep_cell_updates_per_s",
                                                 "relevance_bytes", "F_final")}
            res[name]["sweep_mufu_frac"] = mufu_frac(
                cu, fr.num_cols(c["n_items"], c["n_slots"]), c[name]["sweep_ms"], ex2_per_s)
        out["precision"] = res
    except Exception as ex:  # noqa: BLE001
        out["precision"] = {"error": repr(ex)}
    torch.cuda.synchronize()
    return out


# ---- layered forms against the plain FP32 method ---------------------------------------------
def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def compare_batch(args):
    """256 independent markets: one fr_batch (autotuned buckets, concurrent persistent launches
    under a CUDA graph) against 256 FairRank contexts run one after another; the same S ascent
    steps from theta = 0 in both, F of every market compared."""
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    S, L = max(args.steps, 1) * 8, 50
    ms = synth.markets(256, seed=0)
    sizes = [(m.n_users, m.n_items, m.n_slots) for m in ms]
    rs = [synth.relevance_lowrank_fast(m.n_users, m.n_items, seed=m.seed) for m in ms]
    cells = sum(U * I * fr.num_cols(I, K) for U, I, K in sizes)
    b = fr.FairRankBatch(sizes, sinkhorn_iters=L)
    for j, ((U, I, K), r) in enumerate(zip(sizes, rs)):
        b.set_relevance(j, r)
        b.set_exposure(j, synth.dcg_exposure(K))
    _, tune_s = _timed(b.autotune)
    b.step(2, trace=False)  # warm-up (graph capture)
    b.reset()
    l0 = b.launch_count()
    Fb, t_batch = _timed(lambda: b.step(S))
    launches = b.launch_count() - l0
    ctxs = []
    for (U, I, K), r in zip(sizes, rs):
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L)
        g.set_relevance(r)
        g.set_exposure(synth.dcg_exposure(K))
        g.step(S, trace=False)  # warm-up (graph capture)
        g.reset()
        ctxs.append(g)
    Fs, t_seq = _timed(lambda: [g.step(S) for g in ctxs])
    Fs = np.array(Fs).T
    rel_F = float(np.max(np.abs(Fb[-1] - Fs[-1]) / np.abs(Fs[-1])))
    cu = cells * L * (S + 1)
    return {"compare": "batch", "markets": 256, "ascent_steps": S, "sinkhorn_iters": L,
            "cells": cells, "cell_updates": cu, "batched_s": t_batch, "sequential_s": t_seq,
            "speedup": t_seq / t_batch, "batched_cell_updates_per_s": cu / t_batch,
            "sequential_cell_updates_per_s": cu / t_seq, "max_rel_F_diff_final": rel_F,
            "autotune_s": tune_s, "buckets": b.tuning(), "launches_per_run": launches}


def compare_unrolled(args):
    """|U| = 20000, |I| = 2000, K = 20, L = 100: ascent driven by the unrolled adjoint gradient
    (checkpoints every 10 iterations) against the implicit gradient, same S steps from theta = 0;
    both gradients also taken at one common state."""
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    U, I, K, L, S = 20000, 2000, 20, 100, max(args.steps, 1) * 4
    r = synth.relevance_lowrank_fast(U, I, seed=7)
    out = {"compare": "unrolled", "n_users": U, "n_items": I, "n_slots": K, "sinkhorn_iters": L,
           "ckpt_every": 10, "ascent_steps": S}
    res = {}
    for name, mode in (("implicit", fr.GRAD_IMPLICIT), ("unrolled", fr.GRAD_UNROLLED)):
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, grad_mode=mode,
                        ckpt_every=10)
        g.set_relevance(r)
        g.set_exposure(synth.dcg_exposure(K))
        g.step(2, trace=False)
        g.reset()
        F, t = _timed(lambda: g.step(S))
        kms = g.time_kernels(3)
        g.reset()
        g.impacts()
        res[name] = g.grad()
        out[name] = {"s_per_run": t, "ms_per_step": t / S * 1e3, "F_final": float(F[-1]),
                     "sweep_ms": kms[0], "reduce_ms": kms[1], "grad_ms": kms[2]}
    a, c = res["implicit"].astype(np.float64), res["unrolled"].astype(np.float64)
    out["rel_F_diff_final"] = abs(out["unrolled"]["F_final"] - out["implicit"]["F_final"]) / \
        abs(out["implicit"]["F_final"])
    out["grad_rel_l2_diff_at_theta0"] = float(np.linalg.norm(a - c) / np.linalg.norm(a))
    out["grad_cosine_at_theta0"] = float(a @ c / (np.linalg.norm(a) * np.linalg.norm(c)))
    out["unrolled_over_implicit_time"] = out["unrolled"]["s_per_run"] / out["implicit"]["s_per_run"]
    # free costs (the paper's parametrisation) on the benchmark workload: dL/dc of every cell
    U1, I1, K1, L1, S1 = 2000, 1000, 10, 50, max(args.steps, 1) * 20
    r1 = synth.relevance_lowrank(U1, I1, seed=0).astype(np.float32)
    fc, res1 = {"n_users": U1, "n_items": I1, "n_slots": K1, "sinkhorn_iters": L1, "ckpt_every": 10,
                "ascent_steps": S1}, {}
    for name, mode in (("implicit", fr.GRAD_IMPLICIT), ("unrolled", fr.GRAD_UNROLLED)):
        g = fr.FairRank(U1, I1, K1, param=fr.PARAM_FULL_C, sinkhorn_iters=L1, grad_mode=mode,
                        ckpt_every=10)
        g.set_relevance(r1)
        g.set_exposure(synth.dcg_exposure(K1))
        g.step(2, trace=False)
        g.reset()
        F, t = _timed(lambda: g.step(S1))
        kms = g.time_kernels(3)
        g.reset()
        g.step(3, trace=False)
        res1[name] = g.grad()
        fc[name] = {"s_per_run": t, "ms_per_step": t / S1 * 1e3, "F_final": float(F[-1]),
                    "kernel_ms": list(kms)}
        g.close()
    a, c = res1["implicit"].astype(np.float64).ravel(), res1["unrolled"].astype(np.float64).ravel()
    fc["rel_F_diff_final"] = abs(fc["unrolled"]["F_final"] - fc["implicit"]["F_final"]) / \
        abs(fc["implicit"]["F_final"])
    fc["grad_rel_l2_diff_after_3_steps"] = float(np.linalg.norm(a - c) / np.linalg.norm(a))
    fc["grad_cosine_after_3_steps"] = float(a @ c / (np.linalg.norm(a) * np.linalg.norm(c)))
    fc["unrolled_over_implicit_time"] = fc["unrolled"]["s_per_run"] / fc["implicit"]["s_per_run"]
    out["free_costs"] = fc
    return out


def compare_p1_batch(args):
    """The batching workload's 256 markets (|U| ~ U[100, 4000], |I| ~ U[100, 2000], K in
    {5, 10, 20}) under free costs: one batch (autotuned chunk lengths, one launch per kernel
    variant per step on concurrent branches, graph-captured) against the 256 markets as single
    contexts run one after another, the same S ascent steps from C = 0; F of every market
    compared."""
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    S, L = max(args.steps, 1) * 8, 50
    ms = synth.markets(256, seed=0)
    sizes = [(m.n_users, m.n_items, m.n_slots) for m in ms]
    rs = [synth.relevance_lowrank_fast(m.n_users, m.n_items, seed=m.seed) for m in ms]
    cells = sum(U * I * fr.num_cols(I, K) for U, I, K in sizes)
    b = fr.FairRankBatch(sizes, param=fr.PARAM_FULL_C, sinkhorn_iters=L)
    for j, ((U, I, K), r) in enumerate(zip(sizes, rs)):
        b.set_relevance(j, r)
        b.set_exposure(j, synth.dcg_exposure(K))
    _, tune_s = _timed(b.autotune)
    b.step(2, trace=False)  # warm-up (graph capture)
    b.reset()
    l0 = b.launch_count()
    Fb, t_batch = _timed(lambda: b.step(S))
    launches = b.launch_count() - l0
    tuning = b.tuning()
    b.close()
    Fs, t_seq = [], 0.0
    for (U, I, K), r in zip(sizes, rs):  # one context at a time (its state freed before the next)
        g = fr.FairRank(U, I, K, param=fr.PARAM_FULL_C, sinkhorn_iters=L)
        g.set_relevance(r)
        g.set_exposure(synth.dcg_exposure(K))
        g.step(S, trace=False)  # warm-up (graph capture)
        g.reset()
        F, t = _timed(lambda: g.step(S))
        Fs.append(F)
        t_seq += t
        g.close()
    Fs = np.array(Fs).T
    cu = cells * L * (S + 1)
    return {"compare": "p1-batch", "markets": len(sizes), "ascent_steps": S, "sinkhorn_iters": L,
            "cells": cells, "state_bytes": 3 * 4 * sum(U * fr.num_cols(I, K) * ((I + 7) // 8 * 8)
                                                        for U, I, K in sizes),
            "batch_s": t_batch, "sequential_s": t_seq, "speedup": t_seq / t_batch,
            "batch_cell_updates_per_s": cu / t_batch, "sequential_cell_updates_per_s": cu / t_seq,
            "autotune_s": tune_s, "batch_launches": launches, "buckets": tuning,
            "rel_F_diff_final_max": float(np.max(np.abs(Fb[-1] - Fs[-1]) / np.abs(Fs[-1])))}


def compare_bf16(args):
    """|U| = 200000, |I| = 10^4, K = 20, L = 50: BF16 against FP32 relevance storage, same S steps
    from theta = 0; F of both and the Sinkhorn kernel time."""
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    U, I, K, L, S = 200000, 10000, 20, 50, max(args.steps, 1)
    blk = 20000
    r32 = np.empty((U, I), dtype=np.float32)
    for u0 in range(0, U, blk):
        r32[u0:u0 + blk] = synth.relevance_lowrank_fast(U, I, seed=0, boost_frac=0.05, row0=u0,
                                                        rows=min(blk, U - u0))
    out = {"compare": "bf16", "n_users": U, "n_items": I, "n_slots": K, "sinkhorn_iters": L,
           "ascent_steps": S}
    cu = U * I * fr.num_cols(I, K) * L
    for name, dt in (("fp32", fr.F32), ("bf16", fr.BF16)):
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, rel_dtype=dt)
        g.set_relevance(r32 if dt == fr.F32 else synth.to_bf16_bits(r32))
        g.set_exposure(synth.dcg_exposure(K))
        g.impacts()
        F, t = _timed(lambda: g.step(S))
        kms = g.time_kernels(2)
        out[name] = {"s_per_run": t, "ms_per_step": t / S * 1e3, "F_final": float(F[-1]),
                     "sweep_ms": kms[0], "grad_ms": kms[2], "reduce_ms": kms[1],
                     "sweep_cell_updates_per_s": cu / (kms[0] * 1e-3),
                     "relevance_bytes": U * ((I + 7) // 8 * 8) * (4 if dt == fr.F32 else 2)}
        del g
    out["rel_F_diff_final"] = abs(out["bf16"]["F_final"] - out["fp32"]["F_final"]) / \
        abs(out["fp32"]["F_final"])
    out["sweep_speedup"] = out["fp32"]["sweep_ms"] / out["bf16"]["sweep_ms"]
    return out


def compare_precision(args):
    """The precision workload against the FP64 oracle: |U| = 200000, |I| = 10^4, K = 20, L = 50,
    rank-32 sigmoid relevance with 5% boosted items stored in BF16, S ascent steps from theta = 0
    on the GPU. The oracle then solves a seeded sample of 1000 consumers at the GPU's final theta
    from the GPU's warm start of the last solve (the same L iterations), once on the BF16-rounded
    relevance the GPU used (the kernels' error) and once on the FP32 relevance (with the
    quantisation error): the policy's largest absolute difference and the relative error of the
    sample's impacts and of its NSW (sum_i log of the sample's impacts). With --full-oracle it also
    runs one oracle forward over all consumers (in chunks of 2000; about 2 x 10^12 cell-updates of
    host time) and reports F against the GPU's F of the whole market."""
    import oracle
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    U, I, K, L, S = 200000, 10000, 20, 50, max(args.steps, 1) * 2
    n_sample, blk = 1000, 20000
    r32 = np.empty((U, I), dtype=np.float32)
    for u0 in range(0, U, blk):
        r32[u0:u0 + blk] = synth.relevance_lowrank_fast(U, I, seed=0, boost_frac=0.05, row0=u0,
                                                        rows=min(blk, U - u0))
    rb = synth.to_bf16_bits(r32)
    e = synth.dcg_exposure(K)
    g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, rel_dtype=fr.BF16)
    g.set_relevance(rb)
    g.set_exposure(e)
    g.impacts()
    if S > 1:
        g.step(S - 1, trace=False)
    _, _, _, g0, _ = g.get_state()  # warm start of the last solve
    F_trace = g.step(1)
    theta, _, _, _, t = g.get_state()
    imp_gpu, _, F_gpu = g.impacts()
    sample = np.sort(np.random.default_rng(2026).choice(U, n_sample, replace=False))
    X_gpu = np.stack([g.policy(int(u), 1)[0] for u in sample]).astype(np.float64)
    del g
    nc = fr.num_cols(I, K)
    e_pad = np.r_[e, np.zeros(nc - K)]
    out = {"compare": "precision", "n_users": U, "n_items": I, "n_slots": K, "sinkhorn_iters": L,
           "ascent_steps": S, "relevance": "bf16", "sample_consumers": n_sample,
           "sample": "seeded uniform sample of consumers (numpy default_rng(2026))",
           "F_gpu": float(F_gpu), "F_trace_last": float(F_trace[-1])}
    rs_b = synth.bf16_bits_to_f64(rb[sample])
    for name, r_s in (("vs_bf16_relevance", rs_b), ("vs_fp32_relevance", r32[sample].astype(np.float64))):
        o = oracle.Oracle(n_sample, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=True)
        o.set_relevance(r_s)
        o.set_exposure(e)
        o.set_state(param=theta.astype(np.float64), g=g0[sample].astype(np.float64))
        imp_o, _, F_o = o.impacts()
        X_o = o.policy()
        imp_g = (r_s * (X_gpu @ e_pad)).sum(axis=0)  # the sample's impacts from the GPU policy
        F_g = float(np.sum(np.log(imp_g)))
        out[name] = {"x_max_abs_err": float(np.max(np.abs(X_gpu - X_o))),
                     "sample_imp_max_rel_err": float(np.max(np.abs(imp_g - imp_o) / imp_o)),
                     "sample_F_oracle": float(F_o), "sample_F_gpu_policy": F_g,
                     "sample_F_rel_err": abs(F_g - F_o) / abs(F_o)}
        del o, X_o
    if args.full_oracle:
        chunk, imp_full = 2000, np.zeros(I)
        t0 = time.perf_counter()
        for u0 in range(0, U, chunk):
            u1 = min(U, u0 + chunk)
            o = oracle.Oracle(u1 - u0, I, K, param=oracle.PARAM_ITEM, iters=L, warm_start=True)
            o.set_relevance(synth.bf16_bits_to_f64(rb[u0:u1]))
            o.set_exposure(e)
            o.set_state(param=theta.astype(np.float64), g=g0[u0:u1].astype(np.float64))
            imp_full += o.impacts()[0]
            del o
        F_full = float(np.sum(np.log(imp_full)))
        out["full_oracle"] = {"F_oracle": F_full, "F_rel_err": abs(F_gpu - F_full) / abs(F_full),
                              "imp_max_rel_err": float(np.max(np.abs(imp_gpu - imp_full) / imp_full)),
                              "oracle_seconds": time.perf_counter() - t0,
                              "oracle_threads": os.cpu_count()}
    return out


def compare_p1_scale(args):
    """The free-cost parametrisation (the paper's Problem (8)) at the sizes of the differentiation
    and batching workloads: (a) |U| = 20000, |I| = 2000, K = 20 (21 columns), L = 100, S ascent
    steps (implicit gradient, Adam) from C = 0 with the per-step kernel times; (b) the 256 markets
    of the batching workload's size distribution, each a free-cost context created, advanced S
    steps from C = 0 and destroyed in turn (one market's state on the device at a time)."""
    import torch
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    out = {"compare": "p1-scale"}
    U, I, K, L, S = 20000, 2000, 20, 100, max(args.steps, 1) * 2
    r = synth.relevance_lowrank_fast(U, I, seed=7)
    g = fr.FairRank(U, I, K, sinkhorn_iters=L, lr=0.1)
    g.set_relevance(r)
    g.set_exposure(synth.dcg_exposure(K))
    g.step(1, trace=False)  # warm-up (graph capture)
    g.reset()
    F, t = _timed(lambda: g.step(S))
    kms = g.time_kernels(3)
    nc = fr.num_cols(I, K)
    out["differentiation_size"] = {
        "n_users": U, "n_items": I, "n_slots": K, "n_cols": nc, "sinkhorn_iters": L,
        "ascent_steps": S, "s_per_run": t, "F": [float(x) for x in F],
        "fused_ms": kms[0], "reduce_ms": kms[1], "sweep_only_ms": kms[2],
        "sweep_cell_updates_per_s": U * I * nc * L / (kms[2] * 1e-3),
        "state_bytes": 3 * U * nc * ((I + 7) // 8 * 8) * 4}
    del g
    S2, L2 = max(args.steps, 1) * 8, 50
    ms = synth.markets(256, seed=0)
    cells, t_dev, t_all, Fs = 0, 0.0, 0.0, []
    for m in ms:
        U, I, K = m.n_users, m.n_items, m.n_slots
        r = synth.relevance_lowrank_fast(U, I, seed=m.seed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = fr.FairRank(U, I, K, sinkhorn_iters=L2)
        g.set_relevance(r)
        g.set_exposure(synth.dcg_exposure(K))
        F, t = _timed(lambda: g.step(S2))
        del g
        torch.cuda.synchronize()
        t_all += time.perf_counter() - t0
        t_dev += t
        cells += U * I * fr.num_cols(I, K)
        Fs.append(float(F[-1]))
    cu = cells * L2 * (S2 + 1)
    out["batching_markets"] = {
        "markets": len(ms), "ascent_steps": S2, "sinkhorn_iters": L2, "cells": cells,
        "cell_updates": cu, "step_s": t_dev, "with_setup_s": t_all,
        "cell_updates_per_s": cu / t_dev, "F_min": min(Fs), "F_max": max(Fs),
        "all_F_finite": bool(np.all(np.isfinite(Fs)))}
    return out


def compare_paper_shapes(args):
    """Computation time per ascent step of the free-cost method (the paper's Algorithm 1, K = 10,
    m = 11, L = 50) on the shapes of the paper's timing figure: |U| swept at |I| = 250 and |I|
    swept at |U| = 250, the GPU (100 steps under the step graphs) next to the FP64 oracle on the
    host cores (cpu_baseline leg: 3 steps per shape, per-step time)."""
    import oracle
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    K, L, S = 10, 50, 100
    cores = os.cpu_count() or 1
    shapes = [(U, 250) for U in (250, 500, 1000, 2000, 4000)] + [(250, I) for I in (500, 1000, 2000)]
    points = []
    for U, I in shapes:
        r = synth.relevance_lowrank(U, I, seed=5).astype(np.float32)
        e = synth.dcg_exposure(K)
        g = fr.FairRank(U, I, K, sinkhorn_iters=L, lr=0.1)
        g.set_relevance(r)
        g.set_exposure(e)
        g.step(S, trace=False)  # warm-up, graph capture
        g.reset()
        g.impacts()
        _, t_gpu = _timed(lambda: g.step(S, trace=False))
        o = oracle.Oracle(U, I, K, iters=L, lr=0.1, threads=cores)
        o.set_relevance(r.astype(np.float64))
        o.set_exposure(e)
        o.impacts()
        t0 = time.perf_counter()
        o.step(3)
        t_cpu = (time.perf_counter() - t0) / 3
        points.append({"n_users": U, "n_items": I, "gpu_ms_per_step": t_gpu / S * 1e3,
                       "cpu_ms_per_step": t_cpu * 1e3, "speedup": t_cpu / (t_gpu / S)})
        del g, o
    return {"compare": "paper-shapes", "n_slots": K, "n_cols": K + 1, "sinkhorn_iters": L,
            "cpu_cores": cores, "cpu": "FP64 oracle, OpenMP over consumers", "points": points}


def profile_item(args):
    """Sets up one per-item workload and runs --profile-steps ascent steps (for ncu captures):
    implicit / unrolled: 20000 x 2000, K = 20, L = 100 (checkpoints every 10); bf16: 200000 x 10^4,
    K = 20, L = 50, BF16 relevance; batch: the 256-market workload, L = 50, autotuned and warmed up
    first, the n steps between profiler start and stop (ncu --profile-from-start off); metrics: 20000 x 10^4,
    K = 20, L = 20, then one fr_metrics call (the envy contraction)."""
    import torch
    from paper_2406_10262_gb300 import fairrank as fr
    from paper_2406_10262_gb300 import synth
    n = max(args.profile_steps, 1)
    if args.profile_item == "batch":
        ms = synth.markets(256, seed=0)
        sizes = [(m.n_users, m.n_items, m.n_slots) for m in ms]
        b = fr.FairRankBatch(sizes, sinkhorn_iters=50)
        for j, m in enumerate(ms):
            b.set_relevance(j, synth.relevance_lowrank_fast(m.n_users, m.n_items, seed=m.seed))
            b.set_exposure(j, synth.dcg_exposure(m.n_slots))
        b.autotune()
        b.step(1, trace=False)  # warm-up; captures may start at the profiler start below
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        b.step(n, trace=False)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        launches = b.launch_count()
    elif args.profile_item == "metrics":
        U, I, K = args.profile_users or 20000, args.profile_items or 10000, 20
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=20)
        g.set_relevance(synth.relevance_lowrank_fast(U, I, seed=5))
        g.set_exposure(synth.dcg_exposure(K))
        g.step(n, trace=False)
        g.metrics()
        launches = g.launch_count()
    else:
        bf16 = args.profile_item == "bf16"
        U, I, K, L = (200000, 10000, 20, 50) if bf16 else (20000, 2000, 20, 100)
        U = args.profile_users or U
        r = synth.relevance_lowrank_fast(U, I, seed=0, boost_frac=0.05 if bf16 else 0.0)
        mode = fr.GRAD_UNROLLED if args.profile_item == "unrolled" else fr.GRAD_IMPLICIT
        g = fr.FairRank(U, I, K, param=fr.PARAM_ITEM, sinkhorn_iters=L, grad_mode=mode,
                        ckpt_every=10, rel_dtype=fr.BF16 if bf16 else fr.F32)
        g.set_relevance(synth.to_bf16_bits(r) if bf16 else r)
        g.set_exposure(synth.dcg_exposure(K))
        g.step(n, trace=False)
        launches = g.launch_count()
    torch.cuda.synchronize()
    print(json.dumps({"profile_item": args.profile_item, "profile_steps": n, "launches": launches}))


def main():
    args = parse()
    if args.profile_item:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2406_10262_gb300 import build as frbuild
        frbuild.build()
        profile_item(args)
        return
    if args.compare:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2406_10262_gb300 import build as frbuild
        frbuild.build()
        fn = {"batch": compare_batch, "unrolled": compare_unrolled, "bf16": compare_bf16,
              "paper-shapes": compare_paper_shapes, "p1-scale": compare_p1_scale,
              "precision": compare_precision, "p1-batch": compare_p1_batch}[args.compare]
        print(json.dumps(fn(args)), flush=True)
        return
    w = workload(args.workload)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
