#!/usr/bin/env python3
"""Benchmark of the GAME generation step on one GB300 (or N independent
replicas under torchrun), printing one JSON line.

Workload (default): the large classification set, M = 1,000,000 patterns,
N = 32 correlated features scaled to [-1, 1], Chebyshev degree 8 (K = 257
genes), P = 1024 chromosomes, sign targets with 5% flips; seeded synthetic
data generated on the host and uploaded before timing. One step is one
generation: selection / crossover / mutation kernels, the population pack,
the fused fitness contraction (tensor cores, BF16 operands, FP32
accumulation), the FP64 cross-tile error sum and the re-scoring of the 16 best
candidates (FP64, by the Gram form of the MSE) before the next elitism decision. The plain FP32 CUDA-core
form of the same step is timed beside it, and a sample of chromosomes is
re-scored by the FP64 oracle to state the accuracy of both.

Metric: chromosome-pattern fitness evaluations per second (M * P / step
time), whole job (sum over ranks / max time). `--impl reference` times the
FP64 CPU oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("chromosome-pattern fitness evals/s and generations/s vs plain FP32 GPU "
          "at stated accuracy")
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--M", type=int, default=1_000_000, help="patterns (smaller for profiling)")
    ap.add_argument("--form", choices=["bf16", "bf16x3", "fp8", "fp32", "gram"], default="bf16")
    ap.add_argument("--workload", choices=["classification", "batched", "surrogate", "paper"],
                    default="classification",
                    help="batched: 256 independent runs of uneven shape, one graph per "
                         "generation; surrogate: the 4M-pattern regression set with "
                         "surrogate-screened offspring, against the plain FP32 form; paper: "
                         "the degree x iterations grid of Section 5 in the paper-literal "
                         "mode on a set of the paper's data shape")
    ap.add_argument("--error", choices=["mse", "rmse", "mae"], default="mse",
                    help="classification workload: the fitness's error function (Section 3)")
    ap.add_argument("--oversample", type=int, default=8, metavar="O",
                    help="surrogate workload: offspring per kept child (game_params.oversample)")
    ap.add_argument("--surrogate-steps", type=int, default=8, metavar="S",
                    help="surrogate workload: Adam steps per generation on each stored "
                         "generation (game_params.surrogate_steps)")
    ap.add_argument("--selection", choices=["ranking", "roulette"], default="ranking",
                    help="paper workload: parent selection (Section 5 names both)")
    ap.add_argument("--oracle-run", type=int, default=0, metavar="G",
                    help="surrogate workload: also run G generations of the FP64 oracle GA "
                         "(Gram form) and of the screened GPU GA and compare the best fitness")
    ap.add_argument("--no-fp32-leg", action="store_true")
    ap.add_argument("--no-batched-leg", action="store_true",
                    help="classification workload at one GPU: skip the batched workload's "
                         "leg (256 independent runs, 10 generations) added to the line")
    ap.add_argument("--no-surrogate-leg", action="store_true",
                    help="classification workload at one GPU: skip the surrogate workload's "
                         "legs (4M patterns, screened BF16 vs plain FP32) added to the line")
    ap.add_argument("--surrogate-oracle-run", type=int, default=300, metavar="G",
                    help="surrogate legs: generations of the final-best comparison with the "
                         "FP64 oracle GA (0 = off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--precision-report", type=int, default=4, metavar="G",
                    help="generations of the per-form accuracy report (0 = off)")
    ap.add_argument("--classify-run", type=int, default=200, metavar="G",
                    help="classification workload: after the timed steps, G more generations, "
                         "then accuracy / completeness / contamination of the best chromosome "
                         "(0 = off)")
    return ap.parse_args()


# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture), per workload and form, with the
# digest of the kernel sources the capture ran: reported only while the
# sources are unchanged (null once the kernel has changed since).
NCU_TRAFFIC = {("M1000000_N32_cheb8_P1024_cls", "bf16"): (132.64e6 + 3.21e6, "014c5a2ac9e5a2bc")}
KERNEL_SOURCES = ("fitness_tc.cu", "fitness_tc2.cu", "tc_common.cuh", "tc_ptx.cuh",
                  "basis.cuh")


def kernel_digest():
    """sha256 (first 16 hex digits) of the fused fitness kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1211_5481_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, form):
    entry = NCU_TRAFFIC.get((workload, form))
    if entry is None or entry[1] != kernel_digest():
        return None
    return entry[0]


def max_over_ranks(t, world, dev=None):
    """The slowest rank's time, returned on every rank (t itself when there
    is one rank): the all-reduce runs on dev for NCCL, on the host for gloo."""
    if world <= 1:
        return float(t)
    import torch
    import torch.distributed as dist
    if dev is None or dist.get_backend() == "gloo":
        dev = torch.device("cpu")
    tt = torch.tensor([float(t)], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank, t_step_s, world):
    """Units processed by all ranks (the same per rank: weak scaling) per
    second of the slowest rank's step."""
    return units_per_rank * world / t_step_s


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool = True):
        self.proc = None
        self.index = index
        if enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


def oracle_sample_rate(pr, P_s, target_s=8.0, max_s=25.0):
    """FP64 oracle (direct form, all host cores) evals/s on a bounded sample:
    the first M_s patterns x P_s chromosomes, M_s doubled until one call takes
    target_s seconds."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    pop = oracle.init_population(2, P_s, pr.K)
    M_s = 2000
    while True:
        t0 = time.perf_counter()
        oracle.fitness(pr.X[:M_s], pr.y[:M_s], pop, pr.degree, pr.basis)
        dt = time.perf_counter() - t0
        if dt >= target_s or M_s >= pr.M or dt * 2 > max_s:
            break
        M_s = min(pr.M, M_s * 2 if dt < target_s / 4 else int(M_s * target_s / max(dt, 1e-3)))
    return {"value": M_s * P_s / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {M_s} patterns x {P_s} chromosomes of the workload, "
                      f"direct-form FP64 fitness, {dt:.2f} s"}, M_s


def oracle_extra(pr, M_s, cpu):
    """The direct-form oracle on one core (a 1/cores sample), its estimated
    time per generation of the whole workload on all cores, and the Gram
    form (a different algorithm: G built once, then P K^2 per generation),
    timed on a 100,000-pattern build scaled to M and one full generation."""
    import oracle
    cores = cpu["cores"]
    P = pr.P
    pop = oracle.init_population(2, 16, pr.K)
    M_1 = max(2000, M_s // max(cores, 1))
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.fitness(pr.X[:M_1], pr.y[:M_1], pop, pr.degree, pr.basis)
    t1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    M_g = min(pr.M, 100_000)
    t0 = time.perf_counter()
    gs = oracle.gram(pr.X[:M_g], pr.y[:M_g], pr.degree, pr.basis)
    t_build = (time.perf_counter() - t0) * pr.M / M_g
    popP = oracle.init_population(3, P, pr.K)
    t0 = time.perf_counter()
    oracle.fitness_gram(gs, popP)
    t_gen = time.perf_counter() - t0
    return {"one_core": {"value": M_1 * 16 / t1, "unit": UNIT, "cores": 1,
                         "sample": f"first {M_1} patterns x 16 chromosomes"},
            "direct_generation_s_all_cores": pr.M * P / cpu["value"],
            "gram_form": {"build_s_estimate": t_build, "generation_s": t_gen,
                          "note": "Gram form of the MSE: a different algorithm, G built "
                                  f"once (timed on {M_g} patterns, scaled to M), then "
                                  "P K^2 FP64 per generation"}}


def precision_report(game, g, pr, G, M_sub=10_000, seed=2):
    """Accuracy of every contraction form against the FP64 oracle, per
    generation of the GA run held by handle g: the current population is
    evaluated on the first M_sub patterns by each form (a handle on that
    subset) and by the oracle; reported per form and generation: the max and
    median relative fitness error, the overlap of the form's 10 best with
    the oracle's 10 best (for BF16 and FP8 also after re-scoring the 8 or 16
    best in FP64, as the operators see it) and the Spearman rank correlation
    with the oracle over the whole population."""
    import oracle
    oracle.build()
    forms = {"fp32": game.GAME_PREC_FP32, "bf16": game.GAME_PREC_BF16,
             "bf16x3": game.GAME_PREC_BF16X3, "fp8": game.GAME_PREC_FP8}
    Xs, ys = pr.X[:M_sub], pr.y[:M_sub]
    sub = game.Game(Xs, ys, pr.degree, pr.basis, P=g.P, precision=game.GAME_PREC_FP32)
    rows = {f: [] for f in forms}
    gens = []
    for step in range(G):
        pop, _, gen = g.population()
        ref = oracle.fitness(Xs, ys, pop, pr.degree, pr.basis)
        best = set(np.argsort(ref, kind="stable")[:10])
        for name, prec in forms.items():
            f = sub.eval_fitness(pop, precision=prec)
            rel = np.abs(f - ref) / np.abs(ref)
            row = {"max_rel_err": float(rel.max()), "median_rel_err": float(np.median(rel)),
                   "top10_agreement": len(best & set(np.argsort(f, kind="stable")[:10])) / 10,
                   "spearman_all": spearman(f, ref)}
            if prec in (game.GAME_PREC_BF16, game.GAME_PREC_FP8):
                # the vector the operators rank: the best re-scored in FP64
                for n in (8, 16):
                    fr, _ = sub.rescore_top(pop, f, n)
                    row[f"top10_agreement_rescored_{n}"] = len(
                        best & set(np.argsort(fr, kind="stable")[:10])) / 10
            rows[name].append(row)
        gens.append(int(gen))
        if step + 1 < G:
            game.game_generation(g.h, seed)
    sub.close()
    return {"subset_patterns": M_sub, "generations": gens, "forms": rows}


def workload(M):
    from paper_1211_5481_gb300 import datagen as dg
    pr = dg.large_classification(M=M)
    return pr


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pr = workload(args.M)
    P = pr.P
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    # size one step so that the whole run (warm-up and timed steps) takes
    # about 100 s of CPU work, at most 2 s per step
    target = min(2.0, max(0.01, 100.0 / max(args.steps + args.warmup, 1)))
    _, M_s = oracle_sample_rate(pr, 16, target_s=target, max_s=3 * target)
    pop = oracle.init_population(2, 16, pr.K)
    for _ in range(args.warmup):
        oracle.fitness(pr.X[:M_s], pr.y[:M_s], pop, pr.degree, pr.basis)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fitness(pr.X[:M_s], pr.y[:M_s], pop, pr.degree, pr.basis)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = M_s * 16 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": pr.name, "M": pr.M, "N": pr.N, "degree": pr.degree,
                       "K": pr.K, "P": P, "basis": "chebyshev",
                       "step": f"oracle direct-form fitness of 16 chromosomes over the first "
                               f"{M_s} patterns"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {M_s} patterns x 16 chromosomes per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batched(args, torch, game, dev, world, rank):
    """The batched workload's JSON line (see batched_line)."""
    line = batched_line(args.steps, args.warmup, args.no_clocks, torch, game, dev, world)
    if rank == 0:
        print(json.dumps(line))


def batched_line(steps, warmup, no_clocks, torch, game, dev, world):
    """256 independent GA runs (M log-uniform in [10^3, 2 10^5], N in 4..64,
    Chebyshev or trigonometric basis of degree 2..10, P log-uniform in
    [32, 512], regression targets), advanced together: one step = one
    generation of every run = one CUDA-graph replay (batched operators, pack,
    one persistent tensor-core fitness launch, FP64 reduce). Returns the
    workload's JSON line."""
    from paper_1211_5481_gb300 import datagen as dg
    runs = dg.batched_runs(R=256)
    args_b = [(pr.X, pr.y, pr.degree, pr.basis, pr.P, 1000 + r) for r, pr in enumerate(runs)]
    bs = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    b = game.Batch(args_b, autotune=True, stream=bs)
    create_s = time.perf_counter() - t0
    tiles = b.tiles()
    evals = float(sum(pr.M * pr.P for pr in runs))
    flops = float(sum(2.0 * pr.M * pr.P * (pr.K - 1) + 3.0 * pr.M * pr.P for pr in runs))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(warmup, 3)):
        b.generation()
    b.sync()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")), enabled=not no_clocks)
    ev = []
    with torch.cuda.stream(bs):
        for _ in range(steps):
            flush.zero_()   # L2 flush between steps, outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(bs)
            b.generation()
            e1.record(bs)
            ev.append((e0, e1))
    b.sync()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t_step = max_over_ranks(sum(x.elapsed_time(y) for x, y in ev) / len(ev) * 1e-3, world, dev)
    fit_ms = b.fitness_ms(10)
    peaks, peak_src = load_peaks()
    achieved = flops / (fit_ms * 1e-3) / 1e12
    peak = float(peaks["bf16_tflops"])
    # algorithmic bytes of one launch: features, targets, operand image, partials
    nbytes = float(sum(4.0 * pr.M * pr.N + 4.0 * pr.M + 2.0 * pr.P * (pr.K - 1)
                       + 8.0 * -(-pr.M // 128) * pr.P for pr in runs))
    hbm_gbs = nbytes / (fit_ms * 1e-3) / 1e9
    hbm_peak = float(peaks["hbm_gbs"])
    line = {
        "metric": METRIC, "value": whole_job_rate(evals, t_step, world), "unit": UNIT,
        "n_gpus": world,
        "steps": steps, "warmup": max(warmup, 3), "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "batched_256_runs", "runs": len(runs),
                   "sum_M": int(sum(pr.M for pr in runs)), "sum_MP": evals,
                   "K_range": [int(min(pr.K for pr in runs)), int(max(pr.K for pr in runs))],
                   "step": "one generation of all runs: one CUDA graph replay",
                   "timing": "CUDA events on the batch's stream around each graph replay",
                   "l2": "flushed between steps (256 MB write)",
                   "tiles": {str(t): int((tiles == t).sum()) for t in (32, 64, 128, 256)},
                   "create_s": create_s},
        "generations_per_s": 1.0 / t_step,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{peak_src} bf16_tflops (burst)",
                     "kernel": "fitness_batch_kernel", "kernel_ms": fit_ms,
                     "flops_per_launch": flops},
        "roofline_hbm": {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_gbs / hbm_peak, "algorithmic_bytes": nbytes,
                         "note": "the same launch against the HBM roof (partials counted at "
                                 "128-pattern tiles)"},
        "gpu_launches": 5 * steps,
        "clocks": clk,
    }
    b.close()
    return line


def spearman(a, b):
    ra = np.argsort(np.argsort(a, kind="stable"), kind="stable")
    rb = np.argsort(np.argsort(b, kind="stable"), kind="stable")
    return float(np.corrcoef(ra, rb)[0, 1])


def oracle_ga_best(pr, G):
    """Best fitness after G generations of the FP64 oracle GA on problem pr
    (Gram-form fitness, no surrogate, seed 4), and its host time."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    _, _, best = oracle.train(pr.X, pr.y, pr.degree, pr.basis, pr.P, G, 4, use_gram=True)
    return {"generations": G, "best": float(best[-1]), "seconds": time.perf_counter() - t0,
            "cores": oracle.set_threads(0)}


def surrogate_leg(torch, game, dev, pr, Xd, yd, oversample, steps_per_gen, timed_gens,
                  warmup, oracle_final=None, precision_gens=0, fp32_gens=3, clocks_enabled=True,
                  cpu_reports=True):
    """The surrogate-screened form (BF16 contraction, elite re-scoring,
    oversampled offspring screened by the MLP) against the plain FP32 form
    on the surrogate workload: generations per second of each and their
    ratio, the surrogate's rank correlation with the exact fitness of the
    children it kept and its trust verdicts, per-generation accuracy of the
    contraction forms against the FP64 oracle on 10,000 patterns, and, given
    oracle_final, the best fitness after its G generations of the screened
    GA against the FP64 oracle GA's (oracle_final, from oracle_ga_best)."""
    M, P = pr.M, pr.P
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(h, steps, warm):
        for _ in range(warm):
            game.game_generation(h.h, 4)
        torch.cuda.synchronize(dev)
        h.set_timing(True)
        ev = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            game.game_generation(h.h, 4)
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize(dev)
        tm = h.timing()
        h.set_timing(False)
        return sum(x.elapsed_time(y) for x, y in ev) / len(ev), tm

    kw = dict(stream=stream, P=P, seed=4, precision=game.GAME_PREC_BF16, surrogate=1,
              oversample=oversample, surrogate_steps=steps_per_gen)
    gs = game.Game(Xd, yd, pr.degree, pr.basis, **kw)
    fit_kernel = gs.plan()["kernel"]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")), enabled=clocks_enabled)
    t_sur, tm = timed(gs, timed_gens, warmup)
    clk = clocks.stop()
    g32 = game.Game(Xd, yd, pr.degree, pr.basis, stream=stream, P=P, seed=4,
                    precision=game.GAME_PREC_FP32)
    t_32, _ = timed(g32, fp32_gens, 1)
    g32.close()
    # surrogate rank agreement on the next generations (untimed)
    rho, trust = [], []
    E = 2
    for _ in range(3):
        game.game_generation(gs.h, 4)
        pred, keep, trusted, r = gs.surrogate_last()
        _, fit, _ = gs.population()
        rho.append(spearman(pred[keep.astype(bool)], np.log(fit[E:])))
        trust.append({"trusted": trusted, "pearson_kept": r})
    acc = precision_report(game, gs, pr, precision_gens) if cpu_reports and precision_gens else None
    gs.close()
    final = None
    if oracle_final is not None:
        G = oracle_final["generations"]
        gg = game.Game(Xd, yd, pr.degree, pr.basis, **kw)
        t0 = time.perf_counter()
        gg.train(G)
        t_g = time.perf_counter() - t0
        _, fit_g, _ = gg.population()
        gg.close()
        best_g, best_o = float(fit_g.min()), oracle_final["best"]
        final = {"generations": G, "oracle_best": best_o, "screened_bf16_best": best_g,
                 "rel_diff": (best_g - best_o) / best_o,
                 "oracle": "FP64 GA, Gram-form fitness, no surrogate, same seed",
                 "oracle_s": oracle_final["seconds"], "gpu_s": t_g}
    gen_s, gen32_s = 1e3 / t_sur, 1e3 / t_32
    return {
        "workload": pr.name, "M": M, "N": pr.N, "degree": pr.degree, "K": pr.K, "P": P,
        "form": f"BF16 contraction + elite re-score + surrogate screening, "
                f"{oversample}x oversampled offspring, {steps_per_gen} Adam round(s) "
                f"per generation",
        "oversample": oversample, "surrogate_steps": steps_per_gen,
        "ms_per_generation": t_sur, "generations_per_s": gen_s, "evals_per_s": M * P / (t_sur * 1e-3),
        "fitness_kernel": fit_kernel,
        "fp32_form": {"ms_per_generation": t_32, "generations_per_s": gen32_s},
        "gens_ratio_vs_fp32": gen_s / gen32_s,
        "stage_ms_per_generation": {k.replace("_ms", ""): tm[k] / max(timed_gens, 1)
                                    for k in ("fitness_ms", "pack_ms", "reduce_ms",
                                              "operators_ms", "rescore_ms", "surrogate_ms")},
        "surrogate_rank_spearman_kept": rho, "surrogate_trust": trust,
        "accuracy": acc, "final_best": final, "clocks": clk,
        "timing": "CUDA events around each generation, L2 flushed between generations",
    }


def run_surrogate(args, torch, game, dev, world, rank):
    """The surrogate workload (4M patterns, N = 48, Chebyshev degree 6,
    K = 289, P = 2048) as its own JSON line: value = evaluations per second
    of the screened generation."""
    from paper_1211_5481_gb300 import datagen as dg
    pr = dg.surrogate_regression()
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    cpu = rank == 0 and not args.no_cpu_baseline
    ofinal = oracle_ga_best(pr, args.oracle_run) if cpu and args.oracle_run > 0 else None
    leg = surrogate_leg(torch, game, dev, pr, Xd, yd, args.oversample, args.surrogate_steps,
                        args.steps, max(args.warmup, 3), oracle_final=ofinal,
                        precision_gens=2, fp32_gens=max(3, args.steps // 10),
                        clocks_enabled=not args.no_clocks, cpu_reports=cpu)
    t_sur = leg["ms_per_generation"]
    line = {
        "metric": METRIC, "value": pr.M * pr.P * world / (t_sur * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": t_sur, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": pr.name, "M": pr.M, "N": pr.N, "degree": pr.degree, "K": pr.K,
                   "P": pr.P, "form": leg["form"], "oversample": args.oversample,
                   "surrogate_steps": args.surrogate_steps,
                   "step": "one screened generation: offspring, MLP screening, exact "
                           "fitness of the kept population, MLP training",
                   "l2": "flushed between steps (256 MB write)"},
        "generations_per_s": leg["generations_per_s"],
        "fp32_form": leg["fp32_form"], "gens_ratio_vs_fp32": leg["gens_ratio_vs_fp32"],
        "stage_ms_per_step": leg["stage_ms_per_generation"],
        "surrogate_rank_spearman_kept": leg["surrogate_rank_spearman_kept"],
        "surrogate_trust": leg["surrogate_trust"],
        "accuracy": leg["accuracy"], "final_best": leg["final_best"], "clocks": leg["clocks"],
    }
    if rank == 0:
        print(json.dumps(line))


PAPER_DEGREES = (1, 2, 4, 8)
PAPER_ITERATIONS = (1000, 2000, 4000, 10000, 20000, 40000)


def run_paper(args, torch, game, dev, world, rank):
    """Section 5's grid, degree {1, 2, 4, 8} x iterations {1000 .. 40000},
    with the paper's settings: trigonometric basis, shared genes (Eq. 5),
    P = B N + 1 (Eq. 4), crossover 0.9, mutation 0.2, 2 elites, ranking or
    roulette selection, MSE stop threshold 0.001; on a synthetic set of the
    experiment's shape (2100 patterns, 9 features, +-1 classes). Fitness in
    the Gram form (FP64; K = 2 d + 1). Each cell is one game_train call from
    a fresh handle, timed on the host around the synchronous call; the FP64
    oracle runs a bounded number of generations of the same GA per degree
    on the host cores."""
    from paper_1211_5481_gb300 import datagen as dg
    pr = dg.small_classification()
    sel = {"ranking": game.GAME_SEL_RANKING, "roulette": game.GAME_SEL_ROULETTE}[args.selection]
    prm = dict(P=0, tied=1, elitism=2, pc=0.9, pm=0.2, selection=sel,
               precision=game.GAME_PREC_GRAM, mse_threshold=0.001, check_every=100, seed=11)
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    for d in PAPER_DEGREES:   # warm-up: module load, first launches
        with game.Game(Xd, yd, d, game.GAME_BASIS_TRIG, **prm) as g:
            g.train(max(args.warmup, 3) * 10)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")), enabled=not args.no_clocks)
    grid = []
    total_gen, total_s = 0, 0.0
    for d in PAPER_DEGREES:
        for it in PAPER_ITERATIONS:
            with game.Game(Xd, yd, d, game.GAME_BASIS_TRIG, **prm) as g:
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                ran = g.train(it)
                t = time.perf_counter() - t0
                pop, fit, gen = g.population()
                best = int(np.argmin(fit))
                cls = g.classify(pop[best])
            grid.append({"degree": d, "iterations": it, "generations_run": int(ran),
                         "seconds": t, "best_mse": float(fit[best]),
                         "accuracy": cls["accuracy"], "completeness": cls["completeness"],
                         "contamination": cls["contamination"]})
            total_gen += int(ran)
            total_s += t
    clk = clocks.stop()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = oracle.set_threads(0)
        G_s = 400
        per_degree = []
        t_all = 0.0
        for d in PAPER_DEGREES:
            t0 = time.perf_counter()
            oracle.train_tied(pr.X, pr.y, d, game.GAME_BASIS_TRIG, 2 * pr.N + 1, G_s, 11,
                              oracle.ga_params(elitism=2, pc=0.9, pm=0.2, selection=sel))
            t = time.perf_counter() - t0
            t_all += t
            gpu = [c for c in grid if c["degree"] == d]
            gpu_rate = sum(c["generations_run"] for c in gpu) / sum(c["seconds"] for c in gpu)
            per_degree.append({"degree": d, "oracle_generations_per_s": G_s / t,
                               "gpu_generations_per_s": gpu_rate,
                               "speedup": gpu_rate * t / G_s})
        cpu = {"value": len(PAPER_DEGREES) * G_s / t_all, "unit": "generations/s",
               "cores": cores, "kind": "oracle",
               "sample": f"{G_s} generations per degree of the same GA (FP64, direct "
                         f"shared-gene fitness)", "per_degree": per_degree}
    line = {
        "metric": "GAME generations/s, Section 5 degree x iterations grid (paper-literal mode)",
        "value": total_gen * world / total_s, "unit": "generations/s", "n_gpus": world,
        "steps": len(grid), "warmup": max(args.warmup, 3),
        "ms_per_step": total_s / total_gen * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": pr.name, "M": pr.M, "N": pr.N, "basis": "trigonometric",
                   "genes": "shared (Eq. 5), K = 2 d + 1", "P": 2 * pr.N + 1,
                   "selection": args.selection, "pc": 0.9, "pm": 0.2, "elitism": 2,
                   "stop": "MSE < 0.001, checked every 100 generations",
                   "fitness": "Gram form, FP64",
                   "step": "one generation (ms_per_step is the grid's mean)",
                   "timing": "host clock around each synchronous game_train call",
                   "l2": "inputs of 76 KB stay L2-resident (a latency-bound workload)"},
        "grid": grid,
        "roofline": None,
        "roofline_note": "launch-latency bound: 19 chromosomes x 2100 patterns per generation",
        "cpu_baseline": cpu,
        "gpu_launches": 4 * total_gen,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_1211_5481_gb300 import game

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.workload in ("batched", "surrogate", "paper"):
        game.load()
        {"batched": run_batched, "surrogate": run_surrogate,
         "paper": run_paper}[args.workload](args, torch, game, dev, world, rank)
        if world > 1:
            dist.destroy_process_group()
        return

    pr = workload(args.M)
    M, K, P = pr.M, pr.K, pr.P
    Xd = torch.from_numpy(pr.X).to(dev)
    yd = torch.from_numpy(pr.y).to(dev)
    game.load()
    prec = {"fp32": game.GAME_PREC_FP32, "bf16": game.GAME_PREC_BF16,
            "bf16x3": game.GAME_PREC_BF16X3, "fp8": game.GAME_PREC_FP8,
            "gram": game.GAME_PREC_GRAM}[args.form]
    tensor = prec not in (game.GAME_PREC_FP32, game.GAME_PREC_GRAM)
    errk = {"mse": game.GAME_ERR_MSE, "rmse": game.GAME_ERR_RMSE, "mae": game.GAME_ERR_MAE}[args.error]
    ekw = dict(error=errk, rescore_top=0 if args.error == "mae" else 16)
    t_create = time.perf_counter()
    g = game.Game(Xd, yd, pr.degree, pr.basis, stream=stream, P=P, precision=prec, seed=2, **ekw)
    t_create = time.perf_counter() - t_create
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_steps(handle, steps, warmup):
        for _ in range(warmup):
            game.game_generation(handle.h, 2)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        handle.set_timing(True)
        ms = []
        for _ in range(steps):
            flush.zero_()   # L2 flush between steps, outside the timed events
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            game.game_generation(handle.h, 2)
            b.record(stream)
            ms.append((a, b))
        torch.cuda.synchronize(dev)
        tm = handle.timing()
        handle.set_timing(False)
        step_ms = [x.elapsed_time(y) for x, y in ms]
        if world > 1:
            dist.barrier()
        return step_ms, tm

    # main leg
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    step_ms, tm = timed_steps(g, args.steps, max(args.warmup, 3))
    clk = clocks.stop()
    t_step = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    value = whole_job_rate(M * P, t_step * 1e-3, world)

    peaks, peak_src = load_peaks()
    flops_launch = 2.0 * M * P * (K - 1) + 3.0 * M * P
    fit_ms = tm["fitness_ms"] / max(tm["fitness_launches"], 1)
    achieved_tflops = flops_launch / (fit_ms * 1e-3) / 1e12
    if tensor:
        # FP8 runs at twice the BF16 rate (nominal 4.5 vs 2.25 PFLOP/s dense);
        # bf16x3 issues three BF16 MMAs per useful product
        ratio = 2.0 if prec == game.GAME_PREC_FP8 else 1.0
        mma_per_product = 3.0 if prec == game.GAME_PREC_BF16X3 else 1.0
        peak = float(peaks["bf16_tflops"]) * ratio
        roof = {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak, "traffic": ncu_traffic(pr.name, args.form),
                "kernel_digest": kernel_digest(),
                "algorithmic_bytes": 4.0 * M * pr.N + 4.0 * M + 2.0 * P * (K - 1),
                "peak_source": (f"{peak_src} bf16_tflops (burst)"
                                + (" x 2 (FP8 / BF16 nominal ratio)" if ratio != 1.0 else "")),
                "frac_of_sustained": achieved_tflops / (float(peaks.get(
                    "bf16_tflops_sustained", peaks["bf16_tflops"])) * ratio),
                "mma_tflops": achieved_tflops * mma_per_product,
                "kernel": g.plan()["kernel"], "kernel_ms": fit_ms}
    elif prec == game.GAME_PREC_GRAM:
        # FP64 quadratic forms: 2 P K^2 + 2 P K flop per generation
        gflops = (2.0 * P * K * K + 2.0 * P * K) / (fit_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": gflops, "peak": 1.25, "unit": "TFLOP/s",
                "frac": gflops / 1.25, "traffic": None,
                "peak_source": "nominal GB300 FP64 rate (not in the measured peaks)",
                "kernel": "quad_kernel", "kernel_ms": fit_ms,
                "gram_build_s": t_create,
                "note": "evaluations implicit: fit = (y.y - 2 a.b + a^T G a) / M"}
    else:
        props = torch.cuda.get_device_properties(dev)
        peak = props.multi_processor_count * 128 * 2 * float(peaks["sm_max_mhz"]) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak, "traffic": None,
                "peak_source": "FP32 FFMA: SMs x 128 lanes x 2 flop x max SM clock",
                "kernel": "fitness_fp32_kernel", "kernel_ms": fit_ms}

    # plain FP32 GPU form of the same step, for the "vs plain FP32" ratio
    fp32_leg = None
    if tensor and not args.no_fp32_leg:
        g32 = game.Game(Xd, yd, pr.degree, pr.basis, stream=stream, P=P,
                        precision=game.GAME_PREC_FP32, seed=2, **ekw)
        ms32, tm32 = timed_steps(g32, max(3, args.steps // 4), 3)
        t32 = sum(ms32) / len(ms32)
        k32 = tm32["fitness_ms"] / max(tm32["fitness_launches"], 1)
        # CUDA-core FP32 peak: SMs x 128 FP32 lanes x 2 flop (FFMA) x max SM clock
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = float(clk.get("sm_max_mhz") or 2070.0)
        ffma_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        a32 = (2.0 * M * P * (K - 1) + 3.0 * M * P) / (k32 * 1e-3) / 1e12
        fp32_leg = {"value": whole_job_rate(M * P, t32 * 1e-3, world), "ms_per_step": t32,
                    "fitness_kernel_ms": k32,
                    "roofline": {"bound": "alu", "achieved": a32, "peak": ffma_peak,
                                 "unit": "TFLOP/s", "frac": a32 / ffma_peak,
                                 "peak_source": f"{sms} SMs x 128 FFMA lanes x 2 x {mhz:.0f} MHz"}}
        g32.close()

    # end to end through the public API: a host population (pinned) in, its
    # fitness out, one synchronous call per step
    pin_pop = torch.empty((P, K), dtype=torch.float32).pin_memory()
    pop_np, _, _ = g.population()
    pin_pop.copy_(torch.from_numpy(pop_np))
    pin_fit = torch.empty(P, dtype=torch.float64).pin_memory()
    popv, fitv = pin_pop.numpy(), pin_fit.numpy()
    for _ in range(2):
        g.eval_fitness(popv)
        game.game_eval_fitness(g.h, popv, fitv)
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        game.game_eval_fitness(g.h, popv, fitv)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_t) / len(e2e_t)
    e2e = {"value": M * P * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": P * K * 4,
           "d2h_bytes_per_step": P * 8,
           "call": "game_eval_fitness(host pinned pop[P][K]) -> host fit[P]"}

    # accuracy of the timed forms on a sample of the current population
    acc = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pop_np, fit_np, gen = g.population()
        sample = np.linspace(0, P - 1, 8).astype(int)
        ref = oracle.fitness(pr.X, pr.y, pop_np[sample], pr.degree, pr.basis,
                             err={"mse": oracle.ERR_MSE, "rmse": oracle.ERR_RMSE,
                                  "mae": oracle.ERR_MAE}[args.error])
        f_bf = g.eval_fitness(pop_np, precision=prec)
        f_32 = g.eval_fitness(pop_np, precision=game.GAME_PREC_FP32)
        acc = {"sample_chromosomes": len(sample), "generation": gen,
               "form_max_rel_err": float(np.max(np.abs(f_bf[sample] - ref) / ref)),
               "fp32_max_rel_err": float(np.max(np.abs(f_32[sample] - ref) / ref)),
               "top10_agreement_form_vs_fp32": len(set(np.argsort(f_bf)[:10]) &
                                                    set(np.argsort(f_32)[:10])) / 10}
        cpu, M_s = oracle_sample_rate(pr, 16)
        cpu.update(oracle_extra(pr, M_s, cpu))
        if args.precision_report > 0 and args.error == "mse":
            acc["precision_forms"] = precision_report(game, g, pr, args.precision_report)

    n_launch = tm["fitness_launches"] + tm["pack_launches"] + tm["reduce_launches"] + \
        (1 if P <= 1024 and P * K <= 65536 else 2) * tm["operators_launches"] + \
        3 * tm["rescore_launches"]
    cls = None
    if rank == 0 and args.classify_run > 0:
        # trained model quality (outside the timed region): the best
        # chromosome after G more generations, classified by Out > 0 (labels
        # are +-1), beside the generating polynomial's own score (the 5%
        # flipped labels bound every model)
        g.train(args.classify_run)
        pop_np, fit_np, gen = g.population()
        best = int(np.argmin(fit_np))
        res = g.classify(pop_np[best])
        gen_res = g.classify(pr.coef)
        cls = {"generations": int(gen), "best_fitness": float(fit_np[best]),
               "accuracy": res["accuracy"], "completeness": res["completeness"],
               "contamination": res["contamination"],
               "generating_polynomial": {k: gen_res[k] for k in
                                         ("accuracy", "completeness", "contamination")},
               "definition": "positive: label > 0, predicted positive: Out > 0 (FP64)"}
    sur = None
    if world == 1 and not args.no_surrogate_leg:
        # the surrogate workload (4M patterns, N = 48, degree 6, P = 2048)
        # beside the headline: the screened BF16 form at the workload's
        # literal 8x oversampling and at 2x (milder screening), both with
        # eight Adam rounds per generation, each against the plain FP32
        # form; the FP64 oracle GA's best after G generations is shared by
        # both comparisons
        from paper_1211_5481_gb300 import datagen as dg
        pr4 = dg.surrogate_regression()
        X4 = torch.from_numpy(pr4.X).to(dev)
        y4 = torch.from_numpy(pr4.y).to(dev)
        cpu4 = rank == 0 and not args.no_cpu_baseline
        of = (oracle_ga_best(pr4, args.surrogate_oracle_run)
              if cpu4 and args.surrogate_oracle_run > 0 else None)
        sur = {}
        for o, st in ((8, 8), (2, 8)):
            sur[f"oversample_{o}x_steps_{st}"] = surrogate_leg(
                torch, game, dev, pr4, X4, y4, o, st, 10, 3, oracle_final=of,
                precision_gens=3, fp32_gens=3, clocks_enabled=not args.no_clocks,
                cpu_reports=cpu4)
        if of is not None:
            # the BF16 form without screening, same seed and generations: the
            # precision form alone against the FP64 oracle GA
            with game.Game(X4, y4, pr4.degree, pr4.basis, stream=stream, P=pr4.P, seed=4,
                           precision=game.GAME_PREC_BF16) as gb:
                gb.train(of["generations"])
                best_b = float(gb.population()[1].min())
            sur["unscreened_bf16_final_best"] = {
                "generations": of["generations"], "bf16_best": best_b,
                "oracle_best": of["best"], "rel_diff": (best_b - of["best"]) / of["best"]}
        del X4, y4
    bat = None
    if world == 1 and not args.no_batched_leg:
        # the batched workload (256 independent runs of uneven shape, one
        # CUDA-graph replay per generation of all runs) beside the headline
        bl = batched_line(10, 3, args.no_clocks, torch, game, dev, world)
        bat = {"workload": bl["config"]["workload"], "runs": bl["config"]["runs"],
               "sum_MP": bl["config"]["sum_MP"], "steps": bl["steps"],
               "ms_per_generation": bl["ms_per_step"], "evals_per_s": bl["value"],
               "generations_per_s": bl["generations_per_s"],
               "fitness_kernel": bl["roofline"]["kernel"],
               "fitness_kernel_ms": bl["roofline"]["kernel_ms"],
               "roofline_frac": bl["roofline"]["frac"],
               "roofline_peak": bl["roofline"]["peak"],
               "tiles": bl["config"]["tiles"], "timing": bl["config"]["timing"],
               "l2": bl["config"]["l2"], "clocks": bl["clocks"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3",
                                               "fp8": "e4m3", "gram": "f64"}[args.form],
        "data": "synthetic",
        "config": {"workload": pr.name, "M": M, "N": pr.N, "degree": pr.degree, "K": K, "P": P,
                   "basis": "chebyshev", "contraction": args.form, "error": args.error,
                   "step": ("one generation: operators + pack + fused fitness + FP64 reduce"
                            + (" + elite re-score (16 best: FP64 Gram form)"
                               if tensor else "")),
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"{world} independent replica(s)"},
        "generations_per_s": 1e3 / t_step,
        "vs_fp32": (value / fp32_leg["value"]) if fp32_leg else None,
        "fp32_form": fp32_leg,
        "stage_ms_per_step": {k.replace("_ms", ""): tm[k] / max(args.steps, 1)
                              for k in ("fitness_ms", "pack_ms", "reduce_ms", "operators_ms",
                                        "rescore_ms")},
        "accuracy": acc,
        "classification": cls,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "surrogate_workload": sur,
        "batched_workload": bat,
        "gpu_launches": int(n_launch),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
