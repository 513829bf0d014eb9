"""Benchmark of the APO population update on GB300.

Default workload ("scale"): plain APO at population 4096, D = 100, 2000
iterations, on the four seeded shifted-rotated forms (ill-conditioned
elliptic, chained Rosenbrock, Rastrigin cosine sum, 30/30/40 hybrid).  One
step = one complete run of each of the four forms (4 x 4096 x 2000 candidate
updates, each evaluated exactly once, plus 4 x 4096 initial evaluations),
issued as one apo_run_batch call.  Metric: candidate updates/s (whole job,
all GPUs); true evaluations/s is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--iters T] [--workload scale|single]

Multi-GPU: the runs are independent, so N ranks run N replicas (weak
scaling); torch.distributed only carries the timing barrier and the max over
ranks.  --impl reference times the FP64 CPU oracle (the only reference the
paper's method has here) on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2510_14982_gb300 import inputs  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SMS = 152                 # GB300 streaming multiprocessors
FP32_LANES = 128          # FP32 FMA lanes per SM
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        p["source"] = "measured"
        return p
    except OSError:
        p = dict(FALLBACK)
        p["source"] = "fallback"
        return p


def workload(name, iters):
    """(specs, ps, T, label) of a named workload."""
    if name == "scale":
        return inputs.scale_forms(seed=0, D=100), 4096, iters or 2000, "plain APO ps=4096 D=100 x4 forms"
    if name == "single":
        return [inputs.single_rastrigin(0)], 20, iters or 1000, "plain APO ps=20 D=10 Rastrigin"
    raise SystemExit("unknown workload " + name)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(n_gpus=None):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_setup(backend="nccl"):
    """(world, rank, local rank) from the torchrun environment; with more than
    one rank, joins the process group.  Every rank runs its own replica of the
    workload (the runs share nothing), so the group carries only the timing
    barriers and the max over ranks."""
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def sync_ranks(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cpu"):
    """The maximum of x over all ranks (the slowest replica sets the time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _ctx():
    """(world, rank, local rank, torch, apo) with the process group joined and
    the device selected (idempotent)."""
    import torch
    world, rank, local = replica_setup()
    torch.cuda.set_device(local)
    from paper_2510_14982_gb300 import apo
    return world, rank, local, torch, apo


def replica_seed(step, rank):
    """Seed of a replica's runs in a step: distinct for every (step, rank) below 100 ranks."""
    return 100 * step + rank


def aggregate_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, as it stands, on every host core:
    each step is a bounded sample of the scale workload (31 seeds x the four
    forms at ps 4096, --ref-iters iterations each, one run per task)."""
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    import oracle
    oracle.build()
    specs, ps, T, label = workload(args.workload, args.iters)
    cores = os.cpu_count() or 1
    probs = [oracle.OracleProblem.from_spec(s) for s in specs]

    def sample(iters, step):
        allp = [p for p in probs for _ in range(31)]
        prm = [oracle.params(ps, 1, 0.1, iters, 31 * step + sd, k) for k in range(len(probs)) for sd in range(31)]
        t0 = time.perf_counter()
        oracle.apo_run_many(allp, prm, cores)
        return time.perf_counter() - t0, len(allp)

    for w in range(max(1, min(args.warmup, 1))):
        sample(1, 1000 + w)
    times = []
    n_runs = 0
    for k in range(args.steps):
        dt, n_runs = sample(args.ref_iters, k)
        times.append(dt)
    per_step = statistics.mean(times)
    value = n_runs * ps * args.ref_iters / per_step
    smp = "%d runs (31 seeds x %d forms) x ps %d x %d iterations per step (full run: %d iterations), %d cores" % (
        n_runs, len(specs), ps, args.ref_iters, T, cores)
    line = {"impl": "reference", "metric": "APO candidate updates/s", "value": value, "unit": "updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": label, "sample": smp},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle", "sample": smp},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batched(args):
    """Batched workload: n independent runs (ps ~ U{20..512}, D in {10, 20, 50},
    form ~ U{4 forms}, own o and M, 1000 iterations) as one autotuned persistent
    work-queue launch replayed from a CUDA graph; beside it the same kind of
    runs launched one at a time (a bounded sample, scaled)."""
    world, rank, local, torch, apo = _ctx()
    T = args.iters or 1000
    runs = inputs.batched_runs(args.runs, seed=rank)
    n = len(runs)
    probs = [apo.problem_from_spec(s) for s, _ in runs]
    prms = [apo.apo_params_make(ps, 1, 0.1, T, 17, k) for k, (_, ps) in enumerate(runs)]
    updates = sum(ps for _, ps in runs) * T
    flops = sum(2.0 * s.D * s.D * ps * (T + 1) for s, ps in runs)
    dev = torch.device("cuda", local)
    bx = torch.zeros((n, 50), device=dev)
    bf = torch.zeros(n, dtype=torch.float64, device=dev)
    if args.batch_config:
        # a fixed mapping instead of the autotuner's choice (reproducible
        # profiling: under a profiler the autotuner's timings are distorted)
        smem, cps_sm, cl_ps, cl_sz = (int(v) for v in args.batch_config.split(","))
        b = apo.apo_batch_create(probs, prms, bx, 50, bf, smem_budget=smem, ctas_per_sm=cps_sm, cluster_ps=cl_ps,
                                 cluster_size=cl_sz)
        chosen = {"smem_budget": smem, "ctas_per_sm": cps_sm, "cluster_ps": cl_ps, "cluster_size": cl_sz,
                  "fixed": True}
    else:
        b = apo.apo_batch_create(probs, prms, bx, 50, bf)
        chosen = b.autotune(probe_iters=40)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.launch(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.launch(stream)
    flush = torch.zeros(64 << 20, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    sync_ranks(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms = []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    total_ms = max_over_ranks(sum(ms), world, dev)
    sync_ranks(world)
    value = aggregate_rate(world, args.steps * updates, total_ms * 1e-3)
    # the same kind of runs launched one at a time (one apo_run_device call each)
    k_s = min(args.per_run_sample, n)
    sx = torch.zeros(50, device=dev)
    sf = torch.zeros(1, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    e0.record()
    for k in range(k_s):
        apo.apo_run_device(probs[k], prms[k], sx, sf)
    e1.record()
    torch.cuda.synchronize()
    per_run_rate = sum(runs[k][1] for k in range(k_s)) * T / (e0.elapsed_time(e1) * 1e-3)
    # end to end: problems uploaded from host memory, one apo_run_batch, results read back
    host_bf = torch.empty(n, dtype=torch.float64, pin_memory=True)
    host_bx = torch.empty((n, 50), pin_memory=True)
    h2d = sum(4 * (s.D * s.D + s.D) + 16 * s.D + (0 if s.perm is None else 4 * s.D) for s, _ in runs)
    t0 = time.perf_counter()
    probs2 = [apo.problem_from_spec(s) for s, _ in runs]
    apo.apo_run_batch(probs2, prms, bx, 50, bf)
    host_bx.copy_(bx, non_blocking=True)
    host_bf.copy_(bf, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    del probs2
    pk = peaks()
    fp32_peak = SMS * FP32_LANES * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved = flops / (total_ms / args.steps * 1e-3) / 1e12
    line = {
        "metric": "APO candidate updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched APO: %d runs, ps U{20..512}, D in {10,20,50}, 4 forms, %d iterations, "
                               "one persistent launch replayed from a CUDA graph" % (n, T),
                   "l2": "flushed between steps (256 MiB write)", "autotune": chosen},
        "true_evals_per_s": world * args.steps * sum(ps for _, ps in runs) * (T + 1) / (total_ms * 1e-3),
        "per_run_launch": {"value": per_run_rate, "unit": "updates/s", "sample_runs": k_s,
                           "ratio_batched_over_per_run": value / world / per_run_rate},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None,
                     "kernel": "run_kernel (work queue), 2 D^2 flop per evaluation",
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x max clock (%s)" % pk["source"]},
        "clocks": clk.summary(), "gpu_launches": 2 * args.steps,
        "e2e": {"value": updates / e2e_s, "unit": "updates/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(n * 8 + n * 50 * 4)},
    }
    return line


def run_thresholding(args):
    """Multilevel thresholding: 256 synthetic 4096 x 4096 8-bit images (4 GiB,
    drawn on the device, untimed) -> bit-exact 256-bin histograms -> APO over
    T in {2, 4, 8, 16} Otsu thresholds (ps 100, 500 iterations) for every
    image, 1024 runs in one autotuned persistent launch.  One step = the
    histograms of all images and the 1024 runs."""
    world, rank, local, torch, apo = _ctx()
    dev = torch.device("cuda", local)
    n_img, side = args.images, args.side
    npx = side * side
    T = args.iters or 500
    imgs = inputs.gmm_images_torch(n_img, side, seed=rank, device=dev)
    hist = torch.zeros((n_img, 256), dtype=torch.int32, device=dev)
    apo.apo_histogram_u8(imgs, npx, n_img, hist)
    torch.cuda.synchronize()
    Ts = (2, 4, 8, 16)
    probs = [apo.apo_problem_create(Tk, np.zeros(Tk), np.full(Tk, 255.0), apo.APO_OBJ_OTSU, hist_device=hist[i])
             for i in range(n_img) for Tk in Ts]
    prms = [apo.apo_params_make(100, 1, 0.1, T, 5, k) for k in range(len(probs))]
    n = len(probs)
    bx = torch.zeros((n, 16), device=dev)
    bf = torch.zeros(n, dtype=torch.float64, device=dev)
    b = apo.apo_batch_create(probs, prms, bx, 16, bf)
    chosen = b.autotune(probe_iters=40)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        apo.apo_histogram_u8(imgs, npx, n_img, hist, stream=stream)
        b.launch(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.launch(stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(args.warmup):
        apo.apo_histogram_u8(imgs, npx, n_img, hist)
        graph.replay()
    torch.cuda.synchronize()
    sync_ranks(world)
    hist_ms, apo_ms = [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            ev[0].record()
            apo.apo_histogram_u8(imgs, npx, n_img, hist)
            ev[1].record()
            graph.replay()
            ev[2].record()
            torch.cuda.synchronize()
            hist_ms.append(ev[0].elapsed_time(ev[1]))
            apo_ms.append(ev[1].elapsed_time(ev[2]))
    total_ms = max_over_ranks(sum(hist_ms) + sum(apo_ms), world, dev)
    sync_ranks(world)
    updates = n * 100 * T
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    h_gbs = n_img * npx / (statistics.mean(hist_ms) * 1e-3) / 1e9
    # exactness on the device against bincount of one image (cheap spot check)
    ref = torch.bincount(imgs[0].long(), minlength=256).to(torch.int32)
    exact = bool(torch.equal(ref, hist[0]))
    line = {
        "metric": "APO candidate updates/s", "value": aggregate_rate(world, args.steps * updates, total_ms * 1e-3),
        "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8 histogram, f64 Otsu fitness, f32 positions", "data": "synthetic",
        "config": {"workload": "thresholding: %d images %dx%d (GMM), T in {2,4,8,16}, ps 100, %d iterations, %d runs"
                               % (n_img, side, side, T, n),
                   "l2": "inputs (4 GiB) larger than L2", "autotune": chosen},
        "histogram_ms": statistics.mean(hist_ms), "apo_ms": statistics.mean(apo_ms),
        "histogram_bit_exact_spot_check": exact,
        "roofline": {"bound": "hbm", "achieved": h_gbs, "peak": hbm, "unit": "GB/s", "frac": h_gbs / hbm,
                     "traffic": None, "kernel": "histogram_u8_kernel (1 byte read per pixel)",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % pk["source"]},
        "clocks": clk.summary(), "gpu_launches": 3 * args.steps, "e2e": None,
    }
    return line


def run_surrogate(args):
    """Surrogate-assisted APO on the 10-component composition (D 200, ps 256,
    300 iterations, k 8 candidates screened by the online-trained BF16 MLP).
    One step = one surrogate run.  Beside the throughput: time to the plain
    method's median best (over --seeds seeds), in iterations, true evaluations
    and wall time."""
    world, rank, local, torch, apo = _ctx()
    T = args.iters or 300
    spec = inputs.composition(D=200, seed=0)
    prob = apo.problem_from_spec(spec)
    sp = apo.surrogate_params(k=8, retrain_every=10, archive_cap=50000, train_steps=50, batch=512, lr=1e-3,
                              train_window=1280)

    def plain(seed):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, f, c = apo.apo_run(prob, apo.apo_params_make(256, 1, 0.1, T, seed))
        return f, c, time.perf_counter() - t0

    def surr(seed):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, f, c, st = apo.apo_run_surrogate(prob, apo.apo_params_make(256, 1, 0.1, T, seed), sp)
        return f, c, time.perf_counter() - t0, st

    for k in range(args.warmup):
        surr(1000 + k)
        plain(1000 + k)
    P = [plain(s) for s in range(args.seeds)]
    target = float(np.median([p[0] for p in P]))
    S = []
    torch.cuda.synchronize()
    sync_ranks(world)
    with Clocks(local) as clk:
        for s in range(max(args.steps, args.seeds)):
            S.append(surr(s))
    times = [x[2] for x in S[:args.steps]]
    t_max = max_over_ranks(sum(times), world, torch.device("cuda", local))
    sync_ranks(world)
    stt = S[0][3]

    def iters_to(curve):
        hit = np.nonzero(curve <= target)[0]
        return int(hit[0]) if hit.size else None

    def med_time_to(runs):
        tt = []
        for r in runs:
            it = iters_to(r[1])
            tt.append(r[2] * it / T if it is not None else float("inf"))
        return float(np.median(tt)), [iters_to(r[1]) for r in runs]

    p_t, p_it = med_time_to(P)
    s_t, s_it = med_time_to(S[:args.seeds])
    screened = stt["screened"]
    line = {
        "metric": "APO candidate updates/s", "value": aggregate_rate(world, screened * len(times), t_max), "unit": "updates/s",
        "n_gpus": world, "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 APO, bf16 MLP (fp32 accumulate)",
        "data": "synthetic",
        "config": {"workload": "surrogate-assisted APO: composition of 10 (D 200), ps 256, %d iterations, k 8, retrain "
                               "every 10 on the last 1280 evaluations (50 Adam steps of 512)" % T,
                   "l2": "working set resident (no flush)"},
        "true_evals_per_s": aggregate_rate(world, stt["true_evals"] * len(times), t_max),
        "time_to_target": {"target_best_f": target, "target": "median best of plain APO over %d seeds" % args.seeds,
                           "surrogate_s": s_t, "plain_s": p_t, "ratio": s_t / p_t if p_t > 0 else None,
                           "surrogate_iters": s_it, "plain_iters": p_it,
                           "surrogate_median_best": float(np.median([x[0] for x in S[:args.seeds]])),
                           "note": "wall time to target = run wall time x (first iteration at target / iterations)"},
        "surrogate_stats": stt,
        "roofline": None, "clocks": clk.summary(), "gpu_launches": None, "e2e": None,
    }
    return line


def flush_l2(buf):
    buf.add_(1)   # writes 256 MiB, larger than the 129 MB L2


# The paper's own numbers (Tesla T4 GPU and a sequential Xeon code): context
# for the large-dimension and thresholding workloads, not targets.
PAPER_TABLE2_T4_S = {  # GPU seconds, D 1000, 1000 iterations, by form and ps (1k, 2k, 5k, 10k)
    "bent_cigar": {1000: 35, 2000: 64, 5000: 158, 10000: 345},
    "elliptic": {1000: 67, 2000: 129, 5000: 322, 10000: 673},
    "hgbat": {1000: 34, 2000: 64, 5000: 160, 10000: 345},
    "rosenbrock": {1000: 96, 2000: 190, 5000: 471, 10000: 971},
    "griewank": {1000: 48, 2000: 93, 5000: 232, 10000: 492},
}
PAPER_TABLE3_T4_S = {512: 3, 1024: 13, 2048: 50, 4096: 199}   # ps 100, 1 threshold, 50 iterations


def run_table2(args, steps=None, warmup=None, pss=None):
    """The paper's Table-2 shapes on the large-dimension path: the five seeded
    forms (Bent Cigar, elliptic, HGBat, Rosenbrock, Griewank), D 1000, 1000
    iterations, at each population; one step = the five runs as one
    apo_run_batch call.  Per-stage device time from the library's stage
    timers (one extra, untimed step); the rotation GEMM's roofline counts the
    three fp16 tensor products of every candidate (3 x 2 ps D^2 flop per
    launch) against the measured bf16 tensor peak (fp16 has the same rate)."""
    world, rank, local, torch, apo = _ctx()
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    pss = pss or ((args.ps,) if args.ps else (1000, 10000))
    D, T = 1000, args.iters or 1000
    specs = inputs.table2_forms(seed=rank, D=D)
    probs = [apo.problem_from_spec(s) for s in specs]
    n = len(specs)
    dev = torch.device("cuda", local)
    pk = peaks()
    tensor_peak = float(pk.get("bf16_tflops", 1880.9))
    out = {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for ps in pss:
        bx = torch.zeros((n, D), device=dev)
        bf = torch.zeros(n, dtype=torch.float64, device=dev)
        cv = torch.zeros((n, T + 1), device=dev)

        def step(k):
            prms = [apo.apo_params_make(ps, 1, 0.1, T, replica_seed(k, rank), j) for j in range(n)]
            apo.apo_run_batch(probs, prms, bx, D, bf, cv, T + 1)

        for k in range(warmup):
            step(k)
        torch.cuda.synchronize()
        sync_ranks(world)
        ms = []
        with Clocks(local) as clk:
            for k in range(steps):
                torch.cuda.synchronize()
                e0.record()
                step(warmup + k)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        total_ms = max_over_ranks(sum(ms), world, dev)
        apo.apo_large_stage_timing(True)
        step(warmup + steps)
        torch.cuda.synchronize()
        stages = apo.apo_large_stage_timing(False)
        g = stages["gemm_eval"]
        gemm_flop = 3.0 * 2.0 * ps * D * D * n          # per launch (all five runs)
        gemm_avg_s = g["ms"] / max(g["launches"], 1) * 1e-3
        achieved = gemm_flop / gemm_avg_s / 1e12 if g["launches"] else None
        per_run_s = total_ms / steps * 1e-3
        out[str(ps)] = {
            "value": aggregate_rate(world, steps * n * ps * T, total_ms * 1e-3), "unit": "updates/s",
            "ms_per_step": total_ms / steps, "runs_per_step": n, "ps": ps, "D": D, "iterations": T,
            "stage_ms_per_iteration": {k: v["ms"] / max(v["launches"], 1) for k, v in stages.items()},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": tensor_peak, "unit": "TFLOP/s",
                         "frac": achieved / tensor_peak if achieved else None, "traffic": None,
                         "kernel": "big_gemm_kernel: TMA-staged 128-byte-swizzled fp16 tiles, three tcgen05.mma per "
                                   "K step, objective epilogue from TMEM; 3 x 2 ps D^2 flop per launch",
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (%s; fp16 has the bf16 rate)" % pk["source"]},
            "clocks": clk.summary(),
            "paper_t4_seconds_per_run": {f: PAPER_TABLE2_T4_S[f].get(ps) for f in PAPER_TABLE2_T4_S},
            "seconds_per_run_here": per_run_s / n,
        }
    return {"workload": "Table-2 shapes: 5 forms x D 1000 x %d iterations, one apo_run_batch per step" % T,
            "dtype": "f32 state, fp16 hi+lo tensor products with fp32 accumulation", "by_ps": out,
            "steps": steps, "warmup": warmup}


def run_table3(args):
    """The paper's Table-3 settings: one Otsu threshold, ps 100, 50 iterations,
    on a synthetic 8-bit image of side^2 pixels (the photograph is not
    available); one step = the device histogram and the APO run.  The best
    threshold is checked against the exhaustive optimum over all 256."""
    world, rank, local, torch, apo = _ctx()
    dev = torch.device("cuda", local)
    out = {}
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for side in (512, 1024, 2048, 4096):
        img = inputs.gmm_images_torch(1, side, seed=side + rank, device=dev)
        h = torch.zeros((1, 256), dtype=torch.int32, device=dev)
        bx = torch.zeros(1, device=dev)
        bf = torch.zeros(1, dtype=torch.float64, device=dev)
        hms, ams = [], []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e[0].record()
            apo.apo_histogram_u8(img, side * side, 1, h)
            e[1].record()
            prob = apo.apo_problem_create(1, np.zeros(1), np.full(1, 255.0), apo.APO_OBJ_OTSU, hist_device=h[0])
            apo.apo_run_device(prob, apo.apo_params_make(100, 1, 0.1, 50, k), bx, bf)
            e[2].record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                hms.append(e[0].elapsed_time(e[1]))
                ams.append(e[1].elapsed_time(e[2]))
        hist = h[0].cpu().numpy().astype(np.int64)
        p = hist / hist.sum()
        omega = np.cumsum(p)
        mu = np.cumsum(p * np.arange(256))
        with np.errstate(divide="ignore", invalid="ignore"):
            sb = np.where((omega > 0) & (omega < 1), (mu[-1] * omega - mu) ** 2 / (omega * (1 - omega)), 0.0)
        t_best = int(min(max(np.floor(bx.item()), 0), 255))
        # between-class variance of APO's threshold against the exhaustive
        # maximum (several thresholds tie where the histogram has empty bins)
        out[str(side)] = {"histogram_ms": statistics.mean(hms), "problem_and_apo_ms": statistics.mean(ams),
                          "total_ms": statistics.mean(hms) + statistics.mean(ams),
                          "best_threshold": t_best, "sigma_b2": float(-bf.item()),
                          "exhaustive_sigma_b2": float(sb.max()),
                          "optimal_thresholds": [int(v) for v in np.flatnonzero(sb >= sb.max() * (1 - 1e-12))][:8],
                          "reaches_exhaustive_optimum": bool(abs(-bf.item() - sb.max()) <= 1e-9 * sb.max()),
                          "paper_t4_gpu_seconds": PAPER_TABLE3_T4_S[side]}
    return {"workload": "Table-3 settings: 1 threshold, ps 100, 50 iterations, synthetic GMM images",
            "by_side": out, "steps": args.steps, "warmup": args.warmup}


def run_variants(args, seeds=31):
    """Quality of the variant switches on the scale workload (ps 4096, D 100,
    2000 iterations, the four forms): median best fitness over seeds 0..30 for
    Eq. 13 as printed, its mirrored form (pdr_form 1) and the better / worse
    pair policy of Eq. 6-7 (pair_policy 1)."""
    world, rank, local, torch, apo = _ctx()
    dev = torch.device("cuda", local)
    T = args.iters or 2000
    specs = inputs.scale_forms(seed=0, D=100)
    probs = [apo.problem_from_spec(s) for s in specs]
    variants = {"as_printed": dict(pdr_form=0, pair_policy=0), "pdr_mirrored": dict(pdr_form=1, pair_policy=0),
                "pairs_better_worse": dict(pdr_form=0, pair_policy=1)}
    out = {}
    t0 = time.perf_counter()
    for name, kw in variants.items():
        allp, prm = [], []
        for j, p in enumerate(probs):
            for sd in range(seeds):
                allp.append(p)
                prm.append(apo.apo_params_make(4096, 1, 0.1, T, sd, j, kw["pdr_form"], kw["pair_policy"]))
        bx = torch.zeros((len(allp), 100), device=dev)
        bf = torch.zeros(len(allp), dtype=torch.float64, device=dev)
        apo.apo_run_batch(allp, prm, bx, 100, bf)
        v = bf.cpu().numpy().reshape(len(probs), seeds)
        out[name] = {inputs.FORM_NAMES[s.kind]: float(np.median(v[j])) for j, s in enumerate(specs)}
    return {"workload": "scale forms, ps 4096, D 100, %d iterations, %d seeds per form and variant" % (T, seeds),
            "median_best": out, "seconds": time.perf_counter() - t0}


def cpu_baseline_line(specs, ps, iters_single, iters_all, seeds=31):
    """The oracle as it stands on the host cores: one run per form on one core
    (per-(objective, seed) rates), and 31 seeds x the forms over every core."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    probs = [oracle.OracleProblem.from_spec(s) for s in specs]
    single = {}
    t_single = 0.0
    for k, p in enumerate(probs):
        t0 = time.perf_counter()
        oracle.apo_run_many([p], [oracle.params(ps, 1, 0.1, iters_single, 1000, k)], 1)
        dt = time.perf_counter() - t0
        t_single += dt
        single[inputs.FORM_NAMES[specs[k].kind]] = ps * (iters_single + 1) / dt
    allp, prm = [], []
    for k, p in enumerate(probs):
        for sd in range(seeds):
            allp.append(p)
            prm.append(oracle.params(ps, 1, 0.1, iters_all, sd, k))
    t0 = time.perf_counter()
    oracle.apo_run_many(allp, prm, cores)
    dt = time.perf_counter() - t0
    value = len(allp) * ps * iters_all / dt
    return {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d runs (%d seeds x %d forms) x ps %d x %d iterations (+ initialisation) over %d cores in "
                      "%.1f s; single core, one run per form, %d iterations: %.1f s"
                      % (len(allp), seeds, len(specs), ps, iters_all, cores, dt, iters_single, t_single),
            "single_core_updates_per_s": single}


def run_scale(args):
    """The headline: plain APO at ps 4096, D 100, 2000 iterations on the four
    shifted-rotated forms (one step = one apo_run_batch of the four runs)."""
    world, rank, local, torch, apo = _ctx()
    specs, ps, T, label = workload(args.workload, args.iters)
    n = len(specs)
    Dmax = max(s.D for s in specs)
    probs = [apo.problem_from_spec(s) for s in specs]
    dev = torch.device("cuda", local)
    bx = torch.zeros((n, Dmax), device=dev)
    bf = torch.zeros(n, dtype=torch.float64, device=dev)
    cv = torch.zeros((n, T + 1), device=dev)
    flush = torch.zeros(64 << 20, dtype=torch.float32, device=dev)
    ev_run0 = torch.cuda.Event(enable_timing=True)
    ev_run1 = torch.cuda.Event(enable_timing=True)
    ev_run0.record()   # torch creates the cudaEvent_t on first record
    ev_run1.record()

    def step(k):
        prms = [apo.apo_params_make(ps, 1, 0.1, T, replica_seed(k, rank), j) for j in range(n)]
        apo.apo_run_batch(probs, prms, bx, Dmax, bf, cv, T + 1)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    sync_ranks(world)
    apo.apo_set_timing_events(ev_run0, ev_run1)
    step_ms, run_ms = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            e0.record()
            step(args.warmup + k)
            e1.record()
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            run_ms.append(ev_run0.elapsed_time(ev_run1))
    apo.apo_set_timing_events(None, None)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    sync_ranks(world)
    evals = world * args.steps * n * ps * (T + 1)
    value = aggregate_rate(world, args.steps * n * ps * T, total_ms * 1e-3)

    # end to end through the public API: problem upload from host memory,
    # the batch call, and the results read back into pinned host memory
    e2e = None
    if not args.no_e2e:
        host_bx = torch.empty((n, Dmax), pin_memory=True)
        host_bf = torch.empty(n, dtype=torch.float64, pin_memory=True)
        host_cv = torch.empty((n, T + 1), pin_memory=True)
        h2d = sum(4 * (s.D * s.D + s.D) + 16 * s.D + (0 if s.perm is None else 4 * s.D) for s in specs)
        d2h = host_bx.numel() * 4 + host_bf.numel() * 8 + host_cv.numel() * 4
        e2e_s = []
        for k in range(args.steps):
            flush_l2(flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ps_k = [apo.problem_from_spec(s) for s in specs]
            prms = [apo.apo_params_make(ps, 1, 0.1, T, 7000 + 100 * k + rank, j) for j in range(n)]
            apo.apo_run_batch(ps_k, prms, bx, Dmax, bf, cv, T + 1)
            host_bx.copy_(bx, non_blocking=True)
            host_bf.copy_(bf, non_blocking=True)
            host_cv.copy_(cv, non_blocking=True)
            torch.cuda.synchronize()
            del ps_k
            e2e_s.append(time.perf_counter() - t0)
        e2e_v = n * ps * T * args.steps / sum(e2e_s) * world
        e2e = {"value": e2e_v, "unit": "updates/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    pk = peaks()
    clocks = clk.summary()
    # dominant kernel: the iteration-loop kernel; algorithmic work per launch is
    # the rotation z = M (x - o) of every evaluation, 2 D^2 flop each
    flop_per_launch = sum(2.0 * s.D * s.D * ps * (T + 1) for s in specs)
    run_avg_s = statistics.mean(run_ms) * 1e-3
    achieved = flop_per_launch / run_avg_s / 1e12
    kernel = "grid_kernel" if ps > 1024 or (n == 1 and ps >= 128) else "run_kernel"
    measured = None
    try:
        measured = apo.apo_measure_peaks()
    except Exception:   # instrumentation only; the line stays valid without it
        measured = None
    if measured:
        alu_peak, alu_src = measured["ffma_tflops"], "apo_measure_peaks: FFMA chains on every SM (this run)"
    else:
        alu_peak = SMS * FP32_LANES * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        alu_src = "152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s clock)" % (float(pk.get("sm_max_mhz", 2070.0)),
                                                                           pk["source"])
    D = Dmax
    # algorithmic integer/FP operations per candidate update (a model of the
    # arithmetic the method needs, not of what the kernel issues): ceil(D/2)
    # Philox4x32-10 calls of 10 rounds x 10 operations, the mask k-selection
    # (about 3.5 warp-wide counts over D keys, 3 operations per key), about
    # 12 D operations of candidate arithmetic and clamp, 3 D of the objective
    # epilogue; the rotation itself runs on the tensor cores
    alg_ops = ((D + 1) // 2) * 100 + 3.5 * 3 * D + 12 * D + 3 * D
    alg_achieved = alg_ops * sum(ps * (T + 1) for _ in specs) / run_avg_s / 1e12
    line = {
        "metric": "APO candidate updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": label, "runs_per_step": n, "ps": ps, "D": Dmax, "iterations": T,
                   "np": 1, "pf_max": 0.1, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "true_evals_per_s": evals / (total_ms * 1e-3),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": None,
                     "kernel": "%s: rotation on the tensor cores (3-term fp16 split, fp32 accumulation); "
                               "achieved = 2 D^2 rotation flop per evaluation (FP32-equivalent) / kernel time, "
                               "against the FP32 FMA peak; the kernel is issue-bound in candidate generation "
                               "and ranking" % kernel,
                     "tensor_frac": achieved / (float(pk.get("bf16_tflops", 1880.9))),
                     "peak_source": alu_src, "kernel_ms": statistics.mean(run_ms)},
        "roofline_alu_ops": {"bound": "alu", "achieved": alg_achieved,
                             "peak": measured["alu_tops"] if measured else None, "unit": "Tops/s",
                             "frac": alg_achieved / measured["alu_tops"] if measured else None,
                             "ops_per_update": alg_ops,
                             "model": "ceil(D/2) Philox calls x 100 + mask selection 10.5 D + 12 D candidate + 3 D "
                                      "epilogue integer/FP operations per update, against the measured plain-ALU "
                                      "throughput (apo_measure_peaks)"},
        "measured_peaks": measured,
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(specs, ps, args.cpu_single_iters, args.cpu_all_iters)
    return line


def _brief(line, keys):
    return {k: line.get(k) for k in keys if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="scale",
                    choices=["scale", "single", "batched", "thresholding", "surrogate", "table2", "table3", "variants"])
    ap.add_argument("--images", type=int, default=256, help="thresholding: number of images")
    ap.add_argument("--side", type=int, default=4096, help="thresholding: image side")
    ap.add_argument("--seeds", type=int, default=5, help="surrogate: seeds for the time-to-target comparison")
    ap.add_argument("--runs", type=int, default=1024, help="batched workload: number of runs")
    ap.add_argument("--per-run-sample", type=int, default=24, help="batched: runs timed with one launch each")
    ap.add_argument("--batch-config", default="",
                    help="batched: fixed SMEM_BUDGET,CTAS_PER_SM,CLUSTER_PS,CLUSTER_SIZE instead of autotuning")
    ap.add_argument("--iters", type=int, default=0, help="override the iteration count (profiling)")
    ap.add_argument("--ps", type=int, default=0, help="table2: one population instead of 1000 and 10000")
    ap.add_argument("--ref-iters", type=int, default=2, help="oracle iterations of each run per --impl reference step")
    ap.add_argument("--cpu-single-iters", type=int, default=10,
                    help="cpu_baseline: oracle iterations of the one-core run per form")
    ap.add_argument("--cpu-all-iters", type=int, default=3,
                    help="cpu_baseline: oracle iterations of each of the 31 x 4 runs spread over all cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="scale workload: skip the secondary workloads reported beside the headline")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    runners = {"batched": run_batched, "thresholding": run_thresholding, "surrogate": run_surrogate,
               "table2": run_table2, "table3": run_table3, "variants": run_variants}
    if args.workload in runners:
        line = runners[args.workload](args)
    else:
        line = run_scale(args)
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if args.workload == "scale" and not args.no_extras and world == 1:
            import copy
            sub = copy.copy(args)
            sub.iters = 0
            sub.steps, sub.warmup = 3, 3
            b = run_batched(sub)
            line["batched"] = _brief(b, ["value", "unit", "ms_per_step", "true_evals_per_s", "per_run_launch",
                                         "roofline", "config", "e2e"])
            th = run_thresholding(sub)
            line["thresholding"] = _brief(th, ["value", "unit", "ms_per_step", "histogram_ms", "apo_ms",
                                               "histogram_bit_exact_spot_check", "roofline", "config"])
            sub.steps, sub.warmup = 1, 1
            su = run_surrogate(sub)
            line["surrogate"] = _brief(su, ["value", "unit", "ms_per_step", "true_evals_per_s", "time_to_target",
                                            "config"])
            line["surrogate"]["seeds"] = sub.seeds
            line["table2"] = run_table2(sub, steps=2, warmup=1)
            sub.steps, sub.warmup = 3, 1
            line["table3"] = run_table3(sub)
            line["variants"] = run_variants(sub)
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line))
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
