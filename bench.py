#!/usr/bin/env python
"""Throughput of one separable-dictionary-learning iteration on GB300.

One step = one iteration of Algorithm 1 (two 2D-OMP coding passes with the
fused partial sums, the D1 and D2 least-squares updates and the code
rescale) over the whole training set, through the library's C ABI.  Steps
are timed two ways: per-call launches of sdl_iterate (each kernel timed by
events: the per-kernel split and the roofline), and the batched path
(sdl_batch_iterate: one captured CUDA graph per iteration, autotuned
tilings), which gives the headline value.

Workload: image-patch learning, N = 200000 mean-removed 12x12 FP32 patches
cut at seeded positions from 64 seeded synthetic 512x512 images, D1, D2
12x24 (576 atom pairs), s = 6.  Metric: signals/s per iteration.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (torchrun) every rank runs
an independent replica of the workload on its own GPU ("replicas only": the
one-GPU method has no data-path exchange between GPUs); value aggregates all
ranks.  --impl reference times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "signals/sec per 2D-OMP+TMOD iteration"
UNIT = "signals/s"
W = dict(N=200_000, p1=12, p2=12, n1=24, n2=24, s=6, n_images=64, image_seed=100,
         patch_seed=5, dict_seed=1)
WORKLOAD = ("image-patch learning: N=200000 mean-removed 12x12 FP32 patches from 64 seeded "
            "synthetic 512x512 images, D1,D2 12x24, s=6, one Algorithm-1 iteration per step")
CPU_SAMPLE = 32768          # signals in the timed oracle sample (cpu_baseline)
REF_SAMPLE = 8192           # signals per step of the reference arm
FLUSH_BYTES = 256 << 20     # > 129 MB L2


def make_inputs():
    from paper_2007_03800_gb300 import synth
    imgs = np.stack([synth.synthetic_image(W["image_seed"] + i) for i in range(W["n_images"])])
    Y = synth.random_patches(imgs, W["N"], W["p1"], seed=W["patch_seed"])
    D1, D2 = synth.init_dictionaries(W["p1"], W["p2"], W["n1"], W["n2"], seed=W["dict_seed"])
    return Y, D1, D2


# ------------------------------------------------------------- algorithmic work
def flops_per_signal_pass(p1, p2, n1, n2, s, side):
    """Algorithmic FLOPs of one 2D-OMP coding pass of one signal (with the
    fused partial sums of `side`): correlation C0 = D1^T (Y D2) in the cheaper
    association, the Gram-domain correlation updates sum_t 2 t n1 n2, the
    incremental Cholesky/solves ~2 t^2 per step, and the epilogue sums (B1 takes
    rows of Z = Y D2, B2 rows of W = D1^T Y, both already formed for C0)."""
    c0 = 2 * min(p1 * p2 * n2 + n1 * p1 * n2, n1 * p1 * p2 + n1 * p2 * n2)
    upd = sum(2 * t * n1 * n2 for t in range(s))
    chol = sum(2 * t * t + 4 * t + 4 for t in range(s))
    epi = 2 * (p1 if side == 1 else p2) * s + 3 * s * s
    return c0 + upd + chol + epi


def bytes_per_signal_pass(p1, p2, s, side):
    """Algorithmic HBM bytes: Y read once per pass; codes written by pass 2."""
    return 4 * p1 * p2 + (8 * s + 4 if side == 2 else 0)


def flops_pass_hist(p1, p2, n1, n2, s, side, nnz_hist):
    """Algorithmic FLOPs of one coding pass of signals whose code sizes have
    the histogram nnz_hist (error-driven stop): a signal with no atom skips
    its correlations; one with m atoms pays C0, the score updates of steps
    1..m-1, m Cholesky steps and its epilogue sums."""
    c0 = 2 * min(p1 * p2 * n2 + n1 * p1 * n2, n1 * p1 * p2 + n1 * p2 * n2)
    tot = 0
    for m, count in enumerate(nnz_hist):
        if m == 0 or count == 0:
            continue
        upd = sum(2 * t * n1 * n2 for t in range(m))
        chol = sum(2 * t * t + 4 * t + 4 for t in range(m))
        epi = 2 * (p1 if side == 1 else p2) * m + 3 * m * m if side else 0
        tot += count * (c0 + upd + chol + epi)
    return tot


def flops_ortho_pass(p1, p2, s):
    """Thresholded coding (Remark 1, square dictionaries): C0 = D1^T Y D2 and
    the epilogue sums; no pursuit."""
    return 2 * (p1 * p2 * p2 + p1 * p1 * p2) + 2 * max(p1, p2) * s


def flops_pass3(p, n, s):
    """Three-mode pursuit (Remark 3) of one signal: C0 by three mode
    contractions in the cheapest order, the score updates sum_t 2 t Q over
    Q = n1 n2 n3 triples, the Cholesky steps and the mode-k epilogue."""
    import itertools
    best = None
    for order in itertools.permutations(range(3)):
        dims, cost = list(p), 0
        for m in order:       # mode-m product: every fibre of length p_m becomes one of length n_m
            others = dims[0] * dims[1] * dims[2] // dims[m]
            cost += 2 * others * p[m] * n[m]
            dims[m] = n[m]
        best = cost if best is None else min(best, cost)
    Q = n[0] * n[1] * n[2]
    upd = sum(2 * t * Q for t in range(s))
    chol = sum(2 * t * t + 4 * t + 4 for t in range(s))
    return best + upd + chol + 2 * max(p) * s + 3 * s * s


def alu_roofline(kernel, flops_per_launch, ms_per_launch, peak, basis):
    achieved = flops_per_launch / (ms_per_launch / 1e3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "algorithmic_flops_per_launch": flops_per_launch,
            "ms_per_launch": ms_per_launch, "peak_basis": basis}


PEAK_BASIS = "measured FP32 FMA rate (sdl_fp32_fma_peak, packed fma.rn.f32x2)"


# sources of the coding-pass kernels timed by the roofline (the specialised
# kernel and its shared header): stored DRAM counters are only used while
# these files are unchanged
KERNEL_SOURCES = ("omp_fast.cu", "sdl_internal.cuh")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_03800_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------- CPU oracle
_ORACLE_SNIPPET = r"""
import sys, time, json, os
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle


def code_chunk(args):
    Y, D1, D2, s = args
    r = oracle.omp2d(Y, D1, D2, s)
    return r.support, r.coef


def iterate_pool(pool, nchunks, Y, D1, D2, s):
    # Algorithm 1 with the two coding passes spread over worker processes by
    # signal chunks (each signal's pursuit is independent); the dictionary
    # updates, which sum over all signals, run here
    parts = np.array_split(np.arange(Y.shape[0]), nchunks)

    def code(Da, Db):
        out = pool.map(code_chunk, [(Y[c], Da, Db, s) for c in parts])
        return np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out])

    sa, ca = code(D1, D2)
    upd_a = oracle.update_D1(Y, D1, D2, sa, ca)
    sb, cb = code(upd_a.D, D2)
    return oracle.update_D2(Y, upd_a.D, D2, sb, cb)


if __name__ == "__main__":
    d = np.load(sys.argv[2])
    Y, D1, D2, s, reps, cores = d["Y"], d["D1"], d["D2"], int(d["s"]), int(d["reps"]), int(d["cores"])
    times = []
    if cores <= 1:
        for _ in range(reps):
            t = time.perf_counter()
            r = oracle.iterate(Y, D1, D2, s)
            times.append(time.perf_counter() - t)
        if len(sys.argv) > 3:
            N, p1, p2 = Y.shape
            np.savez(sys.argv[3], D1=r.D1, D2=r.D2, support=r.support, nnz=r.nnz,
                     rmse=np.array([r.rmse_after_D1, r.rmse_after_D2]))
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(code_chunk, [(Y[:8], D1, D2, s)] * cores)      # workers started and warm
            for _ in range(reps):
                t = time.perf_counter()
                iterate_pool(pool, 4 * cores, Y, D1, D2, s)
                times.append(time.perf_counter() - t)
    print(json.dumps(times))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(Y, D1, D2, s, reps, cores=1, result_path=None):
    """Run the FP64 oracle (unmodified) in a child process: one iteration of
    Algorithm 1 per rep, on one host thread (cores = 1; `result_path` then
    receives its dictionaries, codes and RMSEs) or with its coding passes
    spread over `cores` single-threaded worker processes.  Returns the wall
    time of every rep."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.npz")
        script = os.path.join(td, "oracle_run.py")
        with open(script, "w") as f:
            f.write(_ORACLE_SNIPPET)
        np.savez(path, Y=Y, D1=D1, D2=D2, s=s, reps=reps, cores=cores)
        cmd = [sys.executable, script, ROOT, path] + ([result_path] if result_path else [])
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------ arms
def max_over_ranks(value, dist, dev):
    """The largest of every rank's value (the job's time is its slowest
    rank's); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, units_per_rank, ms_per_step):
    """Whole-job throughput of `world` replicas that each process
    `units_per_rank` units per step, the step taking `ms_per_step` on the
    slowest rank."""
    return world * units_per_rank / (ms_per_step / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    Y, D1, D2 = make_inputs()
    sample = Y[:REF_SAMPLE]
    cores = host_cores()
    times = time_oracle(sample, D1, D2, W["s"], args.warmup + args.steps, cores=cores)[args.warmup:]
    per_step = sum(times) / len(times)
    value = REF_SAMPLE / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_signals_per_step": REF_SAMPLE},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {REF_SAMPLE} of the 200000 patches, one full "
                                   "Algorithm-1 iteration per step, FP64 numpy, the coding passes "
                                   f"over {cores} single-threaded worker processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2007_03800_gb300 import sdl

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        dist = None
        torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    p1, p2, n1, n2, s, N = W["p1"], W["p2"], W["n1"], W["n2"], W["s"], W["N"]

    Y, D1, D2 = make_inputs()
    Y32 = np.asarray(Y, dtype=np.float32)
    ctx = sdl.Context(local)
    ctx.reserve(p1, p2, n1, n2, s)
    Yg = sdl.signals(torch.from_numpy(Y32).to(dev))
    D1_0 = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device=dev))
    D2_0 = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device=dev))
    D1g, D2g = sdl.dictionary(D1_0.clone()), sdl.dictionary(D2_0.clone())
    codes = sdl.Codes.empty(N, s, dev)
    rmse = torch.zeros(2, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # the per-call path runs the tiling the tuner measured fastest on these
    # signals (every tiling gives the same codes), or the one --tiling names
    if args.tiling is None:
        tiling, tune_log = ctx.tune_tiling(Yg, D1g, D2g, s)
        tune_log = [dict(tiling=e["tiling"], ctas_per_sm=e["ctas_per_sm"], us=round(e["us"], 1))
                    for e in tune_log]
    else:
        tiling, tune_log = args.tiling, []
        ctx.set_tiling(p1, p2, n1, n2, s, tiling, 2)
    for _ in range(args.warmup):
        ctx.iterate(Yg, D1g, D2g, s, out=codes, rmse_out=rmse)
    ctx.check()
    ctx.profile_collect()                      # reset counters

    # ---- timed regions (L2 flushed between steps, untimed):
    #   A: per-call launches of sdl_iterate, each kernel bracketed by events
    #      (per-kernel split and the roofline of the dominant kernel);
    #   B: the batched path: persistent multi-problem passes, one launch per
    #      update stage, the iteration replayed from one captured CUDA graph,
    #      tilings and CTA split picked by the autotuner (the headline value).
    def timed(step_fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step_fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        total = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, dev)
        return total / args.steps

    batch = sdl.Batch(ctx, [dict(Y=Yg, D1=D1g, D2=D2g, s=s, codes=codes)], autotune=True,
                      graph=True)
    rmse_b = torch.zeros(2, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        batch.iterate(rmse_out=rmse_b)
    ctx.check()
    with ClockSampler(local) as clk:
        # clock pre-roll: identical untimed iterations for ~1.5 s, so that the
        # 100 ms nvidia-smi sampler sees the GPU under this load around the
        # (short) timed regions
        t_end = time.perf_counter() + (0.0 if args.quick else 1.5)
        while time.perf_counter() < t_end:
            for _ in range(8):
                batch.iterate(rmse_out=rmse_b)
            torch.cuda.synchronize()
        ctx.profile_collect()                  # reset counters after the pre-roll
        ctx.profile(True)
        ms_plain = timed(lambda: ctx.iterate(Yg, D1g, D2g, s, out=codes, rmse_out=rmse))
        ctx.profile(False)
        prof = ctx.profile_collect()
        ms_per_step = timed(lambda: batch.iterate(rmse_out=rmse_b))
        prof_b = ctx.profile_collect()
    ctx.check()
    tuning = batch.tuning()
    tuning_log = [dict(shape_id=t["shape_id"], ctas_per_sm=t["ctas_per_sm"], us=round(t["cost_us"], 1))
                  for t in batch.tuning_log()]
    batch.close()
    value = replica_throughput(world, N, ms_per_step)
    value_plain = replica_throughput(world, N, ms_plain)
    final_rmse = rmse_b.cpu().tolist()

    # ---- end to end: host inputs in, results out, every step
    if args.quick:
        print(json.dumps({"quick": True, "ms_per_step": ms_per_step, "ms_per_step_plain": ms_plain,
                          "kernels": prof, "tuning": tuning, "tuning_log": tuning_log,
                          "tiling": tiling, "tune_log": tune_log}), flush=True)
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return 0
    # Every step is an independent job through the public API: H2D of the
    # signals and the starting dictionaries from pinned host memory, one
    # Algorithm-1 iteration (sdl_batch_iterate: the graph-replayed batch of the
    # set's device buffers), D2H of the codes, the dictionaries and the RMSE.
    # Two device buffer sets (a batch each; the context remembers the tuning
    # of the timed batch above) and two copy streams let the copies of step
    # k+1 and the results of step k-1 move while step k computes (a set is
    # refilled only after its previous results have left).  The L2 flush of
    # each step is inside the timed region: it runs on the copy stream after
    # the step's inputs have arrived and before its compute may start, so no
    # input of a step is served from L2, while the previous step computes.
    Yh = torch.from_numpy(np.ascontiguousarray(Y32.transpose(0, 2, 1))).pin_memory()  # (N, p2, p1)
    D1h = torch.tensor(D1, dtype=torch.float32).t().contiguous().pin_memory()   # column-major
    D2h = torch.tensor(D2, dtype=torch.float32).t().contiguous().pin_memory()
    sets = []
    for _ in range(2):
        S = {"Y": torch.empty((N, p2, p1), dtype=torch.float32, device=dev),
             "D1": torch.empty((n1, p1), dtype=torch.float32, device=dev),
             "D2": torch.empty((n2, p2), dtype=torch.float32, device=dev),
             "codes": sdl.Codes.empty(N, s, dev),
             "rmse": torch.zeros(2, dtype=torch.float64, device=dev),
             "in": torch.cuda.Event(), "done": torch.cuda.Event(), "out": torch.cuda.Event()}
        S["host"] = {"D1": torch.empty_like(D1h).pin_memory(), "D2": torch.empty_like(D2h).pin_memory(),
                     "support": torch.empty((N, s), dtype=torch.int32).pin_memory(),
                     "coef": torch.empty((N, s), dtype=torch.float32).pin_memory(),
                     "nnz": torch.empty((N,), dtype=torch.int32).pin_memory(),
                     "rmse": torch.empty(2, dtype=torch.float64).pin_memory()}
        S["batch"] = sdl.Batch(ctx, [dict(Y=S["Y"].transpose(1, 2), D1=S["D1"].t(), D2=S["D2"].t(),
                                          s=s, codes=S["codes"])], autotune=True, graph=True)
        sets.append(S)
    h2d = Yh.numel() * 4 + D1h.numel() * 4 + D2h.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in sets[0]["host"].values())
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    s_run = torch.cuda.Stream(device=dev)

    def put(k):
        S = sets[k % 2]
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(S["out"])            # the set's previous results have left
            S["Y"].view(-1).copy_(Yh.view(-1), non_blocking=True)
            S["D1"].copy_(D1h, non_blocking=True)
            S["D2"].copy_(D2h, non_blocking=True)
            flush.fill_(float(k))
            S["in"].record(s_in)

    def run(k):
        S = sets[k % 2]
        s_run.wait_event(S["in"])
        S["batch"].iterate(rmse_out=S["rmse"], stream=s_run)
        S["done"].record(s_run)
        with torch.cuda.stream(s_out):
            s_out.wait_event(S["done"])
            H = S["host"]
            H["D1"].copy_(S["D1"], non_blocking=True)
            H["D2"].copy_(S["D2"], non_blocking=True)
            H["support"].copy_(S["codes"].support, non_blocking=True)
            H["coef"].copy_(S["codes"].coef, non_blocking=True)
            H["nnz"].copy_(S["codes"].nnz, non_blocking=True)
            H["rmse"].copy_(S["rmse"], non_blocking=True)
            S["out"].record(s_out)

    def pipeline(n):
        put(0)
        for k in range(n):
            if k + 1 < n:
                put(k + 1)
            run(k)

    pipeline(args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    pipeline(args.steps)
    t1.record(s_out)
    t1.synchronize()
    torch.cuda.synchronize()
    ctx.check()
    for S in sets:
        S["batch"].close()
    e2e_total = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    e2e_value = replica_throughput(world, N, e2e_total / args.steps)

    line = None
    if rank == 0:
        peaks = measured_peaks()
        props = torch.cuda.get_device_properties(dev)
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        fp32_derived = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
        # the FP32 FMA peak, measured on this GPU (packed fma.rn.f32x2, as the coders issue)
        fp32_peak, _ = sdl.fp32_fma_peak(packed=True)
        fp32_scalar, _ = sdl.fp32_fma_peak(packed=False)
        kinds = {k: v for k, v in prof.items() if v[1] > 0}
        dom = max(kinds, key=lambda k: kinds[k][0])
        dom_ms, dom_n = kinds[dom]
        side = {"code_D1": 1, "code_D2": 2}.get(dom, 2)
        flops = N * flops_per_signal_pass(p1, p2, n1, n2, s, side)
        achieved = flops / (dom_ms / dom_n / 1e3) / 1e12
        traffic = issue = None
        tpath = os.path.join(ROOT, "profiles", "traffic.json")
        clk = clk.summary()
        if os.path.exists(tpath):
            t = json.load(open(tpath))
            ent = t.get(f"{dom}/tiling{tiling}")
            if ent and ent.get("source_hash") == source_hash() and ent.get("N") == N:
                traffic = ent["dram_bytes_per_launch"]
                inst = ent.get("warp_instructions_per_launch")
                if inst:
                    # instruction-issue bound: every SM sub-partition issues at
                    # most one warp instruction per cycle
                    mhz = (clk or {}).get("sm_mhz") or sm_max
                    bound_ms = inst / (props.multi_processor_count * 4 * mhz * 1e6) * 1e3
                    issue = {"warp_instructions_per_signal": inst / N,
                             "bound_ms": bound_ms, "kernel_ms": dom_ms / dom_n,
                             "frac": bound_ms / (dom_ms / dom_n), "sm_mhz": mhz}
        # the oracle on a bounded sample: one thread (its results also judge
        # the GPU below), and its coding passes spread over every host core
        with tempfile.TemporaryDirectory() as td:
            res_path = os.path.join(td, "oracle.npz")
            cpu_times = time_oracle(Y[:CPU_SAMPLE], D1, D2, s, 1, cores=1, result_path=res_path)
            ores = dict(np.load(res_path))
        cores = host_cores()
        cpu_all = time_oracle(Y[:CPU_SAMPLE], D1, D2, s, 1, cores=cores) if cores > 1 else cpu_times
        # matched RMSE: the same iteration on the GPU over the oracle's sample
        Ys = sdl.signals(torch.from_numpy(Y32[:CPU_SAMPLE]).to(dev))
        D1s, D2s = sdl.dictionary(D1_0.clone()), sdl.dictionary(D2_0.clone())
        rm = torch.zeros(2, dtype=torch.float64, device=dev)
        cs = ctx.iterate(Ys, D1s, D2s, s, rmse_out=rm)
        ctx.check()
        rm = rm.cpu().numpy()
        same = ((cs.support.cpu().numpy() == ores["support"]).all(axis=1) &
                (cs.nnz.cpu().numpy() == ores["nnz"]))
        parity = {"sample": f"first {CPU_SAMPLE} patches, one Algorithm-1 iteration from the same "
                            "start, GPU sdl_iterate (FP32) against the FP64 oracle",
                  "rmse_rel_err": [float(abs(rm[i] - ores["rmse"][i]) / ores["rmse"][i]) for i in range(2)],
                  "dict_max_abs_err": [float(np.abs(D1s.cpu().numpy() - ores["D1"]).max()),
                                       float(np.abs(D2s.cpu().numpy() - ores["D2"]).max())],
                  "supports_identical": float(same.mean()),
                  "tolerance": 1e-4}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "p1": p1, "p2": p2, "n1": n1, "n2": n2,
                       "s": s, "l2": "256 MiB buffer written between timed steps (untimed)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "path": "sdl_batch_iterate (CUDA graph, autotuned tilings)",
                       "final_rmse": final_rmse},
            "gpu_launches": int(sum(v[1] for k, v in prof_b.items() if k != "batch_graph")),
            "variants": {
                "batch_graph_autotuned": {"value": value, "ms_per_step": ms_per_step,
                                          "tuning": tuning, "tuning_log": tuning_log},
                "per_call_launches": {"value": value_plain, "ms_per_step": ms_plain,
                                      "tiling": tiling, "tune_log": tune_log},
            },
            "kernels_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in kinds.items()},
            "roofline": {"bound": "alu", "kernel": f"{dom} (tiling {tiling})", "achieved": achieved,
                         "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                         "peak_basis": "measured: FP32 FMA microbenchmark (sdl_fp32_fma_peak, packed "
                                       f"fma.rn.f32x2; scalar fma.rn.f32 {fp32_scalar:.1f}); derived "
                                       f"{props.multi_processor_count} SMs x 128 lanes x 2 x "
                                       f"{sm_max:.0f} MHz = {fp32_derived:.1f}",
                         "algorithmic_flops_per_launch": flops,
                         "issue": issue,
                         "hbm_gbs": N * bytes_per_signal_pass(p1, p2, s, side) /
                                    (dom_ms / dom_n / 1e3) / 1e9},
            "parity": parity,
            "cpu_baseline": {"value": CPU_SAMPLE / cpu_all[0], "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": f"first {CPU_SAMPLE} of the 200000 patches, one full "
                                       "Algorithm-1 iteration, FP64 numpy, the coding passes over "
                                       f"{cores} single-threaded worker processes",
                             "single_thread": {"value": CPU_SAMPLE / cpu_times[0], "cores": 1}},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_total / args.steps,
                    "path": "sdl_batch_iterate (graph replay) per step from pinned host buffers; copies "
                            "double-buffered on two streams, overlapping the neighbouring steps' compute; "
                            "each step's 256 MiB L2 flush on the input stream after its copies"},
            "clocks": clk,
        }
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ studies
# Extra measurements on the other synthetic workloads (one JSON line each,
# "study": name).  They are not the headline line and touch no oracle.
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _device_dict(D, dev):
    import torch

    from paper_2007_03800_gb300 import sdl
    return sdl.dictionary(torch.tensor(D, dtype=torch.float32, device=dev))


def study_precision(args):
    """Hyperspectral-shaped signals, N = 50000 of 16x64, D1 16x32, D2 64x128,
    s = 10, 15 iterations from the same start in each precision mode: device
    time per iteration, the per-kernel split of one iteration, the RMSE
    trajectory and the entries re-scored in FP32.  Y is 205 MB (> L2), so no
    flush is needed between iterations."""
    import torch

    from paper_2007_03800_gb300 import sdl, synth
    dev = torch.device("cuda:0")
    N, s, iters = 50_000, 10, 15
    Y = synth.hyperspectral(N, seed=31)
    D1, D2 = synth.init_dictionaries(16, 64, 32, 128, seed=1)
    ctx = sdl.Context(0)
    Yg = sdl.signals(torch.tensor(Y, dtype=torch.float32, device=dev))
    codes = sdl.Codes.empty(N, s, dev)
    rmse = torch.zeros(2, dtype=torch.float64, device=dev)
    C = sdl.Context
    modes = {"fp32": C.PREC_FP32, "bf16_rescored": C.PREC_BF16_CORR,
             "fp64_solve": C.PREC_FP64_SOLVE, "bf16_fp64": C.PREC_BF16_CORR | C.PREC_FP64_SOLVE}
    peak, _ = sdl.fp32_fma_peak(packed=True)
    out = {}
    for name, flags in modes.items():
        ctx.set_precision(flags)
        D1w, D2w = _device_dict(D1, dev), _device_dict(D2, dev)
        for _ in range(args.warmup):
            ctx.iterate(Yg, D1w, D2w, s, out=codes, rmse_out=rmse)
        ctx.status()
        ctx.precision_stats()
        D1g, D2g = _device_dict(D1, dev), _device_dict(D2, dev)
        ms, traj, resc, st = [], [], [], []
        for _ in range(iters):
            a, b = _events()
            a.record()
            ctx.iterate(Yg, D1g, D2g, s, out=codes, rmse_out=rmse)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
            traj.append(rmse.tolist())
            resc.append(ctx.precision_stats())
            # a singular normal matrix leaves that dictionary unchanged and is
            # recorded here; the run goes on
            rc = ctx.status()
            st.append(sdl.ERRORS.get(rc, str(rc)) if rc else "ok")
        ctx.profile_collect()
        ctx.profile(True)
        ctx.iterate(Yg, D1w, D2w, s, out=codes, rmse_out=rmse)
        ctx.profile(False)
        prof = {k: v for k, v in ctx.profile_collect().items() if v[1] > 0}
        split = {k: round(v[0], 4) for k, v in prof.items()}
        ctx.status()
        roof = None
        if not flags & C.PREC_BF16_CORR and "code_D1" in prof:
            # the FP32 coding pass (D1 side) against the FP32 FMA peak
            roof = alu_roofline("code_D1 (generic coder, 16x64 signals, 32x128 pairs, s=10)",
                                N * flops_per_signal_pass(16, 64, 32, 128, s, 1),
                                prof["code_D1"][0] / prof["code_D1"][1], peak, PEAK_BASIS)
        out[name] = {"roofline": roof, "ms_per_iteration": statistics.median(ms), "signals_per_s":
                     N / (statistics.median(ms) / 1e3), "final_rmse": traj[-1],
                     "rmse_trajectory_after_D2": [round(t[1], 7) for t in traj],
                     "status_per_iteration": st,
                     "rescored_per_iteration": resc, "kernel_ms_one_iteration": split}
    ref = out["fp32"]["final_rmse"][1]
    for name in out:
        out[name]["final_rmse_rel_vs_fp32"] = out[name]["final_rmse"][1] / ref - 1.0
    ctx.close()
    print(json.dumps({"study": "precision", "workload": "hyperspectral-shaped 16x64 signals, "
                      "N=50000, D1 16x32, D2 64x128, s=10, 15 iterations",
                      "unit": "signals/s per iteration", "modes": out}), flush=True)
    return 0


def study_learned(args):
    """Learned support proposal on the 12x12 separable generative model (s = 6,
    20 dB): dictionaries from 20 plain iterations on 1M training signals,
    labels = the plain 2D-OMP codes of those signals, network 144 -> 512
    (GELU) -> 576 trained on the GPU, then 1M fresh signals of the same model
    coded by both coders (k = 32)."""
    import torch

    from paper_2007_03800_gb300 import learned, sdl
    p, n, s, k, N = 12, 24, 6, 32, 1_000_000
    ctx = sdl.Context(0)
    t0 = time.perf_counter()
    Yg, D1g, D2g, labels = learned.kron_problem(ctx, N, p, n, s, dl_iterations=20)
    Yt = learned.fresh_signals(N, p, n, s)
    t_prep = time.perf_counter() - t0
    net = sdl.MLP(ctx, p, p, n, n, hidden=512, max_batch=65536)
    net.init(seed=3)
    a, b = _events()
    a.record()
    hist = learned.train(net, Yg, labels, epochs=30, batch=4096, lr=2e-3, cosine=True)
    b.record()
    b.synchronize()
    ms_train = a.elapsed_time(b)
    untrained = sdl.MLP(ctx, p, p, n, n, hidden=512, max_batch=65536)
    untrained.init(seed=3)
    base = learned.compare(ctx, untrained, Yt, D1g, D2g, s, k=k, reps=1)
    untrained.close()
    for _ in range(args.warmup):
        learned.compare(ctx, net, Yt[:65536], D1g, D2g, s, k=k, reps=1)
    res = learned.compare(ctx, net, Yt, D1g, D2g, s, k=k, reps=max(args.steps, 1))
    # shortlist recall on the fresh signals: the share of the plain coder's
    # picks inside the k-pair shortlist, per pick and per signal (all picks)
    plain = ctx.sparse_code(Yt, D1g, D2g, s)
    hits, picks, whole = 0, 0, 0
    for r0 in range(0, N, 131072):
        sl = slice(r0, min(N, r0 + 131072))
        cand = ctx.learned_shortlists(net.forward(Yt[sl]), k, k)
        sup = plain.support[sl]
        inside = (cand[:, :, None] == sup[:, None, :]).any(dim=1) | (sup < 0)
        hits += int(((cand[:, :, None] == sup[:, None, :]).any(dim=1) & (sup >= 0)).sum())
        picks += int((sup >= 0).sum())
        whole += int(inside.all(dim=1).sum())
    res.update({"shortlist_recall_per_pick": hits / max(picks, 1),
                "shortlist_holds_every_pick": whole / N})
    ctx.profile_collect()
    ctx.profile(True)
    net.sparse_code(Yt, D1g, D2g, s, k=k)
    ctx.profile(False)
    split = {kk: round(v[0], 4) for kk, v in ctx.profile_collect().items() if v[1] > 0}
    ctx.check()
    net.close()
    ctx.close()
    res.update({"train_loss_per_epoch": [round(h, 4) for h in hist], "ms_train": ms_train, "k": k,
                "train": "30 epochs of 1M pairs, batch 4096, Adam, step 2e-3 with cosine decay",
                "untrained_network": {kk: base[kk] for kk in ("rmse_gap", "fallback_rate",
                                                               "identical_codes", "speedup")},
                "learned_kernel_ms": split, "host_prep_s": t_prep,
                "signals_per_s_plain": N / (res["ms_plain"] / 1e3),
                "signals_per_s_learned": N / (res["ms_learned"] / 1e3)})
    print(json.dumps({"study": "learned", "workload": "12x12 separable model (s=6, 20 dB), "
                      "D 12x24 from 20 plain iterations, 1M training pairs, 1M fresh signals",
                      "result": res}), flush=True)
    return 0


def study_ortho(args):
    """Orthonormal variant (Remark 1) on the bench's 200k 12x12 patches: square
    orthonormal D1, D2 (12 x 12, random orthogonal start from seed 1), s = 6,
    20 iterations of thresholded coding + Procrustes updates; device time per
    iteration and the RMSE trajectory, next to the general variant (D 12x24)
    on the same patches for context."""
    import torch

    from paper_2007_03800_gb300 import sdl
    dev = torch.device("cuda:0")
    Y, D1g_init, D2g_init = make_inputs()
    p, s, N = 12, 6, W["N"]
    rng = np.random.default_rng(1)
    Qs = []
    for _ in range(2):
        Q, R = np.linalg.qr(rng.standard_normal((p, p)))
        Qs.append(Q * np.sign(np.diag(R)))
    ctx = sdl.Context(0)
    Yg = sdl.signals(torch.tensor(Y, dtype=torch.float32, device=dev))
    codes = sdl.Codes.empty(N, s, dev)
    rmse = torch.zeros(2, dtype=torch.float64, device=dev)
    D1w, D2w = _device_dict(Qs[0], dev), _device_dict(Qs[1], dev)
    for _ in range(args.warmup):
        ctx.ortho_iterate(Yg, D1w, D2w, s, out=codes, rmse_out=rmse)
    ctx.check()
    D1g, D2g = _device_dict(Qs[0], dev), _device_dict(Qs[1], dev)
    ms, traj = [], []
    for _ in range(20):
        a, b = _events()
        a.record()
        ctx.ortho_iterate(Yg, D1g, D2g, s, out=codes, rmse_out=rmse)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
        traj.append(round(rmse[1].item(), 5))
    ctx.profile_collect()
    ctx.profile(True)
    ctx.ortho_iterate(Yg, D1w, D2w, s, out=codes, rmse_out=rmse)
    ctx.profile(False)
    prof = {k: v for k, v in ctx.profile_collect().items() if v[1] > 0}
    split = {k: round(v[0], 4) for k, v in prof.items()}
    ctx.check()
    peak, _ = sdl.fp32_fma_peak(packed=True)
    roof = alu_roofline("ortho_code (thresholded coding, 12x12, both sides)",
                        N * flops_ortho_pass(p, p, s), prof["ortho_code"][0] / prof["ortho_code"][1],
                        peak, PEAK_BASIS)
    # general variant, same patches, same number of iterations (context)
    D1a, D2a = _device_dict(D1g_init, dev), _device_dict(D2g_init, dev)
    gen = []
    for _ in range(20):
        ctx.iterate(Yg, D1a, D2a, s, out=codes, rmse_out=rmse)
        gen.append(round(rmse[1].item(), 5))
    ctx.check()
    ctx.close()
    med = statistics.median(ms)
    print(json.dumps({"study": "ortho", "workload": "200000 12x12 patches, orthonormal D 12x12, "
                      "s=6, 20 iterations", "ms_per_iteration": med,
                      "signals_per_s": N / (med / 1e3), "rmse_trajectory": traj,
                      "kernel_ms_one_iteration": split, "roofline": roof,
                      "general_variant_rmse_trajectory_D12x24": gen}), flush=True)
    return 0


def study_nsweep(args):
    """Signals/s per Algorithm-1 iteration against N on the c2 shapes (12x12
    patches of the 64 seeded images, D 12x24, s = 6): the batched path (graph
    replay, autotuned) and per-call sdl_iterate (tuned tiling), L2 flushed
    before every timed iteration, median of steps.  The patches of each N are
    the first N of one seeded stream (chunks of 250 000)."""
    import torch

    from paper_2007_03800_gb300 import sdl, synth
    dev = torch.device("cuda:0")
    p1, p2, n1, n2, s = W["p1"], W["p2"], W["n1"], W["n2"], W["s"]
    imgs = np.stack([synth.synthetic_image(W["image_seed"] + i) for i in range(W["n_images"])])
    sizes = [4096, 16384, 65536, 200_000, 1_000_000, 2_000_000]
    chunks, have = [], 0
    while have < sizes[-1]:
        n = min(250_000, sizes[-1] - have)
        chunks.append(synth.random_patches(imgs, n, p1, seed=W["patch_seed"] + 1000 * len(chunks))
                      .astype(np.float32))
        have += n
    Yall = np.concatenate(chunks)
    D1, D2 = synth.init_dictionaries(p1, p2, n1, n2, seed=W["dict_seed"])
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = sdl.Context(0)
    ctx.reserve(p1, p2, n1, n2, s)
    rows = []
    for N in sizes:
        Yg = sdl.signals(torch.from_numpy(Yall[:N]).to(dev))
        D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device=dev))
        D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device=dev))
        codes = sdl.Codes.empty(N, s, dev)
        rmse = torch.zeros(2, dtype=torch.float64, device=dev)
        tiling, _ = ctx.tune_tiling(Yg, D1g, D2g, s)

        def timed(fn):
            ms = []
            for k in range(max(args.steps, 1)):
                flush.fill_(float(k))
                a, b = _events()
                a.record()
                fn()
                b.record()
                b.synchronize()
                ms.append(a.elapsed_time(b))
            return statistics.median(ms)

        for _ in range(args.warmup):
            ctx.iterate(Yg, D1g, D2g, s, out=codes, rmse_out=rmse)
        ms_plain = timed(lambda: ctx.iterate(Yg, D1g, D2g, s, out=codes, rmse_out=rmse))
        batch = sdl.Batch(ctx, [dict(Y=Yg, D1=D1g, D2=D2g, s=s, codes=codes)], autotune=True,
                          graph=True)
        for _ in range(args.warmup):
            batch.iterate(rmse_out=rmse)
        ms_batch = timed(lambda: batch.iterate(rmse_out=rmse))
        batch.close()
        ctx.check()
        rows.append({"N": N, "ms_batched": round(ms_batch, 4), "signals_per_s_batched": N / (ms_batch / 1e3),
                     "ms_per_call": round(ms_plain, 4), "signals_per_s_per_call": N / (ms_plain / 1e3),
                     "per_call_tiling": tiling})
        del Yg, codes
    ctx.close()
    print(json.dumps({"study": "nsweep", "workload": "12x12 patches of the 64 seeded images, D 12x24, s=6, "
                      "one Algorithm-1 iteration per step, L2 flushed before each", "unit": "signals/s",
                      "rows": rows}), flush=True)
    return 0


def study_gemm(args):
    """The tcgen05 BF16 GEMM on the shapes the library runs it at: the split
    correlations of the 50k hyperspectral-shaped signals (three operand pairs,
    M = 50000, N = n1 n2 = 4096, K = p1 p2 = 1024, summed in one accumulator
    by one launch as the coding pass runs it, and as three accumulating
    launches), the same with one pair (and at K = 512 and 3072: the time per
    round of tiles against K shows whether the main loop or the per-tile
    epilogue sets the pace),
    and the support network's forward GEMMs at a 65536-signal chunk; first a
    16384-row correlation GEMM (C = 268 MB, > L2), the case the kernel's
    profile is captured on.  Device time (CUDA events, median of steps) and
    the fraction of the measured BF16 peak."""
    import torch

    from paper_2007_03800_gb300 import sdl
    dev = torch.device("cuda:0")
    ctx = sdl.Context(0)
    peak = float(measured_peaks().get("bf16_tflops", 1900.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {}
    g = torch.Generator(device=dev).manual_seed(0)
    for name, (M, N, K, terms, fused) in {
            "corr_16384x4096x1024": (16384, 4096, 1024, 1, False),
            "corr_split_50000x4096x1024x3_one_launch": (50000, 4096, 1024, 3, True),
            "corr_split_50000x4096x1024x3": (50000, 4096, 1024, 3, False),
            "corr_50000x4096x1024": (50000, 4096, 1024, 1, False),
            "corr_50000x4096x512": (50000, 4096, 512, 1, False),
            "corr_50000x4096x3072": (50000, 4096, 3072, 1, False),
            "mlp_fwd1_65536x512x144": (65536, 512, 144, 1, False),
            "mlp_fwd2_65536x576x512": (65536, 576, 512, 1, False)}.items():
        A = [torch.randn(M, K, device=dev, generator=g).to(torch.bfloat16) for _ in range(terms)]
        B = [torch.randn(N, K, device=dev, generator=g).to(torch.bfloat16) for _ in range(terms)]
        C = torch.empty(M, N, device=dev)

        def run():
            if fused:
                sdl.gemm_bf16_terms(ctx, A, B, C=C)
                return
            sdl.gemm_bf16(ctx, A[0], B[0], C=C)
            for t in range(1, terms):
                sdl.gemm_bf16(ctx, A[t], B[t], C=C, accumulate=True)

        for _ in range(args.warmup):
            run()
        ms = []
        for _ in range(max(args.steps, 1)):
            a, b = _events()
            a.record()
            run()
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        med = statistics.median(ms)
        tf = 2.0 * M * N * K * terms / (med / 1e3) / 1e12
        # time per round of output tiles (one tile per SM; the launcher's
        # 128 x 256 tiles when N is a multiple of 256 and they fill the SMs)
        mb = -(-M // 128)
        bn = 256 if N % 256 == 0 and mb * (N // 256) >= sms else 128
        rounds = -(-(mb * -(-N // bn)) // sms)
        out[name] = {"ms": med, "tflops": tf, "frac_of_measured_bf16": tf / peak,
                     "launches": 1 if fused else terms,
                     "us_per_tile_round": med * 1e3 / rounds / (1 if fused else terms)}
        del A, B, C
    ctx.check()
    ctx.close()
    print(json.dumps({"study": "gemm", "peak_bf16_tflops_measured": peak, "shapes": out}),
          flush=True)
    return 0


def study_densegram(args):
    """The partial sums of a dictionary update formed densely on tensor cores
    against the fused sparse epilogue of the coding pass, at c2 (200000 12x12
    patches, D 12x24, s = 6; D1 side: P = sum T T^T, B1 = sum Y T^T with
    T_k = X_k D2^T) and c3 (50000 16x64 signals, D1 16x32, D2 64x128, s = 10;
    D2 side: M = sum Z^T Z, B2 = sum Y^T Z with Z_k = D1 X_k).  Fused: the
    coding pass with partial sums minus the same pass without them (CUDA
    events, per-kernel trace).  Dense: T (or Z) materialised in BF16 from the
    codes, then the two products as BF16 GEMMs with FP32 accumulation
    (cuBLAS through torch.matmul, which splits the long K = N p dimension);
    times of both parts, and the HBM floor of writing and reading T once."""
    import torch

    from paper_2007_03800_gb300 import sdl, synth
    dev = torch.device("cuda:0")
    ctx = sdl.Context(0)
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    out = {}

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(reps):
            a, b = _events()
            a.record()
            fn()
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    for name in ("c2", "c3"):
        if name == "c2":
            Y, D1, D2 = make_inputs()
            p1, p2, n1, n2, s, side = 12, 12, 24, 24, 6, 1
        else:
            Y = synth.hyperspectral(50_000, seed=31)
            D1, D2 = synth.init_dictionaries(16, 64, 32, 128, seed=1)
            p1, p2, n1, n2, s, side = 16, 64, 32, 128, 10, 2
        N = Y.shape[0]
        Yg = sdl.signals(torch.tensor(Y, dtype=torch.float32, device=dev))
        D1g, D2g = _device_dict(D1, dev), _device_dict(D2, dev)
        codes = ctx.sparse_code(Yg, D1g, D2g, s)
        ctx.check()
        # fused: per-kernel trace of one iteration (both passes) and of a code-only pass
        kind = "code_D1" if side == 1 else "code_D2"
        it_ms, co_ms = [], []
        for _ in range(max(args.steps, 3)):
            D1w, D2w = _device_dict(D1, dev), _device_dict(D2, dev)
            ctx.profile_collect()
            ctx.profile(True)
            ctx.iterate(Yg, D1w, D2w, s)
            ctx.sparse_code(Yg, D1g, D2g, s, out=codes)
            ctx.profile(False)
            pr = ctx.profile_collect()
            it_ms.append(pr[kind][0] / pr[kind][1])
            co_ms.append(pr["code"][0] / pr["code"][1])
        ctx.status()
        fused = statistics.median(it_ms) - statistics.median(co_ms)
        # dense: materialise T_k = X_k D2^T (n1 x p2) or Z_k = D1 X_k (p1 x n2) in BF16
        sup = codes.support.long()
        valid = sup >= 0
        q = torch.where(valid, sup, torch.zeros_like(sup))
        x = torch.where(valid, codes.coef, torch.zeros_like(codes.coef))
        ii, jj = q % n1, q // n1
        Yf = Yg.float()

        def materialise():
            if side == 1:     # T[k, i, b] = sum_l [i_l = i] x_l D2[b, j_l]
                T = torch.zeros(N, n1, p2, device=dev, dtype=torch.float32)
                vals = x[:, :, None] * D2g.t()[jj]                     # (N, s, p2)
                T.scatter_add_(1, ii[:, :, None].expand(N, s, p2), vals)
            else:             # Z[k, a, j] = sum_l [j_l = j] x_l D1[a, i_l]
                T = torch.zeros(N, n2, p1, device=dev, dtype=torch.float32)
                vals = x[:, :, None] * D1g.t()[ii]                     # (N, s, p1)
                T.scatter_add_(1, jj[:, :, None].expand(N, s, p1), vals)
            return T.to(torch.bfloat16)

        Tm = materialise()
        if side == 1:
            Tp = Tm.permute(1, 0, 2).reshape(n1, N * p2)            # T' = [T_1 ... T_N]
            Yp = Yf.permute(1, 0, 2).reshape(p1, N * p2).to(torch.bfloat16)
        else:
            Tp = Tm.permute(1, 0, 2).reshape(n2, N * p1)            # Z'^T rows j, columns (k, a)
            Yp = Yf.permute(2, 0, 1).reshape(p2, N * p1).to(torch.bfloat16)
        Tp, Yp = Tp.contiguous(), Yp.contiguous()

        def gemms():
            Pm = Tp @ Tp.t()
            Bm = Yp @ Tp.t()
            return Pm, Bm

        ms_mat = timed(materialise, max(args.steps, 3))
        ms_gemm = timed(gemms, max(args.steps, 3))
        t_bytes = Tp.numel() * 2
        out[name] = {"fused_epilogue_ms_per_pass": fused, "pass_with_sums_ms": statistics.median(it_ms),
                     "pass_code_only_ms": statistics.median(co_ms),
                     "dense_materialise_ms": ms_mat, "dense_gemms_ms": ms_gemm,
                     "dense_total_ms": ms_mat + ms_gemm,
                     "dense_hbm_floor_ms": 2 * t_bytes / (hbm * 1e9) * 1e3,
                     "dense_gemm_flops": 2.0 * Tp.shape[0] * Tp.shape[1] * (Tp.shape[0] + Yp.shape[0]),
                     "T_bytes_bf16": t_bytes}
        del Tm, Tp, Yp, Yg
    ctx.close()
    print(json.dumps({"study": "densegram", "unit": "ms", "cases": out}), flush=True)
    return 0


def study_table3(args):
    """The denoising protocol of Table III on synthetic stand-ins for its five
    512x512 test images: sigma in {5, 10, 20, 30, 50}, one noise realisation
    per case, 8x8 patches; general dictionaries 8x16 and orthonormal 8x8
    learned on 4000 noisy patches with s = 6 (50 iterations), error-driven
    coding of all 255 025 patches (eps = 1.15 sigma 8, at most 4 atoms); PSNR
    and SSIM of every case and the device time of each pipeline."""
    import torch

    from paper_2007_03800_gb300 import denoise as dn
    from paper_2007_03800_gb300 import sdl, synth
    dev = torch.device("cuda:0")
    ctx = sdl.Context(0)
    rows = []
    sigmas = (5.0, 10.0, 20.0, 30.0, 50.0)
    for img_seed in range(200, 205):
        clean = synth.synthetic_image(img_seed)
        cg = torch.tensor(clean, dtype=torch.float32, device=dev)
        for sigma in sigmas:
            noisy = clean + np.random.default_rng(img_seed * 100 + int(sigma)).normal(0, sigma, clean.shape)
            ng = torch.tensor(noisy, dtype=torch.float32, device=dev)
            row = {"image_seed": img_seed, "sigma": sigma,
                   "psnr_noisy": sdl.psnr(ng, cg).item()}
            for variant in ("general", "ortho"):
                a, b = _events()
                a.record()
                r = dn.table3_case(ctx, cg, ng, sigma, variant=variant)
                b.record()
                b.synchronize()
                row[variant] = {"psnr": round(r["psnr"].item(), 3), "ssim": round(r["ssim"].item(), 4),
                                "nnz_mean": round(r["nnz_mean"].item(), 3),
                                "ms": round(a.elapsed_time(b), 2)}
            rows.append(row)
    ctx.check()
    ctx.close()
    mean = {}
    for sigma in sigmas:
        sel = [r for r in rows if r["sigma"] == sigma]
        mean[str(sigma)] = {v: {"psnr": round(float(np.mean([r[v]["psnr"] for r in sel])), 3),
                                "ssim": round(float(np.mean([r[v]["ssim"] for r in sel])), 4)}
                            for v in ("general", "ortho")}
        mean[str(sigma)]["psnr_noisy"] = round(float(np.mean([r["psnr_noisy"] for r in sel])), 3)
    print(json.dumps({"study": "table3", "workload": "5 synthetic 512x512 images x sigma "
                      "{5,10,20,30,50}, 8x8 patches, general 8x16 and orthonormal 8x8",
                      "mean_over_images": mean, "cases": rows}), flush=True)
    return 0


def study_tmod3(args):
    """Three-mode learning (Remark 3) on hyperspectral-shaped cubes: 4 x 4
    pixels x 16 bands (every 4th of 64) of the hyperspectral generator,
    N = 50000, D1, D2 4 x 8, D3 16 x 16, s = 8, 10 iterations; device time per
    iteration and the RMSE after each mode update."""
    import torch

    from paper_2007_03800_gb300 import sdl, synth
    dev = torch.device("cuda:0")
    N, s = 50_000, 8
    H = synth.hyperspectral(N, seed=31)                     # (N, 16 pixels, 64 bands)
    Y = H.reshape(N, 4, 4, 64)[..., ::4]                    # (N, 4, 4, 16)
    rng = np.random.default_rng(1)
    Ds = [synth.random_dictionary(4, 8, rng), synth.random_dictionary(4, 8, rng),
          synth.random_dictionary(16, 16, rng)]
    ctx = sdl.Context(0)
    Yg = sdl.signals3(torch.tensor(Y, dtype=torch.float32, device=dev))

    def dicts():
        return [sdl.dictionary(torch.tensor(D, dtype=torch.float32, device=dev)) for D in Ds]

    codes = sdl.Codes.empty(N, s, dev)
    rmse = torch.zeros(3, dtype=torch.float64, device=dev)
    Dw = dicts()
    for _ in range(args.warmup):
        ctx.iterate3(Yg, *Dw, s, out=codes, rmse_out=rmse)
    ctx.check()
    Dg = dicts()
    ms, traj = [], []
    for _ in range(10):
        a, b = _events()
        a.record()
        ctx.iterate3(Yg, *Dg, s, out=codes, rmse_out=rmse)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
        traj.append([round(v, 6) for v in rmse.tolist()])
    ctx.check()
    ctx.profile_collect()
    ctx.profile(True)
    ctx.iterate3(Yg, *Dw, s, out=codes, rmse_out=rmse)
    ctx.profile(False)
    prof = {k: v for k, v in ctx.profile_collect().items() if v[1] > 0}
    ctx.check()
    peak, _ = sdl.fp32_fma_peak(packed=True)
    # the three coding passes of an iteration are traced as code_D1 (mode 1) and code_D2 (2, 3)
    ms3 = sum(prof[k][0] for k in ("code_D1", "code_D2") if k in prof)
    n3 = sum(prof[k][1] for k in ("code_D1", "code_D2") if k in prof)
    roof = alu_roofline("three-mode coding pass (4x4x16 cubes, 8x8x16 triples, s=8)",
                        N * flops_pass3((4, 4, 16), (8, 8, 16), s), ms3 / max(n3, 1), peak, PEAK_BASIS)
    ctx.close()
    med = statistics.median(ms)
    print(json.dumps({"study": "tmod3", "workload": "50000 hyperspectral-shaped 4x4x16 cubes, "
                      "D 4x8, 4x8, 16x16, s=8, 10 iterations", "ms_per_iteration": med,
                      "signals_per_s": N / (med / 1e3), "rmse_after_each_update": traj,
                      "kernel_ms_one_iteration": {k: round(v[0], 4) for k, v in prof.items()},
                      "roofline": roof}),
          flush=True)
    return 0


def study_denoise(args):
    """Denoising with one batch of three patch sizes (8, 12, 16; D p x 2p;
    error-driven stop at 1.15 sigma p, s <= p/2) on a 512x512 synthetic image
    with sigma = 20 noise, 10 iterations: PSNRs and device time of the whole
    pipeline (patch extraction, batch set-up, learning, coding, averaging) and
    of each of those phases.  The timed pipelines run in a context that has
    already tuned the batch (set-up = graph capture); the first pipeline's
    set-up, with the autotuning, is reported on its own."""
    import torch

    from paper_2007_03800_gb300 import denoise as dn
    from paper_2007_03800_gb300 import sdl, synth
    dev = torch.device("cuda:0")
    sigma = 20.0
    clean = synth.synthetic_image(7)
    noisy = clean + np.random.default_rng(8).standard_normal(clean.shape) * sigma
    cg = torch.tensor(clean, dtype=torch.float32, device=dev)
    ng = torch.tensor(noisy, dtype=torch.float32, device=dev)
    ctx = sdl.Context(0)
    # the first pipeline of a context tunes the batch; later ones reuse it
    cold = dn.denoise(ctx, ng, sigma, iterations=1, clean=cg, timing=True)
    for _ in range(args.warmup - 1):
        dn.denoise(ctx, ng, sigma, iterations=1, clean=cg)
    ms, phases = [], []
    r = None
    for _ in range(max(args.steps, 1)):
        a, b = _events()
        a.record()
        r = dn.denoise(ctx, ng, sigma, iterations=10, clean=cg, timing=True)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
        phases.append(r["ms_phases"])
    ctx.check()
    n_patches = sum((512 - p + 1) ** 2 for p, _, _ in dn.DEFAULT_GROUPS)
    # the final coding pass of all patches (one launch of the multi-problem
    # coder, code only): its algorithmic FLOPs from the code sizes it produced
    peak, _ = sdl.fp32_fma_peak(packed=True)
    fl = sum(flops_pass_hist(p, p, n, n, sc, 0, h.tolist())
             for (p, n, sc), h in zip(dn.DEFAULT_GROUPS, r["nnz_hist"]))
    roof = alu_roofline("final coding pass (multi-problem coder, three patch sizes, error-driven)",
                        fl, statistics.median(p["final_code"] for p in phases), peak, PEAK_BASIS)
    res = {"psnr_noisy": sdl.psnr(ng, cg).item(), "psnr_denoised": [x.item() for x in r["psnr"]],
           "nnz_mean": [x.item() for x in r["nnz_mean"]], "rmse_final": r["rmse"][-1].tolist(),
           "ms_pipeline": statistics.median(ms), "patches": n_patches,
           "patch_iterations_per_s": 10 * n_patches / (statistics.median(ms) / 1e3),
           "ms_phases": {k: statistics.median(p[k] for p in phases) for k in phases[0]},
           "ms_setup_first_pipeline": cold["ms_phases"]["setup"],
           "ms_per_learning_iteration": statistics.median(p["iterations"] for p in phases) / 10,
           "roofline": roof, "tuning": r["tuning"],
           "tuning_log": [dict(group=t["group"], shape_id=t["shape_id"], ctas_per_sm=t["ctas_per_sm"],
                               us=round(t["cost_us"], 1)) for t in r["tuning_log"]]}
    ctx.close()
    print(json.dumps({"study": "denoise", "workload": "512x512 synthetic image, sigma=20, "
                      "all 8x8, 12x12, 16x16 patches, 10 iterations", "result": res}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tiling", type=int, default=None,
                    help="pin this coder tiling (sdl_tilings) for the per-call path instead of tuning")
    ap.add_argument("--quick", action="store_true",
                    help="timed region only: no e2e loop, CPU baseline or clock sampling "
                         "(for profiler runs; its numbers are not bench values)")
    ap.add_argument("--study", choices=["precision", "learned", "denoise", "ortho", "gemm", "table3",
                                        "tmod3", "densegram", "nsweep"],
                    help="run one extra study on its own workload instead of the bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.study:
        return {"precision": study_precision, "learned": study_learned,
                "denoise": study_denoise, "ortho": study_ortho,
                "gemm": study_gemm, "table3": study_table3, "densegram": study_densegram,
                "tmod3": study_tmod3, "nsweep": study_nsweep}[args.study](args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
