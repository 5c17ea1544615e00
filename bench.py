"""Throughput of the block-structured cumulant pipeline on GB300.

One step = one pass of the whole hot path over one synthetic dataset:
centring, the moment contraction of every order 2..d_max, the t-chunk
reduction and the cumulant correction, through the C ABI call cum_cumulants.

Default workload ("high-order"): t = 200000 samples x n = 48 variables
(Laplace marginals mixed by a seeded orthogonal matrix, float32), block side
b = 4, orders 2..6, tensor-core FP16x3 contraction.  The metric is stored
block entries x samples per second summed over the orders,
sum_d E_d * t / step time, E_d = C(nbar + d - 1, d) b^d.

Also printed on the same JSON line: the FP64 GPU path on the same data, the
roofline of the dominant kernel (order-6 contraction), per-order rates, an
end-to-end figure through host buffers, the oracle timed on the host cores,
and the paper-scale order-4 point (t = 100000 x n = 60 float64, b = 6) with
its FP64 GPU comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="high-order", t=200_000, n=48, b=4, d_max=6)
PREC_NAMES = {0: "f64", 1: "bf16x3", 2: "fp16x3", 3: "tf32x3"}
METRIC = "moment/cumulant block-entries x samples per s"
UNIT = "block-entries*samples/s"
L2_FLUSH_BYTES = 512 << 20


def entries(n, d, b):
    nbar = -(-n // b)
    return math.comb(nbar + d - 1, d) * b ** d


def total_units(t, n, b, d_max):
    return sum(entries(n, d, b) * t for d in range(2, d_max + 1))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def source_hash(*paths):
    """First 16 hex digits of the sha256 of the code of one or more source files
    (in order): `//` comments, surrounding blanks and empty lines removed, so
    comment edits keep it."""
    import hashlib
    lines = []
    for path in paths:
        for line in open(path).read().splitlines():
            code = line.split("//", 1)[0].strip()
            if code:
                lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def profile_traffic(kernel_file, workload):
    """traffic (bytes per launch) from a committed ncu summary, if it was taken on
    the current kernel source (matching hash), else None."""
    import hashlib
    summary = os.path.join(ROOT, "profiles", f"{kernel_file}_{workload}.txt")
    csrc = os.path.join(ROOT, "paper_1701_05420_gb300", "csrc")
    # the kernel's file and the PTX helpers it inlines (operand splits, waits)
    srcs = [os.path.join(csrc, f"{kernel_file}.cu"), os.path.join(csrc, "tc_ptx.cuh")]
    if not (os.path.exists(summary) and all(os.path.exists(p) for p in srcs)):
        return None
    h = source_hash(*srcs)
    text = open(summary).read()
    m_h = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if m_h and m_t and m_h.group(1) == h:
        return float(m_t.group(1))
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"cumgb_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
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
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(args, world):
    """The `config` object of both arms' JSON lines."""
    return {"workload": WORKLOAD["name"], "t": WORKLOAD["t"], "n": WORKLOAD["n"], "b": WORKLOAD["b"],
            "orders": [2, WORKLOAD["d_max"]], "precision": args.prec,
            "l2": "flushed between timed steps (512 MiB write)",
            "parallelism": ("single GPU" if world == 1 else
                            f"replicas x{world}" if getattr(args, "multi", "sharded") == "replicas" else
                            f"t-sharded x{world} (Alg. 3, NCCL all_reduce of column / residual / moment sums; "
                            f"t = {WORKLOAD['t']} rows per rank)")}


def cpu_sample_plan(X, d_max, seconds_budget=12.0, threads=None, include_special=True):
    """Sampled entries for the oracle on the host cores: a calibration run of the
    oracle on one entry of the highest order sizes each order's sample to about
    seconds_budget / (d_max - 1) seconds on `threads` cores.  Returns the
    centred FP64 data and {d: indices (count x d)}."""
    import numpy as np

    import oracle
    import synth
    threads = threads or len(os.sched_getaffinity(0))
    _, Xc = oracle.center(X.astype(np.float64))
    t, n = Xc.shape
    probe = synth.sample_indices(n, d_max, 1, seed=1, include_special=False)
    t0 = time.perf_counter()
    oracle.cumulant_entries(Xc, probe, threads=1)
    per_entry = max(time.perf_counter() - t0, 1e-4)
    per_order = seconds_budget / (d_max - 1)
    idx = {}
    for d in range(2, d_max + 1):
        cost = per_entry * (2 ** d) / (2 ** d_max)
        count = int(max(threads, min(4096, per_order * threads / cost)))
        idx[d] = synth.sample_indices(n, d, count, seed=100 + d, include_special=include_special)
    return Xc, idx


def cpu_oracle_rate(Xc, idx, threads=None):
    """The oracle (plain C, one entry at a time) on the host cores over the
    sampled entries `idx` of every order: block-entries x samples per second,
    and the oracle's values of those entries."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    threads = threads or cores
    t = Xc.shape[0]
    work, elapsed, sample, values = 0, 0.0, [], {}
    for d, ix in idx.items():
        t0 = time.perf_counter()
        values[d] = oracle.cumulant_entries(Xc, ix, threads=threads)
        elapsed += time.perf_counter() - t0
        work += len(ix) * t
        sample.append(f"{len(ix)} order-{d} entries")
    return work / elapsed, cores, threads, ", ".join(sample) + f" at t={t}", values


def entry_offsets(cum, idx, n, b):
    """Block-storage offsets of multi-indices idx (count x d): rank of the sorted
    block tuple (cum_block_rank) times b^d plus the in-block C-order offset of
    the correspondingly permuted in-block indices."""
    import numpy as np
    idx = np.asarray(idx)
    d = idx.shape[1]
    blk, inb = idx // b, idx % b
    perm = np.argsort(blk, axis=1, kind="stable")
    js = np.take_along_axis(blk, perm, axis=1)
    iis = np.take_along_axis(inb, perm, axis=1)
    w = b ** np.arange(d - 1, -1, -1)
    ranks = np.array([cum.cum_block_rank(list(map(int, j))) for j in js], dtype=np.int64)
    return ranks * b ** d + (iis * w).sum(axis=1)


N_SPECIAL = 6   # the leading multi-indices of each order's sample with few distinct variables


def error_record(got, ref, ref_moments_special):
    """Uniform entries: relF = ||got - ref|| / ||ref|| and relMax = max|got - ref| /
    max|ref|.  The leading entries with few distinct variables, where the cumulant
    is a small difference of large moment and partition terms: their error
    relative to those moments (the cancellation itself is the data's)."""
    import numpy as np
    g, r = got[N_SPECIAL:], ref[N_SPECIAL:]
    diff = g - r
    sp = got[:N_SPECIAL] - ref[:N_SPECIAL]
    return {"relF": float(np.linalg.norm(diff) / np.linalg.norm(r)),
            "relMax": float(np.abs(diff).max() / np.abs(r).max()), "entries": int(len(r)),
            "special_vs_moments": float(np.linalg.norm(sp) / np.linalg.norm(ref_moments_special)),
            "special_entries": N_SPECIAL}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import synth
    t, n, b, d_max = WORKLOAD["t"], WORKLOAD["n"], WORKLOAD["b"], WORKLOAD["d_max"]
    X = synth.high_order()
    import oracle
    oracle.build_c()
    budget = 20.0
    rates = []
    cores = len(os.sched_getaffinity(0))
    Xc, idx = cpu_sample_plan(X, d_max, seconds_budget=budget / (args.warmup + args.steps),
                              include_special=False)
    for i in range(args.warmup + args.steps):
        rate, cores, threads, sample, _ = cpu_oracle_rate(Xc, idx)
        if i >= args.warmup:
            rates.append(rate)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"per step: {sample}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_only_order(args):
    """Centring once, then the order-D contraction (cum_moment_contraction) W + K times:
    the launch sequence a profiler capture of one contraction kernel needs."""
    import torch

    import paper_1701_05420_gb300 as cum
    import synth
    prec = cum.PRECISIONS[args.prec]
    t, n, b, d = args.t or WORKLOAD["t"], WORKLOAD["n"], WORKLOAD["b"], args.only_order
    X = torch.from_numpy(synth.high_order(t=t)).cuda()
    ws = cum.workspace(t, n, d, b, prec)
    M = torch.empty(cum.num_entries(n, d, b), dtype=torch.float64, device="cuda")
    cum.cum_center(X, b, prec, None, ws)
    evs = []
    for i in range(args.warmup + args.steps):
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record()
        cum.cum_moment_contraction(d, t, n, b, prec, M, ws)
        e_.record()
        if i >= args.warmup:
            evs.append((s_, e_))
    torch.cuda.synchronize()
    ms = statistics.median(s_.elapsed_time(e_) for s_, e_ in evs)
    E = entries(n, d, b)
    print(json.dumps({"mode": "only-order", "order": d, "t": t, "n": n, "b": b, "precision": args.prec,
                      "ms": ms, "alg_tflops": 2 * E * t / (ms * 1e-3) / 1e12,
                      "status": cum.cum_device_status(ws), "plan": cum.cum_plan_info(d, t, n, b, prec)}))
    return 0


def run_batch(args):
    """The batch workload on its own JSON line (see batch_record)."""
    rec, line_extra = batch_record(args, args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": PREC_NAMES[cumprec(args)],
        "data": "synthetic (seeded Student-t(5) x U(-1,1) mix, float32, 512 datasets)",
    }
    line.update(rec)
    line.update(line_extra)
    print(json.dumps(line))
    return 0


def cumprec(args):
    import paper_1701_05420_gb300 as cum
    return cum.PRECISIONS[args.prec]


def batch_record(args, steps, warmup):
    """512 independent datasets (t log-uniform in [5000, 200000], n in {16..96},
    Student-t(5) mixed float32), orders 2..4, block side per dataset from the
    autotuner: one captured CUDA graph of cum_batch_run per step, against the
    loop of single-dataset cum_cumulants calls; every dataset's cumulants
    against the FP64 GPU path (held within 1e-10 of the oracle by the tests).
    Returns (record, keys for a stand-alone line)."""
    import numpy as np
    import torch

    import paper_1701_05420_gb300 as cum
    import synth
    from paper_1701_05420_gb300.autotune import AutoTuner
    prec = cum.PRECISIONS[args.prec]
    d_max = 4
    specs = synth.batch_specs(count=args.batch_count)
    tuner = AutoTuner(d_max, prec, cache_path=os.path.join("/tmp", "cumgb_autotune.json"))
    t_tune = time.perf_counter()
    bs = tuner.choose_all([(t, n) for (t, n, _) in specs])
    t_tune = time.perf_counter() - t_tune
    Xs = [torch.from_numpy(synth.batch_dataset(t, n, sd)).cuda() for (t, n, sd) in specs]
    C = [[torch.empty(cum.num_entries(n, d, b), dtype=torch.float64, device="cuda") for d in range(2, d_max + 1)]
         for (t, n, _), b in zip(specs, bs)]
    mean = [torch.empty(n, dtype=torch.float64, device="cuda") for (t, n, _) in specs]
    batch = cum.Batch([t for t, _, _ in specs], [n for _, n, _ in specs], bs, d_max, prec)
    ws = batch.bind(Xs, C, mean)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.run(stream=torch.cuda.current_stream())
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    evs = []
    with Clocks(0) as clk:
        for _ in range(steps):
            flush.fill_(1.0)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            e.record()
            evs.append((a, e))
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(e) for a, e in evs) / len(evs)
    status = cum.cum_device_status(ws)
    work = sum(entries(n, d, b) * t for (t, n, _), b in zip(specs, bs) for d in range(2, d_max + 1))
    # the same datasets through the single-dataset entry point, one call each
    wmax = max(cum.cum_workspace_size(t, n, d_max, b, prec) for (t, n, _), b in zip(specs, bs))
    ws1 = torch.empty(wmax, dtype=torch.uint8, device="cuda")
    for i in range(min(4, len(specs))):
        cum.cum_cumulants(Xs[i], d_max, bs[i], prec, C[i], mean[i], ws1)
    torch.cuda.synchronize()
    flush.fill_(1.0)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(len(specs)):
        cum.cum_cumulants(Xs[i], d_max, bs[i], prec, C[i], mean[i], ws1)
    e.record()
    torch.cuda.synchronize()
    ms_loop = a.elapsed_time(e)
    info = batch.info()
    # accuracy: the last replay's cumulants against the FP64 GPU path, per dataset
    worst = {"relF": 0.0, "dataset": None, "order": None}
    if prec != 0:
        g.replay()
        torch.cuda.synchronize()
        w64 = max(cum.cum_workspace_size(t, n, d_max, b, 0) for (t, n, _), b in zip(specs, bs))
        ws64 = torch.empty(w64, dtype=torch.uint8, device="cuda")
        for i, ((t, n, _), b) in enumerate(zip(specs, bs)):
            C64 = [torch.empty_like(c) for c in C[i]]
            m64 = torch.empty_like(mean[i])
            cum.cum_cumulants(Xs[i].double(), d_max, b, 0, C64, m64, ws64)
            for d in range(2, d_max + 1):
                ref = C64[d - 2]
                rel = float(torch.linalg.norm(C[i][d - 2] - ref) / torch.linalg.norm(ref))
                if not rel <= worst["relF"]:
                    worst = {"relF": rel, "dataset": i, "order": d}
        del ws64
    rec = {
        "value": work / (ms * 1e-3), "ms_per_step": round(ms, 3),
        "config": {"workload": "batch", "datasets": len(specs), "orders": [2, d_max], "precision": args.prec,
                   "t_range": [min(t for t, _, _ in specs), max(t for t, _, _ in specs)],
                   "n_values": sorted(set(n for _, n, _ in specs)), "b_chosen": {str(b): bs.count(b) for b in sorted(set(bs))},
                   "l2": "flushed between timed steps (512 MiB write)", "launch": "one CUDA graph replay per step"},
        "loop_single": {"value": work / (ms_loop * 1e-3), "ms": round(ms_loop, 3),
                        "speedup_of_batch": round(ms_loop / ms, 2)},
        "max_relF_vs_fp64_path": worst,
        "gpu_launches_per_step": info["launches"], "work_units": info["units"],
        "autotune_seconds": round(t_tune, 2), "device_status": status,
    }
    batch.close()
    return rec, {"clocks": clk.summary()}



def fp64_peak_tflops(dev, n=8192, reps=3):
    """FP64 peak of this GPU, measured: cuBLAS DGEMM n^3 (median of `reps`)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b_ = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b_)
    times = []
    for _ in range(reps):
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_.record()
        torch.matmul(a, b_)
        e_.record()
        torch.cuda.synchronize()
        times.append(s_.elapsed_time(e_))
    del a, b_
    return 2.0 * n ** 3 / (statistics.median(times) * 1e-3) / 1e12


def correction_flops(d, E, moment_form=False):
    """FP64 flops of the order-d correction as the library evaluates it: per entry
    one multiply-add per two-part partition, plus the final subtraction.  Order 6
    either sums its 15 three-pair partitions as 5 groups (a multiply and two
    multiply-adds inside, one outer multiply-add), or, in the moment form that
    cum_cumulants uses, has none: 5 of its 25 products take the order-4 moment."""
    two_part = {4: 3, 5: 10, 6: 25}[d]
    three_pair = 5 * (1 + 2 * 2 + 2) if d == 6 and not moment_form else 0
    return E * (2 * two_part + three_pair + 2)


def paper_scale_point(args, cum, prec, dev, stream, flush):
    """Order-4 cumulants of the paper-scale data (t = 100000 x n = 60 float64,
    Student-t(4) mix with 5% outlier rows, b = 6): the split path and the FP64
    GPU path, median of CUDA-event timed runs with an L2 flush before each."""
    import torch

    import synth
    t, n, b, d_max = 100_000, 60, 6, 4
    X = torch.from_numpy(synth.paper_scale()).to(dev)
    C = [torch.empty(cum.num_entries(n, d, b), dtype=torch.float64, device=dev) for d in range(2, d_max + 1)]
    mean = torch.empty(n, dtype=torch.float64, device=dev)
    out = {"workload": "paper-scale", "t": t, "n": n, "b": b, "orders": [2, d_max], "input": "float64"}
    for name, pr in (("split", prec), ("fp64", 0)):
        ws = cum.workspace(t, n, d_max, b, pr, dev)
        cum.cum_cumulants(X, d_max, b, pr, C, mean, ws, stream)
        times = []
        for _ in range(max(3, args.fp64_steps)):
            flush.fill_(1.0)
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record(stream)
            cum.cum_cumulants(X, d_max, b, pr, C, mean, ws, stream)
            e_.record(stream)
            torch.cuda.synchronize()
            times.append(s_.elapsed_time(e_))
        ms = statistics.median(times)
        out[name] = {"precision": PREC_NAMES[pr], "ms_per_step": round(ms, 4),
                     "value": total_units(t, n, b, d_max) / (ms * 1e-3),
                     "d4_alg_tflops": 2 * entries(n, 4, b) * t / (ms * 1e-3) / 1e12}
        del ws
    out["speedup_of_split_path"] = round(out["fp64"]["ms_per_step"] / out["split"]["ms_per_step"], 2)
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_1701_05420_gb300 as cum
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 or args.shard_at_1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = cum.PRECISIONS[args.prec]
    t, n, b, d_max = WORKLOAD["t"], WORKLOAD["n"], WORKLOAD["b"], WORKLOAD["d_max"]

    # N > 1: by default one dataset of N x t samples, each rank holding t rows
    # (weak scaling), through the t-sharded steps (Alg. 3) with NCCL
    # all_reduce of the column, residual and moment sums; with --multi
    # replicas each rank computes the cumulants of its own dataset
    sharded = (world > 1 or args.shard_at_1) and args.multi == "sharded"
    Xh = synth.high_order(seed=synth.BASE_SEED + 4 + rank)
    X = torch.from_numpy(Xh).to(dev)
    ws = cum.workspace(t, n, d_max, b, prec, dev)
    C = [torch.empty(cum.num_entries(n, d, b), dtype=torch.float64, device=dev) for d in range(2, d_max + 1)]
    mean = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    if sharded:
        from paper_1701_05420_gb300.sharded import LibraryOps, sharded_cumulants
        ops = LibraryOps(t, n, d_max, b, prec, dev)
        ws = ops.ws

        def allreduce(x):
            torch.distributed.all_reduce(x)

        def step():
            Cd, m = sharded_cumulants(X, t * world, d_max, allreduce, ops)
            for d in range(2, d_max + 1):
                C[d - 2] = Cd[d]
    else:
        def step():
            cum.cum_cumulants(X, d_max, b, prec, C, mean, ws, stream)

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    if cum.cum_device_status(ws, stream) != cum.CUM_OK:
        raise RuntimeError("device status reported a timeout during warm-up")

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            starts[i].record(stream)
            step()
            ends[i].record(stream)
            flush.fill_(1.0)    # L2 flush between timed steps (not timed)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    status = cum.cum_device_status(ws, stream)
    work = total_units(t, n, b, d_max)
    value = work * world / (ms * 1e-3)

    # entries of the last timed step's cumulants, sampled for the oracle check
    # (the sample is the CPU-baseline leg's: its oracle values time the host)
    do_cpu = rank == 0 and world == 1 and not args.no_cpu
    sample_gpu = None
    if do_cpu:
        Xc_cpu, idx_cpu = cpu_sample_plan(Xh, d_max)
        sample_gpu = {d: C[d - 2][torch.from_numpy(entry_offsets(cum, ix, n, b)).to(dev)].cpu().numpy()
                      for d, ix in idx_cpu.items()}

    # launches per step, from the library's own plan
    launches = cum.cum_plan_info(2, t, n, b, prec)["center_launches"]
    for d in range(2, d_max + 1):
        info = cum.cum_plan_info(d, t, n, b, prec)
        launches += info["moment_launches"] + (1 if d >= 4 else 0)
        if sharded and d == 6 and info["moment_launches"] > 2 + (info["splits"] > 1):
            # cum_moment_sums also contracts order 5 for the order-6 correction
            i5 = cum.cum_plan_info(5, t, n, b, prec)
            launches += 2 + (1 if i5["splits"] > 1 else 0)

    # per-order contraction rates and the dominant kernel (order-6 contraction) roofline
    orders = {}
    Mtmp = torch.empty(cum.num_entries(n, d_max, b), dtype=torch.float64, device=dev)
    cum.cum_center(X, b, prec, None, ws, stream)
    for d in range(2, d_max + 1):
        reps = 3
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        cum.cum_moment_contraction(d, t, n, b, prec, Mtmp, ws, stream)
        for s_, e_ in evs:
            flush.fill_(1.0)
            s_.record(stream)
            cum.cum_moment_contraction(d, t, n, b, prec, Mtmp, ws, stream)
            e_.record(stream)
        torch.cuda.synchronize()
        dms = statistics.median(s_.elapsed_time(e_) for s_, e_ in evs)
        E = entries(n, d, b)
        orders[str(d)] = {"ms": round(dms, 4), "rate": E * t / (dms * 1e-3),
                          "alg_tflops": 2 * E * t / (dms * 1e-3) / 1e12}
    # the order-d_max correction alone, on the cumulants of the last step
    corr = None
    if d_max >= 4:
        low = [C[k - 2] for k in range(2, d_max - 1)]
        Ctmp = torch.empty_like(C[d_max - 2])
        moment_form = d_max == 6   # the form cum_cumulants uses at order 6
        if moment_form:
            M4 = torch.empty(cum.num_entries(n, 4, b), dtype=torch.float64, device=dev)
            cum.cum_moment_blocks(4, t, n, b, prec, M4, ws, stream)

        def correct():   # Mtmp holds the order-d_max moments of the loop above
            if moment_form:
                cum.cum_correct_m4(n, b, Mtmp, low, M4, Ctmp, stream)
            else:
                cum.cum_correct(d_max, n, b, Mtmp, low, Ctmp, stream)
        correct()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        for s_, e_ in evs:
            flush.fill_(1.0)
            s_.record(stream)
            correct()
            e_.record(stream)
        torch.cuda.synchronize()
        cms = statistics.median(s_.elapsed_time(e_) for s_, e_ in evs)
        corr = {"kernel": f"correct_staged_kernel order {d_max}" + (" (moment form)" if moment_form else ""),
                "ms": round(cms, 4),
                "fp64_tflops": correction_flops(d_max, entries(n, d_max, b), moment_form) / (cms * 1e-3) / 1e12}
        del Ctmp
    pk, pk_kind = peaks()
    dom = orders[str(d_max)]
    E6 = entries(n, d_max, b)
    split_products = 4 if prec in (1, 2, 3) else 1
    if prec == 0:
        roof = {"bound": "alu", "achieved": 2 * E6 * t / (dom["ms"] * 1e-3) / 1e12, "peak": None,
                "unit": "TFLOP/s", "frac": None, "traffic": None,
                "note": "FP64 CUDA-core path; peak not measured"}
    else:
        bf16 = pk.get("bf16_tflops", 1900.0)
        peak = bf16   # every split precision runs fp16 or bf16 parts here (fp16 = bf16 rate)
        # achieved / frac: the method's work, 2 E_6 t flops per launch (one
        # multiply-add per stored entry per sample); the split executes three
        # products of that size on the tensor pipe, reported beside it
        achieved = 2 * E6 * t / (dom["ms"] * 1e-3) / 1e12
        kfile = "moment_pair"
        roof = {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": profile_traffic(kfile, WORKLOAD["name"]),
                "peak_kind": f"{pk_kind} bf16 burst" + (" (fp16 = bf16 rate)" if prec in (2, 3) else ""),
                "frac_basis": "method's work: 2 E_6 t flops per launch",
                "kernel": f"moment_pair_kernel order {d_max} (cum_moment_contraction)",
                "flops_per_launch": 2 * E6 * t,
                "split_products": {"achieved": round(split_products * achieved, 2),
                                   "frac": round(split_products * achieved / peak, 4),
                                   "flops_per_launch": split_products * 2 * E6 * t,
                                   "basis": "tensor-pipe work: lo*lo + hi*lo + lo*hi + hi*hi"}}

    # FP64 GPU path on the same data (the comparison of the metric)
    fp64 = None
    if args.fp64_steps > 0 and prec != 0 and world == 1:
        ws64 = cum.workspace(t, n, d_max, b, 0, dev)
        X64 = X.double()
        cum.cum_cumulants(X64, d_max, b, 0, C, mean, ws64, stream)
        torch.cuda.synchronize()
        s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(args.fp64_steps):
            flush.fill_(1.0)
            s_.record(stream)
            cum.cum_cumulants(X64, d_max, b, 0, C, mean, ws64, stream)
            e_.record(stream)
            torch.cuda.synchronize()
            tot += s_.elapsed_time(e_)
        ms64 = tot / args.fp64_steps
        fp64 = {"value": work / (ms64 * 1e-3), "ms_per_step": round(ms64, 3),
                "speedup_of_tensor_path": round(ms64 / ms, 2)}
        del ws64, X64
        # FP64 roofline of that path: its contraction flops per step against a
        # measured FP64 peak (cuBLAS DGEMM in this run)
        peak64 = fp64_peak_tflops(dev)
        flops64 = sum(2 * entries(n, d, b) * t for d in range(2, d_max + 1))
        fp64["roofline"] = {"bound": "fp64", "achieved": round(flops64 / (ms64 * 1e-3) / 1e12, 4),
                            "peak": round(peak64, 4), "unit": "TFLOP/s",
                            "frac": round(flops64 / (ms64 * 1e-3) / 1e12 / peak64, 4),
                            "peak_kind": "cuBLAS DGEMM 8192^3 measured in this run",
                            "flops_per_step": flops64}
        if corr is not None:
            corr["fp64_peak_tflops"] = round(peak64, 4)
            corr["frac"] = round(corr["fp64_tflops"] / peak64, 4)

    paper = paper_scale_point(args, cum, prec, dev, stream, flush) if args.fp64_steps > 0 and world == 1 else None

    # end to end through host buffers: pinned host X -> device, cumulants, all C_d -> pinned host
    Xpin = torch.from_numpy(Xh).pin_memory()
    Cpin = [torch.empty(c.numel(), dtype=torch.float64).pin_memory() for c in C]
    Xd = torch.empty_like(X)
    h2d = Xpin.numel() * Xpin.element_size()
    d2h = sum(c.numel() * 8 for c in C)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xd.copy_(Xpin, non_blocking=True)
        if sharded:
            Cd, _ = sharded_cumulants(Xd, t * world, d_max, allreduce, ops)
            C = [Cd[d] for d in range(2, d_max + 1)]
        else:
            cum.cum_cumulants(Xd, d_max, b, prec, C, mean, ws, stream)
        for hc, dc in zip(Cpin, C):
            hc.copy_(dc, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_val = work * world / (statistics.mean(e2e_ms) * 1e-3)

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch, _ = batch_record(args, 3, 3)

    cpu, errors = None, None
    if do_cpu:
        rate, cores, threads, sample, ref = cpu_oracle_rate(Xc_cpu, idx_cpu)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample}
        import oracle
        refm = {d: oracle.moment_entries(Xc_cpu, idx_cpu[d][:N_SPECIAL]) for d in ref}
        errors = {str(d): error_record(sample_gpu[d], ref[d], refm[d]) for d in ref}
        errors["against"] = "oracle (Eq. cumfmom, FP64) on the cpu_baseline sample of the last timed step's output"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": PREC_NAMES[prec] if prec else "f64",
            "data": "synthetic (seeded Laplace x orthogonal mix, float32)",
            "config": workload_config(args, world),
            "roofline": roof, "cpu_baseline": cpu, "errors": errors,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": round(statistics.mean(e2e_ms), 3)},
            "gpu_launches": launches * args.steps, "gpu_launches_per_step": launches,
            "clocks": clk.summary(), "orders": orders, "correction": corr, "fp64_gpu": fp64,
            "paper_scale_d4": paper, "batch": batch,
            "device_status": status,
        }
        print(json.dumps(line))
    if torch.distributed.is_initialized():
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp16x3", choices=["fp64", "bf16x3", "fp16x3", "tf32x3"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--t", type=int, default=0, help="samples (default: the workload's 200000)")
    ap.add_argument("--only-order", type=int, default=0,
                    help="time only the contraction of this order (profiling mode)")
    ap.add_argument("--workload", default="high-order", choices=["high-order", "batch"])
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--no-batch", action="store_true", help="skip the batch sub-object of the N = 1 line")
    ap.add_argument("--shard-at-1", action="store_true",
                    help="run the t-sharded steps (NCCL) even at N = 1, a check of the multi-GPU path on one GPU")
    ap.add_argument("--multi", default="sharded", choices=["sharded", "replicas"],
                    help="N > 1: one dataset sharded over ranks (Alg. 3, NCCL) or independent replicas")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only_order:
        return run_only_order(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.t:
        WORKLOAD["t"] = args.t
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
