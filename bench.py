#!/usr/bin/env python3
"""Benchmark of the non-negative tensor-train hot path on one GB300.

Workload (one "step" = one job): the 6-way 32^6 FP32 tensor (1.07e9 entries,
4.3 GB) built from random non-negative TT cores U[0,1) with ranks
(1,8,16,16,16,8,1) plus 1% |Gaussian| noise; a job is the whole nTT
(Algorithm 2: five NMFs of 200 multiplicative-update iterations each, hand-off
normalisation, FP64 stage objectives) followed by the relative error of
Eq. (3).  Inputs are synthetic and seeded; the tensor is larger than L2, so
no flush is needed between steps.

  value      NTT jobs/s with A resident in HBM (CUDA events on the stream)
  e2e        the same through the host-buffer C-ABI call (A host->device,
             cores and error device->host inside the timed region)
  roofline   the dominant kernel: the fused MU pass of stage 1
             (32 x 33,554,432, r = 8), algorithmic bytes m n 4 + 8 r n per
             iteration over the measured iteration time, against the
             measured HBM copy bandwidth
  cpu_baseline  the FP64 oracle on the host cores on a bounded sample of the
             same job, extrapolated to jobs/s

Multi-GPU (torchrun): every rank runs its own independent job (the jobs
share nothing), value = all ranks' jobs / max time over ranks.
`--impl reference` times the FP64 oracle instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NMF-MU iterations/sec and HBM GB/s (% roofline) per NTT; NTT jobs/sec, p50/p99"
UNIT = "NTT jobs/s"
WORKLOAD = "c2_32x6"
FP32_FMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: SMs x FP32 lanes x 2 flop x max SM clock

# DRAM traffic of one launch of the dominant kernel from an ncu capture, valid
# only for the engine and kernel source it was measured on (hash of that file).
NCU_TRAFFIC = {"engine": "tc_narrow", "kernel_file": "mu_pass_tcw.cu", "kernel_sha": "8f9c365ea42af363",
               "bytes_per_launch": 6.304e9}   # 788.0 MB on 32 x 4194304, x 8 for 33554432 columns


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _kernel_sha(fname):
    p = os.path.join(ROOT, "paper_2008_01340_gb300", "csrc", fname)
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def max_over_ranks(ms, dist, device):
    """Slowest rank's time: every rank ran the same number of independent jobs."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, ms):
    """Jobs per second of the whole job: `world` ranks each finished one job per `ms`."""
    return world * 1e3 / ms


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=f, stderr=subprocess.DEVNULL)
            self._f = f
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = max(smax, float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the job
# ---------------------------------------------------------------------------

def cpu_model():
    """CPU model of this host (lscpu's model name, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(A, cfg, budget_s=15.0):
    """Time the oracle's MU iterations on column samples of every stage's
    unfolding (about budget_s seconds in total) and extrapolate the whole job
    (iterations x columns)."""
    import numpy as np
    import oracle
    import synth

    dims, ranks, iters = cfg["dims"], cfg["ranks"], cfg["iters"]
    shapes = synth.stage_shapes(dims, ranks)
    per_stage = budget_s / len(shapes)
    total_s = 0.0
    desc = []
    spent = 0.0
    for s, (m, n, r) in enumerate(shapes):
        cols = min(n, max(1024, (1 << 25) // m))        # ~33M entries per sample
        if s == 0:
            X = np.ascontiguousarray(A.reshape(m, n)[:, :cols], dtype=np.float64)
            src = "tensor columns"
        else:
            X = synth.uniform_matrix((m, cols), 900 + s).astype(np.float64)
            src = "U[0,1) stand-in of H_{k-1}; the cost does not depend on the values"
        W0 = synth.uniform_matrix((m, r), 800 + s).astype(np.float64)
        H0 = synth.uniform_matrix((r, cols), 700 + s).astype(np.float64)
        k = 0
        t0 = time.perf_counter()
        W, H = W0, H0
        while True:
            W, H, _ = oracle.nmf_mu(X, W, H, 1)
            k += 1
            el = time.perf_counter() - t0
            if k >= 2 and (el >= per_stage or k >= 50):
                break
        dt = el / k
        spent += el
        total_s += dt * iters * (n / cols)
        desc.append(f"stage {s+1}: {k} iters on {m}x{cols} of {m}x{n} ({src})")
    cores = os.cpu_count() or 1
    return {"value": 1.0 / total_s, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "; ".join(desc) + f"; extrapolated to {iters} iters x all columns per stage "
                      f"(extrapolated job time {total_s:.1f} s; iterations per stage sample until the "
                      f"stage's share of a {budget_s:.0f} s budget or 50 are spent)",
            "seconds_spent": round(spent, 2)}


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import synth
    cfg = synth.CONFIGS[WORKLOAD]
    A, _ = synth.tt_tensor(cfg["dims"], cfg["ranks"], cfg["core_dist"], cfg["noise"],
                           cfg["data_seed"])
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(A, cfg, budget_s=10.0)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "note": "FP64 numpy oracle on host cores"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                         "cpu_model": cb["cpu_model"], "sample": cb["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_stage1_small(args):
    """Stage-1 MU iterations (32 x 4194304, r = 8, FP32) through nmf_mu_step
    (the single-problem pass) or, with --engine group, nmf_mu_many (the grouped
    engine), for profiler captures."""
    import torch

    import synth
    import paper_2008_01340_gb300 as ntt
    from paper_2008_01340_gb300 import _build

    _build.build()
    route = "auto"
    if args.case == "tcn_small":
        # stage-1 shape of the 32^6 job at 2^22 columns (FP32 X): the stacked split tensor-core form
        m, n, r = 32, 1 << 22, 8
        X = torch.from_numpy(synth.uniform_matrix((m, n), 1)).cuda()
        route = "tc"
    elif args.case == "tcs_small":
        # stage-2 shape of the 32^6 job at 2^21 columns (FP32 X): the split tensor-core form
        m, n, r = 256, 1 << 21, 16
        X = torch.from_numpy(synth.uniform_matrix((m, n), 1)).cuda()
        route = "tc"
    elif args.case == "tcb_small":
        # stage-2 shape of the precision form on BF16 X: the tensor-core pass
        m, n, r = 256, 1 << 21, 32
        X = torch.from_numpy(synth.uniform_matrix((m, n), 1)).to(torch.bfloat16).cuda()
    elif args.case == "stage3":
        # stage 3 of the 32^6 job (512 x 32768, r = 16): pass and combine both matter
        m, n, r = 512, 1 << 15, 16
        X = torch.from_numpy(synth.uniform_matrix((m, n), 1)).cuda()
    else:
        m, n, r = 32, 1 << 22, 8
        X = torch.from_numpy(synth.uniform_matrix((m, n), 1)).cuda()
    W = torch.from_numpy(synth.uniform_matrix((m, r), 2)).cuda()
    H = torch.from_numpy(synth.uniform_matrix((r, n), 3)).cuda()
    if args.engine == "group":
        ws = ntt.empty_workspace(ntt.nmf_mu_many_workspace_size([(m, n, r)]))
        run = lambda k: ntt.nmf_mu_many([X], [W], [H], k, workspace=ws)
    else:
        ws = ntt.empty_workspace(ntt.nmf_mu_workspace_size(m, n, r, "bf16" if X.dtype == torch.bfloat16 else "f32",
                                                           route))
        obj = torch.zeros(max(args.steps, args.warmup, 1), dtype=torch.float64, device="cuda")
        run = lambda k: ntt.nmf_mu_step(X, W, H, k, 1e-12, obj, workspace=ws, route=route)
    for _ in range(args.warmup):
        run(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run(args.steps)
    e1.record()
    torch.cuda.synchronize()
    it = e0.elapsed_time(e1) / args.steps / 1e3
    gb = (m * n * X.element_size() + 8 * r * n) / it / 1e9
    print(json.dumps({"case": args.case, "engine": args.engine, "m": m, "n": n, "r": r, "ms_per_iter": it * 1e3,
                      "alg_GBps": round(gb, 1)}), flush=True)
    return 0


def run_stream(args):
    """Out-of-core form: a 256 x 16,777,216 FP32 X (16 GB, a column-scaled
    stage 1 of the paper's large synthetic with its first TT rank 20) in pinned
    host memory, streamed in chunks of 2^20 columns (two 1 GB device buffers)
    every MU iteration.  Reported against the pinned host-to-device copy rate
    measured in the same run (1 GB copies, best of 5)."""
    import torch

    import synth
    import paper_2008_01340_gb300 as ntt
    from paper_2008_01340_gb300 import _build

    _build.build()
    m, n, r, chunk = 256, 1 << 24, 20, 1 << 20
    X = torch.empty((m, n), dtype=torch.float32).pin_memory()
    g = torch.Generator()
    g.manual_seed(6)
    for c0 in range(0, n, 1 << 22):       # U[0,1) fill in slices
        X[:, c0:c0 + (1 << 22)] = torch.rand((m, 1 << 22), generator=g)
    W = torch.from_numpy(synth.uniform_matrix((m, r), 2)).cuda()
    H = torch.from_numpy(synth.uniform_matrix((r, n), 3)).cuda()
    # link rate: pinned host -> device copies of 1 GB
    src = X.view(-1)[: 1 << 28]
    dst = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, (1 << 30) / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del dst
    ws = None
    for _ in range(args.warmup):
        ws = ntt.nmf_mu_step_host(X, W, H, 1, chunk, workspace=ws)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ntt.nmf_mu_step_host(X, W, H, args.steps, chunk, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    it = e0.elapsed_time(e1) / 1e3 / args.steps
    gbs = m * n * 4 / it / 1e9
    line = {
        "metric": METRIC, "value": round(1.0 / it, 3), "unit": "MU iterations/s (X streamed from host memory)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(it * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"out_of_core: {m} x {n} FP32 X (16 GB) in pinned host memory, r = {r}, "
                               f"chunks of {chunk} columns", "chunk_cols": chunk},
        "roofline": {"bound": "host link", "achieved": round(gbs, 1), "peak": round(best, 1), "unit": "GB/s",
                     "frac": round(gbs / best, 4), "traffic": None,
                     "peak_source": "pinned host-to-device copy of 1 GB measured in this run (best of 5)"},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """Batched form: 512 instances x 8 restarts per stage x 300 iterations per step."""
    import numpy as np
    import torch

    import synth
    import paper_2008_01340_gb300 as ntt
    from paper_2008_01340_gb300 import _build

    _build.build()
    inst = synth.batched_instances(512)
    iters = args.batch_iters or 300
    if args.batch_top:
        # profiling subset: the largest instances only
        order = np.argsort([-int(np.prod(i["dims"])) for i in inst], kind="stable")
        inst = [inst[k] for k in order[:args.batch_top]]
    b = ntt.ntt_batch_create([(i["dims"], i["ranks"]) for i in inst], iters, 8, 1e-12, 4)
    A = torch.empty(b.input_floats, dtype=torch.float32).pin_memory()
    An = A.numpy()
    for k, it in enumerate(inst):
        size = int(np.prod(it["dims"]))
        synth.tt_tensor(it["dims"], it["ranks"], "uniform", 0.01, it["data_seed"],
                        out=An[b.input_off[k]:b.input_off[k] + size])
    Ad = A.cuda()
    cores = torch.zeros(b.core_floats, dtype=torch.float32, device="cuda")
    ws = ntt.empty_workspace(b.workspace_bytes)
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        ntt.ntt_decompose_batched(b, Ad, cores, ws, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ntt.ntt_decompose_batched(b, Ad, cores, ws, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # relative error (Eq. 3) of every instance from its cores
    views = b.core_views(cores)
    errs = []
    for k, it in enumerate(inst):
        size = int(np.prod(it["dims"]))
        err = torch.zeros(3, dtype=torch.float64, device="cuda")
        ntt.ntt_rel_error(it["dims"], it["ranks"], [c.contiguous() for c in views[k]],
                          Ad[b.input_off[k]:b.input_off[k] + size], err)
        errs.append(err[0].item())
    line = {
        "metric": METRIC, "value": round(len(inst) * 1e3 / ms, 3), "unit": "NTT instances/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": (f"c4_batched: {len(inst)} nTTs, d~U{{3..6}}, n_k~U{{8..24}}, r_k~U{{2..12}} "
                                f"clamped, U[0,1) cores + 1% noise, 8 restarts/stage, {iters} MU iterations")
                   + (" (profiling subset: largest instances)" if args.batch_top else ""),
                   "input_entries": b.input_floats},
        "rel_error": {"median": float(np.median(errs)), "max": float(np.max(errs))},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Serving form: 1000 Poisson requests (d 4-7, 1e4-1e8 entries, ranks 4-32,
    FP32 or BF16), 100 MU iterations per stage, ticks of 10.  First the
    closed-loop saturation throughput (all requests submitted at once), then an
    open loop at 0.8x that rate with p50/p99 latency from submit to result on
    the host.  Inputs come from pinned host memory; results land in pinned host
    memory: the timed region is host to host."""
    import threading

    import numpy as np
    import torch

    import synth
    import paper_2008_01340_gb300 as ntt
    from paper_2008_01340_gb300 import _build

    _build.build()
    reqs = synth.serving_requests(args.requests)
    # host pools the jobs slice their inputs from (U[0,1) values; the data do
    # not change the work): FP32 and its BF16 rounding, both pinned
    pool_n = 1 << 28
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    pool_dev = torch.rand(pool_n, device="cuda", generator=g)
    pool32 = torch.empty(pool_n, dtype=torch.float32, pin_memory=True)
    pool32.copy_(pool_dev)
    pool16 = torch.empty(pool_n, dtype=torch.bfloat16, pin_memory=True)
    pool16.copy_(pool_dev.to(torch.bfloat16))
    del pool_dev
    torch.cuda.empty_cache()

    def job_input(i, q):
        size = int(np.prod(q["dims"]))
        off = (i * 7919 * 1024) % (pool_n - size) // 64 * 64
        pool = pool16 if q["x_dtype"] == "bf16" else pool32
        return pool[off:off + size]

    budget = int(args.serve_budget_gb * (1 << 30))
    h2d = sum(int(np.prod(q["dims"])) * (2 if q["x_dtype"] == "bf16" else 4) for q in reqs)

    def one_run(arrivals):
        srv = ntt.Server(budget, max_jobs=args.serve_slots, tick_iters=10, stage_iters=100)
        handles = [None] * len(reqs)
        t0 = time.perf_counter()
        if arrivals is None:
            for i, q in enumerate(reqs):
                handles[i] = srv.submit(job_input(i, q), q["dims"], q["ranks"], seed=q["data_seed"])
        else:
            def submitter():
                for i, q in enumerate(reqs):
                    dt = arrivals[i] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                    handles[i] = srv.submit(job_input(i, q), q["dims"], q["ranks"], seed=q["data_seed"])
            th = threading.Thread(target=submitter)
            th.start()
            th.join()
        infos = [srv.wait(h, timeout=3600) for h in handles]
        wall = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        lat = np.array([i["t_done"] - i["t_submit"] for i in infos])
        first = min(i["t_submit"] for i in infos)
        last = max(i["t_done"] for i in infos)
        return {"jobs": len(infos), "makespan_s": last - first, "wall_s": wall,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "ticks": stats["ticks"], "peak_gb": stats["peak_bytes"] / 2**30, "busy_s": stats["busy_s"]}

    sampler = ClockSampler(0)
    sampler.start()
    closed = one_run(None)
    x_sat = closed["jobs"] / closed["makespan_s"]
    base_arr = np.array([q["arrival"] for q in reqs])      # rate-1 Poisson arrival times
    lam = 0.8 * x_sat
    opened = one_run(base_arr / lam)
    sweep = {}
    if args.serve_sweep:
        for f in (0.25, 0.5, 0.95):
            r = one_run(base_arr / (f * x_sat))
            sweep[str(f)] = {"p50_s": r["p50_s"], "p99_s": r["p99_s"]}
    clocks = sampler.stop()
    line = {
        "metric": METRIC, "value": round(x_sat, 3), "unit": "NTT jobs/s (closed loop, host to host)",
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": round(closed["makespan_s"] * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"c5_serving: {len(reqs)} Poisson requests, d~U{{4..7}}, size~logU[1e4,1e8], "
                               "r~U{4..32} clamped, FP32/BF16 p=1/2, 100 MU iterations per stage, ticks of 10",
                   "budget_gb": args.serve_budget_gb, "slots": args.serve_slots},
        "latency": {"lambda_jobs_s": round(lam, 3), "p50_s": round(opened["p50_s"], 4),
                    "p99_s": round(opened["p99_s"], 4),
                    "throughput_jobs_s": round(opened["jobs"] / opened["makespan_s"], 3), "sweep": sweep},
        "closed_loop": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in closed.items()},
        "e2e": {"value": round(x_sat, 3), "unit": "NTT jobs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": sum(4 * sum(q["ranks"][k] * n * q["ranks"][k + 1]
                                                  for k, n in enumerate(q["dims"])) for q in reqs)},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ntt", choices=["ntt", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None, help="jobs in the end-to-end run (default max(steps, 20))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=1000, help="c5_serving: number of requests")
    ap.add_argument("--batch-iters", type=int, default=0, help="c4_batched: MU iterations (profiling runs)")
    ap.add_argument("--batch-top", type=int, default=0, help="c4_batched: only the largest K instances")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-slots", type=int, default=512)
    ap.add_argument("--serve-sweep", action="store_true", help="c5_serving: also 0.25/0.5/0.95 x saturation")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "c3_16x8", "c4_batched", "c5_serving"],
                    help="c3_16x8: precision form on 16^8 (BF16 X per stage, 5 FP32 refinement "
                         "iterations); c4_batched: 512 nTT instances (d 3-6, n_k 8-24, r_k 2-12), 8 "
                         "restarts per stage, 300 MU iterations, one batched decomposition per step; "
                         "c5_serving: 1000 Poisson requests through the serving form")
    ap.add_argument("--engine", default="pass", choices=["pass", "group"],
                    help="stage1_small: single-problem pass or grouped engine")
    ap.add_argument("--case", default="full",
                    choices=["full", "stage1_small", "tcb_small", "tcs_small", "tcn_small", "stage3", "stream"],
                    help="stage1_small: MU iterations of the stage-1 shape on 32 x 4194304 "
                         "(512 MB, larger than L2) for profiler captures")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "stream":
        return run_stream(args)
    if args.case in ("stage1_small", "tcb_small", "tcs_small", "tcn_small", "stage3"):
        return run_stage1_small(args)
    if args.workload == "c4_batched":
        return run_batched(args)
    if args.workload == "c5_serving":
        return run_serving(args)

    import numpy as np
    import torch

    import synth
    import paper_2008_01340_gb300 as ntt
    from paper_2008_01340_gb300 import _build

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    ntt.lib()
    dev = torch.device("cuda", local)

    wl = args.workload
    cfg = synth.CONFIGS[wl]
    dims, ranks, iters = cfg["dims"], cfg["ranks"], cfg["iters"]
    x_dtype, refine = cfg["x_dtype"], cfg.get("refine_iters", 0)
    N = math.prod(dims)
    A_host = torch.empty(N, dtype=torch.float32).pin_memory()
    A_np, info = synth.tt_tensor(dims, ranks, cfg["core_dist"], cfg["noise"], cfg["data_seed"],
                                 out=A_host.numpy())
    Ad = A_host.to(dev, non_blocking=False)
    plan = ntt.ntt_plan_create(dims, ranks, iters, 1e-12, x_dtype, refine, cfg["init_seed"])
    ws = ntt.empty_workspace(plan.workspace_size(), dev)
    ws_rel = ntt.empty_workspace(ntt.ntt_reconstruct_workspace_size(dims, ranks), dev)
    cores = [torch.empty(s, dtype=torch.float32, device=dev) for s in plan.core_shapes()]
    err = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        ntt.ntt_decompose(plan, Ad, cores, ws, stream)
        ntt.ntt_rel_error(dims, ranks, cores, Ad, err, ws_rel, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    stats = ntt.ntt_plan_get_stats(plan)
    rel_err = float(err[0].item())
    ms = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(world, ms)

    # ---- end to end through the host-buffer C-ABI call
    # back-to-back jobs through the host-buffer call: the first job's input copy
    # has no previous job to overlap, so a short run measures that start-up
    # more than the sustained rate; at least 20 jobs (about 6 s)
    e2e_steps = args.e2e_steps or max(args.steps, 20)
    ws_host = ntt.empty_workspace(plan.workspace_size_host(), dev)
    cores_h = [torch.empty(s, dtype=torch.float32).pin_memory() for s in plan.core_shapes()]
    err_h = torch.zeros(3, dtype=torch.float64).pin_memory()
    for _ in range(2):   # warm: one graph per input slot of the host variant
        ntt.ntt_decompose_host(plan, A_host, cores_h, ws_host, err_h, stream)
    torch.cuda.synchronize(dev)

    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        ntt.ntt_decompose_host(plan, A_host, cores_h, ws_host, err_h, stream)
    f1.record(stream)
    enqueue_ms = (time.perf_counter() - t0) * 1e3   # host time to enqueue every step (no waits inside)
    torch.cuda.synchronize(dev)
    e2e_ms = f0.elapsed_time(f1) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    # the host-to-device copy of one step's input alone, for reading the e2e figure
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g0.record(stream)
        Ad.copy_(A_host, non_blocking=True)
        g1.record(stream)
    torch.cuda.synchronize(dev)
    h2d_alone_ms = g0.elapsed_time(g1)
    h2d = N * 4
    d2h = sum(math.prod(s) for s in plan.core_shapes()) * 4 + 3 * 8

    # ---- roofline of the dominant kernel: the fused pass of the stage with the
    # longest MU loop, against HBM bandwidth, or against the FP32 FMA rate when
    # its arithmetic (4 m r + 4 r^2 flops per column) binds first
    peak, peak_src = _peaks()
    dom = max(range(len(stats["stages"])), key=lambda k: stats["stages"][k]["iter_ms"])
    st1 = stats["stages"][dom]
    per_iter_s = st1["iter_ms"] / 1e3 / st1["iters"]
    if per_iter_s <= 0:
        raise RuntimeError("stage timing events did not record")
    achieved = st1["alg_bytes"] / per_iter_s / 1e9
    flops = 4.0 * st1["n"] * (st1["m"] * st1["r"] + st1["r"] ** 2)
    tflops = flops / per_iter_s / 1e12
    traffic = None
    if (NCU_TRAFFIC["engine"] == st1.get("engine") and wl == WORKLOAD
            and NCU_TRAFFIC["kernel_sha"] == _kernel_sha(NCU_TRAFFIC["kernel_file"])):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    kernel_of = {"fma_pass": "mu_pass_kernel", "grouped": "gpass_kernel", "tc_bf16": "mu_pass_tcs_kernel (BF16 form)",
                 "tc_split": "mu_pass_tcs_kernel", "fma_narrow": "mu_pass_narrow_kernel",
                 "tc_narrow": "mu_pass_tcw_kernel"}
    kname = (f"{kernel_of.get(st1.get('engine'), st1.get('engine'))}<m={st1['m']},r={st1['r']},"
             f"{'bf16' if x_dtype == 'bf16' else 'f32'} X> + combine, "
             f"stage {dom + 1} ({st1['m']} x {st1['n']}, r={st1['r']})")
    if achieved / peak >= tflops / FP32_FMA_TFLOPS:
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kname,
                    "alg_bytes_per_launch": st1["alg_bytes"],
                    "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roofline = {"bound": "alu", "achieved": round(tflops, 2), "peak": FP32_FMA_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(tflops / FP32_FMA_TFLOPS, 4), "traffic": traffic, "kernel": kname,
                    "alg_flops_per_launch": flops,
                    "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz",
                    "hbm": {"achieved": round(achieved, 1), "frac": round(achieved / peak, 4)}}

    rel_launches = 0
    # Eq. (3): chain products left and right of the split point, then one residual pass
    s_split = 3
    rel_launches = (s_split - 1) + (len(dims) - 1 - s_split) + 1
    launches = (stats["launches"] + rel_launches) * args.steps

    stage_rows = []
    for s, st in enumerate(stats["stages"]):
        it_s = st["iter_ms"] / 1e3 / st["iters"]
        stage_rows.append({
            "m": st["m"], "n": st["n"], "r": st["r"], "iters": st["iters"],
            "mu_iters_per_s": round(1.0 / it_s, 1) if it_s > 0 else None,
            "alg_GBps": round(st["alg_bytes"] / it_s / 1e9, 1) if it_s > 0 else None,
            "frac_hbm": round(st["alg_bytes"] / it_s / 1e9 / peak, 4) if it_s > 0 else None,
            "stage_ms": round(st["stage_ms"], 3), "engine": st.get("engine"),
            "resid_half_sq": st["resid"], "xnorm2": st["xnorm2"]})

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 X, f32 arithmetic" if x_dtype == "bf16" else "f32",
        "data": "synthetic",
        "config": {"workload": (WORKLOAD + ": 32^6 FP32 tensor from random U[0,1) TT cores, ranks "
                                "(1,8,16,16,16,8,1), 1% |Gaussian| noise; 200 MU iterations per unfolding + Eq. (3)")
                   if wl == WORKLOAD else
                   (wl + ": 16^8 FP32 tensor from random Exp(1) TT cores, ranks (1,16,32,32,32,32,32,16,1), "
                    "1% |Gaussian| noise; per unfolding 200 MU iterations on its BF16 copy then 5 on FP32 + Eq. (3)"),
                   "global_batch": world, "l2_policy": f"inputs larger than L2 ({N * 4 / 1e9:.1f} GB tensor)",
                   "parallelism": f"independent jobs x{world}"},
        "roofline": roofline,
        "e2e": {"value": round(whole_job_rate(world, e2e_ms), 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3), "steps": e2e_steps,
                "host_enqueue_ms": round(enqueue_ms, 2), "h2d_alone_ms": round(h2d_alone_ms, 2),
                "input_pinned": bool(A_host.is_pinned())},
        "gpu_launches": launches,
        "clocks": clocks,
        "rel_error": rel_err,
        "stages": stage_rows,
        "mu_iters_per_s_stage1": stage_rows[0]["mu_iters_per_s"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A_np, cfg)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
