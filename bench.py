#!/usr/bin/env python
"""Throughput of the FRW + MicroWalk capacitance engine on the 3-layer
interconnect workload (24 wires with 10 nm eps-7.0 shells in an eps-2.7 ILD plus
12 eps-5 LDE blocks, lattice N = 24, the three layer masters, 0.5 % 1-sigma
target, budget 1e7 walks per master).

One step = one full extraction of the three capacitance rows: every row of the
hot path (walk issue, Gaussian sampling, first cube and weight, cube sizing,
hybrid dispatch, analytical route, MicroWalk, absorption, exact accumulation and
the stop rule) runs on the GPU for every walk.  The structure is loaded once
and stays resident in HBM; each step uses a fresh request id (new random walks).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_09730_gb300 import workloads as W  # noqa: E402

METRIC = "FRW walks/s and MicroWalk transitions/s at 1% 1\u03c3; request p50/p99 latency"
UNIT = "walks/s"
# algorithmic integer ops of one MicroWalk step: a quarter of a Philox4x32-10 block
# (15: ten rounds of two wide products and two xor-adds, over four words), the
# seven material queries, six weight reads, five prefix adds, the mul-high and five
# compares with four adds, and the move with its boundary test
INT_OPS_PER_MICRO_STEP = 45


# ---------------------------------------------------------------------------
# Profiling workloads (--case): the launches the ncu captures under profiles/
# cover; each prints what its profiled launch processed.

def case_walk():
    """The persistent walk kernel on the interconnect structure (N = 24, FP32
    geometry, masters 3, 11, 19), budget mode, 2^20 walks per master, with the
    launch settings the autotuner picks for this workload (2048 slots per CTA, 1
    analytical hop per epoch, MicroWalk lanes parked once the queue is empty and
    each has made 128 steps): one warm-up launch (fills the analytical-table
    cache), then the profiled launch."""
    from paper_2507_09730_gb300 import binding as B
    s = W.interconnect(0)
    c = B.Context(0, N=24, precision=B.FRW_FP32_GEOM, seed=0)
    c.set_tuning(pool_per_cta=2048, hops_per_epoch=1, suspend_lanes=32, suspend_min_steps=128)
    sid = c.load(s)
    jobs = lambda r: [dict(structure_id=sid, master=m, walk_budget=1 << 20, request_id=r + i)
                      for i, m in enumerate(s.masters)]
    c.extract_batch(jobs(1))
    rows, _ = c.extract_batch(jobs(100))
    walks = sum(r[2]["walks"] for r in rows)
    steps = sum(r[2]["micro_steps"] for r in rows)
    print(f"walk kernel: {walks} walks, {steps} MicroWalk steps, {rows[0][2]['kernel_ms']:.2f} ms")
    c.close()


def case_microwalk():
    """The MicroWalk kernel alone: 2^24 samples from 1024 random N = 16 cubes
    (16384 each, 2-6 blocks, permittivities {2.5, 3.9, 7.0, 25.0}): one warm-up
    launch, then the profiled launch."""
    import torch
    from paper_2507_09730_gb300 import binding as B
    N, n_cubes, spc = 16, 1024, 16384
    cubes = W.random_cubes(n_cubes, N=N, seed=0)
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    ex = torch.empty(n_cubes * spc, dtype=torch.int32, device="cuda")
    st = torch.empty(n_cubes * spc, dtype=torch.int32, device="cuda")
    c = B.Context(0, N=N, slots=1 << 12)
    for r in range(2):
        t0 = time.perf_counter()
        B.frw_microwalk_cubes(c.ctx, N, n_cubes, rec.data_ptr(), cubes.eps, spc, r, ex.data_ptr(), st.data_ptr())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    steps = int(st.to(torch.int64).sum().item())
    print(f"MicroWalk kernel: {n_cubes * spc} samples, {steps} steps, {1e3 * dt:.2f} ms ({steps / dt:.3e} steps/s)")
    c.close()


def case_fdm():
    """The FD-transition kernel of the FRW-FDM comparator alone: 1216 random N = 24
    cubes (2-6 blocks, permittivities as above), one mixed-precision FD solve and
    one sampled panel each: one warm-up launch on 8 cubes, then the profiled
    launch."""
    import torch
    from paper_2507_09730_gb300 import binding as B
    N, n = 24, 1216
    cubes = W.random_cubes(n, N=N, seed=5)
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    c = B.Context(0, N=N, slots=1 << 12)
    B.frw_fdm_cubes(c.ctx, N, 8, rec.data_ptr(), cubes.eps, 0, 0, 0, it.data_ptr())
    B.frw_fdm_cubes(c.ctx, N, n, rec.data_ptr(), cubes.eps, 0, 0, 0, it.data_ptr())
    torch.cuda.synchronize()
    iv = it.cpu().numpy().view(np.uint32)
    print(f"FD transitions: {n} cubes, {int((iv & 0xFFFFFF).sum())} CG iterations, "
          f"{int((iv >> 24).sum())} refinement passes")
    c.close()


PROFILE_CASES = {"walk": case_walk, "microwalk": case_microwalk, "fdm": case_fdm}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15)   # about 1 s timed: several 200 ms clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--N", type=int, default=24)
    ap.add_argument("--sigma", type=float, default=0.005)
    ap.add_argument("--budget", type=int, default=10_000_000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="arrival window of the serving measurement at 200 req/s (0: skip it)")
    ap.add_argument("--case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one profiling workload (the launches the profiles/ captures cover) and exit")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_walks(s, masters, N, seconds, threads, base_request, chunk=200, chunks=None):
    """Run the oracle as it stands on `threads` host threads, for about `seconds`
    or for exactly `chunks` chunks per thread: thread t takes chunks of `chunk`
    walks from its own walk-id range (ids t * 10^9 + ...), masters in turn.
    ctypes releases the GIL during each oracle call, so the threads run in
    parallel.  Returns (walks, seconds)."""
    import concurrent.futures as cf
    from oracle import oracle as O
    O.build()

    def worker(t, t0):
        walks, i = 0, 0
        while (i < chunks) if chunks is not None else (time.perf_counter() - t0 < seconds):
            O.frw_run(s, masters[i % len(masters)], chunk, N=N, seed=0, request=base_request,
                      walk_begin=t * 10**9 + i * chunk, records=False)
            walks += chunk
            i += 1
        return walks

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        total = sum(ex.map(worker, range(threads), [t0] * threads))
    return total, time.perf_counter() - t0


def cpu_baseline(s, masters, N, seconds):
    """The oracle as it stands on a bounded sample of the same workload: first one
    thread, then every host core over disjoint walk-id ranges."""
    cores = os.cpu_count() or 1
    w1, t1 = oracle_walks(s, masters, N, seconds / 3, 1, 900)
    wn, tn = oracle_walks(s, masters, N, 2 * seconds / 3, cores, 901)
    return {"value": wn / tn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": w1 / t1,
            "sample": f"{wn} walks on {cores} threads in {tn:.1f} s (chunks of 200 walks, disjoint walk-id ranges, "
                      f"masters {list(masters)}) of the same interconnect structure at N={N}, FP64; "
                      f"single thread: {w1} walks in {t1:.1f} s"}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    s = W.interconnect(0)
    masters = list(s.masters)
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    # one step: one chunk of walks per host thread (200: a few seconds)
    per_thread = int(os.environ.get("FRW_BENCH_REF_WALKS", "200"))
    for w in range(a.warmup):
        oracle_walks(s, masters, a.N, None, cores, 500 + w, chunk=20, chunks=1)
    t0 = time.perf_counter()
    walks = 0
    for k in range(a.steps):
        n, _ = oracle_walks(s, masters, a.N, None, cores, 600 + k, chunk=per_thread, chunks=1)
        walks += n
    dt = time.perf_counter() - t0
    v = walks / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"interconnect 3-layer/24-wire + shells + 12 LDE, N={a.N}, masters {masters}; "
                                   f"bounded sample: {per_thread} walks per host thread per step",
                       "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{walks} walks in {a.steps} steps on {cores} threads "
                                       f"({per_thread} walks per thread per step, disjoint walk-id ranges)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# DRAM bytes (read + write) per walk of the walk kernel, from one ncu capture of
# this workload (k_walk, 3 x 2^20 walks in budget mode); scaled by the walks a
# launch started.  None once the kernel has changed since the capture.
DRAM_BYTES_PER_WALK = 4878.3
# issue-slot utilisation (smsp__issue_active) and instruction-cache hit rate of the
# walk kernel in the same capture; None once the kernel has changed since
ISSUE_ACTIVE_NCU = 0.494
ICACHE_HIT_NCU = 0.830


def traffic_per_launch(agg, n_launch):
    if DRAM_BYTES_PER_WALK is None:
        return None
    return DRAM_BYTES_PER_WALK * agg["issued"] / n_launch


def microwalk_kernel(alu_peak, steps_timed=3):
    """MicroWalk transition kernel alone (Algorithm 3): 2^24 samples from the
    centres of 1024 random N = 16 cubes (16384 each), 2-6 blocks per cube with
    permittivities from {2.5, 3.9, 7.0, 25.0}; CUDA events on the launch stream."""
    import torch
    from paper_2507_09730_gb300 import binding as B
    N, n_cubes, spc = 16, 1024, 16384
    cubes = W.random_cubes(n_cubes, N=N, seed=0)
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    n = n_cubes * spc
    ex = torch.empty(n, dtype=torch.int32, device="cuda")
    stp = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx = B.Context(0, N=N, slots=1 << 12)
    stream = torch.cuda.current_stream()
    B.frw_set_stream(ctx.ctx, stream.cuda_stream)
    run = lambda r: B.frw_microwalk_cubes(ctx.ctx, N, n_cubes, rec.data_ptr(), cubes.eps, spc, r, ex.data_ptr(),
                                          stp.data_ptr())
    for r in range(3):
        run(r)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in range(steps_timed):
        run(100 + r)
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3 / steps_timed
    steps = int(stp.to(torch.int64).sum().item())
    ctx.close()
    ach = INT_OPS_PER_MICRO_STEP * steps / secs / 1e12
    return {"workload": "2^24 samples, 1024 random N=16 cubes x 16384, eps {2.5,3.9,7.0,25.0}",
            "samples_per_s": n / secs, "micro_transitions_per_s": steps / secs, "ms_per_launch": 1e3 * secs,
            "roofline": {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "Tint-op/s",
                         "frac": ach / alu_peak}}


def fp32_deviation(s, masters, N, sigma, budget):
    """FP32 cube geometry against FP64 geometry on the same requests: the walks
    differ only where a geometric decision differs, so the rows agree within
    their combined standard errors; reported per master as (C32 - C64) / C64 for
    C_ii and that difference in combined standard errors."""
    from paper_2507_09730_gb300 import binding as B
    out = []
    rows = {}
    for prec in (B.FRW_FP32_GEOM, B.FRW_FP64_GEOM):
        ctx = B.Context(0, N=N, precision=prec, seed=0)
        sid = ctx.load(s)
        res, _ = ctx.extract_batch([dict(structure_id=sid, master=m, walk_budget=budget, sigma_target=sigma,
                                         request_id=777 + i) for i, m in enumerate(masters)])
        rows[prec] = res
        ctx.close()
    for m, (C32, se32, _), (C64, se64, _) in zip(masters, rows[B.FRW_FP32_GEOM], rows[B.FRW_FP64_GEOM]):
        d = C32[m] - C64[m]
        out.append({"master": m, "C_ii_fp64": C64[m], "rel_dev": d / C64[m],
                    "dev_in_sigma": d / float(np.hypot(se32[m], se64[m]))})
    return out


def mwe_measurement(s, masters, N, precision, sigma, budget, tuning, rows_mw, steps=2):
    """FRW-MWE: the same extraction with MicroWalk-E (non-stratified later cubes
    expanded 5x, conductors inside them absorbing), timed like the main steps; its
    rows compared with the FRW-MW rows of the main measurement."""
    import torch
    from paper_2507_09730_gb300 import binding as B
    ctx = B.Context(0, N=N, precision=precision, seed=0, mwe_factor=5)
    ctx.set_tuning(**{k: tuning[k] for k in ("pool_per_cta", "hops_per_epoch", "suspend_lanes", "suspend_min_steps")})
    stream = torch.cuda.current_stream()
    B.frw_set_stream(ctx.ctx, stream.cuda_stream)
    sid = ctx.load(s)
    jobs = lambda r: [dict(structure_id=sid, master=m, walk_budget=budget, sigma_target=sigma,
                           request_id=r * 4 + i) for i, m in enumerate(masters)]
    ctx.extract_batch(jobs(70_000))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    walks = hops = 0
    e0.record(stream)
    for k in range(steps):
        res, _ = ctx.extract_batch(jobs(80_000 + k))
        walks += sum(r[2]["walks"] for r in res)
        hops += sum(r[2]["hops"] for r in res)
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    ctx.close()
    dev = []
    for m, (C, se, _), (Cw, sew, _) in zip(masters, res, rows_mw):
        dev.append({"master": m, "C_ii_mwe": C[m], "C_ii_mw": Cw[m], "diff_in_sigma": (C[m] - Cw[m]) / float(np.hypot(se[m], sew[m]))})
    return {"workload": "as the main line, MicroWalk-E (expansion 5) on non-stratified later cubes",
            "walks_per_s": walks / secs, "ms_per_step": 1e3 * secs / steps, "hops_per_walk": hops / max(1, walks),
            "vs_frw_mw": dev}


FDM_BUDGET = 400             # walks per master of the FRW-FDM comparison run
FDM_CUBES = 1216             # random non-stratified cubes of the per-transition comparison


def fdm_measurement(s, masters, N, precision, walks_per_s_mw):
    """FRW-FDM, the paper's comparator (Algorithm 2: each later non-stratified
    transition solves the cube's FD system and samples its SGF), on the same
    structure and masters at a fixed budget of FDM_BUDGET walks per master, timed
    with CUDA events around one batched extraction; and the cost of one transition
    both ways on FDM_CUBES random cubes of the same N (2-6 blocks, permittivities
    {2.5, 3.9, 7.0, 25.0}): FD solves per second against MicroWalk samples per
    second (64 per cube)."""
    import torch
    from paper_2507_09730_gb300 import binding as B
    from paper_2507_09730_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    ctx = B.Context(0, N=N, precision=precision, seed=0, transition=B.FRW_TRANSITION_FDM)
    B.frw_set_stream(ctx.ctx, stream.cuda_stream)
    sid = ctx.load(s)
    jobs = lambda r, b: [dict(structure_id=sid, master=m, walk_budget=b, request_id=r * 4 + i)
                         for i, m in enumerate(masters)]
    ctx.extract_batch(jobs(90_000, 20))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res, _ = ctx.extract_batch(jobs(90_001, FDM_BUDGET))
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    walks = sum(r[2]["walks"] for r in res)
    fd = sum(r[2]["mw_hops"] for r in res)
    ctx.close()
    cubes = W.random_cubes(FDM_CUBES, N=N, seed=5)
    c = B.Context(0, N=N, slots=1 << 12)
    B.frw_set_stream(c.ctx, stream.cuda_stream)
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    it = torch.zeros(FDM_CUBES, dtype=torch.int32, device="cuda")
    spc = 64
    ex = torch.zeros(FDM_CUBES * spc, dtype=torch.int32, device="cuda")
    times = {}
    for name, run in (("fd", lambda: B.frw_fdm_cubes(c.ctx, N, FDM_CUBES, rec.data_ptr(), cubes.eps, 0, 0, 0,
                                                     it.data_ptr())),
                      ("mw", lambda: B.frw_microwalk_cubes(c.ctx, N, FDM_CUBES, rec.data_ptr(), cubes.eps, spc, 5,
                                                           ex.data_ptr(), 0))):
        run()
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        times[name] = e0.elapsed_time(e1) / 1e3
    iv = it.cpu().numpy().view(np.uint32)
    c.close()
    fd_rate = FDM_CUBES / times["fd"]
    mw_rate = FDM_CUBES * spc / times["mw"]
    return {"workload": f"as the main line, FD-based later non-stratified transitions, {FDM_BUDGET} walks per master",
            "walks_per_s": walks / secs, "seconds": secs, "walks": walks, "fd_transitions_per_walk": fd / max(1, walks),
            "frw_mw_over_frw_fdm": walks_per_s_mw / (walks / secs),
            "per_transition": {"cubes": f"{FDM_CUBES} random cubes, N = {N}, 2-6 blocks",
                               "fd_solves_per_s": fd_rate, "microwalk_samples_per_s": mw_rate,
                               "microwalk_over_fd": mw_rate / fd_rate,
                               "cg_iterations_mean": float((iv & 0xFFFFFF).mean()),
                               "refinement_passes_mean": float((iv >> 24).mean())}}


BATCH_BUDGET = 400_000       # walk budget (cap) of one job of the batched configuration


def batched_measurement(N, precision, tuning, steps=1):
    """The batched configuration: 64 structures of 2-200 conductors (2-6 layers,
    generated like the interconnect), every conductor as master (3024 jobs), 1 %
    sigma target capped at BATCH_BUDGET walks per job, run as one captured plan
    (a CUDA graph holding the persistent walk kernel and its set-up).  A short
    batched extraction (5000 walks per job) fills the analytical-table cache,
    then `steps` plan replays with fresh request ids are timed with CUDA events."""
    import torch
    from paper_2507_09730_gb300 import binding as B
    from paper_2507_09730_gb300 import workloads as W
    fam = W.batched_family(64)
    stream = torch.cuda.current_stream()
    ctx = B.Context(0, N=N, precision=precision, seed=0)
    ctx.set_tuning(**{k: tuning[k] for k in ("pool_per_cta", "hops_per_epoch", "suspend_lanes", "suspend_min_steps")})
    B.frw_set_stream(ctx.ctx, stream.cuda_stream)
    sids = [ctx.load(st) for st in fam]
    jobs = [dict(structure_id=sid, master=m, walk_budget=BATCH_BUDGET, sigma_target=0.01, request_id=0)
            for sid, st in zip(sids, fam) for m in range(st.n_cond)]
    for i, j in enumerate(jobs):
        j["request_id"] = i
    ctx.extract_batch([dict(j, walk_budget=5000, request_id=j["request_id"] + 900_000) for j in jobs])
    plan = ctx.plan(jobs)
    try:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        walks = conv = 0
        e0.record(stream)
        for k in range(steps):
            res, _ = plan.run((k + 1) * 10_000)
            walks += sum(r[2]["walks"] for r in res)
            conv += sum(1 for (C, se, st) in res if st["walks"] < BATCH_BUDGET)
        e1.record(stream)
        e1.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
    finally:
        plan.close()
        ctx.close()
    return {"workload": f"64 structures of 2-200 conductors, all {len(jobs)} masters, N={N}, sigma 1 %, "
                        f"budget {BATCH_BUDGET} per job, one CUDA-graph plan per replay",
            "jobs": len(jobs), "walks_per_s": walks / secs, "jobs_per_s": steps * len(jobs) / secs,
            "ms_per_replay": 1e3 * secs / steps, "walks_per_job": walks / (steps * len(jobs)),
            "converged_before_budget": conv / (steps * len(jobs))}




def serving_measurement(N, precision, rate, duration, seed=0):
    """Serving form (paper_2507_09730_gb300.studies.serving_point): Poisson
    arrivals of extraction requests over a pool of 32 structures with 4-200
    conductors, 1-sigma targets U[0.5 %, 2 %], served through frw_submit and, on
    the same arrival times, one request per launch; latency = completion -
    arrival."""
    from paper_2507_09730_gb300 import studies
    return studies.serving_point(N, precision, rate, duration, seed)


def interconnect_seeds(N, precision, sigma, budget, tuning, seeds=(0, 1, 2, 3), steps=2):
    """The interconnect configuration at seeds 0-3 (each seed its own wire widths,
    spacings and LDE blocks; masters the fourth wire of each layer): walks/s of
    the same extraction as the main line (tuned settings of seed 0) and each
    master's self capacitance with its standard error."""
    from paper_2507_09730_gb300 import binding as B
    out = []
    for sd in seeds:
        s = W.interconnect(sd)
        c = B.Context(0, N=N, precision=precision, seed=0)
        c.set_tuning(**{k: tuning[k] for k in ("pool_per_cta", "hops_per_epoch", "suspend_lanes",
                                               "suspend_min_steps")})
        sid = c.load(s)
        jobs = lambda r: [dict(structure_id=sid, master=m, walk_budget=budget, sigma_target=sigma,
                               request_id=r * 4 + i) for i, m in enumerate(s.masters)]
        c.extract_batch(jobs(7))
        walks, kms, rows = 0, 0.0, None
        for k in range(steps):
            rows, _ = c.extract_batch(jobs(100 + k))
            walks += sum(r[2]["walks"] for r in rows)
            kms += rows[0][2]["kernel_ms"]
        c.close()
        out.append({"seed": sd, "walks_per_s": walks / (kms / 1e3),
                    "rows": [{"master": m, "C_ii_fF": float(C[m]), "stderr_fF": float(se[m]), "walks": int(st["walks"])}
                             for m, (C, se, st) in zip(s.masters, rows)]})
    return out


def structure_bytes(s):
    return (s.cond_lo.nbytes + s.cond_hi.nbytes + s.block_lo.nbytes + s.block_hi.nbytes + s.block_mat.nbytes +
            s.eps.nbytes + 48 + 40 * len(s.masters))


def main():
    a = parse()
    if a.case:
        return PROFILE_CASES[a.case]()
    if a.impl == "reference":
        return run_reference(a)
    import torch
    from paper_2507_09730_gb300 import binding as B
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = B.FRW_FP32_GEOM if a.precision == "fp32" else B.FRW_FP64_GEOM
    ctx = B.Context(local, N=a.N, precision=prec, seed=0)
    stream = torch.cuda.current_stream()
    B.frw_set_stream(ctx.ctx, stream.cuda_stream)
    s = W.interconnect(0)
    sid = ctx.load(s)
    masters = list(s.masters)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    # launch settings from the project's autotuner, on this workload in budget mode (results do not depend on them)
    tuning = ctx.autotune([dict(structure_id=sid, master=m, walk_budget=400_000, request_id=90 + i)
                           for i, m in enumerate(masters)], sample_walks=400_000)

    def jobs_for(step):
        rq = 1_000_000 * (rank + 1) + step
        return [dict(structure_id=sid, master=m, walk_budget=a.budget, sigma_target=a.sigma,
                     request_id=rq * 4 + i, batch=a.batch) for i, m in enumerate(masters)]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(a.warmup):
        ctx.extract_batch(jobs_for(10_000 + w))
        flush.zero_()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    agg = dict(walks=0, micro=0, mw_ms=0.0, geom_ms=0.0, fill_ms=0.0, reduce_ms=0.0, kernel_ms=0.0, launches=0,
               hops=0, mw_hops=0, branch=[0, 0, 0], truncated=0,
               strat=0, hom=0, rounds=0, tables=0, mw_jobs=0, walk_launches=0, issued=0)
    rows = None
    ev0.record(stream)
    for k in range(a.steps):
        res, conv = ctx.extract_batch(jobs_for(k))
        for C, se, st in res:
            agg["walks"] += st["walks"]
            agg["issued"] += st["walks_issued"]
            agg["micro"] += st["micro_steps"]
            agg["hops"] += st["hops"]
            agg["mw_hops"] += st["mw_hops"]
            agg["strat"] += st["strat_hops"]
            agg["hom"] += st["hom_hops"]
            agg["truncated"] += st["truncated"]
            for b in range(3):
                agg["branch"][b] += st["branch"][b]
        st0 = res[0][2]
        agg["mw_ms"] += st0["mw_ms"]
        agg["geom_ms"] += st0["geom_ms"]
        agg["fill_ms"] += st0["fill_ms"]
        agg["reduce_ms"] += st0["reduce_ms"]
        agg["kernel_ms"] += st0["kernel_ms"]
        agg["walk_launches"] += st0["launches"]
        agg["launches"] += st0["launches"] + 1     # + the L2 flush
        agg["rounds"] += st0["rounds"]
        agg["tables"] += st0["tables_built"]
        agg["mw_jobs"] += st0["mw_jobs"]
        rows = res
        flush.zero_()
    ev1.record(stream)
    ev1.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clocks = clk.stop()
    barrier()
    t_all = elapsed
    walks_all = agg["walks"]
    if world > 1:
        from paper_2507_09730_gb300 import sharding
        t_all = sharding.reduce_max(elapsed)
        walks_all = int(sharding.reduce_sum(agg["walks"]))
    value = walks_all / t_all

    # end to end through the C ABI with host buffers: load (H2D), extract, rows back (D2H), unload
    e2e = None
    if not a.no_e2e:
        h2d = structure_bytes(s)
        d2h = 2 * 8 * (s.n_cond + 1) * len(masters) + 8 * 17 * len(masters)
        barrier()
        te0 = time.perf_counter()
        ew = 0
        for k in range(a.steps):
            sid2 = ctx.load(s)
            jb = jobs_for(50_000 + k)
            for j in jb:
                j["structure_id"] = sid2
            res, _ = ctx.extract_batch(jb)
            ew += sum(st["walks"] for _, _, st in res)
            ctx.unload(sid2)
        torch.cuda.synchronize()
        te = time.perf_counter() - te0
        e2e = {"value": ew / te * (walks_all / max(1, agg["walks"])) if world > 1 else ew / te, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * 128 * sm_max * 1e6 / 1e12          # Tint-op/s: 128 INT32 lanes per SM at max clock
    # dominant kernel: the persistent walk kernel (one launch per step); algorithmic work =
    # the MicroWalk lattice steps it ran x INT_OPS_PER_MICRO_STEP, over its event-timed duration
    k_s = agg["kernel_ms"] / 1e3
    ops = INT_OPS_PER_MICRO_STEP * agg["micro"]
    achieved = ops / k_s / 1e12 if k_s > 0 else None
    mw_s = agg["mw_ms"] / 1e3
    mw_ach = ops / mw_s / 1e12 if mw_s > 0 else None
    n_l = max(1, agg["walk_launches"])
    roofline = {"kernel": "k_walk (persistent: geometry, table fill, reduction, MicroWalk)", "bound": "alu",
                "achieved": achieved, "peak": alu_peak, "unit": "Tint-op/s",
                "frac": (achieved / alu_peak) if achieved else None, "traffic": traffic_per_launch(agg, n_l),
                "peak_source": f"{n_sm} SMs x 128 INT32 lanes x {sm_max:.0f} MHz ({src} max clock)",
                "launch_ms": agg["kernel_ms"] / n_l, "walks_per_launch": agg["walks"] / n_l,
                "micro_steps_per_launch": agg["micro"] / n_l,
                "phase_share": {"mw": agg["mw_ms"] / max(1e-9, agg["kernel_ms"]),
                                "geom": agg["geom_ms"] / max(1e-9, agg["kernel_ms"]),
                                "fill": agg["fill_ms"] / max(1e-9, agg["kernel_ms"]),
                                "reduce": agg["reduce_ms"] / max(1e-9, agg["kernel_ms"])},
                "mw_phase": {"achieved": mw_ach, "frac": (mw_ach / alu_peak) if mw_ach else None},
                "ncu_capture": {"issue_active": ISSUE_ACTIVE_NCU, "icache_hit": ICACHE_HIT_NCU,
                                "workload": "3 x 2^20 walks, budget mode, same structure and settings"}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_all / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "interconnect 3-layer/24-wire + shells + 12 LDE, N=%d, masters %s, sigma %.3g "
                                   "(the interconnect configuration's target), budget %d/master"
                                   % (a.N, masters, a.sigma, a.budget),
                       "geometry": a.precision, "accumulate": "exact int128 (fp64 in/out)",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"weak x{world}",
                       "tuning": {k: tuning[k] for k in ("pool_per_cta", "hops_per_epoch", "suspend_lanes",
                                                            "suspend_min_steps")}},
            "micro_transitions_per_s": agg["micro"] * (walks_all / max(1, agg["walks"])) / t_all,
            "hops_per_walk": agg["hops"] / max(1, agg["walks"]),
            "mw_hop_fraction": agg["mw_hops"] / max(1, agg["hops"] - agg["walks"]),
            "analytical_hop_fraction": (agg["strat"] + agg["hom"]) / max(1, agg["hops"] - agg["walks"]),
            "first_cube_branches": {"stratified": agg["branch"][0] / max(1, agg["walks"]),
                                    "shrunk": agg["branch"][1] / max(1, agg["walks"]),
                                    "homogenised": agg["branch"][2] / max(1, agg["walks"])},
            "truncated_walks": agg["truncated"],
            "gpu_launches": agg["launches"], "roofline": roofline, "clocks": clocks}
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and world == 1:
        line["frw_mwe"] = mwe_measurement(s, masters, a.N, prec, a.sigma, a.budget, tuning, rows)
        line["frw_fdm"] = fdm_measurement(s, masters, a.N, prec, value)
        line["batched"] = batched_measurement(a.N, prec, tuning)
        line["microwalk_kernel"] = microwalk_kernel(alu_peak)
        line["fp32_vs_fp64"] = fp32_deviation(s, masters, a.N, a.sigma, a.budget)
        line["interconnect_seeds"] = interconnect_seeds(a.N, prec, a.sigma, a.budget, tuning)
    if rank == 0 and world == 1 and a.serve_seconds > 0:
        from paper_2507_09730_gb300 import studies
        line["serving"] = {
            "workload": "Poisson arrivals over 32 structures of 4-200 conductors, N=%d, sigma U[0.5%%, 2%%], "
                        "budget %d per request; served = frw_submit into the running kernel, "
                        "one_job_per_launch = frw_extract in arrival order, same GPU" % (a.N, studies.SERVE_BUDGET),
            "at_200_per_s": serving_measurement(a.N, prec, 200.0, a.serve_seconds),
            "at_25_per_s": serving_measurement(a.N, prec, 25.0, 2.0 * a.serve_seconds)}
    if rank == 0 and world == 1 and not a.no_cpu:
        line["cpu_baseline"] = cpu_baseline(s, masters, a.N, a.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
