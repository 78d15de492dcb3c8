"""Workloads for profiler captures (python -m paper_2507_09730_gb300.profile_cases CASE).

walk       the persistent walk kernel on the interconnect structure (N = 24, FP32
           geometry, masters 3, 11, 19), budget mode, 2^20 walks per master, with
           the launch settings the autotuner picks for this workload (2048 slots
           per CTA, 2 analytical hops per epoch, MicroWalk lanes parked once the
           queue is empty and each has made 64 steps): one warm-up launch (fills
           the analytical-table cache), then the profiled launch.
microwalk  the MicroWalk kernel alone: 2^24 samples from 1024 random N = 16 cubes
           (16384 each, 2-6 blocks, permittivities {2.5, 3.9, 7.0, 25.0}): one
           warm-up launch, then the profiled launch.
fdm        the FD-transition kernel of the FRW-FDM comparator alone: 1216 random
           N = 24 cubes (2-6 blocks, permittivities as above), one mixed-precision
           FD solve and one sampled panel each: one warm-up launch on 8 cubes,
           then the profiled launch.
Prints what the launch processed (walks / samples and MicroWalk steps).
"""
from __future__ import annotations

import sys

from . import binding as B
from . import workloads as W


def walk():
    s = W.interconnect(0)
    c = B.Context(0, N=24, precision=B.FRW_FP32_GEOM, seed=0)
    c.set_tuning(pool_per_cta=2048, hops_per_epoch=2, suspend_lanes=32, suspend_min_steps=64)
    sid = c.load(s)
    jobs = lambda r: [dict(structure_id=sid, master=m, walk_budget=1 << 20, request_id=r + i)
                      for i, m in enumerate(s.masters)]
    c.extract_batch(jobs(1))
    rows, _ = c.extract_batch(jobs(100))
    walks = sum(r[2]["walks"] for r in rows)
    steps = sum(r[2]["micro_steps"] for r in rows)
    print(f"walk kernel: {walks} walks, {steps} MicroWalk steps, {rows[0][2]['kernel_ms']:.2f} ms")
    c.close()


def microwalk():
    import torch
    N, n_cubes, spc = 16, 1024, 16384
    cubes = W.random_cubes(n_cubes, N=N, seed=0)
    rec = torch.from_numpy(B.pack_cubes(cubes)).cuda()
    ex = torch.empty(n_cubes * spc, dtype=torch.int32, device="cuda")
    st = torch.empty(n_cubes * spc, dtype=torch.int32, device="cuda")
    c = B.Context(0, N=N, slots=1 << 12)
    for r in range(2):
        B.frw_microwalk_cubes(c.ctx, N, n_cubes, rec.data_ptr(), cubes.eps, spc, r, ex.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    print(f"MicroWalk kernel: {n_cubes * spc} samples, {int(st.to(torch.int64).sum().item())} steps")
    c.close()


def fdm():
    import numpy as np
    import torch
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


if __name__ == "__main__":
    {"walk": walk, "microwalk": microwalk, "fdm": fdm}[sys.argv[1]]()
