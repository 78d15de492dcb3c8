"""Parametric studies on synthetic inputs (python -m paper_2507_09730_gb300.studies CASE).

tau      the expected MicroWalk length against the lattice edge (Fig. 3a, Eq. 11):
         for each N, random cubes each holding 2-6 axis-aligned blocks placed
         uniformly (voxel ranges) with permittivities drawn from an exponential
         distribution of rate 0.1 (mean 10), background included; the mean number
         of steps of `samples` walks from the centre of each cube, from the
         MicroWalk kernel alone (allocation-free entry point, two cubes and at most
         14 permittivities per launch).  Reports min / mean / max of E(tau) / N^2
         over the cubes: the paper finds O(N^2), 0.3373 N^2 for one dielectric.
nsweep   the interconnect extraction (3 masters, 0.5 % sigma, FP32 geometry)
         at several lattice edges N (Fig. 5a: how the work splits with N):
         walks/s, hops and MicroWalk steps per walk, phase shares of the walk
         kernel.
serving  the serving configuration: Poisson arrivals over a pool of 32
         interconnect-style structures of 4-200 conductors, N = 24, FP32
         geometry, 1-sigma targets U[0.5 %, 2 %], budget 4e6 walks per request;
         served through frw_submit (admitted into the running walk kernel) and,
         on the same arrival times, one request per launch (frw_extract): p50 /
         p99 latency from arrival to completion, walks/s, identical results.
         First the configuration as stated (200 requests/s for 60 s), then a
         rate sweep over shorter windows to find the highest rate the GPU
         sustains (the served p99 stays near the service time instead of
         growing with the window).
Prints one JSON line per case (per N, per rate).
"""
from __future__ import annotations

import json
import sys

import numpy as np

from . import binding as B
from . import workloads as W


def _cube_pair(rng, N, n_cubes):
    """n_cubes (1 or 2) random cube records (64 int32 each) and their permittivities"""
    recs = np.zeros((n_cubes, 64), np.int32)
    eps = []
    for c in range(n_cubes):
        K = int(rng.integers(2, 7))
        recs[c, 0] = len(eps)
        eps.append(float(rng.exponential(10.0)))
        recs[c, 1] = K
        for b in range(K):
            for a in range(3):
                lo, hi = sorted(int(v) for v in rng.integers(0, N + 1, 2))
                if hi == lo:
                    hi = lo + 1 if lo < N else lo
                    lo = hi - 1
                recs[c, 2 + 7 * b + 2 * a] = lo
                recs[c, 3 + 7 * b + 2 * a] = hi
            recs[c, 8 + 7 * b] = len(eps)
            eps.append(float(rng.exponential(10.0)))
    return recs, np.asarray(eps)


def expected_steps(Ns=(8, 12, 16, 20, 24, 32), n_cubes=500, samples=4096, seed=0):
    """Mean MicroWalk length per random cube, for each N (see the module doc)."""
    import torch
    out = []
    stream = torch.cuda.current_stream().cuda_stream
    for N in Ns:
        rng = np.random.default_rng([6, seed, N])
        taus = []
        for g in range(0, n_cubes, 2):
            nc = min(2, n_cubes - g)
            recs, eps = _cube_pair(rng, N, nc)
            d = torch.from_numpy(recs).cuda()
            ex = torch.empty(nc * samples, dtype=torch.int32, device="cuda")
            st = torch.empty(nc * samples, dtype=torch.int32, device="cuda")
            rc = B.frw_microwalk_cubes_noalloc(N, nc, d.data_ptr(), eps, 0, samples, 1000 * N + g, ex.data_ptr(),
                                               st.data_ptr(), stream)
            if rc != B.FRW_OK:
                raise B.FRWError(rc, B.frw_strerror(rc))
            taus.extend(st.view(nc, samples).to(torch.float64).mean(dim=1).cpu().tolist())
        t = np.asarray(taus) / N ** 2
        out.append({"N": N, "cubes": len(taus), "samples_per_cube": samples, "tau_over_N2_min": float(t.min()),
                    "tau_over_N2_mean": float(t.mean()), "tau_over_N2_max": float(t.max())})
    return out


def n_sweep(Ns=(8, 12, 16, 20, 24, 32), sigma=0.005, steps=2):
    """The interconnect extraction at several lattice edges (see the module doc)."""
    import torch
    out = []
    s = W.interconnect(0)
    for N in Ns:
        c = B.Context(0, N=N, precision=B.FRW_FP32_GEOM, seed=0)
        sid = c.load(s)
        jobs = lambda r: [dict(structure_id=sid, master=m, walk_budget=10_000_000, sigma_target=sigma,
                               request_id=r * 4 + i) for i, m in enumerate(s.masters)]
        c.autotune([dict(j, walk_budget=300_000) for j in jobs(0)], sample_walks=300_000)
        c.extract_batch(jobs(1))
        walks = hops = micro = 0
        kms = mw = geom = 0.0
        for k in range(steps):
            res, _ = c.extract_batch(jobs(10 + k))
            walks += sum(r[2]["walks"] for r in res)
            hops += sum(r[2]["hops"] for r in res)
            micro += sum(r[2]["micro_steps"] for r in res)
            kms += res[0][2]["kernel_ms"]
            mw += res[0][2]["mw_ms"]
            geom += res[0][2]["geom_ms"]
        c.close()
        torch.cuda.synchronize()
        out.append({"N": N, "walks_per_s": walks / (kms / 1e3), "hops_per_walk": hops / walks,
                    "micro_steps_per_walk": micro / walks, "mw_share": mw / kms, "geometry_share": geom / kms})
    return out


SERVE_BUDGET = 4_000_000     # walk budget (cap) of one served request


def serving_point(N, precision, rate, duration, seed=0, baseline=True):
    """One serving measurement (see the module doc): requests drawn for `rate`
    per second over `duration` seconds, served, then (baseline) replayed one
    per launch; latency = completion - arrival."""
    import time
    pool = W.serving_pool(32)
    reqs = W.serving_requests(pool, rate=rate, duration=duration, seed=seed)
    ctx = B.Context(0, N=N, precision=precision, seed=0, serve_arena_mb=16384, serve_jobs=4096)
    sids = [ctx.load(st) for st in pool]
    ctx.extract_batch([dict(structure_id=sid, master=m, walk_budget=20000, request_id=1 + m)
                       for sid, st in zip(sids, pool) for m in range(0, st.n_cond, max(1, st.n_cond // 4))])

    def job(i, r):
        return dict(structure_id=sids[r.structure], master=r.master, walk_budget=SERVE_BUDGET, sigma_target=r.sigma,
                    request_id=10_000 + i)

    t0 = time.perf_counter()
    tickets = []
    for i, r in enumerate(reqs):
        dt = r.t - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(ctx.submit(job(i, r)))
    lat, walks, rows = [], 0, []
    for t in tickets:
        C, se, st, conv = ctx.wait(t)
        lat.append(st["seconds"])
        walks += st["walks"]
        rows.append(C)
    span = time.perf_counter() - t0
    out = {"rate_per_s": rate, "arrival_window_s": duration, "requests": len(reqs),
           "walks_per_request": walks / max(1, len(reqs)),
           "served": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                      "walks_per_s": walks / span, "makespan_s": span}}
    if baseline:
        t0 = time.perf_counter()
        lat_b, walks_b, same = [], 0, 0
        for i, r in enumerate(reqs):
            dt = r.t - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            C, se, st, conv = ctx.extract(sids[r.structure], r.master, SERVE_BUDGET, r.sigma, 10_000 + i)
            lat_b.append(time.perf_counter() - t0 - r.t)
            walks_b += st["walks"]
            same += int(np.array_equal(C, rows[i]))
        span_b = time.perf_counter() - t0
        out["one_job_per_launch"] = {"p50_s": float(np.percentile(lat_b, 50)),
                                     "p99_s": float(np.percentile(lat_b, 99)),
                                     "walks_per_s": walks_b / span_b, "makespan_s": span_b}
        out["identical_results"] = same
    ctx.close()
    return out


def serving(N=24, rates=(25, 50, 75, 100, 125, 150, 175), window=15.0):
    """The serving configuration as stated, then the rate sweep (module doc)."""
    out = [dict(case="configuration 4 as stated", **serving_point(N, B.FRW_FP32_GEOM, 200.0, 60.0))]
    for r in rates:
        out.append(dict(case="rate sweep", **serving_point(N, B.FRW_FP32_GEOM, float(r), window)))
    return out


if __name__ == "__main__":
    case = sys.argv[1]
    rows = {"tau": expected_steps, "nsweep": n_sweep, "serving": serving}[case]()
    for r in rows:
        print(json.dumps(r), flush=True)
