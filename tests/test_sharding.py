"""Sharding one extraction over ranks (one process per GPU): shard ranges, the
exact int128 exchange and the row formed from the combined sums.

The host side runs here as two gloo ranks on the CPU, with a stand-in engine
that returns exact integer sums for a walk-id range (signed 127-bit per-walk
terms, so carries across the 64-bit halves and negative totals occur).  The
device side (frw_extract_sums on shards of one GPU, combined) is checked
bit-for-bit against one full run in the GPU test."""
import os
import socket

import numpy as np
import pytest

from paper_2507_09730_gb300 import sharding as S


def _walk_terms(walk, k):
    """stand-in per-walk exact sums (S1, S2 words of k electrodes) for walk id `walk`"""
    rng = np.random.default_rng([walk, 17])
    e = int(rng.integers(0, k))
    s1 = [0] * k
    s2 = [0] * k
    mag = int(rng.integers(0, 1 << 62)) << 62 | int(rng.integers(0, 1 << 62))
    s1[e] = -mag if rng.integers(0, 2) else mag
    s2[e] = mag >> 3
    return s1, s2


def _range_sums(begin, count, k):
    S1 = [0] * k
    S2 = [0] * k
    for w in range(begin, begin + count):
        a, b = _walk_terms(w, k)
        S1 = [x + y for x, y in zip(S1, a)]
        S2 = [x + y for x, y in zip(S2, b)]
    return np.concatenate([S.ints_to_words(S1), S.ints_to_words(S2)]), count


def test_shard_ranges_partition():
    for n in (0, 1, 7, 1000, 12345):
        for world in (1, 2, 3, 8):
            got = [S.shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and sum(c for _, c in got) == n
            for (b0, c0), (b1, _) in zip(got, got[1:]):
                assert b0 + c0 == b1
            assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        S.shard_range(10, 2, 2)


def test_int128_words_roundtrip():
    vals = [0, 1, -1, (1 << 64) - 1, 1 << 64, -(1 << 64), (1 << 127) - 1, -(1 << 127), 123456789012345678901234567]
    assert S.words_to_ints(S.ints_to_words(vals)) == vals


def test_row_from_sums_matches_definition():
    # C = S1 / n and se = sqrt((S2 - S1^2/n) / (n (n - 1))) in fF units
    s1 = [int(0.75 * 2 ** 64) * 8, -int(0.25 * 2 ** 64) * 8]
    s2 = [int(0.75 * 2 ** 40) * 8, int(0.125 * 2 ** 40) * 8]
    C, se = S.row_from_sums(s1, s2, 8)
    assert C[0] == 0.75 and C[1] == -0.25
    assert se[0] == np.sqrt((6.0 - 36.0 / 8) / 56) and se[1] == np.sqrt((1.0 - 4.0 / 8) / 56)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, k, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        begin, count = S.shard_range(n, rank, world)
        words, cnt = _range_sums(begin, count, k)
        parts = S.allgather_sums(words, cnt)
        S1, S2, total = S.combine(parts)
        t = S.reduce_max(float(rank + 1))
        w = S.reduce_sum(float(cnt))
        q.put((rank, [str(x) for x in S1], [str(x) for x in S2], total, t, w))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_exactly():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    n, k, world = 301, 5, 2
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, k, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full, _ = _range_sums(0, n, k)
    F = S.words_to_ints(full)
    for rank, s1, s2, total, t, w in got:
        assert [int(x) for x in s1] == F[:k] and [int(x) for x in s2] == F[k:]
        assert total == n and t == float(world) and w == float(n)


@pytest.mark.gpu
def test_gpu_shards_equal_one_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09730_gb300 import binding as B
    from paper_2507_09730_gb300 import workloads as W
    s = W.interconnect(1)
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=21, slots=1 << 16) as c:
        sid = c.load(s)
        n = 100_003
        parts = []
        for r in range(3):
            begin, count = S.shard_range(n, r, 3)
            words, cnt, _ = B.frw_extract_sums(c.ctx, sid, 11, s.n_cond, count, 5, 4096, begin)
            parts.append((words, cnt))
        C, se = S.row_from_sums(*S.combine(parts))
        Cf, sef, st, _ = c.extract(sid, 11, n, 0.0, 5, 4096)
        np.testing.assert_array_equal(C, Cf)
        np.testing.assert_array_equal(se, sef)
        assert st["walks"] == n


def _dying_rank_main(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=15))
    if rank == 1:
        os._exit(0)          # this rank leaves between steps, before the exchange
    try:
        S.allgather_sums(np.zeros(8, np.uint64), 5)
        q.put((rank, "no error"))
    except Exception as e:   # the collective ends with an error instead of waiting forever
        q.put((rank, type(e).__name__))


def test_lost_rank_ends_the_exchange_with_an_error():
    import multiprocessing as mp
    import time
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_rank_main, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    rank, what = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what != "no error"
    assert time.time() - t0 < 100


# ---------------------------------------------------------------------------
# sigma-target extraction across ranks: the stop rule on the combined batches

def _standin_batch_sums(k, batch, master=0, seed=3):
    """Stand-in engine: walk w ends at electrode e with weight omega (fixed point
    of the library's scales), so that the relative errors fall like 1/sqrt(n)."""
    def walk(w):
        rng = np.random.default_rng([w, seed])
        e = master if rng.random() < 0.6 else int(rng.integers(0, k))
        om = (1.0 if e == master else -0.4) * (0.5 + rng.random())
        return e, int(round(om * 2 ** 64)), int(round(om * om * 2 ** 40))

    def sums(begin, n):
        nb = (n + batch - 1) // batch
        words = np.zeros((nb, 4 * k), np.uint64)
        cnt = np.zeros(nb, np.uint64)
        for b in range(nb):
            s1, s2 = [0] * k, [0] * k
            lo, hi = begin + b * batch, min(begin + (b + 1) * batch, begin + n)
            for w in range(lo, hi):
                e, a, q = walk(w)
                s1[e] += a
                s2[e] += q
            words[b] = np.concatenate([S.ints_to_words(s1), S.ints_to_words(s2)])
            cnt[b] = hi - lo
        return words, cnt
    return sums


def _sigma_rank_main(rank, world, port, k, batch, sigma, budget, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        C, se, used, conv = S.extract_sharded_sigma(_standin_batch_sums(k, batch), k - 1, 0, sigma, budget, batch,
                                                    rank, world, S.allgather_words, batches_per_round=2)
        q.put((rank, C.tolist(), se.tolist(), used, conv))
    finally:
        dist.destroy_process_group()


def test_sigma_fold_matches_a_plain_recomputation():
    """The fold stops at the first full batch where the self term and the largest
    coupling both reach the target; recomputed here in plain floating point from
    the same per-batch sums (exact sums converted once per check)."""
    k, batch, sigma, budget = 4, 64, 0.03, 64 * 200
    sums = _standin_batch_sums(k, batch)
    w, cnt = sums(0, budget)
    F = S.SigmaFold(k - 1, 0, sigma, budget, batch)
    for g in range(w.shape[0]):
        if F.add(g, w[g], int(cnt[g])):
            break
    assert F.decided == 1 and F.used < budget
    tot1 = np.zeros(k, dtype=object)
    tot2 = np.zeros(k, dtype=object)
    stop = None
    for g in range(w.shape[0]):
        v = S.words_to_ints(w[g])
        tot1 += np.array(v[:k], dtype=object)
        tot2 += np.array(v[k:], dtype=object)
        n = (g + 1) * batch
        c = np.array([float(x) / 2 ** 64 for x in tot1]) / n
        var = (np.array([float(x) / 2 ** 40 for x in tot2]) - c * c * n) / (n * (n - 1.0))
        se = np.sqrt(np.maximum(var, 0))
        jb = 1 + int(np.argmax(np.abs(c[1:k - 1])))          # largest coupling, ground (last) excluded
        if se[0] / abs(c[0]) <= sigma and se[jb] / abs(c[jb]) <= sigma:
            stop = n
            break
    assert stop == F.used
    C, se, used, conv = F.row()
    assert conv and used == stop
    C2, se2 = S.row_from_sums([int(x) for x in tot1], [int(x) for x in tot2], stop)
    np.testing.assert_array_equal(C, C2)
    np.testing.assert_array_equal(se, se2)
    # a budget too small to converge: decided by the budget, partial last batch included
    F2 = S.SigmaFold(k - 1, 0, 1e-6, 1000, batch)
    w2, cnt2 = sums(0, 1000)
    done = [F2.add(g, w2[g], int(cnt2[g])) for g in range(w2.shape[0])]
    assert done[-1] and not any(done[:-1]) and F2.decided == 2 and F2.used == 1000


def test_two_gloo_ranks_stop_at_the_single_run_batch():
    import multiprocessing as mp
    k, batch, sigma, budget = 4, 64, 0.03, 64 * 200
    C1, se1, used1, conv1 = S.extract_sharded_sigma(_standin_batch_sums(k, batch), k - 1, 0, sigma, budget, batch)
    assert conv1 and used1 < budget
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sigma_rank_main, args=(r, 2, port, k, batch, sigma, budget, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, C, se, used, conv in got:
        assert used == used1 and conv == conv1
        np.testing.assert_array_equal(np.array(C), C1)
        np.testing.assert_array_equal(np.array(se), se1)


@pytest.mark.gpu
def test_gpu_sigma_shards_equal_one_run():
    """Three shards of a sigma-target extraction on one GPU (the ranks' rounds run
    one after the other) give the row, the walk count and the decision of one
    frw_extract with the same target, bit for bit; the per-batch sums add up to
    frw_extract_sums over the same walks."""
    import itertools
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_09730_gb300 import binding as B
    from paper_2507_09730_gb300 import workloads as W
    s = W.interconnect(1)
    master, batch, sigma, budget, request = 11, 4096, 0.02, 2_000_000, 6
    with B.Context(0, N=16, precision=B.FRW_FP32_GEOM, seed=21, slots=1 << 16) as c:
        sid = c.load(s)

        def sums(begin, n):
            w, cnt, _ = B.frw_extract_batch_sums(c.ctx, sid, master, s.n_cond, n, request, batch, begin)
            return w, cnt

        w, cnt = sums(3 * batch, 5 * batch + 17)
        assert list(cnt) == [batch] * 5 + [17]
        tot, n, _ = B.frw_extract_sums(c.ctx, sid, master, s.n_cond, 5 * batch + 17, request, batch, 3 * batch)
        S1, S2, nn = S.combine([(w[b], cnt[b]) for b in range(w.shape[0])])
        assert nn == n and S.ints_to_words(S1 + S2).tolist() == tot.tolist()
        with pytest.raises(B.FRWError):
            B.frw_extract_batch_sums(c.ctx, sid, master, s.n_cond, batch, request, batch, 5)

        world, m = 3, 2
        rounds = itertools.count()

        def gather(p0):
            r = next(rounds)
            return [p0] + [S.round_payload(sums, s.n_cond, budget, batch, r, q, world, m) for q in range(1, world)]

        C, se, used, conv = S.extract_sharded_sigma(sums, s.n_cond, master, sigma, budget, batch, 0, world, gather, m)
        Cf, sef, st, convf = c.extract(sid, master, budget, sigma, request, batch)
    assert conv and convf and used == st["walks"] < budget
    np.testing.assert_array_equal(C, Cf)
    np.testing.assert_array_equal(se, sef)
