"""One extraction sharded over several GPUs (one process per GPU).

Walks are independent and keyed by (seed, request, walk id, hop), so rank r runs
its own contiguous range of walk ids (``frw_extract_sums`` with ``walk_begin``)
and the ranks exchange their exact sums once, at the end, with one all-gather of
4 (n_cond + 1) + 1 64-bit words each.  The sums are 128-bit integers (S1 in units
of 2^-64 fF, S2 in units of 2^-40 fF^2), so adding them is exact and the combined
row is bit-for-bit the row of a single run over all the walks.  The row is then
formed with the library's own arithmetic: each sum converted to double, C_k =
S1_k / n and the standard error sqrt((S2_k - S1_k^2 / n) / (n (n - 1))).

A sigma-target extraction shards the same way with one exchange per round
(``extract_sharded_sigma``): in round r rank q runs batches r W m + q m .. + m - 1
(W ranks, m batches each, batch = B walk ids), the ranks all-gather those
batches' exact sums, and every rank folds them in walk-id order into the running
sums, testing the stop rule of Sec. IV at every full batch exactly as the walk
kernel does on one GPU (``rel_errors``: the self term and the largest coupling,
ground excluded, each relative standard error at most the target).  All ranks
therefore stop after the same batch, and the row equals the single-GPU
``frw_extract`` row with the same target bit for bit.

Also the cross-rank reductions the benchmark uses (largest time, summed counts).
"""
from __future__ import annotations

import math

import numpy as np

S1_SCALE = 2.0 ** 64
S2_SCALE = 2.0 ** 40


def shard_range(n_walks: int, rank: int, world: int) -> tuple[int, int]:
    """(first walk id, count) of rank `rank` out of `world`: contiguous ranges that
    partition [0, n_walks), the first n_walks % world ranks one walk longer."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the group")
    base, extra = divmod(int(n_walks), world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def words_to_ints(words) -> list[int]:
    """(low, high) uint64 word pairs -> two's complement int128 values."""
    w = [int(x) & 0xFFFFFFFFFFFFFFFF for x in np.asarray(words, dtype=np.uint64).tolist()]
    out = []
    for i in range(0, len(w), 2):
        u = w[i] | (w[i + 1] << 64)
        out.append(u - (1 << 128) if u >= (1 << 127) else u)
    return out


def ints_to_words(values) -> np.ndarray:
    out = np.zeros(2 * len(values), dtype=np.uint64)
    for i, v in enumerate(values):
        u = int(v) & ((1 << 128) - 1)
        out[2 * i] = u & 0xFFFFFFFFFFFFFFFF
        out[2 * i + 1] = u >> 64
    return out


def combine(parts) -> tuple[list[int], list[int], int]:
    """parts: iterable of (sums words, n_walks) -> exact (S1, S2, n) over all parts."""
    S1 = S2 = None
    n = 0
    for words, cnt in parts:
        v = words_to_ints(words)
        half = len(v) // 2
        a, b = v[:half], v[half:]
        S1 = a if S1 is None else [x + y for x, y in zip(S1, a)]
        S2 = b if S2 is None else [x + y for x, y in zip(S2, b)]
        n += int(cnt)
    return S1, S2, n


def row_from_sums(S1, S2, n: int):
    """Capacitance row and standard errors from exact sums (the library's order of
    operations, so the result equals its own row bit for bit)."""
    k = len(S1)
    C = np.zeros(k)
    se = np.zeros(k)
    nn = float(n)
    for i in range(k):
        s1 = float(S1[i]) / S1_SCALE
        s2 = float(S2[i]) / S2_SCALE
        C[i] = s1 / nn if nn > 0 else 0.0
        v = (s2 - s1 * s1 / nn) / (nn * (nn - 1.0)) if nn > 1 else 0.0
        se[i] = math.sqrt(v if v > 0 else 0.0)
    return C, se


def allgather_sums(words, n_walks: int, group=None):
    """Every rank's (sums words, n_walks), gathered on every rank (one all-gather
    of 64-bit words; works with the gloo and nccl backends)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    payload = np.concatenate([np.asarray(words, dtype=np.uint64), np.array([n_walks], dtype=np.uint64)])
    t = torch.from_numpy(payload.view(np.int64).copy())
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    parts = []
    for o in out:
        a = o.cpu().numpy().view(np.uint64)
        parts.append((a[:-1], int(a[-1])))
    return parts


def extract_sharded(ctx, structure_id: int, master: int, n_cond: int, n_walks: int, request_id: int = 0,
                    batch: int = 0, group=None):
    """Budget-mode extraction of `n_walks` walks split over the ranks of `group`;
    every rank returns the same (C, stderr, n_walks)."""
    import torch.distributed as dist
    from . import binding as B
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    begin, count = shard_range(n_walks, rank, world)
    words, n, _ = B.frw_extract_sums(ctx, structure_id, master, n_cond, count, request_id, batch, begin)
    S1, S2, total = combine(allgather_sums(words, n, group))
    C, se = row_from_sums(S1, S2, total)
    return C, se, total


def _words_of(v: int) -> tuple[int, int]:
    u = int(v) & ((1 << 128) - 1)
    return u & 0xFFFFFFFFFFFFFFFF, u >> 64


def i128_to_double_kernel(v: int) -> float:
    """The walk kernel's conversion of a two's complement int128 to double (used
    by its stop rule): magnitude = hi * 2^64 + lo with each 64-bit word converted
    to double first (two roundings), then the sign."""
    lo, hi = _words_of(v)
    neg = hi >= (1 << 63)
    if neg:
        lo = (~lo + 1) & 0xFFFFFFFFFFFFFFFF
        hi = (~hi + (1 if lo == 0 else 0)) & 0xFFFFFFFFFFFFFFFF
    m = float(hi) * 18446744073709551616.0 + float(lo)
    return -m if neg else m


def rel_errors(S1, S2, master: int, n: float) -> tuple[float, float]:
    """Relative standard errors of the self term and of the largest coupling
    (largest |C_j|, j != master, ground excluded; the first on ties) from exact
    running sums, with the walk kernel's arithmetic; inf for a zero estimate."""
    def val(k):
        s1 = i128_to_double_kernel(S1[k]) / S1_SCALE
        s2 = i128_to_double_kernel(S2[k]) / S2_SCALE
        v = (s2 - s1 * s1 / n) / (n * (n - 1.0))
        return s1 / n, math.sqrt(v if v > 0 else 0.0)
    nc = len(S1) - 1
    ci, si = val(master)
    rs = si / abs(ci) if ci != 0.0 else math.inf
    jb, cb = -1, 0.0
    for j in range(nc):
        if j == master:
            continue
        c, _ = val(j)
        if jb < 0 or abs(c) > cb:
            jb, cb = j, abs(c)
    rc = 0.0
    if jb >= 0:
        c, sj = val(jb)
        rc = sj / abs(c) if c != 0.0 else math.inf
    return rs, rc


class SigmaFold:
    """Running exact sums of one extraction, fed batch by batch in walk-id order;
    decides like the walk kernel's stop rule: after a full batch with n >= 2
    walks, stop when both relative errors are at most `sigma`; otherwise stop when
    the budget is used up."""

    def __init__(self, n_cond: int, master: int, sigma: float, budget: int, batch: int):
        self.k = n_cond + 1
        self.master, self.sigma, self.budget, self.batch = master, float(sigma), int(budget), int(batch)
        self.S1 = [0] * self.k
        self.S2 = [0] * self.k
        self.next = 0              # next batch index expected
        self.used = 0
        self.decided = 0           # 1: converged, 2: budget used up

    @property
    def n_batches(self) -> int:
        return (self.budget + self.batch - 1) // self.batch

    def add(self, g: int, words, count: int) -> bool:
        """Fold batch g (its 4 (n_cond + 1) words and walk count); True once decided."""
        if self.decided:
            return True
        if g != self.next:
            raise ValueError("batches must be folded in walk-id order")
        v = words_to_ints(words)
        for i in range(self.k):
            self.S1[i] += v[i]
            self.S2[i] += v[self.k + i]
        self.next += 1
        n = min(self.next * self.batch, self.budget)
        if self.sigma > 0.0 and int(count) == self.batch and n >= 2:
            rs, rc = rel_errors(self.S1, self.S2, self.master, float(n))
            if rs <= self.sigma and rc <= self.sigma:
                self.decided, self.used = 1, n
                return True
        if self.next >= self.n_batches:
            self.decided, self.used = 2, self.budget
            return True
        return False

    def row(self):
        C, se = row_from_sums(self.S1, self.S2, self.used)
        return C, se, self.used, self.decided == 1


def round_payload(batch_sums, n_cond: int, budget: int, batch: int, r: int, rank: int, world: int, m: int):
    """Rank `rank`'s contribution to round r: its m batches r W m + rank m .. + m - 1
    (those below the budget), packed as m blocks of 4 (n_cond + 1) words followed
    by the m walk counts (zeros past the budget)."""
    words_per = 4 * (n_cond + 1)
    n_batches = (int(budget) + batch - 1) // batch
    mine = (r * world + rank) * m
    n_mine = max(0, min(m, n_batches - mine))
    payload = np.zeros(m * (words_per + 1), np.uint64)
    if n_mine > 0:
        w, cnt = batch_sums(mine * batch, min(n_mine * batch, int(budget) - mine * batch))
        w = np.asarray(w, np.uint64).reshape(-1, words_per)
        payload[:n_mine * words_per] = w[:n_mine].reshape(-1)
        payload[m * words_per:m * words_per + n_mine] = np.asarray(cnt, np.uint64)[:n_mine]
    return payload


def extract_sharded_sigma(batch_sums, n_cond: int, master: int, sigma: float, budget: int, batch: int = 16384,
                          rank: int = 0, world: int = 1, gather=None, batches_per_round: int = 4):
    """A sigma-target extraction split over `world` ranks.

    batch_sums(walk_begin, n_walks) -> (words of shape (n_b, 4 (n_cond + 1)),
    walks per batch) runs this rank's walks (walk_begin a multiple of `batch`);
    gather(payload) -> list of every rank's payload for the round (rank order) is
    the all-gather (None: a single rank).  Returns (C, stderr, walks used,
    converged), the same on every rank."""
    m = int(batches_per_round)
    F = SigmaFold(n_cond, master, sigma, budget, batch)
    words_per = 4 * (n_cond + 1)
    for r in range(F.n_batches + 1):
        payload = round_payload(batch_sums, n_cond, budget, batch, r, rank, world, m)
        parts = [payload] if gather is None else gather(payload)
        for q, part in enumerate(parts):
            part = np.asarray(part, np.uint64)
            for i in range(m):
                g = (r * world + q) * m + i
                if g >= F.n_batches:
                    break
                if F.add(g, part[i * words_per:(i + 1) * words_per], int(part[m * words_per + i])):
                    return F.row()
    raise RuntimeError("the fold ended without a decision")


def allgather_words(payload, group=None):
    """all-gather of one uint64 array per rank (gloo or nccl) -> list of arrays"""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.asarray(payload, np.uint64).view(np.int64).copy())
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return [o.cpu().numpy().view(np.uint64) for o in out]


def extract_sharded_sigma_ctx(ctx, structure_id: int, master: int, n_cond: int, sigma: float, budget: int,
                              request_id: int = 0, batch: int = 16384, group=None, batches_per_round: int = 4):
    """extract_sharded_sigma on this process's GPU context over the ranks of `group`."""
    import torch.distributed as dist
    from . import binding as B
    rank, world = dist.get_rank(group), dist.get_world_size(group)

    def sums(begin, n):
        w, cnt, _ = B.frw_extract_batch_sums(ctx, structure_id, master, n_cond, n, request_id, batch, begin)
        return w, cnt

    return extract_sharded_sigma(sums, n_cond, master, sigma, budget, batch, rank, world,
                                 lambda p: allgather_words(p, group), batches_per_round)


def reduce_max(x: float, group=None) -> float:
    """Largest value over the ranks (the benchmark's step time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def reduce_sum(x: float, group=None) -> float:
    """Sum over the ranks (walks processed by the whole job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, group=group)
    return float(t.item())
