"""One extraction sharded over several GPUs (one process per GPU).

Walks are independent and keyed by (seed, request, walk id, hop), so rank r runs
its own contiguous range of walk ids (``frw_extract_sums`` with ``walk_begin``)
and the ranks exchange their exact sums once, at the end, with one all-gather of
4 (n_cond + 1) + 1 64-bit words each.  The sums are 128-bit integers (S1 in units
of 2^-64 fF, S2 in units of 2^-40 fF^2), so adding them is exact and the combined
row is bit-for-bit the row of a single run over all the walks.  The row is then
formed with the library's own arithmetic: each sum converted to double, C_k =
S1_k / n and the standard error sqrt((S2_k - S1_k^2 / n) / (n (n - 1))).

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
