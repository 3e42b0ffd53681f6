"""Trajectory-range sharding across ranks and the merge of tail statistics.

Philox is keyed by the global trajectory id, so rank r running ids
[r n, (r + 1) n) reproduces exactly the trajectories a single process would run
for those ids. The only exchange is a sum of the tail weight sums
(sum_T w, sum_T w^2), from which the merged effective sample size follows;
the merge checks that the ranks' ranges tile the whole range (a missing or
overlapping shard is an error, not a smaller sample).
"""
from __future__ import annotations

import math


def shard_offset(n_per_rank: int, rank: int) -> int:
    """First global trajectory id of `rank` (weak scaling: n_per_rank each)."""
    if n_per_rank < 0 or rank < 0:
        raise ValueError("n_per_rank and rank must be non-negative")
    if (rank + 1) * n_per_rank > (1 << 32):
        raise ValueError("trajectory ids must stay below 2^32")
    return rank * n_per_rank


def tail_sums(hist: dict) -> tuple:
    """(sum_T w, sum_T w^2) of one histogram result (fpt_histogram dict)."""
    sw = hist["p_tail"] * hist["n_total"]
    sw2 = sw * sw / hist["ess_tail"] if hist["ess_tail"] > 0 else 0.0
    return sw, sw2


def ess_of(sw: float, sw2: float) -> float:
    return sw * sw / sw2 if sw2 > 0 else 0.0


class ShardError(RuntimeError):
    """A shard of the trajectory range is missing, duplicated or overlaps
    another, or a rank did not take part in the merge."""


def check_tiling(parts, n_expected: int) -> None:
    """The ranks' trajectory ranges [first, first + count) must tile
    [0, n_expected) exactly; otherwise ShardError names the first gap,
    overlap or empty shard."""
    nxt = 0
    for rank, (first, count) in sorted(enumerate(parts), key=lambda rp: (rp[1][0], rp[0])):
        first, count = int(first), int(count)
        if count <= 0:
            raise ShardError(f"missing shard: rank {rank} reports no trajectories")
        if first > nxt:
            raise ShardError(f"missing shard: trajectories [{nxt}, {first}) were run by no rank")
        if first < nxt:
            raise ShardError(f"overlapping shards: rank {rank} starts at {first}, before {nxt}")
        nxt = first + count
    if nxt != n_expected:
        if nxt < n_expected:
            raise ShardError(f"missing shard: trajectories [{nxt}, {n_expected}) were run by no rank")
        raise ShardError(f"shards cover [0, {nxt}), beyond the expected {n_expected} trajectories")


def merge_shards(sw: float, sw2: float, first: int, count: int, n_expected: int, dist=None,
                 device=None) -> tuple:
    """Merged tail sums (sum_T w, sum_T w^2) of all ranks.

    Every rank contributes (first, count, sw, sw2) for its trajectory range;
    the table is gathered to every rank, checked (check_tiling) and summed in
    rank order, so all ranks raise the same ShardError or return the same
    sums. A rank that does not take part at all makes the collective fail
    (its peers see the connection close, or the process group's timeout),
    which is raised as ShardError as well."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        parts = [(first, count, sw, sw2)]
    else:
        import torch
        t = torch.tensor([float(first), float(count), sw, sw2], dtype=torch.float64, device=device)
        out = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
        try:
            dist.all_gather(out, t)
        except Exception as e:                       # a rank left, or the process-group timeout
            raise ShardError(f"shard merge failed: a rank did not take part ({type(e).__name__}: {e})") from e
        parts = [tuple(float(v) for v in o.cpu().tolist()) for o in out]
    check_tiling([(p[0], p[1]) for p in parts], n_expected)
    return sum(p[2] for p in parts), sum(p[3] for p in parts)


def ess_spread(sw_steps, sw2_steps, n_boot: int = 2000, seed: int = 0) -> dict:
    """Uncertainty of the pooled tail ESS from the per-step tail sums.

    The steps are independent batches, so the pooled ESS = (sum sw)^2 / sum sw2
    is resampled over steps (bootstrap, n_boot resamples with replacement):
    returns the 2.5% and 97.5% quantiles relative to the pooled value, and the
    delete-one-step jackknife relative standard error. With heavy-tailed
    weights a few steps hold most of sum sw2; the spread shows how much the
    pooled figure depends on them."""
    import numpy as np
    a = np.asarray(sw_steps, dtype=np.float64)
    b = np.asarray(sw2_steps, dtype=np.float64)
    K = len(a)
    if K < 2 or b.sum() <= 0:
        return {"lo": None, "hi": None, "rel_se": None, "steps": K}
    pooled = a.sum() ** 2 / b.sum()
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, K, (n_boot, K))
    A, B = a[idx].sum(axis=1), b[idx].sum(axis=1)
    boot = np.where(B > 0, A * A / np.where(B > 0, B, 1.0), 0.0)
    lo, hi = np.quantile(boot, [0.025, 0.975])
    jk = np.array([(a.sum() - a[k]) ** 2 / (b.sum() - b[k]) if b.sum() > b[k] else 0.0 for k in range(K)])
    # pooled over K - 1 steps: scale to K steps before comparing
    jk = jk * K / (K - 1)
    se = math.sqrt((K - 1) / K * float(np.sum((jk - jk.mean()) ** 2)))
    return {"lo": float(lo / pooled), "hi": float(hi / pooled), "rel_se": se / pooled, "steps": K}
