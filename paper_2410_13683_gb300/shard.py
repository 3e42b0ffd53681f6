"""Trajectory-range sharding across ranks and the merge of tail statistics.

Philox is keyed by the global trajectory id, so rank r running ids
[r n, (r + 1) n) reproduces exactly the trajectories a single process would run
for those ids. The only exchange is a sum of the tail weight sums
(sum_T w, sum_T w^2), from which the merged effective sample size follows.
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


def merge_tail_sums(sw: float, sw2: float, dist=None, device=None) -> tuple:
    """All-reduce (sum) of the tail sums over the default process group."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return sw, sw2
    import torch
    t = torch.tensor([sw, sw2], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t[0]), float(t[1])


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
