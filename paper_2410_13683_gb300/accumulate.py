"""Pooling the runs of a long sampling job, with checkpoint and resume.

A job calls fpt_run once per Philox run id k = 0, 1, 2, ... (one seed, one
trajectory range), and fpt_histogram gives each run's per-bin FP64 moments
(count, ln sum w, ln sum w^2, sum ln w, sum (ln w)^2) and its tail set. The
trajectories are keyed by (seed, run id, trajectory id), so the job's whole
state is the next run id and the pooled moments: `save` writes them exactly,
`load` restores them, and a resumed job pools the same runs in the same order
-- bit-identical to one that never stopped. Runs enter in run-id order; a
skipped or repeated run id is an error (its trajectories would be missing or
counted twice).

The pooled estimates are the single-run estimators of Sec. 4.1 over the union
of the runs: the weighted estimator P_b = sum_b w / (n db) with the standard
error of a sample mean, the lognormal-mean estimator (n_b/n) exp(m + s^2/2)/db
with Cox's error on the log combined with the binomial error of n_b/n, and the
tail set's ESS = (sum_T w)^2 / sum_T w^2 and probability sum_T w / n.
"""
from __future__ import annotations

import json
import math

import numpy as np

_ARRAYS = ("count", "log_sum_w", "log_sum_w2", "sum_lw", "sum_lw2")


class RunAccumulator:
    def __init__(self, seed: int, N_lo: float, N_hi: float, n_bins: int, N_tail: float = float("nan")):
        if not (N_hi > N_lo) or n_bins < 1:
            raise ValueError("need N_lo < N_hi and n_bins >= 1")
        self.seed, self.N_lo, self.N_hi, self.n_bins, self.N_tail = int(seed), float(N_lo), float(N_hi), \
            int(n_bins), float(N_tail)
        self.next_run = 0
        self.n_total = 0
        self.n_passed = 0
        self.n_capped = 0
        self.n_tail = 0
        self.tail_sw = 0.0
        self.tail_sw2 = 0.0
        self.count = np.zeros(n_bins, np.int64)
        self.log_sum_w = np.full(n_bins, -np.inf)
        self.log_sum_w2 = np.full(n_bins, -np.inf)
        self.sum_lw = np.zeros(n_bins)
        self.sum_lw2 = np.zeros(n_bins)

    @property
    def db(self) -> float:
        return (self.N_hi - self.N_lo) / self.n_bins

    def add(self, run_id: int, h: dict) -> None:
        """Pool run `run_id`'s histogram (an fpt_histogram result over this
        job's bins and tail threshold)."""
        if run_id != self.next_run:
            raise ValueError(f"run {run_id} added where run {self.next_run} is next: "
                             "runs enter in run-id order, each once")
        if len(h["count"]) != self.n_bins or h.get("db", self.db) != self.db:
            raise ValueError("the run's histogram has other bins than the job's")
        self.n_total += int(h["n_total"])
        self.n_passed += int(h["n_passed"])
        self.n_capped += int(h["n_capped"])
        self.n_tail += int(h["n_tail"])
        self.count += np.asarray(h["count"], np.int64)
        self.log_sum_w = np.logaddexp(self.log_sum_w, np.asarray(h["log_sum_w"], np.float64))
        self.log_sum_w2 = np.logaddexp(self.log_sum_w2, np.asarray(h["log_sum_w2"], np.float64))
        self.sum_lw += np.asarray(h["sum_lw"], np.float64)
        self.sum_lw2 += np.asarray(h["sum_lw2"], np.float64)
        # tail sums of the run: sum_T w = p_tail n, sum_T w^2 = (sum_T w)^2 / ESS
        sw = float(h["p_tail"]) * float(h["n_total"])
        self.tail_sw += sw
        self.tail_sw2 += sw * sw / float(h["ess_tail"]) if h["ess_tail"] > 0 else 0.0
        self.next_run += 1

    def estimates(self) -> dict:
        """Pooled P(N) per bin with both estimators and their errors, and the
        tail set's ESS and probability."""
        n, db, nb = float(self.n_total), self.db, self.n_bins
        pdf, se_w = np.zeros(nb), np.zeros(nb)
        pdf_ln, se_ln = np.full(nb, np.nan), np.full(nb, np.nan)
        for b in range(nb):
            c = float(self.count[b])
            if c <= 0:
                continue
            M = self.log_sum_w[b]                 # scale: sums relative to e^M
            S1, S2 = 1.0, math.exp(self.log_sum_w2[b] - 2.0 * M)
            pdf[b] = math.exp(M - math.log(n * db))
            var = max(S2 - S1 * S1 / n, 0.0) / ((n - 1.0) * n) if n > 1 else 0.0
            se_w[b] = math.exp(M) * math.sqrt(var) / db
            if c >= 2:
                m = self.sum_lw[b] / c
                s2 = max((self.sum_lw2[b] - c * m * m) / (c - 1.0), 0.0)
                pdf_ln[b] = (c / n) * math.exp(m + 0.5 * s2) / db
                cox = math.sqrt(s2 / c + s2 * s2 / (2.0 * (c - 1.0)))
                binom = math.sqrt(max(1.0 - c / n, 0.0) / c)
                se_ln[b] = pdf_ln[b] * math.sqrt(cox * cox + binom * binom)
        ess = self.tail_sw ** 2 / self.tail_sw2 if self.tail_sw2 > 0 else 0.0
        return {"pdf": pdf, "se_w": se_w, "pdf_ln": pdf_ln, "se_ln": se_ln, "count": self.count.copy(),
                "n_total": self.n_total, "n_passed": self.n_passed, "n_capped": self.n_capped,
                "ess_tail": ess, "p_tail": self.tail_sw / n if n > 0 else 0.0, "runs": self.next_run}

    def save(self, path: str) -> None:
        """The job's state: next run id, pooled moments and tail sums (exact)."""
        meta = {k: getattr(self, k) for k in ("seed", "N_lo", "N_hi", "n_bins", "N_tail", "next_run", "n_total",
                                               "n_passed", "n_capped", "n_tail", "tail_sw", "tail_sw2")}
        np.savez(path, meta=json.dumps(meta), **{k: getattr(self, k) for k in _ARRAYS})

    @classmethod
    def load(cls, path: str) -> "RunAccumulator":
        z = np.load(path)
        meta = json.loads(str(z["meta"]))
        acc = cls(meta["seed"], meta["N_lo"], meta["N_hi"], meta["n_bins"], meta["N_tail"])
        for k in ("next_run", "n_total", "n_passed", "n_capped", "n_tail", "tail_sw", "tail_sw2"):
            setattr(acc, k, meta[k])
        for k in _ARRAYS:
            setattr(acc, k, np.array(z[k]))
        return acc
