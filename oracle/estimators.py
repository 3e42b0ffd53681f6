"""FP64 estimators of P(delta N) from first-passage samples.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Plain definitions, written with numpy loops over bins:

* bins: uniform in N over [N_lo, N_hi); passed trajectory j falls in bin
  b = floor((N_j - N_lo) / db), db = (N_hi - N_lo) / n_bins; N_j = n_j dN;
* weighted estimator (Sec. 4.1, importance sampling): P_b = sum_{j in b} w_j / (n db),
  n = all trajectories of the run (capped ones included); its standard error
  from the sample variance of X_j = w_j 1[j in b] / db;
* lognormal estimator (Sec. 4.1: error from the estimate of the mean of a
  lognormal): P_b = (n_b/n) exp(m + s^2/2) / db with m, s^2 the mean and
  unbiased variance of ln w over the bin; relative error from Cox's interval
  sqrt(s^2/n_b + s^4/(2(n_b - 1))) combined with the binomial error of n_b/n;
* jackknife (Sec. 4.1, direct sampling): G = 32 contiguous blocks of
  trajectory index, block(i) = floor(i G / n); delete-one-block estimates of
  P_b and SE = sqrt((G-1)/G sum_g (P_(-g) - mean)^2);
* effective sample size of a set T: ESS_T = (sum_T w)^2 / sum_T w^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

JACKKNIFE_BLOCKS = 32


def _lse(v: np.ndarray) -> float:
    if v.size == 0:
        return -math.inf
    m = float(np.max(v))
    return m + math.log(float(np.sum(np.exp(v - m))))


@dataclass
class Histogram:
    N_lo: float
    N_hi: float
    n_bins: int
    n_total: int
    count: np.ndarray          # [n_bins] int64
    log_sum_w: np.ndarray      # [n_bins] ln sum w   (-inf if empty)
    log_sum_w2: np.ndarray     # [n_bins] ln sum w^2
    sum_lw: np.ndarray
    sum_lw2: np.ndarray
    n_under: int
    n_over: int
    n_capped: int
    jk_count: np.ndarray       # [G, n_bins]
    jk_log_sum_w: np.ndarray   # [G, n_bins]
    jk_n: np.ndarray           # [G] trajectories per block

    @property
    def db(self):
        return (self.N_hi - self.N_lo) / self.n_bins

    @property
    def centers(self):
        return self.N_lo + self.db * (np.arange(self.n_bins) + 0.5)


def bin_index(nsteps: np.ndarray, dN: float, N_lo: float, N_hi: float, n_bins: int):
    db = (N_hi - N_lo) / n_bins
    N = nsteps.astype(np.float64) * dN
    return np.floor((N - N_lo) / db).astype(np.int64)


def histogram(nsteps, logw, status, dN, N_lo, N_hi, n_bins, G=JACKKNIFE_BLOCKS) -> Histogram:
    nsteps = np.asarray(nsteps)
    logw = np.asarray(logw, dtype=np.float64)
    status = np.asarray(status)
    n = len(nsteps)
    b = bin_index(nsteps, dN, N_lo, N_hi, n_bins)
    passed = status == 0
    blk = (np.arange(n, dtype=np.int64) * G) // max(n, 1)
    count = np.zeros(n_bins, np.int64)
    lsw = np.full(n_bins, -math.inf)
    lsw2 = np.full(n_bins, -math.inf)
    slw = np.zeros(n_bins)
    slw2 = np.zeros(n_bins)
    jkc = np.zeros((G, n_bins), np.int64)
    jkl = np.full((G, n_bins), -math.inf)
    for k in range(n_bins):
        sel = passed & (b == k)
        lw = logw[sel]
        count[k] = lw.size
        lsw[k] = _lse(lw)
        lsw2[k] = _lse(2.0 * lw)
        slw[k] = float(np.sum(lw))
        slw2[k] = float(np.sum(lw * lw))
        for g in range(G):
            s2 = sel & (blk == g)
            jkc[g, k] = int(np.sum(s2))
            jkl[g, k] = _lse(logw[s2])
    jk_n = np.bincount(blk, minlength=G).astype(np.int64)
    return Histogram(N_lo, N_hi, n_bins, n, count, lsw, lsw2, slw, slw2,
                     int(np.sum(passed & (b < 0))), int(np.sum(passed & (b >= n_bins))),
                     int(np.sum(~passed)), jkc, jkl, jk_n)


def p_weighted(h: Histogram):
    """P_b = sum w / (n db) and its standard error."""
    n = h.n_total
    P = np.exp(h.log_sum_w - math.log(n * h.db))
    # sample variance of X = w 1_b / db over all n trajectories
    sw = np.exp(h.log_sum_w)
    sw2 = np.exp(h.log_sum_w2)
    var = np.maximum(sw2 - sw * sw / n, 0.0) / (n - 1)
    se = np.sqrt(var / n) / h.db
    return P, se


def p_lognormal(h: Histogram):
    """Lognormal-mean estimator and its standard error (n_b >= 2)."""
    n = h.n_total
    P = np.full(h.n_bins, np.nan)
    se = np.full(h.n_bins, np.nan)
    for k in range(h.n_bins):
        nb = int(h.count[k])
        if nb < 2:
            continue
        m = h.sum_lw[k] / nb
        s2 = max((h.sum_lw2[k] - nb * m * m) / (nb - 1), 0.0)
        P[k] = (nb / n) * math.exp(m + 0.5 * s2) / h.db
        cox = math.sqrt(s2 / nb + s2 * s2 / (2.0 * (nb - 1)))
        binom = math.sqrt(max(1.0 - nb / n, 0.0) / nb)
        se[k] = P[k] * math.sqrt(cox * cox + binom * binom)
    return P, se


def p_jackknife(h: Histogram):
    """Delete-one-block jackknife of the weighted estimator."""
    G = h.jk_count.shape[0]
    sw = np.exp(h.log_sum_w)
    swg = np.exp(h.jk_log_sum_w)
    Pg = (sw[None, :] - swg) / ((h.n_total - h.jk_n[:, None]) * h.db)
    mean = Pg.mean(axis=0)
    se = np.sqrt((G - 1) / G * np.sum((Pg - mean[None, :]) ** 2, axis=0))
    return sw / (h.n_total * h.db), se


def ess(logw: np.ndarray) -> float:
    """(sum w)^2 / sum w^2 from log-weights."""
    lw = np.asarray(logw, dtype=np.float64)
    if lw.size == 0:
        return 0.0
    return math.exp(2.0 * _lse(lw) - _lse(2.0 * lw))


def tail_ess(nsteps, logw, status, dN, N_tail) -> tuple:
    """ESS and probability estimate of the tail set T = {passed, N >= N_tail}."""
    nsteps = np.asarray(nsteps); logw = np.asarray(logw); status = np.asarray(status)
    sel = (status == 0) & (nsteps.astype(np.float64) * dN >= N_tail)
    lw = logw[sel]
    p = math.exp(_lse(lw)) / len(nsteps) if lw.size else 0.0
    return ess(lw), p, int(lw.size)


def mean_N(nsteps, status, dN, logw=None) -> float:
    """Mean first-passage time of passed trajectories (self-normalised with
    weights if logw is given)."""
    nsteps = np.asarray(nsteps); status = np.asarray(status)
    sel = status == 0
    N = nsteps[sel].astype(np.float64) * dN
    if logw is None:
        return float(np.mean(N))
    lw = np.asarray(logw)[sel]
    w = np.exp(lw - np.max(lw))
    return float(np.sum(w * N) / np.sum(w))


def combine(Ps, ses, counts, min_count=10):
    """Per-bin inverse-variance combination of several runs' estimates,
    using only runs with at least ``min_count`` samples in the bin."""
    Ps = np.asarray(Ps); ses = np.asarray(ses); counts = np.asarray(counts)
    ok = (counts >= min_count) & np.isfinite(Ps) & np.isfinite(ses) & (ses > 0)
    wgt = np.where(ok, 1.0 / np.where(ok, ses, 1.0) ** 2, 0.0)
    tot = wgt.sum(axis=0)
    P = np.where(tot > 0, (wgt * np.where(ok, Ps, 0.0)).sum(axis=0) / np.where(tot > 0, tot, 1), np.nan)
    se = np.where(tot > 0, 1.0 / np.sqrt(np.where(tot > 0, tot, 1)), np.nan)
    return P, se
