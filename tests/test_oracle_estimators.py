"""Pins of the FP64 estimators against brute force and special cases."""
import math

import numpy as np
import pytest

from oracle import estimators as E


def _sample(n=997, seed=0):
    rng = np.random.default_rng(seed)
    nsteps = rng.integers(800, 1300, n)
    logw = rng.normal(-3.0, 1.5, n)
    status = (rng.random(n) < 0.03).astype(np.uint8)
    return nsteps, logw, status


def test_histogram_brute_force():
    nsteps, logw, status = _sample()
    h = E.histogram(nsteps, logw, status, 1e-3, 0.9, 1.2, 37)
    db = (1.2 - 0.9) / 37
    cnt = np.zeros(37, int); sw = np.zeros(37); sw2 = np.zeros(37)
    for ns, lw, st in zip(nsteps, logw, status):
        if st:
            continue
        b = math.floor((ns * 1e-3 - 0.9) / db)
        if 0 <= b < 37:
            cnt[b] += 1; sw[b] += math.exp(lw); sw2[b] += math.exp(2 * lw)
    assert np.array_equal(cnt, h.count)
    np.testing.assert_allclose(np.exp(h.log_sum_w), sw, rtol=1e-12)
    np.testing.assert_allclose(np.exp(h.log_sum_w2), sw2, rtol=1e-12)
    assert h.n_capped == int(status.sum())
    assert h.count.sum() + h.n_under + h.n_over + h.n_capped == len(nsteps)
    assert np.array_equal(h.jk_count.sum(axis=0), h.count)


def test_direct_sampling_estimators_agree():
    """w = 1: weighted P = counts/(n db); the lognormal estimator reduces to it;
    jackknife and sample-variance errors agree with the binomial error."""
    rng = np.random.default_rng(1)
    n = 20000
    nsteps = rng.integers(0, 1000, n)
    lw = np.zeros(n)
    st = np.zeros(n, np.uint8)
    h = E.histogram(nsteps, lw, st, 1e-3, 0.0, 1.0, 10)
    P, se = E.p_weighted(h)
    Pl, sel = E.p_lognormal(h)
    Pj, sej = E.p_jackknife(h)
    np.testing.assert_allclose(P, h.count / (n * 0.1), rtol=1e-12)
    np.testing.assert_allclose(Pl, P, rtol=1e-12)
    np.testing.assert_allclose(Pj, P, rtol=1e-12)
    p = h.count / n
    binom = np.sqrt(p * (1 - p) / n) / 0.1
    np.testing.assert_allclose(se, binom, rtol=1e-3)
    np.testing.assert_allclose(sel, binom, rtol=1e-3)
    assert np.all(np.abs(sej / binom - 1) < 0.6)


def test_lognormal_mean_of_lognormal_weights():
    """ln w ~ N(m, s^2) in one bin: the lognormal estimator recovers
    E[w] = exp(m + s^2/2) within its stated error."""
    rng = np.random.default_rng(2)
    n = 50000
    lw = rng.normal(-2.0, 1.0, n)
    h = E.histogram(np.full(n, 500), lw, np.zeros(n, np.uint8), 1e-3, 0.0, 1.0, 1)
    P, se = E.p_lognormal(h)
    assert abs(P[0] - math.exp(-1.5)) < 4 * se[0]


def test_ess_and_tail():
    lw = np.log(np.array([1.0, 1.0, 2.0, 4.0]))
    assert E.ess(lw) == pytest.approx(64 / 22)
    ns = np.array([10, 20, 30, 40]); st = np.zeros(4, np.uint8)
    e, p, k = E.tail_ess(ns, lw, st, 0.1, 2.5)
    assert k == 2 and e == pytest.approx(36 / 20) and p == pytest.approx(6 / 4)


def test_combine_inverse_variance():
    P, se = E.combine([[1.0, 2.0], [3.0, np.nan]], [[1.0, 1.0], [1.0, 1.0]],
                      [[20, 20], [20, 0]])
    assert P[0] == pytest.approx(2.0) and se[0] == pytest.approx(1 / math.sqrt(2))
    assert P[1] == pytest.approx(2.0)


@pytest.mark.parametrize("s,p", [(2.0, 0.5), (0.3, 0.1)])
def test_lognormal_error_matches_the_spread_of_replicates(s, p):
    """The stated error of the lognormal estimator (Cox's term on the log,
    sqrt(s^2/n_b + s^4/(2(n_b - 1))), combined with the binomial error of
    n_b/n) against the spread of K independent replicates: each replicate has
    n trajectories, a fraction p of them in the bin, with ln w ~ N(-3, s^2).
    The variance of ln P over the replicates must equal the mean stated
    relative variance within the chi-square band of K - 1 degrees of freedom.
    At s = 2 the Cox terms dominate (dropping s^4/(2(n_b - 1)) would cut the
    stated variance by 3x); at s = 0.3, p = 0.1 the binomial term dominates."""
    rng = np.random.default_rng(17 + int(10 * s))
    K, n = 1500, 400
    logP, rel2 = np.empty(K), np.empty(K)
    for r in range(K):
        inbin = rng.random(n) < p
        nsteps = np.where(inbin, 500, 1500)               # bin [0.4, 0.6) holds N = 0.5
        lw = rng.normal(-3.0, s, n)
        h = E.histogram(nsteps, lw, np.zeros(n, np.uint8), 1e-3, 0.4, 0.6, 1, G=1)
        P, se = E.p_lognormal(h)
        logP[r] = math.log(P[0])
        rel2[r] = (se[0] / P[0]) ** 2
    emp, stated = logP.var(ddof=1), rel2.mean()
    # chi-square band of the sample variance, 4.5 standard deviations wide
    band = 4.5 * math.sqrt(2.0 / (K - 1))
    print(f"s={s} p={p}: var ln P over replicates {emp:.5g}, stated {stated:.5g}, ratio {emp / stated:.4f}")
    assert abs(emp / stated - 1.0) < band + 0.03
    # the mean of the estimator is the lognormal mean p exp(m + s^2/2)/db (bias O(s^4/n_b))
    mean_P = np.exp(logP).mean()
    assert abs(mean_P / (p * math.exp(-3.0 + 0.5 * s * s) / 0.2) - 1.0) < 0.05
