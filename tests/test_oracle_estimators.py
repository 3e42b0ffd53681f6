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
