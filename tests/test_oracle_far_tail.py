"""Pins of the oracle's importance-sampled far tail against a closed form.

On the exponential test model (V = V0 e^{mu phi}, attractor pi = -mu exact,
constant noise s, no correlation) the field performs an exact Gaussian random
walk with drift -mu per e-fold, monitored every dN. Its first-passage time
through x = 0 from x_0 = a is, for continuous monitoring, inverse Gaussian
IG(mean a/mu, shape a^2/s^2); discrete monitoring is accounted for by moving
the barrier away by 0.5826 s sqrt(dN) (Siegmund 1979; Broadie, Glasserman and
Kou 1997): P(walk above 0 at steps 1..m) = P(tau_a' > m dN). A trajectory with
step count n >= k has stayed above at steps 1..k-1, so
    P(N >= k dN) = IG_sf((k - 1) dN; a'/mu, a'^2/s^2),   a' = a + 0.5826 s sqrt(dN).

The importance-sampling machinery (the biased step of Eq. 4.7 with constant
amplitude A, the weight of Eqs. 4.4-4.5, the weighted tail estimator of
Sec. 4.1) is checked against this law where the metric is scored: at tail
probabilities 1e-12 and 1e-20, with ln w near -33 and -54. A bias of the
estimator that grows with |ln w| (a wrong quadratic term of the weight, a
dropped sqrt(dN), single-precision accumulation) moves the estimate far
outside the bar. The bar is 10% and, tighter, 4 standard errors (about 1%
each) plus 2% for the residual of the first-order monitoring correction; the
estimate must also lie closer to the shifted law than to the unshifted one,
which differs by 5-6% at these points.
The closed form comes from scipy.stats.invgauss, cross-checked at 50 digits
with mpmath.
"""
import math

import numpy as np
import pytest
from scipy import optimize, stats

import workloads as W
from oracle import estimators as E
from oracle import stepper as S
from oracle import tables as T

SIEGMUND = 0.5826      # -zeta(1/2)/sqrt(2 pi)
TARGETS = (1e-12, 1e-20)


def ig_law(shift=True):
    m = W.BM.model
    a = m.phi_in - m.phi_end
    if shift:
        a += SIEGMUND * W.BM_S * math.sqrt(m.dN)
    mean, lam = a / W.BM_MU, a * a / W.BM_S ** 2
    return stats.invgauss(mu=mean / lam, scale=lam), mean, lam


def tail_point(p):
    """Grid time k dN with P(N >= k dN) closest to p from above, and the law's value there."""
    d, _, _ = ig_law()
    dN = W.BM.model.dN
    t = optimize.brentq(lambda t: d.logsf(t) - math.log(p), 5.0, 20.0)
    k = int(math.floor(t / dN)) + 1
    return k, float(d.sf((k - 1) * dN))


def is_estimate(k, n, seed):
    """Constant-bias IS estimate of P(N >= k dN) on n oracle trajectories,
    with the proposal's mean passage time 0.1 e-fold beyond the point."""
    m = W.BM.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    a = m.phi_in - m.phi_end
    A = (W.BM_MU - a / (k * m.dN + 0.1)) / W.BM_S
    tr = S.run(m, res, tab, seed=seed, run_id=0, n=n, A=A)
    assert (tr.status == 0).all()
    sel = tr.nsteps >= k
    lw = tr.logw[sel]
    M = lw.max()
    w = np.exp(lw - M)
    p = math.exp(M) * w.sum() / n
    # standard error of the mean of X = w 1[N >= k dN] over all n trajectories
    var = (np.sum(w * w) - w.sum() ** 2 / n) / (n - 1)
    se = math.exp(M) * math.sqrt(max(var, 0.0) / n)
    _, p_fn, _ = E.tail_ess(tr.nsteps, tr.logw, tr.status, m.dN, k * m.dN - 0.5 * m.dN)
    assert p_fn == pytest.approx(p, rel=1e-12)
    return p, se, A, float(lw.mean())


@pytest.mark.parametrize("p", TARGETS)
def test_closed_form_is_accurate_in_the_deep_tail(p):
    """scipy's IG survival function against the IG law written out at 50 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    d, mean, lam = ig_law()
    k, ref = tail_point(p)
    t = mp.mpf((k - 1) * W.BM.model.dN)
    m_, l_ = mp.mpf(mean), mp.mpf(lam)
    cdf = mp.ncdf(mp.sqrt(l_ / t) * (t / m_ - 1)) + mp.exp(2 * l_ / m_) * mp.ncdf(-mp.sqrt(l_ / t) * (t / m_ + 1))
    assert float(1 - cdf) == pytest.approx(ref, rel=1e-9)
    assert 0.5 * p < ref < 2.0 * p


@pytest.mark.parametrize("p", TARGETS)
def test_importance_sampled_tail_matches_inverse_gaussian(p):
    k, ref = tail_point(p)
    est, se, A, mean_lw = is_estimate(k, 1 << 17, seed=101 + int(-math.log10(p)))
    rel = abs(est / ref - 1.0)
    print(f"P(N >= {k * 1e-3:.3f}) = {est:.4e} +- {se / est:.2%} (A = {A:.3f}, mean ln w {mean_lw:.1f}); "
          f"inverse Gaussian {ref:.4e}; relative error {rel:.2%}")
    assert se / est < 0.02                       # the comparison resolves a few per cent
    assert rel <= 0.10                           # the tail-error bar
    assert abs(est - ref) <= 4.0 * se + 0.02 * ref
    # the discrete monitoring is resolved: the continuous-monitoring law is farther off
    d0, _, _ = ig_law(shift=False)
    ref0 = float(d0.sf((k - 1) * W.BM.model.dN))
    assert abs(ref0 / ref - 1.0) > 0.04
    assert abs(est - ref) < abs(est - ref0)


def test_tail_estimate_does_not_depend_on_the_proposal():
    """Two constant amplitudes that put the proposal's typical passage time on
    either side of the 1e-20 point estimate the same tail probability."""
    k, ref = tail_point(1e-20)
    m = W.BM.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    a = m.phi_in - m.phi_end
    ests = []
    for j, dt in enumerate((-0.05, 0.3)):
        A = (W.BM_MU - a / (k * m.dN + dt)) / W.BM_S
        tr = S.run(m, res, tab, seed=131 + j, run_id=0, n=1 << 16, A=A)
        sel = tr.nsteps >= k
        M = tr.logw[sel].max()
        w = np.exp(tr.logw[sel] - M)
        n = len(tr.nsteps)
        se = math.exp(M) * math.sqrt(max((np.sum(w * w) - w.sum() ** 2 / n) / (n - 1), 0.0) / n)
        ests.append((math.exp(M) * w.sum() / n, se))
    (p1, s1), (p2, s2) = ests
    assert abs(p1 - p2) <= 4.0 * math.hypot(s1, s2)
    for pe, s in ests:
        assert abs(pe / ref - 1.0) <= 0.10
