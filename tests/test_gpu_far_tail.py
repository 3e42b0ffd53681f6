"""The GPU's importance-sampled far tail against the closed form and the oracle.

On the exponential test model the first-passage law is inverse Gaussian with
the discrete-monitoring shift of the barrier (the law and its derivation are
in test_oracle_far_tail.py). Here the tail probabilities P(N >= N_t) at
1e-12 and 1e-20 are estimated through the C ABI (fpt_run with a constant
bias, fpt_histogram's tail set) at 2^22 trajectories and compared with that
law; the first 2^16 trajectories of the same run are compared with the FP64
oracle one by one, and the two tail estimates on them must agree.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt

from gpu_common import compare, gpu_run, require_gpu
from test_oracle_far_tail import TARGETS, ig_law, tail_point

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def _bias(k):
    m = W.BM.model
    a = m.phi_in - m.phi_end
    return (W.BM_MU - a / (k * m.dN + 0.1)) / W.BM_S


@pytest.mark.parametrize("p", TARGETS)
def test_gpu_tail_matches_inverse_gaussian(torch, p):
    m = W.BM.model
    k, ref = tail_point(p)
    A = _bias(k)
    N_tail = (k - 0.5) * m.dN                  # between the grid times (k-1) dN and k dN
    n = 1 << 22
    S, T = np.full(16, W.BM_S), np.zeros(16)
    seed = 140 + int(-math.log10(p))
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, S, T)
        assert fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=seed, run_id=0, A=A)]) == fpt.FPT_OK
        assert fpt.fpt_sync(ctx) == fpt.FPT_OK
        h = fpt.fpt_histogram(ctx, 0, 0.0, 12.0, 512, N_tail=N_tail)
        # the first 2^16 trajectories with host outputs, for the oracle comparison
        n_o = 1 << 16
        st, g = gpu_run(ctx, [fpt.run_desc(0, n_o, seed=seed, run_id=0, A=A)], [n_o])
        assert st == fpt.FPT_OK
    est, ess = h["p_tail"], h["ess_tail"]
    se = est * math.sqrt(max(1.0 / ess - 1.0 / n, 0.0))
    print(f"GPU P(N >= {k * m.dN:.3f}) = {est:.5e} +- {se / est:.3%} (ESS {ess:.0f}); "
          f"inverse Gaussian {ref:.5e}; relative error {est / ref - 1:+.3%}")
    assert se / est < 0.005
    assert abs(est / ref - 1.0) <= 0.10
    assert abs(est - ref) <= 4.0 * se + 0.02 * ref
    d0, _, _ = ig_law(shift=False)
    assert abs(est - ref) < abs(est - float(d0.sf((k - 1) * m.dN)))

    # the oracle on the same trajectories: per-trajectory parity, same tail estimate
    res = OT.resolve(m)
    o = OS.run(m, res, OT.user_table(S, T, -0.1, 0.2), seed=seed, run_id=0, n=n_o, A=A)
    o.phi_end_value = res.phi_end
    compare(g[0], o, res.phi_in - res.phi_end, f"far tail p={p}")

    def tail_p(nsteps, logw):
        sel = nsteps >= k
        M = logw[sel].max()
        return math.exp(M) * np.exp(logw[sel] - M).sum() / len(nsteps)

    pg, po = tail_p(g[0]["nsteps"], g[0]["logw"]), tail_p(o.nsteps, o.logw)
    assert pg == pytest.approx(po, rel=2e-3)


def test_gpu_direct_law_is_the_shifted_inverse_gaussian(torch):
    """The bulk of the GPU's first-passage law against the closed form, not
    through the oracle: 2^22 direct paths of the exponential model binned per
    50 steps over [3.5, 6.5] e-folds. A path with n > k steps stayed above the
    end surface at steps 1..k, so P(n > k) = IG_sf(k dN) with the shifted
    barrier (Siegmund), and a bin (k1, k2] holds IG_sf(k1 dN) - IG_sf(k2 dN)
    of the paths. The counts must pass a chi-square test against that law and
    fail it against the continuous-monitoring law; the mean must match Wald's
    identity with the Siegmund overshoot (to its first drift correction)."""
    from scipy import stats as sst
    m = W.BM.model
    n = 1 << 22
    S, T = np.full(16, W.BM_S), np.zeros(16)
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, S, T)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=151, run_id=0)], [n])
    assert st == fpt.FPT_OK and np.all(g[0]["status"] == fpt.FPT_TRAJ_PASSED)
    k = g[0]["nsteps"].astype(np.int64)
    edges = np.arange(3500, 6501, 50)
    obs = np.array([np.sum((k > a) & (k <= b)) for a, b in zip(edges[:-1], edges[1:])], np.float64)

    def chi2_p(law):
        sf = law.sf(edges * m.dN)
        exp = n * (sf[:-1] - sf[1:])
        keep = exp >= 50
        c2 = float(np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep]))
        return c2, float(sst.chi2.sf(c2, int(keep.sum()) - 1)), int(keep.sum())

    d, mean, lam = ig_law()
    c2, p, nb = chi2_p(d)
    d0, _, _ = ig_law(shift=False)
    c20, p0, _ = chi2_p(d0)
    print(f"chi2 {c2:.1f} over {nb} bins (p = {p:.3g}); continuous monitoring: chi2 {c20:.1f} (p = {p0:.3g})")
    assert p > 1e-3
    assert p0 < 1e-6
    # Wald: mu E[N] = a + E[overshoot]; the overshoot is 0.5826 s sqrt(dN) in the
    # limit of a small drift per step, which here is theta = mu sqrt(dN)/s = 0.32 of the
    # step's noise: the first correction, ~theta/4 of s sqrt(dN), moves E[N] by ~2.5e-4
    N = k * m.dN
    assert abs(N.mean() - mean) < 4.0 * N.std() / math.sqrt(n) + 5e-4
