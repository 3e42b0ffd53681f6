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
