"""GPU parity of the full-rank (2-D) noise stepper (Eq. 2.24 with S = sqrt(Xi),
Eq. 3.9) and its importance-sampling weight (Eq. 4.5 with B = S beta) against
the FP64 oracle, trajectory by trajectory."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt
from paper_2410_13683_gb300 import train as TR

from gpu_common import compare, gpu_run, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def _upload2(ctx, tab, model=0):
    M = len(tab.Spp)
    fpt.fpt_noise_table2(ctx, model, fpt.FPT_TABLE_USER2, M, 1.0, tab.phi_lo, tab.phi_lo + tab.h * (M - 1),
                         (tab.Spp, tab.Spq, tab.Sqq))


@pytest.fixture(scope="module")
def usr_numeric():
    m = W.USR_MODEL
    res = OT.resolve(m)
    return m, res, OT.numeric_table(m, res, 129, 1.0)


@pytest.mark.parametrize("betas", [[(0.0, 0.0), (0.5, -0.3), (0.0, 1.0)]])
def test_2d_usr_parity(torch, usr_numeric, betas):
    """Sudden-transition model with the numerically matched full-rank noise
    (sigma = 1): direct and two constant standardised biases in one launch;
    5000 trajectories per run (a ragged tail of the 32-lane refill); capped
    paths carry the CAPPED status on both sides."""
    m, res, tab = usr_numeric
    n = 5000
    with fpt.fpt_init_model([m]) as ctx:
        _upload2(ctx, tab)
        runs = [fpt.run_desc(0, n, seed=80, run_id=r, A=b1, A2=b2) for r, (b1, b2) in enumerate(betas)]
        st, g = gpu_run(ctx, runs, [n] * len(runs))
        # the bias (0.5, -0.3) holds ~10% of the paths above phi_end until the step cap
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    for r, (b1, b2) in enumerate(betas):
        o = OS.run2(m, res, tab, seed=80, run_id=r, n=n, A=b1, A2=b2)
        o.phi_end_value = res.phi_end
        # The matched noise changes by x4 across [phi_end, phi_in], so a field
        # error grows multiplicatively along a path; FP32 and FP64 paths longer
        # than 4x the median (20000 steps) are compared in law.
        mism, near = compare(g[r], o, res.phi_in - res.phi_end, f"2-D usr beta=({b1},{b2})",
                             pathwise_max_steps=20000)
        print(f"2-D usr beta=({b1},{b2}): mismatch {mism:.4%}, near-ties {near:.4%}")
        if b1 or b2:
            assert np.std(o.logw) > 0.1


def test_2d_brownian_full_rank_parity(torch):
    """Exponential potential with a constant full-rank S: pi fluctuates about
    -mu; large biases exercise the weight (|ln w| up to tens)."""
    m = W.BM.model
    a, b, c = 1e-3, 3e-4, 5e-4
    tab = OT.user_table2(np.full(16, a), np.full(16, b), np.full(16, c), -0.1, 0.2)
    res = OT.resolve(m)
    betas = [(0.0, 0.0), (0.6, -0.8), (2.0, 1.5)]
    n = 3000
    with fpt.fpt_init_model([m]) as ctx:
        _upload2(ctx, tab)
        runs = [fpt.run_desc(0, n, seed=81, run_id=r, A=b1, A2=b2) for r, (b1, b2) in enumerate(betas)]
        st, g = gpu_run(ctx, runs, [n] * len(runs))
        assert st == fpt.FPT_OK
    for r, (b1, b2) in enumerate(betas):
        o = OS.run2(m, res, tab, seed=81, run_id=r, n=n, A=b1, A2=b2)
        o.phi_end_value = res.phi_end
        compare(g[r], o, res.phi_in - res.phi_end, f"2-D bm beta=({b1},{b2})")


def test_2d_numeric_table_matches_oracle_and_runs(torch):
    """The library's own NUMERIC table (host FP64 build) agrees with the
    oracle's numerical matching, and the run on it agrees with the oracle run
    on the oracle's table."""
    m = W.USR_MODEL
    res = OT.resolve(m)
    M, n = 65, 4096
    tab = OT.numeric_table(m, res, M, 1.0)
    with fpt.fpt_init_model([m]) as ctx:
        Spp, Spq, Sqq = fpt.fpt_noise_table2(ctx, 0, fpt.FPT_TABLE_NUMERIC, M, 1.0)
        np.testing.assert_allclose(Spp, tab.Spp, rtol=1e-7)
        np.testing.assert_allclose(Spq, tab.Spq, rtol=1e-7, atol=1e-7 * np.max(np.abs(tab.Spq)))
        np.testing.assert_allclose(Sqq, tab.Sqq, rtol=1e-7)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=82, A=0.7, A2=0.2)], [n])
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    o = OS.run2(m, res, tab, seed=82, run_id=0, n=n, A=0.7, A2=0.2)
    o.phi_end_value = res.phi_end
    compare(g[0], o, res.phi_in - res.phi_end, "2-D numeric table")


def _rand_params(seed, out_scale):
    p = W.mlp_init(seed, out_scale=out_scale)
    rng = np.random.default_rng(seed + 100)
    p["b1"] = rng.normal(0, 0.3, 64)
    p["b2"] = rng.normal(0, 0.3, 64)
    p["b3"] = rng.normal(0, 0.3, 2)
    v = fpt.canonical_params(p)
    return v, fpt.params_dict(v)


def test_2d_mlp_statistics_match_oracle(torch):
    """Learned proposal on 2-D noise: beta = (clamp(o1), clamp(o2)) held per
    segment. The network evaluates in bf16 on tensor cores and the oracle in
    FP64 on bf16-rounded operands, so single trajectories may part; the
    laws (mean N, mean ln w) agree within Monte Carlo error and most
    trajectories take the identical number of steps."""
    m = W.BM.model
    a, b, c = 1e-3, 3e-4, 5e-4
    tab = OT.user_table2(np.full(16, a), np.full(16, b), np.full(16, c), -0.1, 0.2)
    res = OT.resolve(m)
    v, p = _rand_params(21, out_scale=0.3)
    n = 1 << 13
    shift, scale, seg, amax = (0.0, 0.0, 0.0), (20.0, 100.0, 0.2), 64, 2.0
    with fpt.fpt_init_model([m]) as ctx:
        _upload2(ctx, tab)
        prop = TR.new_proposal(ctx, v, shift=shift, scale=scale, segment=seg, alpha_max=amax)
        out = dict(nsteps=np.zeros(n, np.int32), logw=np.zeros(n), status=np.zeros(n, np.uint8))
        assert fpt.fpt_run(ctx, [prop.desc(0, n, seed=83, run_id=0)], [out]) == fpt.FPT_OK
    mlp = OS.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, alpha_max=amax, round_bf16=True)
    o = OS.run2(m, res, tab, seed=83, run_id=0, n=n, mlp=mlp)
    same = out["nsteps"] == o.nsteps
    assert same.mean() > 0.8
    se = math.hypot(np.std(o.nsteps), np.std(out["nsteps"])) / math.sqrt(n)
    assert abs(out["nsteps"].mean() - o.nsteps.mean()) < 4 * se
    sl = math.hypot(np.std(o.logw), np.std(out["logw"])) / math.sqrt(n)
    assert abs(out["logw"].mean() - o.logw.mean()) < 4 * sl
    rel = np.abs(out["logw"][same] - o.logw[same]) / np.maximum(1.0, np.abs(o.logw[same]))
    assert np.median(rel) < 1e-3
    assert np.std(o.logw) > 0.01


def test_2d_mlp_constant_output_is_exact(torch):
    """A network with a zero last layer outputs b3: the learned 2-D run equals
    the constant-bias run with beta = clamp(b3), trajectory by trajectory."""
    m = W.BM.model
    a, b, c = 1e-3, 3e-4, 5e-4
    tab = OT.user_table2(np.full(16, a), np.full(16, b), np.full(16, c), -0.1, 0.2)
    res = OT.resolve(m)
    p = W.mlp_init(22, out_scale=0.0)
    p["b3"] = np.array([0.625, -2.5])          # bf16/fp32-exact; the second clamps to -2
    v = fpt.canonical_params(p)
    n = 4096
    with fpt.fpt_init_model([m]) as ctx:
        _upload2(ctx, tab)
        prop = TR.new_proposal(ctx, v, shift=(0, 0, 0), scale=(1, 1, 1), segment=32, alpha_max=2.0)
        out = dict(nsteps=np.zeros(n, np.int32), logw=np.zeros(n), status=np.zeros(n, np.uint8),
                   N=np.zeros(n))
        assert fpt.fpt_run(ctx, [prop.desc(0, n, seed=84, run_id=0)], [out]) == fpt.FPT_OK
    o = OS.run2(m, res, tab, seed=84, run_id=0, n=n, A=0.625, A2=-2.0)
    o.phi_end_value = res.phi_end
    compare(out, o, res.phi_in - res.phi_end, "2-D mlp constant")


def test_2d_call_rules(torch):
    """1-D and 2-D tables do not mix in one call; A2 needs a 2-D table; an
    empty run is fine."""
    m = W.BM.model
    a = np.full(16, 1e-3)
    with fpt.fpt_init_model([m, m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, a, np.zeros(16))
        fpt.fpt_noise_table2(ctx, 1, fpt.FPT_TABLE_USER2, 16, 1.0, -0.1, 0.2, (a, a * 0.1, a * 0.5))
        with pytest.raises(fpt.FptError):
            fpt.fpt_run(ctx, [fpt.run_desc(0, 64, seed=1), fpt.run_desc(1, 64, seed=1, run_id=1)])
        with pytest.raises(fpt.FptError):
            fpt.fpt_run(ctx, [fpt.run_desc(0, 64, seed=1, A=0.5, A2=0.1)])
        st, g = gpu_run(ctx, [fpt.run_desc(1, 0, seed=1), fpt.run_desc(1, 64, seed=1, run_id=1)], [0, 64])
        assert st == fpt.FPT_OK and (g[1]["status"] == fpt.FPT_TRAJ_PASSED).all()
        # a 2-D table replaces the 1-D one of the same model
        fpt.fpt_noise_table2(ctx, 0, fpt.FPT_TABLE_USER2, 16, 1.0, -0.1, 0.2, (a, a * 0.1, a * 0.5))
        st, _ = gpu_run(ctx, [fpt.run_desc(0, 64, seed=1), fpt.run_desc(1, 64, seed=1, run_id=1)], [64, 64])
        assert st == fpt.FPT_OK


def test_2d_mlp_gradient_matches_oracle(torch):
    """Rank-2 mode of the backward kernel (beta = clamp(o), two output
    gradients per record) against the FP64 backward: relative L2 error <= 2e-2,
    cosine >= 0.999, and a clamped component passes no gradient."""
    from oracle import mlp as OM
    v, p = _rand_params(23, out_scale=1.0)
    n = 5000
    s = W.random_states(n, 24)
    db = np.random.default_rng(25).normal(0, 1, (n, 2))
    amax = 0.4                                   # about 14% of the outputs clamp
    s32 = s.astype(np.float32).astype(np.float64)
    o, _ = OM.forward(p, s32, round_bf16=True)
    assert 0.05 < np.mean(np.abs(o) >= amax) < 0.95
    # outputs within 1e-2 of the clamp may fall on either side in bf16 arithmetic:
    # they carry no gradient, so the comparison tests the mask, not the rounding
    db[np.abs(np.abs(o) - amax) < 1e-2] = 0.0
    m = W.BM.model
    with fpt.fpt_init_model([m]) as ctx:
        g = fpt.fpt_mlp_grad2(ctx, v, s, db, amax)
    gr = OM.beta_grad(p, s32, amax, db.astype(np.float32).astype(np.float64), round_bf16=True)
    ref = fpt.canonical_params(gr).astype(np.float64)
    got = g.astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cos = float(got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref)))
    assert rel < 2e-2, rel
    assert cos > 0.999, cos


def test_2d_training_learns_the_exponential_tilt(torch):
    """Training on 2-D noise: with S = diag(s, 0) the field is the drifted
    walk and beta_2 moves nothing but adds weight variance, so the
    zero-variance proposal for the target e^{lambda N} P is beta_1 = the Esscher
    tilt alpha* = (mu - sqrt(mu^2 - 2 lambda s^2))/s and beta_2 = 0. Training from
    a random second output must find both."""
    mu, s_, lam = W.BM_MU, W.BM_S, 9.5
    alpha_star = (mu - math.sqrt(mu * mu - 2 * lam * s_ * s_)) / s_
    p0 = W.mlp_init(16, out_scale=0.0)
    p0["b3"] = np.array([0.0, 0.8])
    v0 = fpt.canonical_params(p0)
    m = W.BM.model
    z = np.zeros(16)
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table2(ctx, 0, fpt.FPT_TABLE_USER2, 16, 1.0, -0.1, 0.2, (np.full(16, s_), z, z))
        prop = TR.new_proposal(ctx, v0, shift=(0.025, -0.01, 3.0), scale=(40.0, 100.0, 0.3),
                               segment=64, alpha_max=4.0)
        TR.train(ctx, prop, 0, rounds=120, n_traj=1 << 13, seed=18, lam=lam, N_cut=lambda r: 1e9, lr=1e-2)
        h = prop.history
        N = np.linspace(0.5, 4.5, 64)
        x = 0.05 - (mu - alpha_star * s_) * N
        st = np.stack([x, np.full(64, -mu), N], axis=1)
        sn = (st - np.array(prop.shift)) * np.array(prop.scale)
        _, o = fpt.fpt_mlp_eval(ctx, prop.blob, sn, np.zeros(64), 4.0)
    o = o.reshape(64, 2)
    print(f"2-D training: loss {h[0]['loss']:.3g} -> {h[-1]['loss']:.3g}, beta1 median "
          f"{np.median(o[:, 0]):.4f} (alpha* {alpha_star:.4f}), |beta2| max {np.max(np.abs(o[:, 1])):.4f}")
    assert h[-1]["loss"] < 0.1 * h[0]["loss"]
    assert abs(np.median(o[:, 0]) / alpha_star - 1) < 0.1
    assert np.all(np.abs(o[:, 0] / alpha_star - 1) < 0.3)
    assert np.max(np.abs(o[:, 1])) < 0.15 * alpha_star
