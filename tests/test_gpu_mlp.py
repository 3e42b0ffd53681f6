"""GPU tests of the learned proposal: the tensor-core forward and backward
against the FP64 oracle, the unbiasedness of MLP-biased runs, and training
against the exponential-tilt closed form."""
import math
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import mlp as OM
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt
from paper_2410_13683_gb300 import train as TR

from gpu_common import gpu_run, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def bm_ctx():
    m = W.BM.model
    ctx = fpt.fpt_init_model([m])
    fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, np.full(16, W.BM_S), np.zeros(16))
    return ctx


def rand_params(seed, out_scale=1.0):
    p = W.mlp_init(seed, out_scale=out_scale)
    rng = np.random.default_rng(seed + 100)
    p["b1"] = rng.normal(0, 0.3, 64)
    p["b2"] = rng.normal(0, 0.3, 64)
    p["b3"] = rng.normal(0, 0.3, 2)
    v = fpt.canonical_params(p)
    return v, fpt.params_dict(v)          # the fp32 values both sides use


def test_mlp_forward_matches_oracle(torch):
    v, p = rand_params(1)
    s = W.random_states(4096 + 17, 2)                        # several warps and a ragged tail
    t = np.random.default_rng(3).uniform(-0.5, 0.5, len(s))
    with bm_ctx() as ctx:
        blob = torch.zeros(fpt.FPT_MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
        fpt.fpt_mlp_pack(ctx, v, blob)
        alpha, o = fpt.fpt_mlp_eval(ctx, blob, s, t, 50.0)
    s32 = s.astype(np.float32).astype(np.float64)
    t32 = t.astype(np.float32).astype(np.float64)
    o_ref, _ = OM.forward(p, s32, round_bf16=True)
    a_ref = OM.alpha_of(o_ref, t32, 50.0)
    scale = max(1.0, float(np.max(np.abs(o_ref))))
    err = np.abs(o - o_ref) / scale
    # bf16 operands (8 significant bits) through two 64-wide layers
    assert err.max() < 2e-2 and err.mean() < 3e-3
    assert np.max(np.abs(alpha - a_ref)) / scale < 2e-2


def test_mlp_clamp(torch):
    v, p = rand_params(4, out_scale=3.0)
    s = W.random_states(256, 5)
    t = np.zeros(len(s))
    with bm_ctx() as ctx:
        blob = torch.zeros(fpt.FPT_MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
        fpt.fpt_mlp_pack(ctx, v, blob)
        alpha, o = fpt.fpt_mlp_eval(ctx, blob, s, t, 0.25)
    assert np.all(np.abs(alpha) <= 0.25 + 1e-7)
    assert np.any(np.abs(alpha) == np.float32(0.25))


def test_mlp_gradient_matches_oracle(torch):
    """Backward kernel (bf16 tensor-core tiles, fp32 accumulation) against the
    FP64 hand-derived backward: relative L2 error <= 2e-2, cosine >= 0.999."""
    v, p = rand_params(6)
    n = 5000                                                   # 78 tiles of 64 + a ragged tail
    s = W.random_states(n, 7)
    rng = np.random.default_rng(8)
    t = rng.uniform(-0.3, 0.3, n)
    da = rng.normal(0, 1, n)
    with bm_ctx() as ctx:
        g = fpt.fpt_mlp_grad(ctx, v, s, t, da, 50.0)
    s32 = s.astype(np.float32).astype(np.float64)
    gr = OM.alpha_grad(p, s32, t.astype(np.float32).astype(np.float64), 50.0,
                       da.astype(np.float32).astype(np.float64), round_bf16=True)
    ref = fpt.canonical_params(gr).astype(np.float64)
    got = g.astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cos = float(got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref)))
    assert rel < 2e-2, rel
    assert cos > 0.999, cos
    # every parameter block is covered
    d = fpt.params_dict(got - ref)
    r = fpt.params_dict(ref)
    for k in d:
        assert np.linalg.norm(d[k]) <= 5e-2 * max(np.linalg.norm(r[k]), 1e-12), k


def test_mlp_gradient_respects_clamp(torch):
    v, p = rand_params(9, out_scale=3.0)
    s = W.random_states(512, 10)
    t = np.zeros(512)
    da = np.ones(512)
    with bm_ctx() as ctx:
        blob = torch.zeros(fpt.FPT_MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
        fpt.fpt_mlp_pack(ctx, v, blob)
        alpha, o = fpt.fpt_mlp_eval(ctx, blob, s, t, 1e-6)        # everything clamped
        g = fpt.fpt_mlp_grad(ctx, v, s, t, da, 1e-6)
    assert np.all(g == 0.0)


def test_mlp_biased_run_is_unbiased(torch):
    """Importance sampling with the learned proposal keeps E_Q[w] = 1 and
    E_Q[w N] = E_P[N] (here with random network weights)."""
    m = W.BM.model
    v, p = rand_params(11, out_scale=0.3)
    n = 1 << 15
    with bm_ctx() as ctx:
        prop = TR.new_proposal(ctx, v, shift=(0, 0, 0), scale=(20.0, 100.0, 0.2), segment=64, alpha_max=2.0)
        out = dict(nsteps=np.zeros(n, np.int32), logw=np.zeros(n), status=np.zeros(n, np.uint8))
        st = fpt.fpt_run(ctx, [prop.desc(0, n, seed=12, run_id=0)], [out])
        assert st == fpt.FPT_OK
        dout = dict(nsteps=np.zeros(n, np.int32), logw=np.zeros(n), status=np.zeros(n, np.uint8))
        fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=13, run_id=0)], [dout])
    w = np.exp(out["logw"])
    N = out["nsteps"] * m.dN
    Nd = dout["nsteps"] * m.dN
    assert abs(w.mean() - 1) < 4 * w.std() / math.sqrt(n)
    assert abs((w * N).mean() - Nd.mean()) < 4 * math.hypot((w * N).std() / math.sqrt(n), Nd.std() / math.sqrt(n))
    assert np.std(out["logw"]) > 0.01          # the proposal did act


def test_mlp_run_statistics_match_oracle(torch):
    """MLP-biased run vs the FP64 oracle with the same network (bf16 operands):
    mean first-passage time and mean log-weight within Monte Carlo error, and
    most trajectories take the identical number of steps."""
    m = W.BM.model
    v, p = rand_params(14, out_scale=0.3)
    n = 1 << 13
    shift, scale, seg, amax = (0.0, 0.0, 0.0), (20.0, 100.0, 0.2), 64, 2.0
    with bm_ctx() as ctx:
        prop = TR.new_proposal(ctx, v, shift=shift, scale=scale, segment=seg, alpha_max=amax)
        out = dict(nsteps=np.zeros(n, np.int32), logw=np.zeros(n), status=np.zeros(n, np.uint8))
        fpt.fpt_run(ctx, [prop.desc(0, n, seed=15, run_id=0)], [out])
    res = OT.resolve(m)
    tab = OT.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    mlp = OS.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, alpha_max=amax, round_bf16=True)
    o = OS.run(m, res, tab, seed=15, run_id=0, n=n, mlp=mlp)
    same = out["nsteps"] == o.nsteps
    assert same.mean() > 0.8
    se = math.hypot(np.std(o.nsteps), np.std(out["nsteps"])) / math.sqrt(n)
    assert abs(out["nsteps"].mean() - o.nsteps.mean()) < 4 * se
    sl = math.hypot(np.std(o.logw), np.std(out["logw"])) / math.sqrt(n)
    assert abs(out["logw"].mean() - o.logw.mean()) < 4 * sl
    # where the paths agree the weights agree closely
    rel = np.abs(out["logw"][same] - o.logw[same]) / np.maximum(1.0, np.abs(o.logw[same]))
    assert np.median(rel) < 1e-3


def test_training_learns_the_exponential_tilt(torch):
    """Random walk with drift -mu and diffusion s, target e^{lambda N} P: the
    zero-variance proposal is the constant Esscher tilt
    alpha* = (mu - sqrt(mu^2 - 2 lambda s^2)) / s. Training from alpha = 0 must
    cut the loss by 10x and bring alpha to alpha* along the states the paths
    visit (x ~ x0 - (mu - alpha* s) N)."""
    mu, s_, lam = W.BM_MU, W.BM_S, 9.5
    alpha_star = (mu - math.sqrt(mu * mu - 2 * lam * s_ * s_)) / s_
    v0 = fpt.canonical_params(W.mlp_init(16, out_scale=0.0))
    with bm_ctx() as ctx:
        prop = TR.new_proposal(ctx, v0, shift=(0.025, -0.01, 3.0), scale=(40.0, 100.0, 0.3),
                               segment=64, alpha_max=4.0)
        TR.train(ctx, prop, 0, rounds=120, n_traj=1 << 13, seed=17, lam=lam, N_cut=lambda r: 1e9, lr=1e-2)
        h = prop.history
        N = np.linspace(0.5, 4.5, 64)
        x = 0.05 - (mu - alpha_star * s_) * N
        st = np.stack([x, np.full(64, -mu), N], axis=1)
        sn = (st - np.array(prop.shift)) * np.array(prop.scale)
        alpha, _ = fpt.fpt_mlp_eval(ctx, prop.blob, sn, np.zeros(64), 4.0)
    assert h[-1]["loss"] < 0.1 * h[0]["loss"]
    assert abs(np.median(alpha) / alpha_star - 1) < 0.1, (np.median(alpha), alpha_star)
    assert np.all(np.abs(alpha / alpha_star - 1) < 0.3)


def test_train_select_keeps_the_best_checkpoint(torch):
    """Model selection on held-out runs: one pooled measurement (two runs)
    per checkpoint, the kept parameters are the ones with the most tail ESS
    per EM step, and running them again on the same held-out trajectories
    reproduces that figure (the blob was re-packed from the kept
    parameters)."""
    m = W.BM.model
    N_tail = 5.6
    v0 = fpt.canonical_params(W.mlp_init(16, out_scale=0.0))
    with bm_ctx() as ctx:
        prop = TR.new_proposal(ctx, v0, shift=(0.025, -0.01, 3.0), scale=(40.0, 100.0, 0.3),
                               segment=64, alpha_max=4.0)
        TR.train_select(ctx, prop, 0, rounds=60, checkpoints=[20, 40], val_traj=1 << 14, val_seed=91,
                        N_tail=N_tail, max_steps=m.max_steps, dN=m.dN, val_runs=2,
                        n_traj=1 << 13, seed=17, lam=9.5, N_cut=lambda r: 1e9, lr=1e-2)
        sel = prop.selection
        assert [v["round"] for v in sel] == [20, 40, 60]
        assert all(v["ess_tail"] > 0 and v["p_tail"] > 0 for v in sel)
        best = max(sel, key=lambda v: v["ess_per_step"])
        again = TR.tail_ess(ctx, prop, 0, 1 << 14, 91, [0, 1], N_tail, m.max_steps, m.dN)
        # the pooled figure is the ESS of the two runs' tail sums together
        one = TR.tail_ess(ctx, prop, 0, 1 << 14, 91, 0, N_tail, m.max_steps, m.dN)
        two = TR.tail_ess(ctx, prop, 0, 1 << 14, 91, 1, N_tail, m.max_steps, m.dN)
    sw = one["p_tail"] * (1 << 14) + two["p_tail"] * (1 << 14)
    sw2 = (one["p_tail"] * (1 << 14)) ** 2 / one["ess_tail"] + (two["p_tail"] * (1 << 14)) ** 2 / two["ess_tail"]
    assert again["ess_tail"] == pytest.approx(sw * sw / sw2, rel=1e-9)
    assert again["steps"] == pytest.approx(one["steps"] + two["steps"], rel=1e-12)
    assert again["ess_per_step"] == pytest.approx(best["ess_per_step"], rel=1e-9)
    assert again["steps"] == pytest.approx(best["steps"], rel=1e-12)


def test_training_is_deterministic(torch):
    """Two trainings from the same parameters on the same trajectories give
    the same network bit for bit: segment records are put in a fixed order
    (trajectory, segment) before the backward, per-block partial gradients are
    added in block order and the loss sums are reduced without atomics. The
    stepper appends the records in an order that depends on warp timing, and
    chunks of different sizes and launch shapes change it, which must not
    change the result."""
    v0 = fpt.canonical_params(W.mlp_init(16, out_scale=0.2))
    nets = []
    for block in (384, 128):
        with bm_ctx() as ctx:
            fpt.fpt_set_launch(ctx, block=block)
            prop = TR.new_proposal(ctx, v0, shift=(0.025, -0.01, 3.0), scale=(40.0, 100.0, 0.3),
                                   segment=64, alpha_max=4.0)
            TR.train(ctx, prop, 0, rounds=4, n_traj=1 << 13, seed=19, lam=9.5, N_cut=lambda r: 1e9, lr=1e-2)
            nets.append((prop.params.cpu().numpy().copy(), [h["loss"] for h in prop.history],
                         [h["grad_norm"] for h in prop.history]))
    (p1, l1, g1), (p2, l2, g2) = nets
    assert np.array_equal(p1.view(np.uint32), p2.view(np.uint32))
    assert l1 == l2 and g1 == g2
    assert not np.array_equal(p1, v0)


def test_batch_training_equals_single_runs(torch):
    """fpt_mlp_train_batch trains several networks, on different models, in
    one generation launch; each network's round equals fpt_mlp_train_round on
    its run alone (one chunk), bit for bit: the same paths, the run's records
    in the same order, the same coefficients and the same tiles."""
    from dataclasses import replace
    m0 = W.BM.model
    m1 = replace(m0, mu=0.012, pi_in=-0.012)
    S, T = np.full(16, W.BM_S), np.zeros(16)
    inits = [fpt.canonical_params(W.mlp_init(40 + k, out_scale=0.2)) for k in range(3)]
    shifts = [(0.025, -0.01, 3.0)] * 3
    scales = [(40.0, 100.0, 0.3), (30.0, 80.0, 0.3), (40.0, 100.0, 0.2)]
    models = [0, 1, 0]
    n = 3000
    with fpt.fpt_init_model([m0, m1]) as ctx:
        for i in range(2):
            fpt.fpt_noise_table(ctx, i, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, S, T)
        props, P, B = TR.new_proposals(ctx, inits, shifts, scales, segment=64, alpha_max=4.0)
        alones = [TR.new_proposal(ctx, inits[k], shift=shifts[k], scale=scales[k], segment=64, alpha_max=4.0)
                  for k in range(3)]
        moms = [(torch.zeros_like(a.params), torch.zeros_like(a.params)) for a in alones]
        for r in range(2):
            # the paths of each run in the batched launch equal the run alone
            runs = [props[k].desc(models[k], n, seed=23, run_id=r * 3 + k) for k in range(3)]
            _, together = gpu_run(ctx, runs, [n] * 3)
            for k in range(3):
                _, alone_out = gpu_run(ctx, [alones[k].desc(models[k], n, seed=23, run_id=r * 3 + k)], [n])
                assert np.array_equal(alone_out[0]["nsteps"], together[k]["nsteps"]), (r, k, "paths")
                assert np.array_equal(alone_out[0]["logw"], together[k]["logw"]), (r, k, "paths")
            hist = TR.train_batch(ctx, props, P, B, models, rounds=1, n_traj=n, seed=23, lam=9.5,
                                  N_cuts=[1e9, 1e9, 1e9], lr=1e-2, first_round=r)
            got = P.cpu().numpy().copy()
            for k in range(3):
                run = alones[k].desc(models[k], n, seed=23, run_id=r * 3 + k)
                st = fpt.fpt_mlp_train_round(ctx, run, n, 9.5, 1e9, dict(lr=1e-2, step=r + 1), alones[k].params,
                                             moms[k][0], moms[k][1], alones[k].blob)
                assert st["n_records"] == hist[0][k]["n_records"], (r, k)
                assert st["loss"] == pytest.approx(hist[0][k]["loss"], rel=1e-12), (r, k)
                assert np.array_equal(alones[k].params.cpu().numpy().view(np.uint32), got[k].view(np.uint32)), (r, k)
    assert not np.array_equal(got[0], got[2])


def test_records_with_a_deadline_are_unaffected(torch):
    """A launch with a deadline keeps its clock origin in its own flag words:
    a record-mode run under a (generous) deadline returns the same records
    and outputs as one without, and no record-overflow error."""
    v, p = rand_params(11, out_scale=0.3)
    n = 512
    with bm_ctx() as ctx:
        prop = TR.new_proposal(ctx, v, shift=(0, 0, 0), scale=(20.0, 100.0, 0.2), segment=64, alpha_max=2.0)
        ref = fpt.fpt_run_records(ctx, prop.desc(0, n, seed=21, run_id=0), cap=1 << 16)
        fpt.fpt_set_launch(ctx, deadline_s=60.0)
        rec = fpt.fpt_run_records(ctx, prop.desc(0, n, seed=21, run_id=0), cap=1 << 16)
        st, g = gpu_run(ctx, [prop.desc(0, n, seed=21, run_id=0)], [n])
        assert st == fpt.FPT_OK
        fpt.fpt_set_launch(ctx, deadline_s=0.0)
        st, g0 = gpu_run(ctx, [prop.desc(0, n, seed=21, run_id=0)], [n])
    assert rec["n_records"] == ref["n_records"] > 0
    for k in ("in", "raw", "sum_xi", "unit", "n0"):
        assert np.array_equal(rec[k], ref[k]), k
    for k in ("nsteps", "logw", "status"):
        assert np.array_equal(g[0][k], g0[0][k]), k
