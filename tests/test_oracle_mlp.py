"""Pins of the FP64 learned-proposal reference: finite differences and the
two independent forward implementations (numpy, C)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mlp as M
from oracle import stepper as S
from oracle import tables as T


def _params(seed=3, out_scale=0.3):
    return W.mlp_init(seed, out_scale=out_scale)


def test_backward_matches_finite_differences():
    p = _params()
    s = W.random_states(7, 1)
    t = np.linspace(-0.2, 0.3, 7)
    da = np.linspace(-1.0, 1.0, 7)
    g = M.alpha_grad(p, s, t, 50.0, da)
    f = lambda q: float(np.sum(da * M.alpha_of(M.forward(q, s)[0], t, 50.0)))
    rng = np.random.default_rng(0)
    for k in M.KEYS:
        for _ in range(4):
            idx = tuple(rng.integers(0, d) for d in p[k].shape)
            h = 1e-6
            q = {kk: v.copy() for kk, v in p.items()}
            q[k][idx] += h
            fp = f(q)
            q[k][idx] -= 2 * h
            fm = f(q)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_c_and_numpy_forward_agree():
    p = _params()
    mlp = S.MLPBias(p, segment=64, in_shift=[0.1, -0.2, 0.3], in_scale=[2.0, 0.5, 1.5],
                    round_bf16=False)
    for s in W.random_states(5, 2):
        oc = S.mlp_forward_c(mlp, s)
        on, _ = M.forward(p, M.normalise(s[None, :], [0.1, -0.2, 0.3], [2.0, 0.5, 1.5]))
        np.testing.assert_allclose(oc, on[0], rtol=1e-12, atol=1e-14)


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: the spacing just above 1 is 2^-7
    v = np.array([1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 1.0 + 3 * 2 ** -8, -3.14159])
    r = M.bf16(v)
    assert r[0] == 1.0                       # tie -> even (mantissa 0)
    assert r[1] == 1.0                       # below half
    assert r[2] == 1.0 + 2 ** -7             # above half
    assert r[3] == 1.0 + 2 ** -6             # tie -> even (mantissa 2)
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)


def test_log_variance_gradient_by_finite_differences():
    """dL/dtheta from the segment records equals the finite-difference
    derivative of Var[ln w_theta + lambda N] over the same recorded paths."""
    wl = W.BM
    m = wl.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    p = _params(out_scale=0.2)
    shift, scale = [0.0, 0.0, 0.0], [20.0, 100.0, 0.2]
    seg = 64
    mlp = S.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, round_bf16=False)
    trajs = [S.run_segments(m, res, tab, mlp, seed=5, run_id=0, traj=j) for j in range(24)]
    lam = 0.3
    loss, g = M.logvar_loss_grad(p, trajs, m.dN, lam, shift, scale, 20.0)
    # recorded ln w equals the off-policy formula at the sampling parameters
    for tr in trajs:
        assert M.logw_at(p, tr, m.dN, shift, scale, 20.0, seg) == pytest.approx(tr["logw"], rel=1e-9, abs=1e-9)

    def L(q):
        Y = np.array([M.logw_at(q, tr, m.dN, shift, scale, 20.0, seg) + lam * tr["nsteps"] * m.dN
                      for tr in trajs])
        return float(np.mean((Y - Y.mean()) ** 2))

    assert L(p) == pytest.approx(loss, rel=1e-9)
    rng = np.random.default_rng(4)
    for k in M.KEYS:
        for _ in range(3):
            idx = tuple(rng.integers(0, d) for d in p[k].shape)
            h = 1e-6
            q = {kk: v.copy() for kk, v in p.items()}
            q[k][idx] += h
            fp = L(q)
            q[k][idx] -= 2 * h
            fd = (fp - L(q)) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9


def test_log_variance_gradient_2d_by_finite_differences():
    """2-D noise (Eq. 4.5 with B = S beta): dL/dtheta from the two noise sums
    per segment equals the finite-difference derivative of
    Var[ln w_theta + lambda N] over the same recorded full-rank paths, and the
    recorded ln w equals the off-policy formula at the sampling parameters."""
    m = W.BM.model
    res = T.resolve(m)
    tab = T.user_table2(np.full(16, 1e-3), np.full(16, 3e-4), np.full(16, 5e-4), -0.1, 0.2)
    p = _params(out_scale=0.2)
    shift, scale = [0.0, 0.0, 0.0], [20.0, 100.0, 0.2]
    seg = 64
    mlp = S.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, alpha_max=0.05, round_bf16=False)
    trajs = [S.run2_segments(m, res, tab, mlp, seed=6, run_id=0, traj=j) for j in range(24)]
    lam = 0.3
    loss, g = M.logvar_loss_grad2(p, trajs, m.dN, lam, shift, scale, 0.05)
    for tr in trajs:
        assert M.logw_at2(p, tr, m.dN, shift, scale, 0.05, seg) == pytest.approx(tr["logw"], rel=1e-9, abs=1e-9)
    assert any(np.any(np.abs(tr["beta"]) == 0.05) for tr in trajs)      # the clamp is exercised

    def L(q):
        Y = np.array([M.logw_at2(q, tr, m.dN, shift, scale, 0.05, seg) + lam * tr["nsteps"] * m.dN
                      for tr in trajs])
        return float(np.mean((Y - Y.mean()) ** 2))

    assert L(p) == pytest.approx(loss, rel=1e-9)
    rng = np.random.default_rng(5)
    for k in M.KEYS:
        for _ in range(3):
            idx = tuple(rng.integers(0, d) for d in p[k].shape)
            h = 1e-8      # small: no output may cross the clamp within the difference
            q = {kk: v.copy() for kk, v in p.items()}
            q[k][idx] += h
            fp = L(q)
            q[k][idx] -= 2 * h
            fd = (fp - L(q)) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-7


@pytest.mark.parametrize("round_bf16", [False, True])
def test_log_field_input_rebuilt_from_the_random_walk(round_bf16):
    """The ln x input of the learned proposal (FPT_MLP_LOG_X), pinned on the
    exponential model, where the field is an exact Gaussian random walk: with
    the recorded alpha of each held segment, x_n = x_0 + sum_i (-mu + alpha_s s)
    dN + s sqrt(dN) xi_i rebuilds the path from the Philox stream alone. At
    every segment start the recorded network input must be ln of that x (the
    natural log of phi - phi_end, not of phi, not x itself), and the recorded
    alpha must be the numpy network's clamped projection at (ln x, pi, N).
    A network with large input weights on ln x makes alpha move with it."""
    wl = W.BM
    m = wl.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    p = _params(seed=9, out_scale=0.5)
    x_in = m.phi_in - m.phi_end
    shift, scale, seg, amax = [math.log(x_in), -W.BM_MU, 0.0], [2.0, 50.0, 0.2], 32, 0.4
    mlp = S.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, alpha_max=amax,
                    round_bf16=round_bf16, log_x=True)
    sdN = math.sqrt(m.dN)
    clamped = 0
    for j in range(6):
        tr = S.run_segments(m, res, tab, mlp, seed=23, run_id=1, traj=j)
        n = tr["nsteps"]
        xi = np.concatenate([S.normals4(23, 1, j, b) for b in range((n + 3) // 4)])[:n]
        alpha = np.repeat(tr["alpha"], seg)[:n]
        x = x_in + np.concatenate([[0.0], np.cumsum((-W.BM_MU + alpha * W.BM_S) * m.dN + W.BM_S * sdN * xi)])
        starts = np.arange(0, n, seg)
        assert len(starts) == len(tr["alpha"])
        # (the rebuilt sum rounds differently from the step-by-step field: 1e-10 of x)
        np.testing.assert_allclose(tr["state"][:, 0], np.log(x[starts]), rtol=0, atol=1e-8)
        np.testing.assert_allclose(tr["state"][:, 1], -W.BM_MU, rtol=0, atol=0)
        np.testing.assert_allclose(tr["state"][:, 2], starts * m.dN, rtol=1e-15, atol=0)
        s = M.normalise(np.stack([np.log(x[starts]), np.full(len(starts), -W.BM_MU), starts * m.dN], 1),
                        shift, scale)
        o, _ = M.forward(p, s, round_bf16)
        a = M.alpha_of(o, np.zeros(len(starts)), amax)
        np.testing.assert_allclose(tr["alpha"], a, rtol=1e-7, atol=1e-9)
        clamped += int(np.sum(np.abs(a) >= amax))
        # the input really is the log: alpha taken at x itself would differ
        s_lin = M.normalise(np.stack([x[starts], np.full(len(starts), -W.BM_MU), starts * m.dN], 1),
                            shift, scale)
        assert np.max(np.abs(M.alpha_of(M.forward(p, s_lin, round_bf16)[0], np.zeros(len(starts)), amax) - a)) > 1e-3
    assert clamped > 0
