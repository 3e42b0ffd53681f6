"""Pins of the full-rank (2-D) noise oracle: numerical matching (Eq. 3.9),
the symmetric square root S of Xi, and the 2-D stepper with the weight of
Eq. (4.5) for a standardised bias B = S beta."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import stats

import workloads as W
from oracle import stepper as S
from oracle import tables as T

SIEGMUND = 0.5826


def test_sqrt_psd2_squares_to_xi():
    """S symmetric, positive semi-definite and S S = Xi, including the singular
    (rank-1) and diagonal cases."""
    rng = np.random.default_rng(0)
    cases = [(1.0, 0.0, 0.0), (2.0, 0.0, 3.0), (1.0, -2.0, 4.0), (1e-12, 3e-12, 9e-12)]
    for _ in range(50):
        L = rng.normal(size=(2, 2))
        X = L @ L.T
        cases.append((X[0, 0], X[0, 1], X[1, 1]))
    for a, b, c in cases:
        p, q, r = T.sqrt_psd2(a, b, c)
        Sm = np.array([[p, q], [q, r]])
        X = np.array([[a, b], [b, c]])
        assert np.allclose(Sm @ Sm, X, rtol=1e-12, atol=1e-14 * max(a, c))
        assert p >= 0 and r >= 0 and p * r - q * q >= -1e-12 * max(a, c)


@pytest.fixture(scope="module")
def desitter():
    """No kink (a_- = a_+ = 1e-3): nu = 3/2 to O(eps), massless de Sitter modes."""
    m = dataclasses.replace(W.USR_MODEL, a_minus=W.USR_MODEL.a_plus, n_in=1.0, n_end=3.0)
    return m, T.resolve(m)


@pytest.mark.parametrize("sigma", [1.0, 0.3])
def test_numerical_matching_de_sitter_closed_form(desitter, sigma):
    """Massless de Sitter Bunch-Davies mode at -k eta = sigma:
    delta phi = H/sqrt(2k^3) (1 - i sigma) e^{i sigma}, delta pi = -H/sqrt(2k^3) sigma^2 e^{i sigma},
    so Xi of Eq. (3.9) is (H/2pi)^2 [[1 + sigma^2, -sigma^2], [-sigma^2, sigma^4]]."""
    m, r = desitter
    for ph in (r.phi_in, 0.5 * (r.phi_in + r.phi_end)):
        xpp, xpq, xqq, a, H, k = T.xi_numeric_at_phi(m, r, ph, sigma)
        P = (H / (2 * math.pi)) ** 2
        assert xpp / P == pytest.approx(1 + sigma ** 2, abs=1e-3)
        assert xpq / P == pytest.approx(-sigma ** 2, abs=1e-3)
        assert xqq / P == pytest.approx(sigma ** 4, abs=1e-3 * sigma ** 2)


@pytest.mark.parametrize("sigma", [1.0, 0.3])
def test_numerical_matching_determinant_is_wronskian(sigma):
    """det Xi = (k^3/2pi^2)^2 (Im dphi* dpi)^2, and the Wronskian a^3 H Im(dphi* dpi)
    = -1/2 of the Bunch-Davies mode (|dphi|^2 = 1/(2k a^2), dpi = -i k/(aH) dphi)
    is conserved, through the kink too (the jump in dpi is proportional to dphi):
    det Xi = (k^3/2pi^2)^2 / (4 a^6 H^2), exactly, at any phi of the USR model."""
    m = W.USR_MODEL
    r = T.resolve(m)
    for ph in (r.phi_in, 0.5 * (r.phi_in + r.phi_end), r.phi_end):
        xpp, xpq, xqq, a, H, k = T.xi_numeric_at_phi(m, r, ph, sigma)
        det = xpp * xqq - xpq * xpq
        pred = (k ** 3 / (2 * math.pi ** 2)) ** 2 / (4 * a ** 6 * H ** 2)
        assert det / pred == pytest.approx(1.0, abs=1e-6)


def test_numerical_matching_after_kink_departs_from_growing_mode():
    """Just after the sudden transition the full mode carries the decaying
    solution: dpi ~ -3 dphi (the kink kicks d(dphi)/dN by -3 dphi for
    a_+ >> a_-), so Xi_phipi / Xi_phiphi ~ -3 while the growing mode alone has
    tan theta = nu - 3/2 ~ 0 (Sec. 3.3: the noise there is genuinely 2-D)."""
    m = W.USR_MODEL
    r = T.resolve(m)
    xpp, xpq, xqq, a, H, k = T.xi_numeric_at_phi(m, r, r.phi_in, 0.1)
    assert -3.3 < xpq / xpp < -2.7
    nm = T.noise_at_phi(m, r, r.phi_in, 0.1)
    assert abs(nm.T / nm.S) < 1e-5


# ---------------------------------------------------------------------------
# 2-D stepper
# ---------------------------------------------------------------------------
def _bm2(a, b, c, n, seed, A=0.0, A2=0.0, mlp=None, model=None):
    m = model or W.BM.model
    res = T.resolve(m)
    tab = T.user_table2(np.full(16, a), np.full(16, b), np.full(16, c), -0.1, 0.2)
    return m, res, S.run2(m, res, tab, seed=seed, run_id=0, n=n, A=A, A2=A2, mlp=mlp)


def test_2d_walk_uses_the_documented_normals():
    """S = diag(s, 0): pi = -mu stays fixed and phi is a Gaussian walk driven by
    normal 2(i & 1) of Philox block i >> 1, with bias s beta_1 (beta_2 moves nothing)."""
    s, b1, b2 = W.BM_S, 0.7, 0.4
    m, res, tr = _bm2(s, 0.0, 0.0, 64, W.BM.seed, A=b1, A2=b2)
    sdN = math.sqrt(m.dN)
    for j in range(64):
        n = int(tr.nsteps[j])
        z = np.concatenate([S.normals4(W.BM.seed, 0, j, q) for q in range((n + 1) // 2)])
        xi1 = z.reshape(-1, 2)[:, 0][:n]
        path = m.phi_in + np.cumsum((-W.BM_MU + b1 * s) * m.dN + s * sdN * xi1)
        assert abs(tr.phi_final[j] - path[-1]) < 1e-12
        assert tr.pi_final[j] == -W.BM_MU
        assert path[-1] <= 0.0 and np.all(path[:-1] > 0.0)


def test_2d_log_weight_identity():
    """beta = (A, 0), S = diag(s, 0): ln w = A^2 N/2 - (A/s)(x_n - x_0 + mu N)."""
    A = 0.9
    m, res, tr = _bm2(W.BM_S, 0.0, 0.0, 2048, 3, A=A)
    N = tr.N
    pred = 0.5 * A * A * N - (A / W.BM_S) * (tr.phi_final - m.phi_in + W.BM_MU * N)
    assert np.all(np.abs(tr.logw - pred) <= 1e-9 * np.maximum(1, np.abs(pred)))


def test_2d_inverse_gaussian_law():
    """S = [[s, 0], [0, 0]]: the first-passage law of the drifted walk (inverse
    Gaussian with the discrete-monitoring shift)."""
    m, res, tr = _bm2(W.BM_S, 0.0, 0.0, 1 << 15, 5)
    a = m.phi_in - m.phi_end + SIEGMUND * W.BM_S * math.sqrt(m.dN)
    mean, lam = a / W.BM_MU, a * a / W.BM_S ** 2
    assert stats.kstest(tr.N, stats.invgauss(mu=mean / lam, scale=lam).cdf).pvalue > 1e-3


@pytest.mark.parametrize("beta", [(0.6, -0.8), (0.0, 1.2)])
def test_2d_importance_sampling_identity(beta):
    """Full-rank constant S: E_Q[w] = 1, E_Q[w N] = E_P[N], E_Q[w N^2] = E_P[N^2]
    (Eq. 4.5 is the likelihood ratio of the Gaussian steps; a dropped term of
    beta . (beta dN/2 + xi sqrt(dN)) biases all three)."""
    a, b, c = 1e-3, 3e-4, 5e-4
    m, _, direct = _bm2(a, b, c, 1 << 15, 21)
    _, _, tr = _bm2(a, b, c, 1 << 15, 22, A=beta[0], A2=beta[1])
    assert (direct.status == 0).all() and (tr.status == 0).all()
    w = np.exp(tr.logw)
    n = len(w)
    for f, g in [(np.ones(n), np.ones(len(direct.N))), (tr.N, direct.N), (tr.N ** 2, direct.N ** 2)]:
        est, se = np.mean(w * f), np.std(w * f) / math.sqrt(n)
        ref, se_ref = np.mean(g), np.std(g) / math.sqrt(len(g))
        assert abs(est - ref) < 4 * math.hypot(se, se_ref)
    # the bias really moved the sample: a different law under Q
    assert stats.ks_2samp(tr.N, direct.N).pvalue < 1e-6


def test_2d_rank_one_noise_reduces_to_1d_in_law():
    """Xi = s^2 (1, t)(1, t)^T has S = s/sqrt(1+t^2) (1,t)(1,t)^T; with
    beta = A (1, t)/sqrt(1+t^2) the 2-D step is the 1-D step of Eq. (4.7) driven
    by xi = (xi_1 + t xi_2)/sqrt(1+t^2) and the weights agree step by step, so the
    2-D and 1-D samplers give the same joint law of (N, ln w)."""
    s, t, A = 3e-3, -0.5, 0.6
    m = W.LINEAR.model
    res = T.resolve(m)
    n = 1 << 15
    one = T.user_table(np.full(16, s), np.full(16, t * s), -0.1, 0.2)
    tr1 = S.run(m, res, one, seed=31, run_id=0, n=n, A=A)
    k = s / math.sqrt(1 + t * t)
    two = T.user_table2(np.full(16, k), np.full(16, k * t), np.full(16, k * t * t), -0.1, 0.2)
    u = A / math.sqrt(1 + t * t)
    tr2 = S.run2(m, res, two, seed=32, run_id=0, n=n, A=u, A2=u * t)
    assert stats.ks_2samp(tr1.N, tr2.N).pvalue > 1e-3
    assert stats.ks_2samp(tr1.logw, tr2.logw).pvalue > 1e-3
    q = np.quantile(tr1.N, 0.9)
    e1 = np.exp(tr1.logw) * (tr1.N > q)
    e2 = np.exp(tr2.logw) * (tr2.N > q)
    assert abs(e1.mean() - e2.mean()) < 4 * math.hypot(e1.std(), e2.std()) / math.sqrt(n)


def test_2d_mlp_with_constant_output_is_constant_bias():
    """An MLP whose last layer is zero outputs its bias b3 exactly: beta = b3
    (clamped to +-alpha_max) reproduces the constant-bias run bit for bit."""
    rng = np.random.default_rng(1)
    H = 64
    p = dict(W1=rng.normal(size=(H, 3)), b1=rng.normal(size=H), W2=rng.normal(size=(H, H)) / 8,
             b2=rng.normal(size=H), W3=np.zeros((2, H)), b3=np.array([0.6, -0.8]))
    a, b, c = 1e-3, 3e-4, 5e-4
    for amax, beta in ((5.0, (0.6, -0.8)), (0.5, (0.5, -0.5))):
        mlp = S.MLPBias(p, segment=8, in_shift=[0, 0, 0], in_scale=[1, 1, 1], alpha_max=amax)
        _, _, t1 = _bm2(a, b, c, 256, 7, mlp=mlp)
        _, _, t2 = _bm2(a, b, c, 256, 7, A=beta[0], A2=beta[1])
        assert np.array_equal(t1.nsteps, t2.nsteps)
        assert np.array_equal(t1.logw, t2.logw)
