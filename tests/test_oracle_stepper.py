"""Pins of the FP64 oracle stepper against closed forms, exact identities and
the noise-free classical limit."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import workloads as W
from oracle import estimators as E
from oracle import stepper as S
from oracle import tables as T

SIEGMUND = 0.5826  # -zeta(1/2)/sqrt(2 pi): mean overshoot of a Gaussian walk in step-std units


def _bm(A=0.0, n=1 << 16, seed=11):
    wl = W.BM
    m = wl.model
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    return m, res, tab, S.run(m, res, tab, seed=seed, run_id=0, n=n, A=A)


def test_bm_walk_is_exact_gaussian_random_walk():
    """pi = -mu is a fixed point, so phi_n = phi_0 + n(-mu + A s) dN + s sqrt(dN) sum xi."""
    m, res, tab, tr = _bm(A=0.7, n=64)
    sdN = math.sqrt(m.dN)
    for j in range(64):
        n = int(tr.nsteps[j])
        xi = np.concatenate([S.normals4(W.BM.seed, 0, j, b) for b in range((n + 3) // 4)])[:n]
        phi = m.phi_in + n * (-W.BM_MU + 0.7 * W.BM_S) * m.dN + W.BM_S * sdN * xi.sum()
        assert abs(tr.phi_final[j] - phi) < 1e-12
        assert tr.pi_final[j] == -W.BM_MU
        # the walk was above the end surface before step n and at/below it at n
        path = m.phi_in + np.cumsum((-W.BM_MU + 0.7 * W.BM_S) * m.dN + W.BM_S * sdN * xi)
        assert path[-1] <= 0.0 and np.all(path[:-1] > 0.0)


def test_bm_log_weight_identity():
    """ln w = A^2 N/2 - (A/s)(x_n - x_0 + mu N), exact for the random walk."""
    A = 0.9
    m, res, tab, tr = _bm(A=A, n=2048)
    N = tr.N
    pred = 0.5 * A * A * N - (A / W.BM_S) * (tr.phi_final - m.phi_in + W.BM_MU * N)
    assert np.all(np.abs(tr.logw - pred) <= 1e-9 * np.maximum(1, np.abs(pred)))


def test_bm_mean_wald_siegmund():
    """Wald: mu E[N] = a + E[overshoot]; overshoot -> 0.5826 s sqrt(dN)."""
    m, res, tab, tr = _bm()
    a = m.phi_in - m.phi_end
    pred = (a + SIEGMUND * W.BM_S * math.sqrt(m.dN)) / W.BM_MU
    se = tr.N.std() / math.sqrt(len(tr.N))
    assert abs(tr.N.mean() - pred) < 4 * se
    # and the raw continuous-time mean a/mu is off by more than the shift allows for
    assert (tr.status == 0).all()


def test_bm_inverse_gaussian_law():
    """First-passage law of Brownian motion with drift: inverse Gaussian with
    mean a'/mu and shape a'^2/s^2, a' = a + 0.5826 s sqrt(dN) (discrete monitoring)."""
    m, res, tab, tr = _bm()
    a = m.phi_in - m.phi_end + SIEGMUND * W.BM_S * math.sqrt(m.dN)
    mean, lam = a / W.BM_MU, a * a / W.BM_S ** 2
    ig = stats.invgauss(mu=mean / lam, scale=lam)
    assert stats.kstest(tr.N, ig.cdf).pvalue > 1e-3
    assert abs(tr.N.var() - mean ** 3 / lam) < 5 * mean ** 3 / lam * math.sqrt(2.0 / len(tr.N)) * 1.5


@pytest.mark.parametrize("A", [0.5, 1.0])
def test_importance_sampling_identity(A):
    """E_Q[w] = 1, E_Q[w N] = E_P[N], E_Q[w N^2] = E_P[N^2] (likelihood ratio
    of Gaussian steps with a bounded stopping time)."""
    m, res, tab, direct = _bm(n=1 << 15, seed=21)
    _, _, _, tr = _bm(A=A, n=1 << 15, seed=22)
    w = np.exp(tr.logw)
    n = len(w)
    for f, g in [(np.ones(n), np.ones(len(direct.N))), (tr.N, direct.N), (tr.N ** 2, direct.N ** 2)]:
        est, se = np.mean(w * f), np.std(w * f) / math.sqrt(n)
        ref, se_ref = np.mean(g), np.std(g) / math.sqrt(len(g))
        assert abs(est - ref) < 4 * math.hypot(se, se_ref)


def test_linear_slow_roll_inverse_gaussian():
    """Slow-roll linear case: N ~ IG with mean ~ 5.0029 and variance ~ 0.0422."""
    wl = W.LINEAR
    m = wl.model
    res = T.resolve(m)
    assert abs(res.pi_in - (-0.0099950)) < 1e-7
    tab = T.desitter_table(m, res, 4096, wl.table.phi_lo, wl.table.phi_hi)
    tr = S.run(m, res, tab, seed=wl.seed, run_id=0, n=wl.n_traj)
    assert (tr.status == 0).all()
    se = tr.N.std() / math.sqrt(len(tr.N))
    assert abs(tr.N.mean() - 5.0029) < 4 * se
    assert abs(tr.N.var() - 0.04225) < 4 * 4.7e-4


def _euler_noise_free(m, res, dN):
    phi, pi, n = res.phi_in, res.pi_in, 0
    while True:
        phi, pi = phi + pi * dN, pi - (3 - 0.5 * pi * pi) * (pi + T.dlnV(m, phi)) * dN
        n += 1
        if phi <= res.phi_end:
            return n * dN


def test_noise_off_limit_is_classical():
    """S = 0: every trajectory is the deterministic Euler solution, within 2 dN
    of the ODE's event time, with first-order convergence in dN."""
    wl = W.LINEAR
    m = wl.model
    res = T.resolve(m)
    tab0 = T.user_table(np.zeros(8), np.zeros(8), 0.0, 0.06)
    tr = S.run(m, res, tab0, seed=0, run_id=0, n=16)
    assert np.all(tr.nsteps == tr.nsteps[0]) and np.all(tr.logw == 0)
    rhs = lambda N, y: [y[1], -(3 - 0.5 * y[1] ** 2) * (y[1] + T.dlnV(m, y[0]))]
    ev = lambda N, y: y[0] - res.phi_end
    ev.terminal = True
    s = integrate.solve_ivp(rhs, (0, 20), [res.phi_in, res.pi_in], method="DOP853",
                            rtol=1e-12, atol=1e-15, events=ev)
    N_ode = float(s.t_events[0][0])
    assert abs(tr.N[0] - N_ode) <= 2 * m.dN
    assert abs(N_ode - 5.00125) < 2e-3          # slow-roll closed form (phi + A phi^2/2)/A
    assert tr.N[0] == pytest.approx(_euler_noise_free(m, res, m.dN), abs=1e-12)
    errs = [abs(_euler_noise_free(m, res, dN) - N_ode) for dN in (4e-3, 2e-3, 1e-3)]
    assert errs[2] < errs[0]


def test_cap_censors_and_reports():
    wl = W.BM
    m = W.BM.model.__class__(**{**W.BM.model.__dict__, "max_steps": 1000})
    res = T.resolve(m)
    tab = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    tr = S.run(m, res, tab, seed=1, run_id=0, n=32)
    assert np.all(tr.status == 1) and np.all(tr.nsteps == 1000)


def test_near_tie_diagnostics():
    m, res, tab, tr = _bm(n=256)
    assert np.all(tr.phi_final <= 0.0)
    assert np.all((tr.xmin_pre > 0) | (tr.nsteps == 1))


def test_noise_window_random_walk_identity():
    """N-indexed noise with a window (noise on for N in [0, N_w], then the
    classical completion): on the exponential model every path satisfies
    phi_n = phi_0 - mu n dN + s sqrt(dN) sum_{i < n, i dN <= N_w} xi_i exactly."""
    m = W.BM.model
    res = T.resolve(m)
    Nw = 2.0
    tab = T.user_table_N(np.full(16, W.BM_S), np.zeros(16), 0.0, Nw)
    tr = S.run(m, res, tab, seed=9, run_id=0, n=200)
    sdN = math.sqrt(m.dN)
    late = 0
    for j in range(200):
        n = int(tr.nsteps[j])
        xi = np.concatenate([S.normals4(9, 0, j, b) for b in range((n + 3) // 4)])[:n]
        on = np.arange(n) <= math.floor(Nw / m.dN + 1e-9)     # integer window of steps
        phi = m.phi_in - n * W.BM_MU * m.dN + W.BM_S * sdN * xi[on].sum()
        assert abs(tr.phi_final[j] - phi) < 1e-12
        late += n * m.dN > Nw
    assert late > 150          # most paths finish after the window, classically
    # after the window the remaining field falls by exactly mu dN per step
    full = T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2)
    tr_full = S.run(m, res, full, seed=9, run_id=0, n=200)
    assert not np.array_equal(tr.nsteps, tr_full.nsteps)


def test_noise_window_covering_the_run_equals_phi_indexed():
    m = W.BM.model
    res = T.resolve(m)
    a = S.run(m, res, T.user_table_N(np.full(16, W.BM_S), np.zeros(16), 0.0, 100.0), seed=3, run_id=0, n=256)
    b = S.run(m, res, T.user_table(np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2), seed=3, run_id=0, n=256)
    assert np.array_equal(a.nsteps, b.nsteps) and np.array_equal(a.logw, b.logw)


def test_noise_window_weight_acts_only_on_noisy_steps():
    """Outside the window the step is classical: no noise, no bias and no
    weight change, so ln w = -sum over window steps of A (A dN/2 + xi sqrt(dN))."""
    m = W.BM.model
    res = T.resolve(m)
    A, Nw = 0.8, 1.5
    tab = T.user_table_N(np.full(16, W.BM_S), np.zeros(16), 0.25, Nw)
    tr = S.run(m, res, tab, seed=10, run_id=0, n=100, A=A)
    sdN = math.sqrt(m.dN)
    lo, hi = math.ceil(0.25 / m.dN - 1e-9), math.floor(Nw / m.dN + 1e-9)
    for j in range(100):
        n = int(tr.nsteps[j])
        xi = np.concatenate([S.normals4(10, 0, j, b) for b in range((n + 3) // 4)])[:n]
        idx = np.arange(n)
        win = (idx >= lo) & (idx <= hi)
        lw = -np.sum(A * (0.5 * A * m.dN + xi[win] * sdN))
        assert abs(tr.logw[j] - lw) < 1e-9 * max(1.0, abs(lw))
        phi = m.phi_in - n * W.BM_MU * m.dN + np.sum(W.BM_S * (A * m.dN + sdN * xi[win]))
        assert abs(tr.phi_final[j] - phi) < 1e-12
