"""Pins of the Gaussian-bump model (Sec. 4.3) in the FP64 oracle: the
potential's derivatives, the onset of ultra-slow roll, the mode equation
(time-translation mode and Wronskian), the V0 normalisation, the consistency
relation of the Bessel-matched noise, the noise-off limit of the stepper and
the importance-sampling identity."""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import stepper as S
from oracle import tables as T

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bump():
    m = W.BUMP_MODEL
    return m, T.resolve(m)


def test_bump_potential_derivatives():
    """V'/V and V''/V against central differences of V itself."""
    m = W.BUMP_MODEL
    for phi in (2.15, 2.18812, 2.2031, 2.21, 2.3, 2.6):
        h = 1e-4
        V = [T.V_of(m, phi + j * h) for j in (-2, -1, 0, 1, 2)]
        d1 = (V[0] - 8 * V[1] + 8 * V[3] - V[4]) / (12 * h) / V[2]
        d2 = (-V[0] + 16 * V[1] - 30 * V[2] + 16 * V[3] - V[4]) / (12 * h * h) / V[2]
        assert T.dlnV(m, phi) == pytest.approx(d1, rel=1e-7, abs=1e-10)
        assert T.d2V_over_V(m, phi) == pytest.approx(d2, rel=1e-5, abs=1e-6)


def test_bump_ultra_slow_roll_onset(bump):
    """N_T is the first time eps2 = 2 pi'/pi reaches -3; the phase lasts until
    eps2 climbs back through -3, about 2.4 e-folds later."""
    m, r = bump
    bg = r.bg

    def eps2(N):
        ph, pi, br = bg.state(N)
        return T.flow(m, ph, pi, br)[1]

    assert eps2(r.N_T) == pytest.approx(-3.0, abs=1e-8)
    assert all(eps2(N) > -3.0 for N in np.linspace(0.0, r.N_T - 1e-3, 200))
    later = np.linspace(r.N_T + 0.05, r.N_T + 3.0, 600)
    e = np.array([eps2(N) for N in later])
    end = later[np.argmax(e > -3.0)]
    assert 2.3 < end - r.N_T < 2.5
    assert e.min() < -6.0                     # a genuine ultra-slow-roll phase


def test_bump_superhorizon_mode_is_time_translation(bump):
    """For k -> 0 the mode equation (Eq. 2.4 with V''/V of the bump) is solved
    exactly by delta phi = pi, the time shift of the background: started as
    (pi, pi') the mode stays equal to pi through the whole transition. A wrong
    V''/V or mass term breaks this."""
    m, r = bump
    bg = r.bg
    N0, N1 = r.N_T - 1.0, r.N_T + 5.0
    ph0, pi0, _ = bg.state(N0)
    dpi0 = T.flow(m, ph0, pi0, None)[3]
    k = 1e-12 * math.exp(N0) * T.hubble(m, ph0, pi0)
    for N in (r.N_T, r.N_T + 1.5, N1):
        u, du, _ = T.evolve_mode(m, bg, k, N0, N, complex(pi0), complex(dpi0))
        ph, pi, _ = bg.state(N)
        assert u.real / pi == pytest.approx(1.0, abs=1e-7)
        assert du.real / T.flow(m, ph, pi, None)[3] == pytest.approx(1.0, abs=1e-6)


def test_bump_wronskian_conserved(bump):
    m, r = bump
    bg = r.bg
    Ns = r.N_T + 1.5
    ph, pi, _ = bg.state(Ns)
    k = math.exp(Ns) * T.hubble(m, ph, pi)
    N0 = Ns - math.log(100.0)
    ws = []
    for N1 in (N0 + 1.0, r.N_T, Ns, r.N_T + 4.0):
        _, _, y = T.mode_at(m, bg, k, N0, N1)
        ws.append(T.wronskian(m, N1, y, None))
    assert np.allclose(ws, ws[0], rtol=1e-8)


def test_bump_v0_normalisation():
    """V0 makes the linear power spectrum peak at 5e-3 (bump_v0.json)."""
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_bump_v0.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "golden", "bump_v0.json")) as f:
        g = json.load(f)
    assert W.BUMP_V0 == pytest.approx(g["V0"], rel=1e-5)
    m = W.BUMP_MODEL
    r = T.resolve(m)
    d = g["peak_crossing_after_N_T"]
    p = mk.power_spectrum(m, r, d)
    assert p == pytest.approx(5e-3, rel=1e-5)
    assert mk.power_spectrum(m, r, d - 0.1) < p and mk.power_spectrum(m, r, d + 0.1) < p


@pytest.mark.parametrize("frac", [0.0, 0.5, 1.0])
def test_bump_consistency_relation(bump, frac):
    """Eq. (3.1) for the Bessel-matched growing mode at sigma = 1 across the
    simulated range (the paper's criterion for choosing the mode range)."""
    m, r = bump
    ph = r.phi_in + frac * (r.phi_end - r.phi_in)
    assert T.consistency_ratio(m, r, ph, 1.0) == pytest.approx(1.0, abs=0.025)


def test_bump_noise_angle_is_nontrivial(bump):
    """nu varies across the range, so tan(theta_n) = nu - 3/2 is far from zero
    (0.25 .. 0.38 at sigma = 1): the correlated pi-noise matters here."""
    m, r = bump
    t = []
    for frac in (0.0, 0.5, 1.0):
        nm = T.noise_at_phi(m, r, r.phi_in + frac * (r.phi_end - r.phi_in), 1.0)
        t.append(nm.T / nm.S)
    assert 0.2 < t[0] < t[1] < t[2] < 0.45


def test_bump_noise_off_is_the_background(bump):
    """Zero noise: every trajectory is the classical Euler path, which reaches
    phi_end after n_end - n_in e-folds of the background (first-order Euler
    error) -- the C stepper's V'/V against the Python background."""
    m, r = bump
    tab = T.user_table(np.zeros(8), np.zeros(8), r.phi_end, r.phi_in)
    tr = S.run(m, r, tab, seed=1, run_id=0, n=4, A=0.0)
    assert np.all(tr.nsteps == tr.nsteps[0])
    assert abs(tr.N[0] - (m.n_end - m.n_in)) < 0.01


def test_bump_importance_sampling_identity(bump):
    m, r = bump
    tab = T.bessel_table(m, r, 64, 1.0, processes=4)
    n = 1 << 14
    d = S.run(m, r, tab, seed=41, run_id=0, n=n)
    q = S.run(m, r, tab, seed=42, run_id=0, n=n, A=1.0)
    w = np.exp(q.logw)
    assert abs(w.mean() - 1) < 4 * w.std() / math.sqrt(n)
    est, se = np.mean(w * q.N), np.std(w * q.N) / math.sqrt(n)
    assert abs(est - d.N.mean()) < 4 * math.hypot(se, d.N.std() / math.sqrt(n))
