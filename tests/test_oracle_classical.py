"""Pins of the classical-delta-N oracle (Sec. 2.2): the constant-eps2 PDF of
Eq. (2.20), the variance sigma_R^2 of Eq. (2.18) in slow roll, and linear
theory against the stochastic simulation near the peak of P(delta N)."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate, stats

import workloads as W
from oracle import classical as C
from oracle import stepper as S
from oracle import tables as T


@pytest.mark.parametrize("s2", [0.01, 1.0])
@pytest.mark.parametrize("eps2", [0.3, 0.745, 2.0, -0.5])
def test_pdf_mass_is_the_reachable_gaussian_mass(s2, eps2):
    """R = -(2/eps2)(1 - e^{-eps2 dN/2}) maps the real line onto one side of
    -2/eps2, so Eq. (2.20) integrates to Phi(2/(|eps2| sigma_R))."""
    f = lambda d: float(C.pdf_constant_eps2(np.array([d]), s2, eps2)[0])
    w = math.sqrt(s2)
    if eps2 > 0:
        edges = [-40 * w, -5 * w, 0.0, 5 * w, 40 * w, 400.0 / eps2]
    else:
        edges = [400.0 / eps2, -40 * w, -5 * w, 0.0, 5 * w, 40 * w]
    mass = sum(integrate.quad(f, a, b, limit=500, epsabs=1e-14)[0] for a, b in zip(edges[:-1], edges[1:]))
    assert mass == pytest.approx(stats.norm.cdf(2.0 / (abs(eps2) * math.sqrt(s2))), abs=1e-9)


def test_pdf_is_the_gaussian_of_R_times_the_jacobian():
    """P(dN) = N(R(dN); sigma_R^2) |dR/d dN|, checked with a numerical derivative."""
    s2, eps2 = 0.02, 0.745
    R = lambda d: -(2.0 / eps2) * (1.0 - np.exp(-0.5 * eps2 * d))
    d = np.linspace(-0.4, 2.0, 25)
    h = 1e-6
    jac = np.abs((R(d + h) - R(d - h)) / (2 * h))
    ref = stats.norm.pdf(R(d), scale=math.sqrt(s2)) * jac
    np.testing.assert_allclose(C.pdf_constant_eps2(d, s2, eps2), ref, rtol=1e-7)


def test_pdf_gaussian_limit():
    d = np.linspace(-1, 1, 11)
    np.testing.assert_allclose(C.pdf_constant_eps2(d, 0.1, 1e-7), C.pdf_constant_eps2(d, 0.1, 0.0), rtol=1e-6)
    np.testing.assert_allclose(C.pdf_constant_eps2(d, 0.1, 0.0), stats.norm.pdf(d, scale=math.sqrt(0.1)),
                               rtol=1e-14)


def test_sigma_R2_slow_roll():
    """No kink (a_- = a_+): slow roll with eps1 = a_+^2/2 to O(eps), where
    P_R = (H/2pi)^2 / (2 eps1) (Eq. 2.8 with the massless de Sitter mode) is
    flat, so sigma_R^2 = P_R (N_end - N_in)."""
    m = dataclasses.replace(W.USR_MODEL, a_minus=W.USR_MODEL.a_plus, n_in=1.0, n_end=3.0)
    r = T.resolve(m)
    s2 = C.sigma_R2(m, r, 1.0, n_k=9)
    ph, pi, br = r.bg.state(0.5 * (r.N_in + r.N_end))
    H = T.hubble(m, ph, pi, br)
    PR = (H / (2 * math.pi)) ** 2 / (pi * pi)
    assert s2 == pytest.approx(PR * (r.N_end - r.N_in), rel=2e-3)


def test_linear_theory_matches_the_simulation_near_the_peak():
    """Gaussian bump: the first-passage time of the stochastic run has the
    variance that linear theory gives, Var(N) = sigma_R^2 (Sec. 4.3: the
    Gaussian of Eq. 2.18 fits the peak), and its mean is n_end - n_in."""
    m = W.BUMP_MODEL
    r = T.resolve(m)
    s2 = C.sigma_R2(m, r, 1.0, n_k=17)
    tab = T.bessel_table(m, r, 128, 1.0, processes=4)
    tr = S.run(m, r, tab, seed=12, run_id=0, n=1 << 15)
    N = tr.N
    se = N.var() * math.sqrt(2.0 / len(N))
    assert abs(N.var() - s2) < 4 * se
    assert abs(N.mean() - (m.n_end - m.n_in)) < 0.02
