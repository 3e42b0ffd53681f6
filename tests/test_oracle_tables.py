"""Pins of the FP64 noise-table oracle (background, modes, Bessel matching)."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import special

import workloads as W
from oracle import tables as T


@pytest.fixture(scope="module")
def usr():
    m = W.USR_MODEL
    return m, T.resolve(m)


def test_usr_endpoints(usr):
    m, r = usr
    # N_T: 0.02 / a_plus e-folds of slow roll; attractor pi = -a_plus
    assert abs(r.N_T - 20.0) < 0.01
    assert abs(r.phi_in - 0.9999171) < 1e-7
    assert abs(r.pi_in - (-7.516e-4)) < 1e-6
    assert abs(r.phi_end - 0.9996620) < 1e-7
    # USR: pi decays as exp(-3 (N - N_T)) right after the transition
    _, piT, _ = r.bg.state(r.N_T + 1e-9)
    _, pi1, _ = r.bg.state(r.N_T + 1.0)
    assert abs(pi1 / piT - math.exp(-3.0)) < 0.01


def test_no_kink_limit_is_de_sitter_bunch_davies():
    """a_- = a_+: nu -> 3/2, |B_k|^2 -> pi/4 and S -> H/2pi (Eqs. 3.6, 3.3, 3.12)."""
    m = dataclasses.replace(W.USR_MODEL, a_minus=W.USR_MODEL.a_plus, n_in=1.0, n_end=3.0)
    r = T.resolve(m)
    for ph in (r.phi_in, 0.5 * (r.phi_in + r.phi_end), r.phi_end):
        nm = T.noise_at_phi(m, r, ph, 1.0)
        assert abs(nm.nu - 1.5) < 1e-5
        assert abs(abs(nm.B) ** 2 / (math.pi / 4) - 1) < 2e-4   # BD start at k/aH=100
        assert abs(nm.S / (nm.H / (2 * math.pi)) - 1) < 2e-4


def test_constant_nu_bunch_davies_reduces_to_eq_3_8():
    """With B_k at its Bunch-Davies value, Eq. (3.12) equals Eq. (3.8)."""
    for nu in (1.2, 1.5, 1.9):
        for sigma in (0.01, 0.3, 1.0):
            B = math.sqrt(math.pi) / 2 * complex(math.cos((nu + 1.5) * math.pi / 2),
                                                   math.sin((nu + 1.5) * math.pi / 2))
            eq312 = (4 * abs(B) ** 2 / math.pi) * (special.gamma(nu) / special.gamma(1.5)) ** 2 \
                * (sigma / 2) ** (3 - 2 * nu)
            eq38 = (special.gamma(nu) / special.gamma(1.5)) ** 2 * (sigma / 2) ** (3 - 2 * nu)
            assert eq312 == pytest.approx(eq38, rel=1e-14)


def test_bessel_match_reconstructs_mode():
    """(A, B) from the matching formula reproduce u and du/dN through the ansatz
    of Eq. (3.5) differentiated numerically in N (z = sigma exp(-(N - N_sigma)))."""
    u, du, nu, sigma = complex(0.3, -1.1), complex(-0.7, 0.4), 1.4999, 1.0
    A, B = T.bessel_match(u, du, nu, sigma, prefac=1.0)
    # ansatz in units where p(N_sigma) = 1: p(N) = exp(-3/2 (N - N_s))
    def f(dN):
        z = sigma * math.exp(-dN)
        return math.exp(-1.5 * dN) * (A * special.jv(nu, z) + B * special.yv(nu, z))
    h = 1e-5
    assert abs(f(0.0) - u) < 1e-12
    assert abs((f(h) - f(-h)) / (2 * h) - du) < 1e-8


def test_kink_jump_keeps_superhorizon_mode_on_background(usr):
    """For k -> 0 the growing solution of the mode equation is u ~ pi(N) (the
    separate-universe solution, Eq. 2.7): it must stay proportional to pi
    through the kink."""
    m, r = usr
    bg = r.bg
    N0, N1 = bg.N_T - 1.0, bg.N_T + 2.0
    ph0, pi0, b0 = bg.state(N0)
    _, _, _, dpi0 = T.flow(m, ph0, pi0, b0)
    k = 1e-8 * math.exp(N0) * T.hubble(m, ph0, pi0, b0)
    u, du, y = T.evolve_mode(m, bg, k, N0, N1, complex(pi0), complex(dpi0))
    _, pi1, _ = bg.state(N1)
    assert abs(u.real / pi1 - 1.0) < 1e-8
    # a jump of the opposite sign would leave u far from pi
    assert abs(pi1 / pi0) < 0.1


def test_wronskian_conserved_through_kink(usr):
    m, r = usr
    bg = r.bg
    N_s = r.N_T + 0.5
    ph, pi, br = bg.state(N_s)
    k = math.exp(N_s) * T.hubble(m, ph, pi, br)
    N0 = N_s - math.log(100.0)
    ph0, pi0, b0 = bg.state(N0)
    kaH = k / (math.exp(N0) * T.hubble(m, ph0, pi0, b0))
    y0 = [ph0, pi0, 1.0, -1.0, 0.0, -kaH]
    w0 = T.wronskian(m, N0, y0, b0)
    u, du, y1 = T.evolve_mode(m, bg, k, N0, N_s, 1.0 + 0j, complex(-1.0, -kaH))
    w1 = T.wronskian(m, N_s, y1, -1)
    assert abs(w1 / w0 - 1) < 1e-8


@pytest.mark.parametrize("frac", [0.0, 0.05, 0.3, 0.7, 1.0])
def test_consistency_relation(usr, frac):
    """Eq. (3.1): the Bessel-matched growing mode reproduces the late-time
    power spectrum within 1% for every post-transition table mode."""
    m, r = usr
    ph = r.phi_end + frac * (r.phi_in - r.phi_end)
    assert abs(T.consistency_ratio(m, r, ph, 1.0) - 1.0) < 0.01


def test_table_values_and_noise_angle(usr):
    m, r = usr
    tab = T.bessel_table(m, r, 4096, 1.0, indices=[0, 1, 2048, 4094, 4095])
    assert tab.phi_lo == r.phi_end and abs(tab.phi_lo + 4095 * tab.h - r.phi_in) < 1e-15
    H2pi = math.sqrt(m.V0 / 3) / (2 * math.pi)
    # late modes are Bunch-Davies-like; early ones carry the transition
    assert abs(tab.S[0] / H2pi - 1) < 1e-3
    assert 0.2 < tab.S[4095] / H2pi < 0.8
    # ultra-slow roll on a linear potential: nu = 3/2 up to eps1 terms
    assert np.all(np.abs(tab.T[[0, 1, 2048, 4094, 4095]] / tab.S[[0, 1, 2048, 4094, 4095]]) < 1e-5)


def test_desitter_table(usr):
    wl = W.LINEAR
    m = wl.model
    r = T.resolve(m)
    tab = T.desitter_table(m, r, 5, 0.0, 0.06)
    for j in range(5):
        ph = 0.06 * j / 4
        V = m.V0 * (1 + m.a_plus * ph)
        pa = m.a_plus / (1 + m.a_plus * ph)
        assert tab.S[j] == pytest.approx(math.sqrt(V / (3 - pa * pa / 2)) / (2 * math.pi), rel=1e-14)
    assert np.all(tab.T == 0)
