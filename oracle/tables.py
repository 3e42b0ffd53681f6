"""FP64 noise-table oracle: background, mode functions, Bessel matching.

TEST INFRASTRUCTURE ONLY -- the product library never imports this module.

Everything is restated from arXiv:2410.13683 with SciPy as the ODE solver
(``solve_ivp``, DOP853) and for Bessel/Gamma functions (``scipy.special``):

* background: Eq. (2.21) without noise, phi' = pi,
  pi' = -(3 - pi^2/2)(pi + V'/V), with e-fold time N = ln a; H^2 = V/(3 - pi^2/2)
  from the Friedmann constraint Eq. (2.2) written in N;
* mode functions: Eq. (2.4) rewritten in N,
  u'' + (3 - eps1) u' + [k^2/(aH)^2 + V''/H^2 - (3 - eps1) pi^2 - 2 pi pi'] u = 0,
  started in the Bunch-Davies state of Eq. (2.5) at k/(aH) = 100 / sigma
  e-folds before matching (i.e. N_0 = N_sigma - ln(100/sigma));
* the potential kink of Eq. (4.11) (V'' = V0 (a_+ - a_-) delta(phi - phi_*))
  is crossed with the jump du'/dN -> du'/dN - (V0/H_T^2)(a_+ - a_-)/|pi_T| u,
  which follows from integrating the mode equation across N_T;
* Bessel matching, Eq. (3.10), with the ansatz of Eq. (3.5) at -k eta = sigma
  and d(-k eta)/dN = -(-k eta); the combination multiplying Y_nu in the
  numerators is (3/2) u + du/dN (differentiating Eq. 3.5 gives this sign;
  Eq. 3.10 prints (3/2) u - du/dN);
* nu^2 from the exact Eq. (3.13) at N_sigma;
* noise amplitude from Eq. (3.12): S = sqrt(Xi_phiphi)
  = (H/2pi) (2|B_k|/sqrt(pi)) [Gamma(nu)/Gamma(3/2)] (sigma/2)^(3/2 - nu),
  and S_pi = (nu - 3/2) S, i.e. tan(theta_n) = nu - 3/2 (Eqs. 3.12, 2.26);
* de Sitter noise, Eq. (3.3): S = H/2pi on phi only, with H evaluated on the
  slow-roll attractor pi = -V'/V.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize, special

RTOL_BG = 1e-13
ATOL_BG = 1e-16
RTOL_MODE = 1e-11
BD_RATIO = 100.0       # k / (aH) at the Bunch-Davies start, times sigma


# --------------------------------------------------------------------------
# Potential (Eq. 4.11 with relative slopes; exponential test model)
# --------------------------------------------------------------------------
def _bump_parts(m, phi):
    """Gaussian bump (Sec. 4.3): V = V0 f (1 + g), f = phi^2/(m^2 + phi^2),
    g = K exp(-(phi - phi0)^2/(2 w^2)). Returns f'/f, f''/f, g, g', g''."""
    m2, w2 = m.bump_m ** 2, m.bump_width ** 2
    d = phi - m.bump_phi0
    g = m.bump_K * math.exp(-0.5 * d * d / w2)
    q = m2 + phi * phi
    f1 = 2.0 * m2 / (phi * q)
    f2 = 2.0 * m2 * (m2 - 3.0 * phi * phi) / (phi * phi * q * q)
    g1 = -g * d / w2
    g2 = g * (d * d / w2 - 1.0) / w2
    return f1, f2, g, g1, g2


def dlnV(m, phi: float, branch: int | None = None) -> float:
    """V'/V. ``branch`` = +1/-1 forces the side of the kink."""
    if m.kind == 1:
        return m.mu
    if m.kind == 2:
        f1, _, g, g1, _ = _bump_parts(m, phi)
        return f1 + g1 / (1.0 + g)
    above = (phi >= m.phi_star) if branch is None else (branch > 0)
    a = m.a_plus if above else m.a_minus
    return a / (1.0 + a * (phi - m.phi_star))


def d2V_over_V(m, phi: float, branch: int | None = None) -> float:
    """V''/V away from the kink (zero for the piecewise-linear potential)."""
    if m.kind == 1:
        return m.mu * m.mu
    if m.kind == 2:
        f1, f2, g, g1, g2 = _bump_parts(m, phi)
        return f2 + 2.0 * f1 * g1 / (1.0 + g) + g2 / (1.0 + g)
    return 0.0


def V_of(m, phi: float, branch: int | None = None) -> float:
    if m.kind == 1:
        return m.V0 * math.exp(m.mu * phi)
    if m.kind == 2:
        _, _, g, _, _ = _bump_parts(m, phi)
        return m.V0 * phi * phi / (m.bump_m ** 2 + phi * phi) * (1.0 + g)
    above = (phi >= m.phi_star) if branch is None else (branch > 0)
    a = m.a_plus if above else m.a_minus
    return m.V0 * (1.0 + a * (phi - m.phi_star))


def hubble(m, phi, pi, branch=None):
    """H from the Friedmann constraint in e-fold time: H^2 = V/(3 - pi^2/2)."""
    return math.sqrt(V_of(m, phi, branch) / (3.0 - 0.5 * pi * pi))


# --------------------------------------------------------------------------
# Background (Eq. 2.21 without noise)
# --------------------------------------------------------------------------
@dataclass
class Background:
    model: object
    N_T: float                 # transition time (kink crossing, or USR onset); nan if none
    pre: object                # OdeSolution for N <= N_T (branch +)
    post: object               # OdeSolution for N >= N_T (branch -)
    N_max: float
    kink: bool = True          # False: smooth potential, N_T only marks the USR onset

    def state(self, N: float):
        sol, br = (self.pre, +1) if (not math.isnan(self.N_T) and N < self.N_T) else (self.post, -1)
        if math.isnan(self.N_T) or not self.kink:
            br = None
        y = sol(N)
        return float(y[0]), float(y[1]), br


def _bg_rhs(branch):
    def f(N, y, m):
        phi, pi = y
        return [pi, -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi, branch))]
    return f


def _eps2(m, phi, pi):
    dpi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi))
    return 2.0 * dpi / pi


def solve_background(m, phi0: float, N_max: float) -> Background:
    """Background from phi0 on the slow-roll attractor pi0 = -V'/V(phi0).

    Piecewise-linear potential: N_T is the kink crossing phi = phi_star.
    Gaussian bump: N_T is the onset of ultra-slow roll, the first time
    eps2 = 2 pi'/pi falls to -3 (Sec. 4.3); the background then continues
    smoothly to N_T + N_max."""
    pi0 = -dlnV(m, phi0)
    if m.kind == 2:
        ev = lambda N, y, m: _eps2(m, y[0], y[1]) + 3.0
        ev.terminal, ev.direction = True, -1
        s1 = integrate.solve_ivp(_bg_rhs(None), (0.0, 200.0), [phi0, pi0], method="DOP853",
                                 rtol=RTOL_BG, atol=ATOL_BG, dense_output=True, events=ev, args=(m,))
        if s1.status != 1:
            raise ValueError("the background never enters ultra-slow roll (eps2 > -3 throughout)")
        N_T = float(s1.t_events[0][0])
        s2 = integrate.solve_ivp(_bg_rhs(None), (N_T, N_T + N_max), s1.y_events[0][0], method="DOP853",
                                 rtol=RTOL_BG, atol=ATOL_BG, dense_output=True, args=(m,))
        return Background(m, N_T, s1.sol, s2.sol, N_T + N_max, kink=False)
    if m.kind == 0 and phi0 > m.phi_star:
        ev = lambda N, y, m: y[0] - m.phi_star
        ev.terminal, ev.direction = True, -1
        s1 = integrate.solve_ivp(_bg_rhs(+1), (0.0, N_max), [phi0, pi0], method="DOP853",
                                 rtol=RTOL_BG, atol=ATOL_BG, dense_output=True,
                                 events=ev, args=(m,))
        if s1.status != 1:
            raise ValueError("background never reaches phi_star")
        N_T = float(s1.t_events[0][0])
        yT = s1.y_events[0][0]
        s2 = integrate.solve_ivp(_bg_rhs(-1), (N_T, N_T + N_max), [m.phi_star, yT[1]],
                                 method="DOP853", rtol=RTOL_BG, atol=ATOL_BG,
                                 dense_output=True, args=(m,))
        return Background(m, N_T, s1.sol, s2.sol, N_T + N_max)
    s = integrate.solve_ivp(_bg_rhs(None), (0.0, N_max), [phi0, pi0], method="DOP853",
                            rtol=RTOL_BG, atol=ATOL_BG, dense_output=True, args=(m,))
    return Background(m, float("nan"), s.sol, s.sol, N_max)


@dataclass
class Resolved:
    phi_in: float
    pi_in: float
    phi_end: float
    N_T: float
    N_in: float
    N_end: float
    bg: Background | None


def resolve(m) -> Resolved:
    """Start point and end surface of a model.

    Explicit phi_in / phi_end are used as given (pi_in = NaN means the
    attractor value -V'/V(phi_in)). With the sudden-transition rule the
    background starts at bg_phi0 on the attractor; phi_in, pi_in are its values
    n_in e-folds after the transition time N_T, and phi_end is its field value
    n_end e-folds after N_T.
    """
    if not math.isnan(m.n_in):
        span = (m.n_end + 10.0) if m.kind == 2 else max(60.0, 2 * m.n_end + 40.0)
        bg = solve_background(m, m.bg_phi0, N_max=span)
        N_in = bg.N_T + m.n_in
        N_end = bg.N_T + m.n_end
        phi_in, pi_in, _ = bg.state(N_in)
        phi_end, _, _ = bg.state(N_end)
        return Resolved(phi_in, pi_in, phi_end, bg.N_T, N_in, N_end, bg)
    pi_in = m.pi_in if not math.isnan(m.pi_in) else -dlnV(m, m.phi_in)
    return Resolved(m.phi_in, pi_in, m.phi_end, float("nan"), float("nan"), float("nan"), None)


def N_of_phi(bg: Background, phi: float, N_lo: float, N_hi: float) -> float:
    """Background time at which the (monotone) post-transition field equals phi."""
    f = lambda N: bg.state(N)[0] - phi
    return optimize.brentq(f, N_lo, N_hi, xtol=1e-14, rtol=4 * np.finfo(float).eps, maxiter=400)


# --------------------------------------------------------------------------
# Hubble-flow quantities and nu^2 (Eq. 3.13)
# --------------------------------------------------------------------------
def flow(m, phi, pi, branch):
    """eps1, eps2, H, pi' at a background point."""
    H = hubble(m, phi, pi, branch)
    dpi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi, branch))
    eps1 = 0.5 * pi * pi
    eps2 = 2.0 * dpi / pi
    return eps1, eps2, H, dpi


def nu_squared(m, phi, pi, branch) -> float:
    """Exact nu^2 of Eq. (3.13) with V''/V of the model (zero away from the
    kink of the piecewise-linear potential)."""
    eps1, eps2, H, _ = flow(m, phi, pi, branch)
    v1 = dlnV(m, phi, branch)
    v2 = d2V_over_V(m, phi, branch)
    return 2.25 - eps1 - 0.5 * eps1 * eps2 * eps2 / (3.0 - eps1) + (eps1 - 3.0) * (v2 - v1 * v1)


# --------------------------------------------------------------------------
# Mode function (Eq. 2.4 in e-fold time)
# --------------------------------------------------------------------------
def _mode_rhs(N, y, m, k, branch):
    """y = (phi, pi, ur, ur', ui, ui'); background integrated alongside."""
    phi, pi, ur, urp, ui, uip = y
    V = V_of(m, phi, branch)
    H2 = V / (3.0 - 0.5 * pi * pi)
    eps1 = 0.5 * pi * pi
    dpi = -(3.0 - 0.5 * pi * pi) * (pi + dlnV(m, phi, branch))
    v2 = d2V_over_V(m, phi, branch)                     # V''/V
    mass = (k * k) / (math.exp(2.0 * N) * H2) + v2 * V / H2 - (3.0 - eps1) * pi * pi - 2.0 * pi * dpi
    return [pi, dpi,
            urp, -(3.0 - eps1) * urp - mass * ur,
            uip, -(3.0 - eps1) * uip - mass * ui]


def evolve_mode(m, bg: Background, k: float, N0: float, N1: float, u0: complex,
                du0: complex, rtol=RTOL_MODE):
    """Integrate the mode equation from (u0, du0) at N0 to N1, background
    integrated alongside from its state at N0; crosses the kink at N_T with
    the jump du/dN -> du/dN - (V0/H_T^2)(a_+ - a_-)/|pi_T| u.
    Returns (u, du/dN, final state vector)."""
    phi0, pi0, br0 = bg.state(N0)
    y = [phi0, pi0, u0.real, du0.real, u0.imag, du0.imag]
    if not bg.kink or math.isnan(bg.N_T):
        segments = [(N0, N1, None)]
    elif N0 < bg.N_T < N1:
        segments = [(N0, bg.N_T, +1), (bg.N_T, N1, -1)]
    elif not math.isnan(bg.N_T):
        segments = [(N0, N1, +1 if N0 < bg.N_T else -1)]
    else:
        segments = [(N0, N1, None)]
    atol = 1e-14 * max(1.0, abs(u0), abs(du0))
    for (a_, b_, br) in segments:
        if a_ != N0:
            # V'' = V0 (a_+ - a_-) delta(phi - phi_*), delta(phi - phi_*) = delta(N - N_T)/|pi_T|
            piT = y[1]
            HT2 = m.V0 / (3.0 - 0.5 * piT * piT)
            jump = -(m.V0 / HT2) * (m.a_plus - m.a_minus) / abs(piT)
            y[3] += jump * y[2]
            y[5] += jump * y[4]
            y[0] = m.phi_star
        s = integrate.solve_ivp(_mode_rhs, (a_, b_), y, method="DOP853", rtol=rtol,
                                atol=[1e-16, 1e-18, atol, atol, atol, atol], args=(m, k, br))
        if not s.success:
            raise RuntimeError(s.message)
        y = list(s.y[:, -1])
    return complex(y[2], y[4]), complex(y[3], y[5]), y


def mode_at(m, bg: Background, k: float, N0: float, N1: float, rtol=RTOL_MODE):
    """One mode from the Bunch-Davies state of Eq. (2.5) at N0 to N1.

    Normalised so that u(N0) = 1: the physical mode is u / (exp(N0) sqrt(2k)).
    delta phi_BD = exp(-i k eta)/(a sqrt(2k)) gives du/dN = u (-1 - i k/(aH)).
    """
    phi0, pi0, br0 = bg.state(N0)
    kaH = k / (math.exp(N0) * hubble(m, phi0, pi0, br0))
    return evolve_mode(m, bg, k, N0, N1, 1.0 + 0j, complex(-1.0, -kaH), rtol)


def wronskian(m, N, y, branch):
    """exp(3N) H Im(conj(u) u'), conserved by the mode equation."""
    phi, pi, ur, urp, ui, uip = y
    H = hubble(m, phi, pi, branch)
    return math.exp(3.0 * N) * H * (ur * uip - ui * urp)


def bessel_match(u: complex, du: complex, nu: float, z: float, prefac: complex = 1.0):
    """Bessel coefficients (A_k, B_k) of Eq. (3.10).

    With p = sqrt(-eta)/a the ansatz of Eq. (3.5) is u = p [A J + B Y] and,
    since d ln p / dN = -3/2 and d z / dN = -z,
    du/dN = p [-(3/2)(A J + B Y) - z (A J' + B Y')].
    ``prefac`` = 1/p in the units of u.
    """
    J, Y = special.jv(nu, z), special.yv(nu, z)
    Jp, Yp = special.jvp(nu, z), special.yvp(nu, z)
    U = u * prefac                                  # A J + B Y
    Vv = -(1.5 * u + du) * prefac / z               # A J' + B Y'
    W = J * Yp - Jp * Y                             # = 2/(pi z)
    A = (U * Yp - Vv * Y) / W
    B = (Vv * J - U * Jp) / W
    return A, B


@dataclass
class ModeNoise:
    phi: float
    N_sigma: float
    k: float
    H: float
    nu: float
    A: complex
    B: complex
    S: float
    T: float


def noise_at_phi(m, res: Resolved, phi: float, sigma: float) -> ModeNoise:
    """Semi-analytical (Bessel-matched) noise at field value phi."""
    bg = res.bg
    N_s = N_of_phi(bg, phi, bg.N_T, bg.N_max)
    ph, pi, br = bg.state(N_s)
    H = hubble(m, ph, pi, br)
    k = sigma * math.exp(N_s) * H
    N0 = N_s - math.log(BD_RATIO / sigma)
    if N0 < 0.0:
        raise ValueError("Bunch-Davies start precedes the background start")
    u, du, _ = mode_at(m, bg, k, N0, N_s)
    nu = math.sqrt(nu_squared(m, ph, pi, br))
    # physical mode = u / (exp(N0) sqrt(2k)); p = sqrt(-eta)/a = sqrt(z/k)/a
    # => mode / p = u exp(N_s - N0) / sqrt(2 z)
    prefac = math.exp(N_s - N0) / math.sqrt(2.0 * sigma)
    A, B = bessel_match(u, du, nu, sigma, prefac)
    S = (H / (2.0 * math.pi)) * (2.0 * abs(B) / math.sqrt(math.pi)) \
        * (special.gamma(nu) / special.gamma(1.5)) * (sigma / 2.0) ** (1.5 - nu)
    return ModeNoise(phi, N_s, k, H, nu, A, B, S, (nu - 1.5) * S)


@dataclass
class NoiseTable:
    phi_lo: float              # first grid coordinate (phi, or N for n_indexed)
    h: float
    S: np.ndarray
    T: np.ndarray
    n_indexed: bool = False    # indexed by time since the start; zero noise outside

    @property
    def n_points(self):
        return len(self.S)


def grid(n_points: int, phi_lo: float, phi_hi: float):
    h = (phi_hi - phi_lo) / (n_points - 1)
    return phi_lo + h * np.arange(n_points), h


def _table_range(res: Resolved, phi_lo, phi_hi):
    lo = res.phi_end if (phi_lo is None or math.isnan(phi_lo)) else phi_lo
    hi = res.phi_in if (phi_hi is None or math.isnan(phi_hi)) else phi_hi
    return lo, hi


def desitter_table(m, res: Resolved, n_points: int, phi_lo=None, phi_hi=None) -> NoiseTable:
    """S = H/2pi with H^2 = V/(3 - pi_att^2/2), pi_att = -V'/V (Eq. 3.3)."""
    lo, hi = _table_range(res, phi_lo, phi_hi)
    phis, h = grid(n_points, lo, hi)
    S = np.empty(n_points)
    for j, ph in enumerate(phis):
        pa = -dlnV(m, ph)
        S[j] = math.sqrt(V_of(m, ph) / (3.0 - 0.5 * pa * pa)) / (2.0 * math.pi)
    return NoiseTable(lo, h, S, np.zeros(n_points))


def _bessel_worker(args):
    m, res, ph, sigma = args
    r = noise_at_phi(m, res, ph, sigma)
    return r.S, r.T


def bessel_table(m, res: Resolved, n_points: int, sigma: float, phi_lo=None, phi_hi=None,
                 indices=None, processes: int = 0) -> NoiseTable:
    """Bessel-matched table on the uniform grid; ``indices`` restricts the
    computation to those grid points (others are NaN)."""
    lo, hi = _table_range(res, phi_lo, phi_hi)
    phis, h = grid(n_points, lo, hi)
    idx = range(n_points) if indices is None else list(indices)
    S = np.full(n_points, np.nan)
    T = np.full(n_points, np.nan)
    jobs = [(m, res, float(phis[j]), sigma) for j in idx]
    if processes and processes > 1 and len(jobs) > 8:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            out = pool.map(_bessel_worker, jobs, chunksize=max(1, len(jobs) // (4 * processes)))
    else:
        out = [_bessel_worker(j) for j in jobs]
    for j, (s, t) in zip(idx, out):
        S[j], T[j] = s, t
    return NoiseTable(lo, h, S, T)


def noise_at_time(m, res: Resolved, N_since_start: float, sigma: float) -> ModeNoise:
    """Bessel-matched noise of the mode that crosses sigma a H at background
    time N_in + N_since_start (the paper's global-time indexing, Sec. 4.1)."""
    bg = res.bg
    N_s = res.N_in + N_since_start
    ph, pi, br = bg.state(N_s)
    return noise_at_phi(m, res, ph, sigma)


def _bessel_time_worker(args):
    m, res, N, sigma = args
    r = noise_at_time(m, res, N, sigma)
    return r.S, r.T


def bessel_table_N(m, res: Resolved, n_points: int, sigma: float, N_lo: float, N_hi: float,
                   indices=None, processes: int = 0) -> NoiseTable:
    """Noise along the classical background on a uniform grid of the time
    since the start, N_j = N_lo + j h; zero outside [N_lo, N_hi] (window)."""
    Ns, h = grid(n_points, N_lo, N_hi)
    idx = range(n_points) if indices is None else list(indices)
    S = np.full(n_points, np.nan)
    T = np.full(n_points, np.nan)
    jobs = [(m, res, float(Ns[j]), sigma) for j in idx]
    if processes and processes > 1 and len(jobs) > 8:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            out = pool.map(_bessel_time_worker, jobs, chunksize=max(1, len(jobs) // (4 * processes)))
    else:
        out = [_bessel_time_worker(j) for j in jobs]
    for j, (sv, tv) in zip(idx, out):
        S[j], T[j] = sv, tv
    return NoiseTable(N_lo, h, S, T, n_indexed=True)


def user_table_N(S, T, N_lo, N_hi) -> NoiseTable:
    S = np.asarray(S, float)
    T = np.asarray(T, float)
    return NoiseTable(N_lo, (N_hi - N_lo) / (len(S) - 1), S, T, n_indexed=True)


def user_table(S, T, phi_lo, phi_hi) -> NoiseTable:
    S = np.asarray(S, float)
    T = np.asarray(T, float)
    return NoiseTable(phi_lo, (phi_hi - phi_lo) / (len(S) - 1), S, T)


def growing_mode(nm: ModeNoise, sigma: float, N0: float):
    """Homogeneous growing mode of Eq. (3.11) at N_sigma, in the units of
    mode_at (u = physical mode x exp(N0) sqrt(2k)); d/dN = (nu - 3/2) x."""
    prefac = math.exp(nm.N_sigma - N0) / math.sqrt(2.0 * sigma)
    dphi_over_p = -nm.B * special.gamma(nm.nu) / math.pi * (sigma / 2.0) ** (-nm.nu)
    u_h = dphi_over_p / prefac
    return u_h, (nm.nu - 1.5) * u_h


def consistency_ratio(m, res: Resolved, phi: float, sigma: float,
                      frozen_after: float = 8.0) -> float:
    """P_R from the matched growing mode via Eqs. (2.9)-(2.10) divided by P_R
    of the full mode, Eq. (2.8) (the criterion of Eq. 3.1).

    Both are evaluated at N_e = max(N_end, N_sigma + frozen_after): the full
    spectrum is compared once the mode is far outside the Hubble radius (at
    N_sigma itself a sigma = 1 mode still carries its gradient term)."""
    bg = res.bg
    nm = noise_at_phi(m, res, phi, sigma)
    N0 = nm.N_sigma - math.log(BD_RATIO / sigma)
    Ns = nm.N_sigma
    Ne = max(res.N_end, Ns + frozen_after)
    u_h, du_h = growing_mode(nm, sigma, N0)
    ph, pi, br = bg.state(Ns)
    eps1, eps2, H, _ = flow(m, ph, pi, br)
    # a_*^3 H_* int_{N*}^{Ne} dN/(2 eps1 a^3 H) with a = e^N, scaled by a_*^3
    def f(N):
        p_, q_, b_ = bg.state(N)
        e1, _, h_, _ = flow(m, p_, q_, b_)
        return math.exp(3.0 * (Ns - N)) / (2.0 * e1 * h_)
    I = integrate.quad(f, Ns, Ne, epsabs=0.0, epsrel=1e-10, limit=400)[0] * H
    r2e = math.sqrt(2.0 * eps1)
    C = u_h / r2e - r2e * (0.5 * eps2 * u_h - du_h) * I
    u_end, _, _ = mode_at(m, bg, nm.k, N0, Ne)
    phe, pie, _ = bg.state(Ne)
    P_full = abs(u_end) ** 2 / (pie * pie)          # |dphi|^2 / (2 eps1)
    return abs(C) ** 2 / P_full



# --------------------------------------------------------------------------
# Full-rank (2-D) noise: numerical matching, Eq. (3.9)
# --------------------------------------------------------------------------
@dataclass
class NoiseTable2:
    """phi-indexed 2x2 noise matrices S = sqrt(Xi) (symmetric): components
    S_phiphi, S_phipi, S_pipi at phi_j = phi_lo + j h; end values held outside."""
    phi_lo: float
    h: float
    Spp: np.ndarray
    Spq: np.ndarray
    Sqq: np.ndarray


def sqrt_psd2(a, b, c):
    """Symmetric square root of the PSD matrix [[a, b], [b, c]]:
    S = (X + sqrt(det) I) / sqrt(tr + 2 sqrt(det))."""
    det = max(a * c - b * b, 0.0)
    sd = math.sqrt(det)
    den = math.sqrt(a + c + 2.0 * sd)
    if den == 0.0:
        return 0.0, 0.0, 0.0
    return (a + sd) / den, b / den, (c + sd) / den


def xi_numeric_at_phi(m, res: Resolved, phi: float, sigma: float):
    """Covariance of Eq. (3.9): the full mode delta phi_k and delta pi_k =
    d(delta phi_k)/dN at k = sigma a H, Xi = k^3/(2 pi^2) (|dphi|^2,
    Re(dphi dpi*), |dpi|^2). Returns (Xi_pp, Xi_pq, Xi_qq, a, H, k)."""
    bg = res.bg
    N_s = N_of_phi(bg, phi, bg.N_T, bg.N_max)
    ph, pi, br = bg.state(N_s)
    H = hubble(m, ph, pi, br)
    k = sigma * math.exp(N_s) * H
    N0 = N_s - math.log(BD_RATIO / sigma)
    u, du, _ = mode_at(m, bg, k, N0, N_s)
    # physical mode = u / (exp(N0) sqrt(2k))
    norm = 1.0 / (math.exp(2.0 * N0) * 2.0 * k)
    pref = k ** 3 / (2.0 * math.pi ** 2) * norm
    xpp = pref * abs(u) ** 2
    xpq = pref * (u * du.conjugate()).real
    xqq = pref * abs(du) ** 2
    return xpp, xpq, xqq, math.exp(N_s), H, k


def numeric_table(m, res: Resolved, n_points: int, sigma: float, phi_lo=None, phi_hi=None,
                  indices=None) -> NoiseTable2:
    lo, hi = _table_range(res, phi_lo, phi_hi)
    phis, h = grid(n_points, lo, hi)
    idx = range(n_points) if indices is None else list(indices)
    A = np.full(n_points, np.nan); B = np.full(n_points, np.nan); Cq = np.full(n_points, np.nan)
    for j in idx:
        xpp, xpq, xqq, _, _, _ = xi_numeric_at_phi(m, res, float(phis[j]), sigma)
        A[j], B[j], Cq[j] = sqrt_psd2(xpp, xpq, xqq)
    return NoiseTable2(lo, h, A, B, Cq)


def user_table2(Spp, Spq, Sqq, phi_lo, phi_hi) -> NoiseTable2:
    Spp = np.asarray(Spp, float)
    return NoiseTable2(phi_lo, (phi_hi - phi_lo) / (len(Spp) - 1), Spp, np.asarray(Spq, float),
                       np.asarray(Sqq, float))
