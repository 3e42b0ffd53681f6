"""FP64 classical-delta-N oracle: the linear power spectrum over the simulated
mode range, its variance sigma_R^2 and the constant-eps2 first-passage PDF.

TEST INFRASTRUCTURE ONLY -- the product library never imports this module.

Restated from arXiv:2410.13683, Sec. 2.2:
* P_R(k) = k^3/(2 pi^2) |delta phi_k|^2 / (2 eps1), Eq. (2.8), of the mode from
  its Bunch-Davies state (Eq. 2.5) read once it is outside the Hubble radius;
* sigma_R^2(k_S) = int_{k_in}^{k_S} P_R(k) d ln k, Eq. (2.18), over the modes
  that reach k = sigma a H between the start and the end of the simulation;
* for constant eps2 the non-linear relation
  R = -(2/eps2)(1 - exp(-eps2 dN/2)), Eq. (2.19), turns the Gaussian R into
  P(dN) = exp[-(2/(sigma_R^2 eps2^2))(1 - e^{-eps2 dN/2})^2 - eps2 dN/2] / (sqrt(2 pi) sigma_R),
  Eq. (2.20); eps2 -> 0 is the Gaussian of variance sigma_R^2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

from . import tables as T

LATE = 4.0          # e-folds after N_end at which P_R is read (frozen modes)


def power_spectrum_at(m, res, N_s: float, sigma: float, N_eval: float) -> float:
    """P_R of the mode with k = sigma a H at background time N_s, read at N_eval."""
    bg = res.bg
    ph, pi, br = bg.state(N_s)
    k = sigma * math.exp(N_s) * T.hubble(m, ph, pi, br)
    N0 = N_s - math.log(T.BD_RATIO / sigma)
    u, _, _ = T.mode_at(m, bg, k, N0, N_eval)
    _, pie, _ = bg.state(N_eval)
    return k ** 3 / (2 * math.pi ** 2) * abs(u) ** 2 / (math.exp(2 * N0) * 2 * k) / (pie * pie)


def sigma_R2(m, res, sigma: float = 1.0, n_k: int = 65, N_eval: float | None = None) -> float:
    """Eq. (2.18) over the modes reaching sigma a H in [N_in, N_end]:
    d ln k = (1 - eps1) dN_s along the background; Simpson's rule in N_s."""
    if N_eval is None:
        N_eval = res.N_end + LATE
    Ns = np.linspace(res.N_in, res.N_end, n_k)
    f = []
    for N in Ns:
        ph, pi, br = res.bg.state(N)
        f.append(power_spectrum_at(m, res, N, sigma, N_eval) * (1.0 - 0.5 * pi * pi))
    return float(integrate.simpson(np.array(f), x=Ns))


def eps2_at(m, res, N: float) -> float:
    ph, pi, br = res.bg.state(N)
    return T.flow(m, ph, pi, br)[1]


def pdf_constant_eps2(dN, s2: float, eps2: float):
    """Eq. (2.20); eps2 = 0 gives the Gaussian of variance s2."""
    dN = np.asarray(dN, dtype=float)
    if eps2 == 0.0:
        return np.exp(-dN * dN / (2 * s2)) / math.sqrt(2 * math.pi * s2)
    R = -(2.0 / eps2) * (1.0 - np.exp(-0.5 * eps2 * dN))
    return np.exp(-R * R / (2 * s2) - 0.5 * eps2 * dN) / math.sqrt(2 * math.pi * s2)
