"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds parameters and random draws only: model constants, seeds,
trajectory counts, bias amplitudes and seeded weight initialisations. It
contains none of the method's arithmetic (no potentials, no noise model, no
stepping), so that the CUDA library and the FP64 oracle, which both read their
inputs from here, share no computation.

Model conventions (all workloads):
  * piecewise-linear potential with relative slopes,
        V(phi) = V0 * [1 + a_plus  * (phi - phi_star)]   for phi >= phi_star,
        V(phi) = V0 * [1 + a_minus * (phi - phi_star)]   for phi <  phi_star,
    the form of the paper's Eq. (potential_starobinsky) (Sec. 4.2) with the
    slopes divided by V0; a_plus == a_minus gives the plain linear potential
    V0 (1 + A phi) of the slow-roll test case;
  * the exponential potential V = V0 exp(mu phi) is a test model whose
    attractor pi = -mu is exact, so the dynamics reduce to a Gaussian random
    walk (used to pin the sampler against first-passage closed forms);
  * the Gaussian-bump potential (Sec. 4.3),
        V(phi) = V0 phi^2/(m^2 + phi^2) [1 + K exp(-(phi - phi0)^2 / (2 width^2))],
    with the paper's K, m, width and phi0; V0 is not printed and is fixed by
    normalising the peak of the linear power spectrum;
  * e-fold step dN = 1e-3 throughout (the paper prints no step size).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

# Potential kinds (mirrors FPT_POT_* in include/fpt.h; values are plain ints).
POT_PWLINEAR = 0
POT_EXP = 1
POT_BUMP = 2

# Noise-table kinds (mirrors FPT_TABLE_*).
TABLE_DESITTER = 0
TABLE_BESSEL = 1
TABLE_USER = 2

# Bias kinds (mirrors FPT_BIAS_*).
BIAS_NONE = 0
BIAS_CONST = 1
BIAS_MLP = 2

NAN = float("nan")


@dataclass(frozen=True)
class Model:
    """One potential + start point + end surface.

    ``phi_in``/``pi_in``/``phi_end`` may be given directly, or (for the
    sudden-transition workloads) resolved from a background solve: the
    background starts at ``bg_phi0`` on the slow-roll attractor, and
    ``phi_in``/``pi_in`` are the background values ``n_in`` e-folds after the
    transition time N_T (phi = phi_star), ``phi_end`` the background field
    value ``n_end`` e-folds after N_T. ``pi_in = NaN`` with explicit
    ``phi_in`` means "on the attractor pi = -V'/V(phi_in)".
    """

    kind: int = POT_PWLINEAR
    V0: float = 1.0
    a_plus: float = 0.0
    a_minus: float = 0.0
    phi_star: float = 0.0
    mu: float = 0.0
    phi_in: float = NAN
    pi_in: float = NAN
    phi_end: float = NAN
    bg_phi0: float = NAN
    n_in: float = NAN
    n_end: float = NAN
    dN: float = 1e-3
    max_steps: int = 1 << 20
    # POT_BUMP: V0 phi^2/(m^2 + phi^2) [1 + K exp(-(phi - phi0)^2 / (2 width^2))]
    bump_K: float = 0.0
    bump_m: float = 0.0
    bump_width: float = 0.0
    bump_phi0: float = 0.0


@dataclass(frozen=True)
class Table:
    kind: int
    n_points: int = 4096
    sigma: float = 1.0
    # NaN: the table spans [phi_end, phi_in] of the resolved model.
    phi_lo: float = NAN
    phi_hi: float = NAN


@dataclass(frozen=True)
class Workload:
    name: str
    model: Model
    table: Table
    n_traj: int
    seed: int
    run_id: int = 0
    biases: tuple = (0.0,)
    n_bins: int = 512
    notes: str = ""


# --- slow-roll linear case: V = V0 (1 + A phi), V0 = 1e-4, A = 1e-2 --------
LINEAR = Workload(
    name="linear_slow_roll",
    model=Model(kind=POT_PWLINEAR, V0=1e-4, a_plus=1e-2, a_minus=1e-2,
                phi_star=0.0, phi_in=0.05, pi_in=NAN, phi_end=0.0,
                dN=1e-3, max_steps=1 << 16),
    table=Table(kind=TABLE_DESITTER, n_points=4096, phi_lo=0.0, phi_hi=0.06),
    n_traj=16384, seed=0, run_id=0,
    notes="16384 trajectories, direct sampling, de Sitter noise H/2pi",
)

# --- sudden transition to ultra-slow roll (relative slopes) -----------------
USR_MODEL = Model(kind=POT_PWLINEAR, V0=2e-10, a_plus=1e-3, a_minus=1e-6,
                  phi_star=1.0, bg_phi0=1.02, n_in=math.log(1.1), n_end=5.0,
                  dN=1e-3, max_steps=1 << 18)
USR_TABLE = Table(kind=TABLE_BESSEL, n_points=4096, sigma=1.0)

USR_DIRECT = Workload(
    name="usr_direct", model=USR_MODEL, table=USR_TABLE,
    n_traj=1 << 22, seed=2, run_id=0,
    notes="2^22 trajectories, direct sampling, Bessel-matched noise table",
)

USR_FIXED_BIAS = Workload(
    name="usr_fixed_bias", model=USR_MODEL, table=USR_TABLE,
    n_traj=1 << 24, seed=3,
    biases=(0.5, 1.0, 2.0, 3.0, 4.0, 6.0, 8.0, 10.0), n_bins=512,
    notes="2^24 trajectories per bias amplitude, run_id = bias index",
)

USR_LEARNED = Workload(
    name="usr_learned", model=USR_MODEL, table=USR_TABLE,
    n_traj=1 << 26, seed=4, n_bins=512,
    notes="MLP proposal: 20 rounds x 2^20 training trajectories, then 2^26",
)
LEARNED_ROUNDS = 20
LEARNED_TRAIN_TRAJ = 1 << 20

# --- Gaussian bump (Sec. 4.3): smooth transition to ultra-slow roll ---------
# K, m, width, phi0 as printed; V0 (not printed) makes the linear power
# spectrum peak at 5e-3 (tests/golden/make_bump_v0.py -> bump_v0.json).
# The background starts at phi = 2.6 on the attractor; N_T is the onset of
# ultra-slow roll (eps2 = -3). The simulated modes start half-way through the
# ultra-slow-roll phase (which lasts 2.4 e-folds) and span 4 e-folds.
BUMP_V0 = 7.76487e-11
BUMP_MODEL = Model(kind=POT_BUMP, V0=BUMP_V0, bump_K=1.17e-3, bump_m=0.5,
                   bump_width=1.59e-2, bump_phi0=2.18812, bg_phi0=2.6,
                   n_in=1.2, n_end=5.2, dN=1e-3, max_steps=1 << 18)
BUMP_TABLE = Table(kind=TABLE_BESSEL, n_points=4096, sigma=1.0)

# --- exponential test model: exact Gaussian random walk ---------------------
# V = V0 exp(mu phi) has V'/V = mu, so pi = -mu is an exact fixed point of the
# momentum equation; with a USER table of constant S = s and zero pi-noise the
# field performs a Gaussian random walk with drift -mu per e-fold.
BM_MU = 0.01
BM_S = 1e-3
BM = Workload(
    name="brownian_exp",
    model=Model(kind=POT_EXP, V0=1e-4, mu=BM_MU, phi_in=0.05, pi_in=-BM_MU,
                phi_end=0.0, dN=1e-3, max_steps=1 << 16),
    table=Table(kind=TABLE_USER, n_points=16, phi_lo=-0.1, phi_hi=0.2),
    n_traj=1 << 14, seed=11,
)


def batch_models(n_models: int = 64, seed: int = 5) -> List[Model]:
    """The batched-sweep model family: a_minus log-uniform in [1e-7, 1e-4],
    phi_star uniform in [0.9, 1.1], V0 log-uniform in [1e-11, 1e-9],
    a_plus = 1e-3; start/end points follow the sudden-transition rule."""
    rng = np.random.default_rng(seed)
    a_minus = 10.0 ** rng.uniform(-7.0, -4.0, n_models)
    phi_star = rng.uniform(0.9, 1.1, n_models)
    V0 = 10.0 ** rng.uniform(-11.0, -9.0, n_models)
    out = []
    for i in range(n_models):
        out.append(replace(USR_MODEL, V0=float(V0[i]), a_minus=float(a_minus[i]),
                           phi_star=float(phi_star[i]),
                           bg_phi0=float(phi_star[i]) + 0.02,
                           max_steps=1 << 23))
    return out


def mlp_init(seed: int, hidden: int = 64, n_in: int = 3, n_out: int = 2,
             out_scale: float = 0.0) -> dict:
    """Seeded initial weights for the 3 -> 64 -> 64 -> 2 SiLU proposal MLP.

    Layout: W1 [hidden, n_in], b1 [hidden], W2 [hidden, hidden], b2 [hidden],
    W3 [n_out, hidden], b3 [n_out], row-major (out, in), float64.
    ``out_scale`` scales the last layer (0 gives a zero initial bias).
    """
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, 1.0 / math.sqrt(n_in), (hidden, n_in))
    b1 = np.zeros(hidden)
    W2 = rng.normal(0.0, 1.0 / math.sqrt(hidden), (hidden, hidden))
    b2 = np.zeros(hidden)
    W3 = rng.normal(0.0, 1.0 / math.sqrt(hidden), (n_out, hidden)) * out_scale
    b3 = np.zeros(n_out)
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def random_states(n: int, seed: int) -> np.ndarray:
    """Seeded MLP input points (x_hat, pi_hat, N_hat), used to compare MLP
    forward/backward implementations on identical inputs."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(-0.5, 1.5, n), rng.uniform(-1.5, 0.5, n),
                     rng.uniform(0.0, 3.0, n)], axis=1)
