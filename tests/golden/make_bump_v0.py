"""Writes bump_v0.json: the potential scale V0 of the Gaussian-bump workload.

Sec. 4.3 gives K, m, width and phi0 of the bump potential but not V0; it
states that the linear power spectrum peaks at P_R ~ 5e-3. V0 is fixed here
by that statement: P_R(k) = k^3/(2 pi^2) |delta phi_k|^2 / (2 eps1) of the
mode from its Bunch-Davies state (Eqs. 2.4-2.5, 2.8), evaluated 1.9 e-folds
after the workload's end surface (outside the Hubble radius, frozen),
maximised over the Hubble-crossing time of k; P_R is proportional to V0 at
fixed shape, so V0 = 5e-3 / max P_R(V0 = 1). Only the FP64 oracle is used.

Run: python tests/golden/make_bump_v0.py   (a few seconds)
"""
import json
import math
import os
import sys
from dataclasses import replace

from scipy import optimize

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import tables as T  # noqa: E402

PEAK = 5e-3
LATE = 1.9          # e-folds after N_end at which P_R is read


def power_spectrum(m, r, dNc):
    """P_R of the mode that crosses the Hubble radius at N_T + dNc."""
    bg = r.bg
    Nc = r.N_T + dNc
    ph, pi, br = bg.state(Nc)
    k = math.exp(Nc) * T.hubble(m, ph, pi, br)
    N0 = Nc - math.log(T.BD_RATIO)
    N_late = r.N_end + LATE
    u, _, _ = T.mode_at(m, bg, k, N0, N_late)
    _, pie, _ = bg.state(N_late)
    return k ** 3 / (2 * math.pi ** 2) * abs(u) ** 2 / (math.exp(2 * N0) * 2 * k) / (pie * pie)


def main():
    m1 = replace(W.BUMP_MODEL, V0=1.0)
    r = T.resolve(m1)
    opt = optimize.minimize_scalar(lambda d: -power_spectrum(m1, r, d), bounds=(0.5, 3.0),
                                   method="bounded", options=dict(xatol=1e-6))
    p1 = -opt.fun
    out = {"V0": PEAK / p1, "P_R_peak": PEAK, "peak_crossing_after_N_T": opt.x,
           "P_R_peak_at_V0_1": p1, "read_at": f"N_end + {LATE}",
           "note": "V0 such that the linear P_R peaks at 5e-3 (Sec. 4.3); FP64 oracle only"}
    with open(os.path.join(HERE, "bump_v0.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
