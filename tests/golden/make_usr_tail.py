"""Writes usr_tail.json: the tail thresholds of the sudden-transition workload.

N_12 and N_20 are the first-passage times at which the complementary CDF of N
reaches 1e-12 and 1e-20; they define the tail sets T = {N >= N_12} of the
effective-sample-size metric and {N >= N_20} of its far-tail leg. Both are
estimated here with the FP64 oracle alone: importance sampling with the
constant diffusion-based bias A (Eq. 4.10; A = 0.5 for N_12, A = 0.55 for
N_20, which sends more paths past 250 e-folds), the weighted estimator of P(N)
and its standard error, on a 0.1 e-fold grid.

Run: python tests/golden/make_usr_tail.py [n_traj [n_traj_20]]   (about twelve minutes on 8 cores)
"""
import json
import math
import os
import sys
from dataclasses import replace

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import estimators as E  # noqa: E402
from oracle import stepper as S  # noqa: E402
from oracle import tables as T  # noqa: E402


def ccdf_of(tr, dN, lo=0.0, hi=600.0, nb=6000):
    """CCDF of N on a 0.1 e-fold grid and its variance (the bins' weighted sums
    are sums over disjoint sets of trajectories; their errors add in quadrature)."""
    h = E.histogram(tr.nsteps, tr.logw, tr.status, dN, lo, hi, nb, G=1)
    P, se = E.p_weighted(h)
    mass = P * h.db
    ccdf = np.cumsum(mass[::-1])[::-1]
    var = np.cumsum((se * h.db)[::-1] ** 2)[::-1]
    return ccdf, var, h.db


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1 << 19
    n20 = int(sys.argv[2]) if len(sys.argv) > 2 else 1 << 20
    A = 0.5
    m = replace(W.USR_MODEL, max_steps=1 << 19)
    res = T.resolve(m)
    tab = T.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=os.cpu_count())
    tr = S.run(m, res, tab, seed=1001, run_id=0, n=n, A=A)
    ccdf, var, db = ccdf_of(tr, m.dN)
    k = int(np.argmax(ccdf < 1e-12))
    N12 = k * db
    out = dict(N_12=round(N12, 1), ccdf_at_N_12=float(ccdf[k]), rel_se_at_N_12=float(math.sqrt(var[k]) / ccdf[k]),
               A=A, n_traj=n, seed=1001, max_steps=m.max_steps,
               ccdf_at=dict((str(x), float(ccdf[int(round(x / db))])) for x in (10, 20, 50, 100, 150, 200)))
    A20 = 0.55
    tr20 = S.run(m, res, tab, seed=1002, run_id=0, n=n20, A=A20)
    c20, v20, _ = ccdf_of(tr20, m.dN)
    k20 = int(np.argmax(c20 < 1e-20))
    out.update(N_20=round(k20 * db, 1), ccdf_at_N_20=float(c20[k20]),
               rel_se_at_N_20=float(math.sqrt(v20[k20]) / c20[k20]), A_20=A20, seed_20=1002, n_traj_20=n20,
               n_capped_20=int(np.sum(tr20.status != 0)),
               ccdf_at_20=dict((str(x), float(c20[int(round(x / db))])) for x in (150, 200, 250)))
    with open(os.path.join(HERE, "usr_tail.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
