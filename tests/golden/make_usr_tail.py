"""Writes usr_tail.json: the tail threshold of the sudden-transition workload.

N_12 is the first-passage time at which the complementary CDF of N reaches
1e-12; it defines the tail set T = {N >= N_12} of the effective-sample-size
metric. It is estimated here with the FP64 oracle alone: importance sampling
with the constant diffusion-based bias A (Eq. 4.10), the weighted estimator of
P(N), and its standard error, on a 0.1 e-fold grid.

Run: python tests/golden/make_usr_tail.py [n_traj]   (about a minute on 8 cores)
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


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1 << 19
    A = 0.5
    m = replace(W.USR_MODEL, max_steps=1 << 19)
    res = T.resolve(m)
    tab = T.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=os.cpu_count())
    tr = S.run(m, res, tab, seed=1001, run_id=0, n=n, A=A)
    lo, hi, nb = 0.0, 400.0, 4000
    h = E.histogram(tr.nsteps, tr.logw, tr.status, m.dN, lo, hi, nb, G=1)
    P, se = E.p_weighted(h)
    mass = P * h.db
    ccdf = np.cumsum(mass[::-1])[::-1]
    var = np.cumsum((se * h.db)[::-1] ** 2)[::-1]      # bins are independent sums
    k = int(np.argmax(ccdf < 1e-12))
    N12 = lo + k * h.db
    out = dict(N_12=round(N12, 1), ccdf_at_N_12=float(ccdf[k]), rel_se_at_N_12=float(math.sqrt(var[k]) / ccdf[k]),
               A=A, n_traj=n, seed=1001, max_steps=m.max_steps,
               ccdf_at=dict((str(x), float(ccdf[int(x / h.db)])) for x in (10, 20, 50, 100, 150, 200)))
    with open(os.path.join(HERE, "usr_tail.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
