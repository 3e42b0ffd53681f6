"""The tail golden file (usr_tail.json, written by make_usr_tail.py with the
oracle's importance-sampled estimator at A = 0.5) against brute force: direct
sampling of the same workload by the oracle, with no bias and no weights,
must give the same complementary CDF of N where direct sampling can reach
it (N = 10 and 20 e-folds, CCDF 7e-2 and 2e-3)."""
import json
import math
import os
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import stepper as OS
from oracle import tables as OT

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.slow
def test_importance_sampled_ccdf_matches_direct_sampling():
    with open(os.path.join(HERE, "golden", "usr_tail.json")) as f:
        tail = json.load(f)
    m = replace(W.USR_MODEL, max_steps=tail["max_steps"])
    res = OT.resolve(m)
    # 512 points instead of 4096: the table is smooth on this range, and the
    # interpolation difference is far below the sampling error here
    tab = OT.bessel_table(m, res, 512, W.USR_TABLE.sigma, processes=min(8, os.cpu_count() or 1))
    n = 1 << 16
    tr = OS.run(m, res, tab, seed=4242, run_id=0, n=n)
    assert np.all(tr.status == 0)          # every path passed (1 = capped)
    for x in ("10", "20"):
        k = int(round(float(x) / m.dN))
        p = float(np.mean(tr.nsteps >= k))
        se = math.sqrt(p * (1.0 - p) / n)
        g = tail["ccdf_at"][x]
        # 4 standard errors of the direct estimate, plus 3% for the golden's own error
        assert abs(p - g) < 4.0 * se + 0.03 * g, (x, p, se, g)
