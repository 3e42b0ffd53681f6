"""Pins of the oracle's random-number chain (Philox4x32-10 -> uniforms ->
Box-Muller normals)."""
import math
import os

import numpy as np
from scipy import stats

from oracle import stepper as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert S.philox4x32_10(ctr, key) == out


def test_normals_are_standard_normal():
    # 4 * 20000 normals from distinct counters: moments and KS against N(0,1)
    z = np.concatenate([S.normals4(7, 3, t, b) for t in range(200) for b in range(100)])
    assert abs(z.mean()) < 4 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 4 * math.sqrt(2.0 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # Box-Muller pairs are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 4 / math.sqrt(len(zz))


def test_normals_depend_on_every_key_and_counter_word():
    base = S.normals4(1, 2, 3, 4)
    for args in [(1 + (1 << 32), 2, 3, 4), (2, 2, 3, 4), (1, 3, 3, 4), (1, 2, 4, 4), (1, 2, 3, 5)]:
        assert not np.allclose(S.normals4(*args), base)
