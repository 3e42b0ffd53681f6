"""Host arithmetic of bench.py on CPU: the clock-record parser (throttle
reasons decide whether a number stands), the issue roofline, the step count
of runs where no path passed, the constant-amplitude sweep's pick, the ESS
spread, and the reference arm's JSON line."""
import math

import numpy as np

import pytest

import bench


def test_parse_clocks_reasons_and_median():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1010.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1010.5, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
        "garbage",
    ]
    c = bench.parse_clocks(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.parse_clocks(["0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clocks([])["sm_mhz"] is None


def test_roofline_arithmetic():
    # 152 SMs x 128 lanes x 2070 MHz = 40.27 T lane-instructions/s; 1e10 steps
    # of 66 instructions in 32.77 ms is half of it
    r = bench.roofline(1e10, 66e10 / (0.5 * 152 * 128 * 2070e6) * 1e3, 152, 2070.0, None, 66)
    assert r["peak"] == pytest.approx(40.274, abs=1e-3)
    assert r["frac"] == pytest.approx(0.5, abs=1e-4)
    assert r["bound"] == "alu" and r["unit"] == "Tinst/s"


def test_passed_steps_without_passed_paths():
    assert bench.passed_steps({"N_mean": float("nan"), "n_passed": 0}, 1e-3) == 0.0
    assert bench.passed_steps({"N_mean": 5.0, "n_passed": 10}, 1e-3) == pytest.approx(5e4)


class _FakeFpt:
    """fpt stand-in: the tail ESS and step counts of each amplitude."""

    def __init__(self, table):
        self.table = table
        self.last = None

    def run_desc(self, model, n, seed, run_id, A, traj_offset):
        return A

    def fpt_run(self, ctx, runs, stream=None):
        self.last = runs[0]

    def fpt_histogram(self, ctx, run, lo, hi, bins, N_tail, stream=None):
        ess, n_passed, N_mean, n_capped = self.table[self.last]
        return {"ess_tail": ess, "n_passed": n_passed, "N_mean": N_mean, "n_capped": n_capped}


def test_fixed_sweep_prices_ess_per_step():
    class M:
        dN = 1e-3
        max_steps = 1000
    # A = 1 has more tail ESS but spends far more steps (capped paths)
    table = {0.5: (100.0, 10, 5.0, 0), 1.0: (150.0, 2, 50.0, 8), 2.0: (0.0, 0, math.nan, 10)}
    out = bench.fixed_sweep(_FakeFpt(table), None, None, 1, 0, 150.0, M, (0.5, 1.0, 2.0), 1e9, n=10)
    rows = out["per_A"]
    assert rows["0.5"]["em_steps"] == pytest.approx(5e4)
    assert rows["1.0"]["em_steps"] == pytest.approx(1e5 + 8000)
    assert rows["2.0"]["em_steps"] == pytest.approx(1e4) and rows["2.0"]["ess_tail_per_s"] == 0.0
    assert rows["0.5"]["ess_tail_per_s"] == pytest.approx(100.0 / 5e4 * 1e9)
    assert out["best_A"] == 0.5


def test_ess_spread_of_identical_steps_is_zero():
    from paper_2410_13683_gb300 import shard
    r = shard.ess_spread([2.0] * 8, [0.5] * 8)
    assert r["lo"] == pytest.approx(1.0) and r["hi"] == pytest.approx(1.0) and r["rel_se"] == pytest.approx(0.0, abs=1e-12)


def test_ess_spread_covers_the_repeat_to_repeat_scatter():
    """Steps with lognormal tail sums: the jackknife error of one set of 20
    steps matches the scatter of the pooled ESS over independent sets, and a
    step holding most of sum w^2 widens the bootstrap interval."""
    from paper_2410_13683_gb300 import shard
    rng = np.random.default_rng(3)
    pooled, ses = [], []
    for _ in range(400):
        w = np.exp(rng.normal(0.0, 1.0, (20, 50)))
        sw, sw2 = w.sum(axis=1), (w * w).sum(axis=1)
        pooled.append(sw.sum() ** 2 / sw2.sum())
        ses.append(shard.ess_spread(sw, sw2, n_boot=200)["rel_se"])
    scatter = np.std(pooled) / np.mean(pooled)
    assert 0.6 < np.mean(ses) / scatter < 1.5
    sw, sw2 = np.ones(10), np.ones(10)
    sw2[3] = 50.0
    r = shard.ess_spread(sw, sw2)
    assert r["lo"] < 0.5 and r["hi"] > 1.2


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one
    JSON line with the contract's keys, on a small sample."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--ref-traj", "2048"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
