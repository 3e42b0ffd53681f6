"""Pooling a sampling job's runs (paper_2410_13683_gb300.accumulate) on CPU.

Per-run histograms come from the FP64 oracle's estimators on synthetic
weighted runs; the pooled estimates must equal the oracle's estimators on the
union of the runs' trajectories (weighted and lognormal estimators with their
errors, the tail set's ESS and probability), a job checkpointed after three
runs and resumed must equal one that never stopped bit for bit, and runs out
of order or with other bins are refused."""
import math

import numpy as np
import pytest

from oracle import estimators as E
from paper_2410_13683_gb300.accumulate import RunAccumulator

DN, N_LO, N_HI, NB, N_TAIL = 1e-3, 0.0, 8.0, 64, 5.0


def synthetic_run(k, n=4000):
    rng = np.random.default_rng(100 + k)
    nsteps = rng.gamma(6.0, 700.0, n).astype(np.int32) + 1
    logw = rng.normal(-0.002 * nsteps, 0.8)
    status = np.where(rng.random(n) < 0.01, 1, 0).astype(np.uint8)     # 1% capped
    return nsteps, logw, status


def run_hist(nsteps, logw, status):
    h = E.histogram(nsteps, logw, status, DN, N_LO, N_HI, NB)
    ess, p, k = E.tail_ess(nsteps, logw, status, DN, N_TAIL)
    return {"count": h.count, "log_sum_w": h.log_sum_w, "log_sum_w2": h.log_sum_w2, "sum_lw": h.sum_lw,
            "sum_lw2": h.sum_lw2, "n_total": h.n_total, "n_passed": int(np.sum(status == 0)),
            "n_capped": h.n_capped, "n_tail": k, "p_tail": p, "ess_tail": ess, "db": h.db}


def test_pooled_runs_equal_the_estimators_on_the_union():
    runs = [synthetic_run(k) for k in range(5)]
    acc = RunAccumulator(seed=7, N_lo=N_LO, N_hi=N_HI, n_bins=NB, N_tail=N_TAIL)
    for k, r in enumerate(runs):
        acc.add(k, run_hist(*r))
    est = acc.estimates()
    ns, lw, st = (np.concatenate([r[i] for r in runs]) for i in range(3))
    h = E.histogram(ns, lw, st, DN, N_LO, N_HI, NB)
    P, se = E.p_weighted(h)
    Pl, sel = E.p_lognormal(h)
    ess, p, _ = E.tail_ess(ns, lw, st, DN, N_TAIL)
    assert np.array_equal(est["count"], h.count) and est["n_total"] == len(ns)
    np.testing.assert_allclose(est["pdf"], P, rtol=1e-11)
    np.testing.assert_allclose(est["se_w"], se, rtol=1e-8, atol=1e-12 * np.max(se))
    np.testing.assert_allclose(est["pdf_ln"], Pl, rtol=1e-10, equal_nan=True)
    np.testing.assert_allclose(est["se_ln"], sel, rtol=1e-10, equal_nan=True)
    assert est["ess_tail"] == pytest.approx(ess, rel=1e-11)
    assert est["p_tail"] == pytest.approx(p, rel=1e-11)
    assert est["n_capped"] == int(np.sum(st != 0)) > 0


def test_checkpointed_job_resumes_bit_for_bit(tmp_path):
    hs = [run_hist(*synthetic_run(k)) for k in range(5)]
    full = RunAccumulator(seed=7, N_lo=N_LO, N_hi=N_HI, n_bins=NB, N_tail=N_TAIL)
    for k, h in enumerate(hs):
        full.add(k, h)
    part = RunAccumulator(seed=7, N_lo=N_LO, N_hi=N_HI, n_bins=NB, N_tail=N_TAIL)
    for k in range(3):
        part.add(k, hs[k])
    path = str(tmp_path / "job.npz")
    part.save(path)
    res = RunAccumulator.load(path)
    assert res.next_run == 3 and res.seed == 7 and math.isclose(res.N_tail, N_TAIL)
    for k in range(res.next_run, 5):
        res.add(k, hs[k])
    a, b = full.estimates(), res.estimates()
    for key in a:
        if isinstance(a[key], np.ndarray):
            assert np.array_equal(a[key], b[key], equal_nan=True), key
        else:
            assert a[key] == b[key], key


def test_runs_out_of_order_or_with_other_bins_are_refused():
    hs = [run_hist(*synthetic_run(k)) for k in range(2)]
    acc = RunAccumulator(seed=7, N_lo=N_LO, N_hi=N_HI, n_bins=NB, N_tail=N_TAIL)
    with pytest.raises(ValueError, match="order"):
        acc.add(1, hs[1])                     # run 0 skipped
    acc.add(0, hs[0])
    with pytest.raises(ValueError, match="order"):
        acc.add(0, hs[0])                     # run 0 twice
    other = dict(hs[1], db=hs[1]["db"] * 2)
    with pytest.raises(ValueError, match="bins"):
        acc.add(1, other)
    assert acc.next_run == 1
