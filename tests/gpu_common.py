"""Shared helpers of the GPU tests: library loading and per-trajectory
comparison of CUDA results with the FP64 oracle."""
import math

import numpy as np
import pytest

from paper_2410_13683_gb300 import build as B
from paper_2410_13683_gb300 import fpt

NEAR_TIE_REL = 1e-5        # tau = 1e-5 * (phi_in - phi_end)
MAX_MISMATCH = 0.01        # mismatched step counts allowed only for near-ties, <= 1%
LOGW_TOL = 1e-4            # |d ln w| <= 1e-4 max(1, |ln w|)


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    fpt.load()
    return torch


def gpu_run(ctx, runs, n_list, stream=None):
    """fpt_run with host output arrays; returns (status, [dict per run])."""
    outs = []
    for n in n_list:
        outs.append(dict(nsteps=np.zeros(n, np.int32), logw=np.zeros(n), status=np.zeros(n, np.uint8),
                         N=np.zeros(n)))
    st = fpt.fpt_run(ctx, runs, outs, stream)
    return st, outs


class _Sub:
    pass


def _subset(o, keep):
    s = _Sub()
    for k in ("nsteps", "logw", "status", "phi_final", "pi_final", "xmin_pre"):
        setattr(s, k, getattr(o, k)[keep])
    s.dN = o.dN
    s.phi_end_value = o.phi_end_value
    return s


def compare(g, o, x_in, label="", max_mismatch=MAX_MISMATCH, max_step_diff=None, pathwise_max_steps=None):
    """Per-trajectory parity of GPU outputs ``g`` with oracle trajectories ``o``.

    Step counts must be equal except for near-ties: trajectories whose FP64
    path had a pre-passage step within tau of the end surface or ended within
    tau below it (tau = 1e-5 x_in); those may differ and must stay <= 1%.
    Matching trajectories must agree in status, N (exactly: N = n dN) and
    ln w to 1e-4 max(1, |ln w|). Returns (mismatch fraction, near-tie fraction).

    pathwise_max_steps: trajectories longer than this (on either side) are
    compared in law only -- their numbers must agree within 4 binomial
    standard errors. Where the noise amplitude depends steeply on the field,
    a field error grows multiplicatively along the path, so FP32 and FP64
    paths of very long trajectories part by more than tau.
    """
    tau = NEAR_TIE_REL * x_in
    n = len(o.nsteps)
    assert len(g["nsteps"]) == n
    x_final = o.phi_final - o.phi_end_value
    near = (o.xmin_pre <= tau) | (x_final > -tau)
    mism = g["nsteps"].astype(np.int64) != o.nsteps
    if pathwise_max_steps is not None:
        lg, lo_ = g["nsteps"] > pathwise_max_steps, o.nsteps > pathwise_max_steps
        p = max(lo_.mean(), 1.0 / n)
        assert abs(int(lg.sum()) - int(lo_.sum())) <= 4 * math.sqrt(n * p * (1 - p)) + 1, \
            f"{label}: {lg.sum()} vs {lo_.sum()} trajectories longer than {pathwise_max_steps} steps"
        keep = ~(lg | lo_)
        g = {k: v[keep] for k, v in g.items()}
        o = _subset(o, keep)
        x_final = x_final[keep]
        near = near[keep]
        mism = mism[keep]
        n = int(keep.sum())
    bad = mism & ~near
    if bad.any():
        j = np.flatnonzero(bad)[:5]
        detail = ", ".join(f"#{i}: gpu {g['nsteps'][i]} oracle {o.nsteps[i]} xmin_pre/tau "
                           f"{o.xmin_pre[i] / tau:.3g} x_final/tau {x_final[i] / tau:.3g}" for i in j)
        raise AssertionError(f"{label}: {bad.sum()} non-near-tie step mismatches: {detail}")
    assert mism.mean() <= max_mismatch, f"{label}: mismatch fraction {mism.mean():.4f}"
    if max_step_diff is not None and mism.any():
        d = np.abs(g["nsteps"].astype(np.int64) - o.nsteps)[mism]
        assert d.max() <= max_step_diff, f"{label}: near-tie step difference {d.max()}"
    ok = ~mism
    assert np.array_equal(g["status"][ok], o.status[ok]), label
    np.testing.assert_array_equal(g["N"][ok], o.nsteps[ok] * o.dN)
    lw_err = np.abs(g["logw"][ok] - o.logw[ok])
    lim = LOGW_TOL * np.maximum(1.0, np.abs(o.logw[ok]))
    assert np.all(lw_err <= lim), f"{label}: max ln w error {np.max(lw_err / lim):.3g} x tolerance"
    return float(mism.mean()), float(near.mean())
