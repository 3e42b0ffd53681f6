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


def compare(g, o, x_in, label="", max_mismatch=MAX_MISMATCH, max_step_diff=None):
    """Per-trajectory parity of GPU outputs ``g`` with oracle trajectories ``o``.

    Step counts must be equal except for near-ties: trajectories whose FP64
    path had a pre-passage step within tau of the end surface or ended within
    tau below it (tau = 1e-5 x_in); those may differ and must stay <= 1%.
    Matching trajectories must agree in status, N (exactly: N = n dN) and
    ln w to 1e-4 max(1, |ln w|). Returns (mismatch fraction, near-tie fraction).
    """
    tau = NEAR_TIE_REL * x_in
    n = len(o.nsteps)
    assert len(g["nsteps"]) == n
    x_final = o.phi_final - o.phi_end_value
    near = (o.xmin_pre <= tau) | (x_final > -tau)
    mism = g["nsteps"].astype(np.int64) != o.nsteps
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
