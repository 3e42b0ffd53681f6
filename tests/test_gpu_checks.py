"""The bounds-checked debug build (libfpt_checks.so, -DFPT_CHECKS) on the GPU.

Every stepper variant and the histogram run once under the checked build in a
child process (FPT_CHECKS=1 selects the library): no check may fire (a fired
check turns fpt_sync or the histogram into FPT_E_STATE), and the results must
equal the plain build's bit for bit -- the checks only observe. The variants:
the sudden-transition model on its Bessel table (shared-memory table, direct
and constant bias), two models in one launch (tables read from global memory),
the full-rank 2-D noise table, the Gaussian bump (cubic drift table), the
N-indexed noise window, and the learned proposal.
"""
import os
import subprocess
import sys
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from paper_2410_13683_gb300 import build as B

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_cases():
    """Small runs of each variant through the library this process loaded;
    returns {case: array} with step counts, ln w and status, and histograms."""
    from paper_2410_13683_gb300 import fpt
    from paper_2410_13683_gb300 import train as TR
    from gpu_common import gpu_run

    out = {}

    def keep(name, g):
        for r, d in enumerate(g):
            for k in ("nsteps", "logw", "status"):
                out[f"{name}_{r}_{k}"] = d[k]

    n = 2048
    usr = replace(W.USR_MODEL, max_steps=1 << 16)
    with fpt.fpt_init_model([usr]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=5, run_id=0), fpt.run_desc(0, n, seed=5, run_id=1, A=2.0)],
                        [n, n])
        keep("usr", g)
        h = fpt.fpt_histogram(ctx, 1, 0.0, 20.0, 64, N_tail=8.0)
        out["usr_hist"] = np.concatenate([h["count"].astype(np.float64), h["pdf"], [h["p_tail"], h["ess_tail"]]])
        v = fpt.canonical_params(W.mlp_init(3, out_scale=0.5))
        prop = TR.new_proposal(ctx, v, shift=(0, 0, 0), scale=(2000.0, 1000.0, 0.2), segment=64, alpha_max=2.0)
        st, g = gpu_run(ctx, [prop.desc(0, n, seed=6, run_id=2)], [n])
        keep("mlp", g)
    two = W.batch_models(2, seed=9)
    two = [replace(m, max_steps=1 << 16) for m in two]
    with fpt.fpt_init_model(two) as ctx:
        for i in range(2):
            fpt.fpt_noise_table(ctx, i, fpt.FPT_TABLE_BESSEL, 256, 1.0)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=7, run_id=0, A=1.0), fpt.run_desc(1, n, seed=7, run_id=1)],
                        [n, n])
        keep("two", g)
    with fpt.fpt_init_model([usr]) as ctx:
        fpt.fpt_noise_table2(ctx, 0, fpt.FPT_TABLE_NUMERIC, 65, 1.0)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=8, A=0.7, A2=0.2)], [n])
        keep("rank2", g)
    bump = replace(W.BUMP_MODEL, max_steps=1 << 16)
    with fpt.fpt_init_model([bump]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        st, g = gpu_run(ctx, [fpt.run_desc(0, 512, seed=9, A=2.0)], [512])
        keep("bump", g)
    bm = W.BM.model
    with fpt.fpt_init_model([bm]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER_N, 16, 1.0, 0.25, 1.5, np.full(16, W.BM_S), np.zeros(16))
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=10, run_id=0), fpt.run_desc(0, n, seed=10, run_id=1, A=0.8)],
                        [n, n])
        keep("window", g)
    out["version"] = np.frombuffer(fpt.fpt_version().encode(), np.uint8)
    return out


def _child(path):
    np.savez(path, **run_cases())


def test_checked_build_fires_no_check_and_changes_nothing(torch, tmp_path):
    B.build(checks=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, FPT_CHECKS="1")
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_gpu_checks as t; t._child(%r)"
            % (HERE, ROOT, path))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    checked = dict(np.load(path))
    assert b"FPT_CHECKS" in checked.pop("version").tobytes()
    plain = run_cases()
    assert b"FPT_CHECKS" not in plain.pop("version").tobytes()
    assert sorted(checked) == sorted(plain)
    for k in plain:
        assert np.array_equal(checked[k], plain[k], equal_nan=True), k


@pytest.fixture(scope="module")
def torch():
    return require_gpu()
