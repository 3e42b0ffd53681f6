"""Batched launches: several models (each with its own noise table, read
through L1 instead of shared memory) and biases in one persistent launch,
checked trajectory by trajectory against the FP64 oracle."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt

from gpu_common import compare, gpu_run, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def test_multi_model_launch_parity(torch):
    fam = [replace(m, max_steps=1 << 15) for m in W.batch_models(64)[:4]]
    lin = W.LINEAR.model
    models = fam + [lin]
    n_pts = 256
    runs, expect = [], []
    with fpt.fpt_init_model(models) as ctx:
        for i, m in enumerate(fam):
            fpt.fpt_noise_table(ctx, i, fpt.FPT_TABLE_BESSEL, n_pts, 1.0)
        fpt.fpt_noise_table(ctx, len(fam), fpt.FPT_TABLE_DESITTER, 1024, 1.0, 0.0, 0.06)
        n = 1024
        for i in range(len(models)):
            A = 0.0 if i % 2 == 0 else 0.5
            runs.append(fpt.run_desc(i, n, seed=50, run_id=i, A=A, traj_offset=7 * i))
            expect.append(A)
        st, g = gpu_run(ctx, runs, [n] * len(runs))
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    for i, m in enumerate(models):
        res = OT.resolve(m)
        if i < len(fam):
            tab = OT.bessel_table(m, res, n_pts, 1.0, processes=8)
        else:
            tab = OT.desitter_table(m, res, 1024, 0.0, 0.06)
        o = OS.run(m, res, tab, seed=50, run_id=i, n=n, A=expect[i], traj0=7 * i)
        o.phi_end_value = res.phi_end
        compare(g[i], o, res.phi_in - res.phi_end, f"model {i}")


def test_many_runs_one_model_match_separate_calls(torch):
    """64 runs (the maximum) in one launch equal the same runs launched one
    by one: the binary search from launch unit to run is exact."""
    m = W.BM.model
    S, T = np.full(16, W.BM_S), np.zeros(16)
    sizes = [(i * 37) % 200 for i in range(64)]          # uneven, including empty runs
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, S, T)
        runs = [fpt.run_desc(0, n, seed=60, run_id=i, A=0.1 * (i % 5)) for i, n in enumerate(sizes)]
        _, together = gpu_run(ctx, runs, sizes)
        for i, r in enumerate(runs):
            if sizes[i] == 0:
                continue
            _, alone = gpu_run(ctx, [r], [sizes[i]])
            assert np.array_equal(alone[0]["nsteps"], together[i]["nsteps"])
            assert np.array_equal(alone[0]["logw"], together[i]["logw"])
