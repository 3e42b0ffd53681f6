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
    """128 runs (the maximum) in one launch equal the same runs launched one
    by one: the binary search from launch unit to run is exact."""
    m = W.BM.model
    S, T = np.full(16, W.BM_S), np.zeros(16)
    sizes = [(i * 37) % 200 for i in range(128)]         # uneven, including empty runs
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


def test_runs_with_their_own_networks_match_separate_calls(torch):
    """One launch with learned-proposal runs that carry different networks,
    input normalisations and clamps, next to constant-bias and direct runs,
    on two models (tables through L1) and on one model (staged table): every
    run equals the same run launched alone with its own network, bit for bit
    (a lane's network output depends only on its own inputs), and the learned
    runs differ from one another."""
    from paper_2410_13683_gb300 import train as TR
    m = W.BM.model
    S, T = np.full(16, W.BM_S), np.zeros(16)
    nets = []
    for k, (sd, sc, amax, seg) in enumerate([(31, 0.4, 2.0, 64), (32, 0.3, 1.0, 64), (33, 0.5, 3.0, 64)]):
        nets.append((fpt.canonical_params(W.mlp_init(sd, out_scale=sc)), amax,
                     (0.02 * k, -0.01, 1.0), (30.0 + 5 * k, 100.0, 0.2 + 0.1 * k)))
    for two_models in (False, True):
        models = [m, m] if two_models else [m]
        with fpt.fpt_init_model(models) as ctx:
            for i in range(len(models)):
                fpt.fpt_noise_table(ctx, i, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, S * (1 + 0.1 * i), T)
            props = [TR.new_proposal(ctx, v, shift=sh, scale=sc, segment=64, alpha_max=amax)
                     for v, amax, sh, sc in nets]
            sizes = [3000, 2500, 0, 2000, 1500, 1200]
            runs = [props[0].desc(0, sizes[0], seed=71, run_id=0),
                    fpt.run_desc(len(models) - 1, sizes[1], seed=71, run_id=1, A=0.7),
                    props[1].desc(0, sizes[2], seed=71, run_id=2),
                    props[1].desc(len(models) - 1, sizes[3], seed=71, run_id=3),
                    fpt.run_desc(0, sizes[4], seed=71, run_id=4),
                    props[2].desc(0, sizes[5], seed=71, run_id=5)]
            st, together = gpu_run(ctx, runs, sizes)
            assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
            for i, r in enumerate(runs):
                if sizes[i] == 0:
                    continue
                st, alone = gpu_run(ctx, [r], [sizes[i]])
                assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
                assert np.array_equal(alone[0]["nsteps"], together[i]["nsteps"]), (two_models, i)
                assert np.array_equal(alone[0]["logw"], together[i]["logw"]), (two_models, i)
            # the networks make a difference: same ids under networks 0 and 2
            st, a0 = gpu_run(ctx, [props[0].desc(0, 1000, seed=72, run_id=0)], [1000])
            st, a2 = gpu_run(ctx, [props[2].desc(0, 1000, seed=72, run_id=0)], [1000])
            assert not np.array_equal(a0[0]["logw"], a2[0]["logw"])
            # a different segment length in one call is refused
            bad = props[1].desc(0, 100, seed=71, run_id=9)
            bad.mlp_segment = 128
            with pytest.raises(fpt.FptError) as e:
                fpt.fpt_run(ctx, [props[0].desc(0, 100, seed=71, run_id=8), bad])
            assert e.value.status == fpt.FPT_E_INVALID and "mlp_segment" in str(e.value)
