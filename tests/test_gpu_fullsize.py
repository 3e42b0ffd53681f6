"""Parity at the full sizes of the benchmark workloads, through the same
launch path the benchmark times: the GPU runs every trajectory, the FP64
oracle recomputes a sample of them one by one (spread over the whole range,
plus the last ids of each run, where the refill ends ragged)."""
import os
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt
from paper_2410_13683_gb300 import train as TR

from gpu_common import compare, require_gpu

pytestmark = pytest.mark.gpu
PROCS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


class _Traj:
    pass


def oracle_sample(m, res, tab, seed, run_id, ids, A=0.0, mlp=None):
    """Oracle trajectories for the given ids, one call each."""
    rows = [OS.run(m, res, tab, seed=seed, run_id=run_id, n=1, traj0=int(i), A=A, mlp=mlp) for i in ids]
    o = _Traj()
    for k in ("nsteps", "logw", "status", "phi_final", "pi_final", "xmin_pre"):
        setattr(o, k, np.concatenate([getattr(r, k) for r in rows]))
    o.dN = m.dN
    o.phi_end_value = res.phi_end
    return o


def sample_ids(n, k, seed):
    rng = np.random.default_rng(seed)
    ids = np.unique(np.concatenate([rng.integers(0, n, k), np.arange(max(0, n - 64), n)]))
    return ids


def device_out(torch, n):
    return dict(nsteps=torch.zeros(n, dtype=torch.int32, device="cuda"),
                logw=torch.zeros(n, dtype=torch.float64, device="cuda"),
                status=torch.zeros(n, dtype=torch.uint8, device="cuda"),
                N=torch.zeros(n, dtype=torch.float64, device="cuda"))


def gather(torch, out, ids):
    idx = torch.as_tensor(ids, device="cuda")
    return {k: v[idx].cpu().numpy() for k, v in out.items()}


@pytest.fixture(scope="module")
def usr4096():
    m = W.USR_MODEL
    res = OT.resolve(m)
    return m, res, OT.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=PROCS)


def test_full_usr_direct_2e22(torch, usr4096):
    """Sudden transition, 4096-point Bessel table, 2^22 trajectories, direct."""
    m, res, tab = usr4096
    n = 1 << 22
    with fpt.fpt_init_model([m]) as ctx:
        S, Sp = fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 4096, 1.0)
        np.testing.assert_allclose(S, tab.S, rtol=1e-8)
        out = device_out(torch, n)
        assert fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=2, run_id=0)], [out]) == fpt.FPT_OK
        torch.cuda.synchronize()
        ids = sample_ids(n, 1024, 1)
        g = gather(torch, out, ids)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 400.0, 512)
    assert h["n_total"] == n and h["n_passed"] + h["n_capped"] == n
    o = oracle_sample(m, res, tab, 2, 0, ids)
    mism, near = compare(g, o, res.phi_in - res.phi_end, "full usr direct")
    print(f"full usr direct: {len(ids)} sampled, mismatch {mism:.4%}, near-ties {near:.4%}")


def test_full_usr_eight_biases_one_launch(torch, usr4096):
    """The constant-bias sweep: 8 amplitudes x 2^24 trajectories (2^27) in one
    persistent launch with uneven lengths and capped paths."""
    m, res, tab = usr4096
    n = 1 << 24
    As = W.USR_FIXED_BIAS.biases
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 4096, 1.0)
        outs = [device_out(torch, n) for _ in As]
        runs = [fpt.run_desc(0, n, seed=3, run_id=r, A=A) for r, A in enumerate(As)]
        assert fpt.fpt_run(ctx, runs, outs) in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
        torch.cuda.synchronize()
        samples = []
        for r in range(len(As)):
            ids = sample_ids(n, 48, 10 + r)
            samples.append((ids, gather(torch, outs[r], ids)))
        del outs
    for r, A in enumerate(As):
        ids, g = samples[r]
        o = oracle_sample(m, res, tab, 3, r, ids, A=A)
        mism, near = compare(g, o, res.phi_in - res.phi_end, f"full usr A={A}")
        print(f"full usr A={A}: {len(ids)} sampled, mismatch {mism:.4%}, near-ties {near:.4%}")


def test_full_usr_learned_2e26(torch, usr4096):
    """The learned-proposal configuration at its production size, 2^26
    trajectories, with a fixed random network (bf16 on tensor cores against the
    oracle's FP64 forward on bf16-rounded operands: paths may part where the
    two networks' outputs differ in the last bits, so the bar is the one of the
    statistical MLP test, per sampled trajectory)."""
    m, res, tab = usr4096
    n = 1 << 26
    p = W.mlp_init(31, out_scale=0.3)
    v = fpt.canonical_params(p)
    p32 = fpt.params_dict(v)
    x_in = res.phi_in - res.phi_end
    shift, scale, seg, amax = (0.0, 0.0, 0.0), (1.0 / x_in, 1.0 / abs(res.pi_in), 0.2), 64, 2.0
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 4096, 1.0)
        prop = TR.new_proposal(ctx, v, shift=shift, scale=scale, segment=seg, alpha_max=amax)
        out = device_out(torch, n)
        assert fpt.fpt_run(ctx, [prop.desc(0, n, seed=4, run_id=0)], [out]) in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
        torch.cuda.synchronize()
        ids = sample_ids(n, 512, 2)
        g = gather(torch, out, ids)
        del out
    mlp = OS.MLPBias(p32, segment=seg, in_shift=shift, in_scale=scale, alpha_max=amax, round_bf16=True)
    o = oracle_sample(m, res, tab, 4, 0, ids, mlp=mlp)
    same = g["nsteps"] == o.nsteps
    assert same.mean() > 0.8, same.mean()
    rel = np.abs(g["logw"][same] - o.logw[same]) / np.maximum(1.0, np.abs(o.logw[same]))
    assert np.median(rel) < 1e-3
    assert np.std(o.logw) > 0.01
    print(f"full learned: {len(ids)} sampled, identical steps {same.mean():.2%}")


def test_full_batched_64_models(torch):
    """The batched sweep: 64 models (sudden-transition family) x 2^20
    trajectories in one launch, tables read through L1; 64-point Bessel tables
    on both sides keep the oracle's table build short."""
    models = W.batch_models(64)
    n, pts = 1 << 20, 64
    with fpt.fpt_init_model(models) as ctx:
        for i in range(len(models)):
            fpt.fpt_noise_table(ctx, i, fpt.FPT_TABLE_BESSEL, pts, 1.0)
        outs = [device_out(torch, n) for _ in models]
        runs = [fpt.run_desc(i, n, seed=5, run_id=i) for i in range(len(models))]
        assert fpt.fpt_run(ctx, runs, outs) in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
        torch.cuda.synchronize()
        samples = []
        for i in range(len(models)):
            ids = sample_ids(n, 8, 100 + i)
            samples.append((ids, gather(torch, outs[i], ids)))
        del outs
    mism_all = []
    for i, m in enumerate(models):
        res = OT.resolve(m)
        tab = OT.bessel_table(m, res, pts, 1.0, processes=PROCS)
        ids, g = samples[i]
        o = oracle_sample(m, res, tab, 5, i, ids)
        mism, _ = compare(g, o, res.phi_in - res.phi_end, f"batched model {i}", max_mismatch=1.0)
        mism_all.append(mism)
    assert np.mean(mism_all) <= 0.02
