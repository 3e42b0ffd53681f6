"""Per-trajectory parity of the learned-proposal stepper in the configuration
the benchmark times.

Configuration: the sudden-transition model with the 4096-point Bessel table,
step cap 2^19, network inputs (ln x, pi, N) shifted and scaled
(FPT_MLP_LOG_X, ln x floored at 2^-14 x_in), alpha held for 128-step
segments, |alpha| <= 8, and a
trained network: tests/golden/mlp_usr_trained.json, trained by the FP64
oracle (tests/golden/make_mlp_usr.py). 2^22 trajectories run through the C ABI
in one launch; the oracle recomputes a sample (random blocks of ids and the
last ids of the run) with the same network, its fp32 weights rounded to bf16
and its activations rounded to bf16 as the tensor cores take them.

The bar is the one of the constant-bias steppers: step counts identical except
near-ties and network partings, at most 1% of the sample; on identical step
counts |ln w_gpu - ln w_oracle| <= 1e-4 max(1, |ln w|) on every trajectory
that no network parting explains. A network parting: the two sides round a
network input or activation to bf16 in different directions (their values
differ by FP32 against FP64 arithmetic, ~1e-7 relative, and a value that close
to a rounding boundary goes either way), so alpha of one segment differs by a
bf16 step instead of ~1e-6. It is shown per trajectory: the GPU's alpha along
its own path (fpt_run_records) differs from the oracle's by more than the
forward tolerance at some segment, and the ln w difference that those alpha
differences predict, sum_s dalpha_s d ln w/d alpha_s with d ln w/d alpha_s =
-(alpha_s m_s dN + sqrt(dN) sum of xi over s) from the oracle's segment
records, accounts for the observed one within the bar. The log-field input is
floored (ln max(x, 2^-14 x_in)): without the floor, ln x of the two sides
differed by up to 1e-3 a step before passage.

Why partings happen at all on these paths: the GPU's FP32 Box-Muller normals
carry a mean error of about -1e-8 per draw against the FP64 ones (the segment
sums of xi show it, test below), so over a 150k-step path the field drifts by
~1e-10 from the oracle's. Near the end surface that moves the bf16-rounded
ln x input across a rounding boundary at a few segments per path (each parting
moves alpha by ~5e-3 for one segment and ln w by a few 1e-3), and it makes the
passage step of about 1% of the paths differ. On the constant-bias workloads,
30 times shorter, the same drift stays far below the near-tie band. So the
learned-proposal bar keeps every ln w within 1e-4 max(1, |ln w|) or explained
to that accuracy by its partings, and allows 2% step mismatches, each a near-tie
or after a parting.
"""
import json
import math
import os
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt
from paper_2410_13683_gb300 import train as TR

from gpu_common import LOGW_TOL, NEAR_TIE_REL, gpu_run, require_gpu

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "mlp_usr_trained.json")
FWD_TOL = 1e-5          # |alpha_gpu - alpha_oracle| <= FWD_TOL max(1, |alpha|) without a parting
MAX_MISMATCH = 0.02     # step-count mismatches (each a near-tie or after a parting)
MAX_PARTED_PATHS = 0.5  # paths with at least one parting


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.fixture(scope="module")
def setup():
    with open(FIXTURE) as f:
        fx = json.load(f)
    p = {k: np.asarray(fx["params"][k], np.float64).reshape(fx["shapes"][k]) for k in fx["params"]}
    m = replace(W.USR_MODEL, max_steps=1 << 19)
    res = OT.resolve(m)
    tab = OT.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=min(16, os.cpu_count() or 1))
    return fx, p, m, res, tab


def _sample_ids(n, blocks, width, seed):
    rng = np.random.default_rng(seed)
    starts = rng.integers(0, n // width - 1, blocks) * width
    return [(int(s), width) for s in np.unique(starts)] + [(n - width, width)]


def test_learned_stepper_matches_oracle_per_trajectory(torch, setup):
    fx, p, m, res, tab = setup
    n = 1 << 22
    seed = 4
    shift, scale = tuple(fx["shift"]), tuple(fx["scale"])
    seg, amax = int(fx["segment"]), float(fx["alpha_max"])
    v = fpt.canonical_params(p)
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
        prop = TR.new_proposal(ctx, v, shift=shift, scale=scale, segment=seg, alpha_max=amax,
                               flags=fpt.FPT_MLP_LOG_X, x_floor=fx["x_floor"])
        out = dict(nsteps=torch.zeros(n, dtype=torch.int32, device="cuda"),
                   logw=torch.zeros(n, dtype=torch.float64, device="cuda"),
                   status=torch.zeros(n, dtype=torch.uint8, device="cuda"))
        st = fpt.fpt_run(ctx, [prop.desc(0, n, seed=seed, run_id=0)], [out])
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
        assert fpt.fpt_sync(ctx) in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
        blocks = _sample_ids(n, 10, 64, 7)
        ids = np.concatenate([np.arange(s, s + w) for s, w in blocks])
        idx = torch.as_tensor(ids, device="cuda")
        g = {k: t[idx].cpu().numpy() for k, t in out.items()}
        del out

        mlp = OS.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, alpha_max=amax, round_bf16=True,
                         log_x=True, x_floor=fx["x_floor"])
        rows = [OS.run(m, res, tab, seed=seed, run_id=0, n=w, traj0=s, mlp=mlp) for s, w in blocks]
        o = {k: np.concatenate([getattr(r, k) for r in rows])
             for k in ("nsteps", "logw", "status", "phi_final", "xmin_pre")}
        tau = NEAR_TIE_REL * (res.phi_in - res.phi_end)
        near = (o["xmin_pre"] <= tau) | (o["phi_final"] - res.phi_end > -tau)
        same = g["nsteps"].astype(np.int64) == o["nsteps"]
        lw_err = np.abs(g["logw"] - o["logw"])
        lim = LOGW_TOL * np.maximum(1.0, np.abs(o["logw"]))
        bad = ~same | (lw_err > lim)

        # each trajectory off the bar: explained by a network parting (or, for a
        # step mismatch, a near-tie)
        explained, parted = 0, 0
        details = []
        for j in np.flatnonzero(bad):
            tid = int(ids[j])
            tr = OS.run_segments(m, res, tab, mlp, seed=seed, run_id=0, traj=tid, cap=1 << 13)
            assert tr["nsteps"] == o["nsteps"][j] and tr["logw"] == pytest.approx(o["logw"][j], rel=1e-12)
            # the GPU's own alpha along its path (segment records of the same trajectory)
            rec = fpt.fpt_run_records(ctx, prop.desc(0, 1, seed=seed, run_id=0, traj_offset=tid), cap=1 << 13)
            k = min(len(rec["raw"]), len(tr["alpha"]))
            d = np.zeros(len(tr["alpha"]))
            d[:k] = np.clip(rec["raw"][:k], -amax, amax) - tr["alpha"][:k]
            part = np.abs(d) > FWD_TOL * np.maximum(1.0, np.abs(tr["alpha"]))
            k = len(tr["alpha"])
            msteps = np.full(k, float(seg))
            msteps[-1] = tr["nsteps"] - seg * (k - 1)
            dlw_da = -(tr["alpha"] * msteps * m.dN + math.sqrt(m.dN) * tr["sum_xi"])
            pred = float(np.sum(d * dlw_da))
            if part.any():
                parted += 1
            if same[j]:
                ok = part.any() and abs(g["logw"][j] - o["logw"][j] - pred) <= lim[j]
            else:
                ok = bool(near[j]) or part.any()
            explained += int(ok)
            details.append(f"#{tid}: steps {g['nsteps'][j]}/{o['nsteps'][j]} dlnw {g['logw'][j] - o['logw'][j]:+.3g} "
                           f"pred {pred:+.3g} partings {int(part.sum())}/{k} first {int(np.argmax(part)) if part.any() else -1}"
                           f" near {bool(near[j])}")
    print(f"learned parity: {len(ids)} sampled, identical steps {same.mean():.3%}, "
          f"off the bar {bad.sum()}, explained {explained}, parted {parted}; mean N {o['nsteps'].mean() * m.dN:.1f}, "
          f"ln w in [{o['logw'].min():.1f}, {o['logw'].max():.1f}]")
    for line in details[:20]:
        print("  " + line)
    assert explained == bad.sum(), "unexplained trajectories:\n" + "\n".join(details)
    assert np.mean(~same) <= MAX_MISMATCH
    # partings are bf16 rounding decisions; their number follows the field's FP32
    # drift near the end surface (see the module docstring), bounded loosely here
    assert parted <= MAX_PARTED_PATHS * len(ids)
    # the configuration is the one timed: long tail paths with spread-out weights
    assert o["nsteps"].mean() * m.dN > 20.0
    assert np.std(o["logw"]) > 1.0


def test_network_forward_matches_oracle_on_trained_weights(torch, setup):
    """The stepper's device forward (fpt_mlp_eval) against the oracle's FP64
    forward with bf16 operands, on states along oracle paths of the trained
    network: all but a small fraction agree within the forward tolerance, and
    the rest differ by about one bf16 step of one activation."""
    fx, p, m, res, tab = setup
    shift, scale = tuple(fx["shift"]), tuple(fx["scale"])
    seg, amax = int(fx["segment"]), float(fx["alpha_max"])
    mlp = OS.MLPBias(p, segment=seg, in_shift=shift, in_scale=scale, alpha_max=amax, round_bf16=True, log_x=True,
                     x_floor=fx["x_floor"])
    S_, A_, T_ = [], [], []
    for j in range(24):
        tr = OS.run_segments(m, res, tab, mlp, seed=77, run_id=0, traj=j, cap=1 << 13)
        S_.append(tr["state"]); A_.append(tr["alpha"]); T_.append(tr["tan_theta"])
    st, al, tt = np.concatenate(S_), np.concatenate(A_), np.concatenate(T_)
    s_norm = ((st - np.asarray(shift)) * np.asarray(scale)).astype(np.float32)
    with fpt.fpt_init_model([m]) as ctx:
        blob = torch.zeros(fpt.FPT_MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
        fpt.fpt_mlp_pack(ctx, torch.tensor(fpt.canonical_params(p), device="cuda"), blob)
        a = np.asarray(fpt.fpt_mlp_eval(ctx, blob, s_norm, tt.astype(np.float32), amax)[0], np.float64)
    d = np.abs(a - al)
    off = d > FWD_TOL * np.maximum(1.0, np.abs(al))
    print(f"forward on {len(al)} path states: {off.mean():.3%} beyond {FWD_TOL:g}; "
          f"median diff {np.median(d):.2e}, max {d.max():.2e}; alpha in [{al.min():.2f}, {al.max():.2f}]")
    assert off.mean() < 0.05
    assert np.all(d < 5e-2 * np.maximum(1.0, np.abs(al)))


def test_learned_segments_match_oracle(torch, setup):
    """Segment by segment along whole learned-proposal paths of the timed
    configuration: the GPU's segment records (fpt_run_records: network inputs,
    tan theta, alpha, sum of xi, first step) against the oracle's segments of
    the same trajectories. Inputs agree to FP32 rounding, alpha to the forward
    tolerance except at partings, the noise sums to FP32 Box-Muller accuracy.
    The ln w that the GPU's own records imply, -sum_s [alpha_s sqrt(dN) S_s +
    alpha_s^2 m_s dN / 2] in FP64, is compared with the GPU's accumulated ln w
    and with the oracle's: this splits a ln w difference into what the path
    (alpha, noise) did and what the in-kernel accumulation did."""
    fx, p, m, res, tab = setup
    shift, scale = np.asarray(fx["shift"]), np.asarray(fx["scale"])
    seg, amax = int(fx["segment"]), float(fx["alpha_max"])
    v = fpt.canonical_params(p)
    mlp = OS.MLPBias(p, segment=seg, in_shift=tuple(shift), in_scale=tuple(scale), alpha_max=amax,
                     round_bf16=True, log_x=True, x_floor=fx["x_floor"])
    ids = [232901, 232907, 232908, 232918, 232933, 944513, 5, 77]
    sdN = math.sqrt(m.dN)
    rows = []
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
        prop = TR.new_proposal(ctx, v, shift=tuple(shift), scale=tuple(scale), segment=seg, alpha_max=amax,
                               flags=fpt.FPT_MLP_LOG_X, x_floor=fx["x_floor"])
        for tid in ids:
            d = prop.desc(0, 1, seed=4, run_id=0, traj_offset=tid)
            st, g = gpu_run(ctx, [d], [1])
            rec = fpt.fpt_run_records(ctx, d, cap=1 << 13)
            tr = OS.run_segments(m, res, tab, mlp, seed=4, run_id=0, traj=tid, cap=1 << 13)
            k = min(len(rec["raw"]), len(tr["alpha"]))
            s_or = (tr["state"][:k] - shift) * scale
            din = np.abs(rec["in"][:k] - s_or).max(axis=0)
            a_gpu = np.clip(rec["raw"][:k], -amax, amax)
            da = np.abs(a_gpu - tr["alpha"][:k])
            dxi = np.abs(rec["sum_xi"][:k] - tr["sum_xi"][:k])
            steps = np.diff(np.append(rec["n0"][:k], g[0]["nsteps"][0]))
            lw_rec = -float(np.sum(a_gpu * sdN * rec["sum_xi"][:k] + 0.5 * a_gpu ** 2 * steps * m.dN))
            rows.append((tid, int(g[0]["nsteps"][0]), int(tr["nsteps"]), float(g[0]["logw"][0]), lw_rec,
                         float(tr["logw"]), din, float(np.max(da)), float(np.median(da)), int(np.sum(da > 1e-5)),
                         float(np.max(dxi)), float(np.mean(rec["sum_xi"][:k] - tr["sum_xi"][:k]))))
    for r in rows:
        print(f"#{r[0]}: steps {r[1]}/{r[2]}; ln w gpu {r[3]:.6f} from gpu records {r[4]:.6f} oracle {r[5]:.6f}; "
              f"max |d in| {r[6][0]:.2e} {r[6][1]:.2e} {r[6][2]:.2e}; |d alpha| max {r[7]:.2e} median {r[8]:.2e} "
              f"(> 1e-5: {r[9]}); |d sum xi| max {r[10]:.2e} mean d {r[11]:+.2e}")
    for r in rows:
        lim = LOGW_TOL * max(1.0, abs(r[5]))
        # the GPU's accumulated ln w equals what its own records imply
        assert abs(r[3] - r[4]) <= lim, r[0]
        # pi and N inputs agree to FP32 rounding; alpha to 1e-6 on most segments
        assert r[6][1] < 1e-6 and r[6][2] < 1e-6, r[0]
        assert r[8] < 1e-6, r[0]
        # noise sums (paths of equal length): FP32 Box-Muller error, a mean offset of
        # order 1e-6 per 128 normals
        if r[1] == r[2]:
            assert abs(r[11]) < 5e-6, r[0]
