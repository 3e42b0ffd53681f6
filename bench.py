#!/usr/bin/env python
"""Benchmark: effective first-passage samples per second in the far tail.

Workload: the sudden-transition (ultra-slow-roll) piecewise-linear model with
relative slopes (V0 = 2e-10, a+ = 1e-3, a- = 1e-6, phi* = 1; start 0.0953
e-folds and end 5 e-folds after the transition on the background), the
4096-point Bessel-matched noise table at sigma = 1, dN = 1e-3. One step is a
full pass of the sampler over a fresh batch of trajectories: the persistent
Euler-Maruyama launch with the importance-sampling proposal (noise, table
lookup, drift, bias, update, log-weight, passage, refill) followed by the
weighted histogram and its FP64 finalisation. The metric is the effective
sample size of the tail set T = {N >= N_12} (CCDF(N_12) = 1e-12) per second:
ESS_T = (sum_T w)^2 / sum_T w^2, summed over all steps and ranks.

The proposal is the learned MLP bias (trained first, untimed, by the
library's own forward/backward kernels and reported separately); the
constant-bias proposal (the comparison run) and direct sampling are measured on the
same GPU for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own trajectory range (weak scaling); the
only exchange is a sum of the tail weight sums. ``--impl reference`` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from dataclasses import replace

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "effective first-passage samples/sec at tail P(dN)<=1e-12"
USR_MODEL_TEXT = "piecewise-linear USR, V0=2e-10 a+=1e-3 a-=1e-6, phi*=1"
UNIT = "samples/s"
TAIL_P = 1e-12

# Source-level operation count of one Euler-Maruyama step of the weighted
# stepper (thread instructions): table lookup 10, drift 9, momentum update 4,
# field increment + compensated add 7, log-weight (Kahan) 5, counter + passage
# 5, predication 2, Philox4x32-10 (40 per 4 steps) 10, uniforms + Box-Muller
# (32 per 4 normals) 8. The learned proposal adds one network evaluation per
# 128-step segment: 44 mma + 61 fragment loads + 128 SiLU (4 each) + 64 packs +
# ~40 shuffles/selects per lane = ~760, i.e. 6 per step.
INSTR_PER_STEP = 60
# The learned proposal's roofline counts the same 60 algorithmic slots per step
# (the step itself); the network's amortised cost (~8 per step with the
# exponential-based SiLU) is reported beside it as frac_incl_network.
INSTR_PER_STEP_MLP = 60
INSTR_NETWORK_PER_STEP = 8
# Full-rank (2-D) stepper, per step: Philox (40 per 2 steps) 20, uniforms +
# Box-Muller for 2 normals 16, two-entry table lookup + 3 interpolations 16,
# drift 9, (phi, pi) update 8, field compensated add 4, log-weight (Kahan) 7,
# counter + passage 5, predication 2.
INSTR_PER_STEP_2D = 87
# Bump stepper: the plain step with the drift from the cubic table (index 5,
# Horner 3, load 1) instead of the closed form (6), and the compensated
# momentum (+3).
INSTR_PER_STEP_BUMP = 66
# Noise-window stepper: the plain step with the table coordinate from the
# step count (+1) and the window test with its four selects (+6).
INSTR_PER_STEP_NIDX = 67
# Training recipe of the learned proposal (log-variance loss towards
# e^{lambda min(N, N_cut)} P, N_cut raised to N_12 by a curriculum), then
# model selection: from round select_from on, every select_every rounds, the
# proposal runs val_runs times on val_traj held-out trajectories (Philox seed
# val_seed) and the checkpoint with the most pooled tail ESS per EM step is
# kept.
TRAIN = dict(rounds=550, n_traj=1 << 18, lam=0.25, alpha_max=8.0, segment=128, lr0=3e-3, lr_min=3e-4,
             select_from=450, select_every=25, val_traj=1 << 22, val_runs=4, val_seed=31337)
SM_LANES = 128
# Floor of the log-field network input, relative to x_in: ln max(x, 2^-14 x_in)
X_FLOOR_REL = 2.0 ** -14
# Constant amplitudes compared with the learned proposal. Larger ones send the
# paths past the step cap (2^19 steps): at A = 1 85% of them, at A >= 3 all.
FIXED_SWEEP = (0.25, 0.375, 0.5, 0.625, 0.75, 1.0)


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def load_tail():
    with open(os.path.join(ROOT, "tests", "golden", "usr_tail.json")) as f:
        return json.load(f)


def usr_model():
    return replace(W.USR_MODEL, max_steps=1 << 19)


class Clocks:
    """nvidia-smi sampler for the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            os.unlink(self.path)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clocks(f)
        os.unlink(self.path)
        return out


def parse_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in
    nvidia-smi samples of Clocks.FIELDS (csv, noheader, nounits)."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        p = [x.strip() for x in line.split(",")]
        if len(p) < 9:
            continue
        try:
            sm.append(float(p[1]))
            smax.append(float(p[2]))
        except ValueError:
            continue
        for name, v in zip(names, p[5:9]):
            if v.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def roofline(steps_per_launch, launch_ms, sm_count, sm_max_mhz, traffic, instr_per_step):
    """Issue-slot roofline of the stepper: thread instructions per second."""
    achieved = steps_per_launch * instr_per_step / (launch_ms * 1e-3) / 1e12
    peak = sm_count * SM_LANES * sm_max_mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "Tinst/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "kernel": "em_kernel<weighted, smem table, MLP>", "instr_per_step": instr_per_step,
            "peak_source": f"{sm_count} SMs x {SM_LANES} lanes x {sm_max_mhz:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)"}


def pipe_fractions(steps_per_s, sm_count, sm_max_mhz):
    """FP32-pipe, XU (special-function) and executed-issue fractions of the
    learned stepper at the measured EM-step rate, from the per-step pipe counts
    of its ncu capture (profiles/em_kernel_mlp_usr_timed.json, taken at the
    timed configuration): thread instructions per step on the FMA pipes
    against SMs x 128 lanes x clock, on the XU against SMs x 16 x clock, and
    all executed thread instructions against the issue peak."""
    path = os.path.join(ROOT, "profiles", "em_kernel_mlp_usr_timed.json")
    try:
        with open(path) as f:
            pr = json.load(f)
    except (OSError, ValueError):
        return None
    clk = sm_max_mhz * 1e6
    per = pr.get("per_step", {})
    out = {"pipes_source": f"profiles/em_kernel_mlp_usr_timed.json (ncu, commit {pr.get('commit', '?')})"}
    if "thread_inst_fma" in per:
        out["fp32_pipe_frac"] = round(per["thread_inst_fma"] * steps_per_s / (sm_count * SM_LANES * clk), 4)
    if "thread_inst_xu" in per:
        out["xu_frac"] = round(per["thread_inst_xu"] * steps_per_s / (sm_count * 16 * clk), 4)
    if "thread_inst" in per:
        out["executed_instr_per_step"] = per["thread_inst"]
        out["issue_frac_executed"] = round(per["thread_inst"] * steps_per_s / (sm_count * SM_LANES * clk), 4)
    return out


def cpu_oracle_sample(model_res_tab, A, N_tail, n, seed=7):
    """The FP64 oracle on the host cores: ESS_T per second on n trajectories."""
    from oracle import estimators as E
    from oracle import stepper as OS
    m, res, tab = model_res_tab
    t0 = time.perf_counter()
    tr = OS.run(m, res, tab, seed=seed, run_id=0, n=n, A=A)
    dt = time.perf_counter() - t0
    e, p, k = E.tail_ess(tr.nsteps, tr.logw, tr.status, m.dN, N_tail)
    return e, dt, OS.max_threads(), int(tr.nsteps.sum())


def reference_arm(args, rank):
    if rank != 0:
        return 0
    from oracle import tables as OT
    tail = load_tail()
    m = usr_model()
    res = OT.resolve(m)
    tab = OT.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=os.cpu_count())
    A = tail["A"]
    n = args.ref_traj
    for _ in range(args.warmup):
        cpu_oracle_sample((m, res, tab), A, tail["N_12"], max(256, n // 8))
    tot_e = tot_t = 0.0
    cores = 1
    for k in range(args.steps):
        e, dt, cores, _ = cpu_oracle_sample((m, res, tab), A, tail["N_12"], n, seed=100 + k)
        tot_e += e
        tot_t += dt
    v = tot_e / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "usr_fixed_bias_tail", "model": USR_MODEL_TEXT,
                       "proposal": f"constant A={A} (the paper's bias; the learned network is a GPU training product)",
                       "n_traj_per_step": n, "N_tail": tail["N_12"], "table_points": W.USR_TABLE.n_points,
                       "dN": m.dN, "max_steps": m.max_steps},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} trajectories per step, FP64 C oracle, OpenMP"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def train_proposal(ctx, fpt, TR, info, N_tail, seed=4):
    """Train the learned proposal (untimed): returns (proposal, seconds)."""
    import torch
    x_in = info["phi_in"] - info["phi_end"]
    p_in = abs(info["pi_in"])
    v0 = fpt.canonical_params(W.mlp_init(21, out_scale=0.0))
    prop = TR.new_proposal(ctx, v0, shift=(math.log(x_in), 0.0, 0.0), scale=(0.2, 1.0 / p_in, 0.01),
                           segment=TRAIN["segment"], alpha_max=TRAIN["alpha_max"], flags=fpt.FPT_MLP_LOG_X,
                           x_floor=x_in * X_FLOOR_REL)
    lr = lambda r: TRAIN["lr0"] if r < 20 else max(TRAIN["lr_min"], TRAIN["lr0"] * 0.98 ** (r - 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = usr_model()
    TR.train_select(ctx, prop, 0, rounds=TRAIN["rounds"],
                    checkpoints=range(TRAIN["select_from"], TRAIN["rounds"], TRAIN["select_every"]),
                    val_traj=TRAIN["val_traj"], val_seed=TRAIN["val_seed"], val_runs=TRAIN["val_runs"],
                    N_tail=N_tail,
                    max_steps=m.max_steps, dN=m.dN,
                    n_traj=TRAIN["n_traj"], seed=seed, lam=TRAIN["lam"],
                    N_cut=lambda r: min(N_tail, 10.0 * 1.3 ** r), lr=lr, chunk=1 << 18)
    torch.cuda.synchronize()
    return prop, time.perf_counter() - t0


# The far-tail leg (tail probability 1e-20): the proposal trained for N_12 is
# trained further towards N_20 (warm start, N_cut raised from N_12 to N_20),
# with held-out selection, then timed on steps of 2^22 trajectories.
FAR = dict(rounds=200, n_traj=1 << 18, lam=0.25, lr=1e-3, select_from=150, select_every=25,
           val_traj=1 << 21, val_runs=2, val_seed=31338, steps=4, warmup=1)


def far_tail_leg(fpt, torch, TR, shard, ctx, prop12, m, tail, n, seed, rank, stream, dist=None, world=1):
    """Learned proposal at the 1e-20 point of the same workload: tail ESS rate
    over T20 = {N >= N_20} and the tail probability against the oracle's."""
    import torch as _t
    N20 = tail["N_20"]
    prop = TR.new_proposal(ctx, prop12.params.detach().cpu().numpy(), shift=prop12.shift, scale=prop12.scale,
                           segment=prop12.segment, alpha_max=prop12.alpha_max, flags=prop12.flags,
                           x_floor=prop12.x_floor)
    N12 = tail["N_12"]
    t0 = time.perf_counter()
    TR.train_select(ctx, prop, 0, rounds=FAR["rounds"],
                    checkpoints=range(FAR["select_from"], FAR["rounds"], FAR["select_every"]),
                    val_traj=FAR["val_traj"], val_seed=FAR["val_seed"], val_runs=FAR["val_runs"],
                    N_tail=N20, max_steps=m.max_steps, dN=m.dN, n_traj=FAR["n_traj"], seed=seed + 40,
                    lam=FAR["lam"], N_cut=lambda r: min(N20, N12 * 1.01 ** r), lr=FAR["lr"], chunk=1 << 17)
    _t.cuda.synchronize()
    train_s = time.perf_counter() - t0
    d = lambda k: prop.desc(0, n, seed=seed + 41, run_id=k, traj_offset=rank * n)

    def one(k):
        fpt.fpt_run(ctx, [d(k)], stream=stream)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 600.0, 512, N_tail=N20, stream=stream)
        return shard.tail_sums(h), passed_steps(h, m.dN) + h["n_capped"] * float(m.max_steps)

    for k in range(FAR["warmup"]):
        one(1000 + k)
    _t.cuda.synchronize()
    e0, e1 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
    e0.record(stream)
    sums, steps = [], 0.0
    for k in range(FAR["steps"]):
        (a, b), st = one(k)
        sums.append((a, b))
        steps += st
    e1.record(stream)
    _t.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    sw, sw2 = sum(a for a, _ in sums), sum(b for _, b in sums)
    sw, sw2 = shard.merge_shards(sw, sw2, rank * n, n, world * n, dist, device="cuda")
    ess = shard.ess_of(sw, sw2)
    n_tot = float(n) * FAR["steps"] * world
    p20 = sw / n_tot
    rel_se = math.sqrt(max(0.0, 1.0 / ess - 1.0 / n_tot)) if ess > 0 else None
    spread = shard.ess_spread([a for a, _ in sums], [b for _, b in sums])
    return {"N_20": N20, "n_traj_per_step": n, "steps": FAR["steps"], "seconds": t,
            "train": {"rounds": FAR["rounds"], "seconds": round(train_s, 2), "traj_per_round": FAR["n_traj"],
                      "warm_start": "the N_12 proposal", "N_cut": f"N_12 * 1.01^r up to {N20}",
                      "kept_round": max(prop.selection, key=lambda v: v["ess_per_step"])["round"]},
            "ess_tail": ess, "ess_tail_per_s": ess / t, "ess_tail_per_s_incl_training": ess / (t + train_s),
            "value_rel_se": spread["rel_se"],
            "p_tail": {"value": p20, "rel_se": rel_se, "oracle": tail["ccdf_at_N_20"],
                       "oracle_rel_se": tail["rel_se_at_N_20"],
                       "rel_diff": p20 / tail["ccdf_at_N_20"] - 1.0},
            "em_steps_per_s": steps / t}


def save_proposal(prop, path):
    """Store a trained proposal (fp32 parameters and its input normalisation)."""
    np.savez(path, params=prop.params.detach().cpu().numpy(), shift=np.asarray(prop.shift),
             scale=np.asarray(prop.scale), segment=prop.segment, alpha_max=prop.alpha_max, flags=prop.flags,
             x_floor=prop.x_floor)


def load_proposal(ctx, fpt, TR, path):
    """A proposal stored by save_proposal, packed for this context."""
    z = np.load(path)
    return TR.new_proposal(ctx, z["params"], shift=tuple(z["shift"]), scale=tuple(z["scale"]),
                           segment=int(z["segment"]), alpha_max=float(z["alpha_max"]), flags=int(z["flags"]),
                           x_floor=float(z["x_floor"]) if "x_floor" in z else 0.0)


def peak_pdf(fpt, ctx, run, stream, N_lo, N_hi, bins=48):
    h = fpt.fpt_histogram(ctx, run, N_lo, N_hi, bins, stream=stream)
    return np.asarray(h["pdf"]), np.asarray(h["se_jk"]), h["N_mean"]


def noise_2d_leg(fpt, torch, shard, m, stream, seed, rank, N_tail, A, sm_count, sm_max, autotune=True):
    """Full-rank noise (numerical matching of Eq. 3.9 at sigma = 1, 4096
    points) on the same model: direct-sampling throughput of the 2-D stepper,
    its issue roofline, the tail ESS rate with the constant standardised bias
    beta = (A, 0), and the 1-D vs 2-D comparison of P(delta N) near the peak
    (direct runs, same sigma)."""
    nd = 1 << 22
    out = {"table": "numerical matching, sigma = 1, 4096 points", "n_traj_per_run": nd}
    ctx2 = fpt.fpt_init_model([m, m], device=torch.cuda.current_device())
    t0 = time.perf_counter()
    fpt.fpt_noise_table2(ctx2, 0, fpt.FPT_TABLE_NUMERIC, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
    out["table_build_s"] = round(time.perf_counter() - t0, 3)
    fpt.fpt_noise_table(ctx2, 1, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
    if autotune:
        fpt.fpt_autotune(ctx2, [fpt.run_desc(0, nd, seed=seed + 5, run_id=99)], fraction=0.25)
    d2 = lambda k, A_=0.0: fpt.run_desc(0, nd, seed=seed + 5, run_id=k, A=A_, traj_offset=rank * nd)
    fpt.fpt_run(ctx2, [d2(100)], stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 0.0
    ms = []
    for k in range(3):
        e0.record(stream)
        fpt.fpt_run(ctx2, [d2(k)], stream=stream)
        e1.record(stream)
        h = fpt.fpt_histogram(ctx2, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        steps += passed_steps(h, m.dN)
    t = sum(ms) * 1e-3
    out["direct_traj_per_s"] = 3 * nd / t
    out["em_steps_per_s"] = steps / t
    out["roofline"] = roofline(steps / 3, float(np.mean(ms)), sm_count, sm_max, None, INSTR_PER_STEP_2D)
    out["roofline"]["kernel"] = "em2_kernel<direct, smem table>"
    # 1-D vs 2-D near the peak: the same seed range, direct sampling, at the
    # workload's sigma = 1 and at the paper's sigma << 1 (Sec. 3.3 matches the
    # full noise numerically at small sigma, where the decaying solution has died
    # away by the time a mode is coarse-grained)
    out["peak_1d_vs_2d_sigma1"] = peak_compare(fpt, ctx2, stream, nd, seed + 6, rank, W.USR_TABLE.sigma)
    c3 = fpt.fpt_init_model([m, m], device=torch.cuda.current_device())
    fpt.fpt_noise_table2(c3, 0, fpt.FPT_TABLE_NUMERIC, W.USR_TABLE.n_points, PEAK_SIGMA)
    fpt.fpt_noise_table(c3, 1, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, PEAK_SIGMA)
    fpt.fpt_run(c3, [fpt.run_desc(0, nd, seed=seed + 8, run_id=0, traj_offset=rank * nd)], stream=stream)
    out["peak_1d_vs_2d"] = peak_compare(fpt, c3, stream, nd, seed + 9, rank, PEAK_SIGMA)
    fpt.fpt_sync(c3)
    c3.close()
    # importance sampling on 2-D noise: beta = (A, 0)
    nb = 1 << 22
    fpt.fpt_run(ctx2, [fpt.run_desc(0, nb, seed=seed + 7, run_id=50, A=A, traj_offset=rank * nb)],
                stream=stream)
    e0.record(stream)
    sw = sw2 = 0.0
    for k in range(3):
        fpt.fpt_run(ctx2, [fpt.run_desc(0, nb, seed=seed + 7, run_id=k, A=A, traj_offset=rank * nb)],
                    stream=stream)
        h = fpt.fpt_histogram(ctx2, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        a, b = shard.tail_sums(h)
        sw += a
        sw2 += b
    e1.record(stream)
    torch.cuda.synchronize()
    out["fixed_bias"] = {"beta": [A, 0.0], "n_traj_per_run": nb,
                         "ess_tail_per_s": shard.ess_of(sw, sw2) / (e0.elapsed_time(e1) * 1e-3)}
    fpt.fpt_sync(ctx2)
    ctx2.close()
    return out


def batched_bias_leg(fpt, torch, shard, m, stream, seed, rank, N_tail, sm_count, sm_max, autotune=True,
                     n=1 << 20):
    """The constant-bias sweep in one launch: the eight amplitudes A in
    {0.5, 1, 2, 3, 4, 6, 8, 10} as eight runs of n trajectories each (uneven
    lengths: A >= 2 sends every path to the step cap), block shape and refill
    interval from the autotuner, replayed as a captured CUDA graph. EM steps
    per second of the mixed launch, its issue roofline, and per amplitude the
    tail probability and tail ESS at N_12 with the inverse-variance
    combination over amplitudes (Sec. 4.1: overlapping amplitudes)."""
    As = W.USR_FIXED_BIAS.biases
    ctx = fpt.fpt_init_model([m], device=torch.cuda.current_device())
    fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
    runs = lambda k: [fpt.run_desc(0, n, seed=seed + 60, run_id=8 * k + r, A=A, traj_offset=rank * n)
                      for r, A in enumerate(As)]
    launch = fpt.fpt_autotune(ctx, runs(100), fraction=0.125) if autotune else fpt.fpt_get_launch(ctx)
    fpt.fpt_run(ctx, runs(101), stream=stream)
    fpt.fpt_sync(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fpt.fpt_run(ctx, runs(0), stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    per, steps = {}, 0.0
    Ps, ses, cnt = [], [], []
    for r, A in enumerate(As):
        h = fpt.fpt_histogram(ctx, r, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        steps += passed_steps(h, m.dN) + h["n_capped"] * float(m.max_steps)
        sw, sw2 = shard.tail_sums(h)
        ess = shard.ess_of(sw, sw2)
        p = h["p_tail"]
        rel = math.sqrt(max(0.0, 1.0 / ess - 1.0 / n)) if ess > 0 else None
        per[str(A)] = {"p_tail": p, "rel_se": rel, "ess_tail": ess, "n_capped": int(h["n_capped"])}
        if rel is not None and ess >= 10:
            Ps.append(p)
            ses.append(p * rel)
    comb = None
    if Ps:
        wts = [1.0 / s ** 2 for s in ses]
        comb = {"p_tail": sum(w * p for w, p in zip(wts, Ps)) / sum(wts), "rel_se": None}
        comb["rel_se"] = 1.0 / math.sqrt(sum(wts)) / comb["p_tail"]
    fpt.fpt_sync(ctx)
    ctx.close()
    rl = roofline(steps, ms, sm_count, sm_max, None, INSTR_PER_STEP)
    rl["kernel"] = "em_kernel<weighted, smem table> (eight runs, one launch)"
    return {"biases": list(As), "n_traj_per_bias": n, "launch": launch, "launch_ms": ms,
            "traj_per_s": 8 * n / (ms * 1e-3), "em_steps_per_s": steps / (ms * 1e-3), "roofline": rl,
            "per_bias": per, "combined_at_N_12": comb,
            "note": "1/16 of the 2^24-per-amplitude workload (at 2^24 its capped paths alone are 5e13 EM steps, "
                    "two minutes per launch); the rates are per EM step and per trajectory"}


def model_family_leg(fpt, torch, TR, prop, stream, seed, rank, sm_count, sm_max, autotune=True, n=1 << 11,
                     pts=256, A_fallback=4.0, rounds=20):
    """The batched sweep over 64 piecewise-linear models (a- log-uniform in
    [1e-7, 1e-4], phi* in [0.9, 1.1], V0 log-uniform in [1e-11, 1e-9]), each
    with its own learned proposal and its constant-bias fallback A = 4: 128
    runs of uneven lengths (step cap 2^23) in one persistent launch, tables read
    through L1, one network per run, block shape and refill interval from the
    autotuner, replayed as a captured CUDA graph.

    Proposals: the network trained on the sudden-transition model, in each
    model's own normalisation (ln x / x_in, pi / |pi_in|), then trained further
    per model -- all 64 networks in one generation launch per round
    (fpt_mlp_train_batch) -- towards e^{lambda min(N, N_cut)} with N_cut = 30 <N>
    of the model's direct paths (the sudden-transition model's N_12 is 30 <N>),
    at most 200 e-folds (which keeps a round's segment records in the buffer). Per model: tail ESS over {N >= N_cut} of the learned
    run against its fallback run in the same launch."""
    models = W.batch_models(64)
    K = len(models)
    ctx = fpt.fpt_init_model(models, device=torch.cuda.current_device())
    t0 = time.perf_counter()
    for i in range(K):
        fpt.fpt_noise_table(ctx, i, fpt.FPT_TABLE_BESSEL, pts, 1.0)
    table_s = time.perf_counter() - t0
    # pilot: direct paths of every model in one launch give <N> and the tail points
    fpt.fpt_run(ctx, [fpt.run_desc(i, n, seed=seed + 69, run_id=i) for i in range(K)], stream=stream)
    cuts = []
    for i in range(K):
        h = fpt.fpt_histogram(ctx, i, 0.0, 1e4, 64, stream=stream)
        meanN = h["N_mean"] if h["n_passed"] > 0 else models[i].max_steps * models[i].dN
        cuts.append(float(min(30.0 * meanN, 200.0, 0.5 * models[i].max_steps * models[i].dN)))
    infos = [fpt.fpt_model_get_info(ctx, i) for i in range(K)]
    x_ins = [inf["phi_in"] - inf["phi_end"] for inf in infos]
    v = prop.params.detach().cpu().numpy()
    props, P, B = TR.new_proposals(ctx, [v] * K, [(math.log(x), 0.0, 0.0) for x in x_ins],
                                   [(prop.scale[0], 1.0 / abs(inf["pi_in"]), prop.scale[2]) for inf in infos],
                                   segment=prop.segment, alpha_max=prop.alpha_max, flags=prop.flags,
                                   x_floors=[x * X_FLOOR_REL for x in x_ins])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    TR.train_batch(ctx, props, P, B, list(range(K)), rounds=rounds, n_traj=n // 2, seed=seed + 71, lam=0.25,
                   N_cuts=cuts, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    def runs(k):
        out = []
        for i in range(K):
            out.append(props[i].desc(i, n, seed=seed + 70, run_id=2 * (64 * k + i), traj_offset=rank * n))
            out.append(fpt.run_desc(i, n, seed=seed + 70, run_id=2 * (64 * k + i) + 1, A=A_fallback,
                                    traj_offset=rank * n))
        return out

    launch = fpt.fpt_autotune(ctx, runs(100), fraction=0.25) if autotune else fpt.fpt_get_launch(ctx)
    fpt.fpt_run(ctx, runs(101), stream=stream)
    fpt.fpt_sync(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fpt.fpt_run(ctx, runs(0), stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    steps, capped = 0.0, 0
    gains, ess_l, ess_f, with_l = [], 0.0, 0.0, 0
    for i in range(K):
        m = models[i]
        e = []
        for r in (2 * i, 2 * i + 1):
            h = fpt.fpt_histogram(ctx, r, 0.0, 1e4, 64, N_tail=cuts[i], stream=stream)
            steps += passed_steps(h, m.dN) + h["n_capped"] * float(m.max_steps)
            capped += int(h["n_capped"])
            e.append(float(h["ess_tail"]))
        ess_l += e[0]
        ess_f += e[1]
        with_l += int(e[0] > 0)
        if e[1] > 0:
            gains.append(e[0] / e[1])
    fpt.fpt_sync(ctx)
    ctx.close()
    rl = roofline(steps, ms, sm_count, sm_max, None, INSTR_PER_STEP)
    rl["kernel"] = "em_kernel<weighted, tables via L1, MLP, one network per run>"
    return {"models": K, "runs": 2 * K, "n_traj_per_run": n, "table_points": pts,
            "table_build_s": round(table_s, 2), "launch": launch, "launch_ms": ms,
            "traj_per_s": 2 * K * n / (ms * 1e-3), "em_steps_per_s": steps / (ms * 1e-3),
            "roofline": rl, "censored_fraction": capped / float(2 * K * n),
            "train": {"rounds": rounds, "seconds": round(train_s, 2), "traj_per_model_per_round": n // 2,
                      "launches_per_round": 1,
                      "N_cut": "30 <N> of the model's direct paths, at most 200 e-folds and half the cap"},
            "tail_ess_learned_total": ess_l, "tail_ess_fallback_total": ess_f,
            "models_with_learned_tail": with_l, "models_with_fallback_tail": len(gains),
            "tail_ess_gain_median_where_fallback_reaches": float(np.median(gains)) if gains else None,
            "proposal": "per-model networks (warm start: the sudden-transition network in the model's "
                        "normalisation); fallback A = %g" % A_fallback,
            "note": "2^11 trajectories per run instead of 2^20: the A = 4 fallback sends most paths to the "
                    "2^23-step cap (at 2^20 per run that alone is 5.6e14 EM steps)"}


PEAK_SIGMA = 0.05


def peak_compare(fpt, ctx2, stream, nd, seed, rank, sigma, lo=4.0, hi=6.0):
    """P(delta N) near the peak from the full-rank table (model 0, the
    context's last run, direct) against the 1-D Bessel table (model 1, direct,
    Philox seed `seed`: independent of the first run): per-bin z-scores over
    bins above 1e-3 of the peak."""
    pdf2, se2, mean2 = peak_pdf(fpt, ctx2, 0, stream, lo, hi)
    fpt.fpt_run(ctx2, [fpt.run_desc(1, nd, seed=seed, run_id=0, traj_offset=rank * nd)], stream=stream)
    pdf1, se1, mean1 = peak_pdf(fpt, ctx2, 0, stream, lo, hi)
    ok = (se1 > 0) & (se2 > 0) & (pdf1 > 1e-3 * pdf1.max())
    z = np.abs(pdf2 - pdf1)[ok] / np.hypot(se1, se2)[ok]
    return {"sigma": sigma, "N_mean_1d": mean1, "N_mean_2d": mean2,
            "pdf_max_1d": float(pdf1.max()), "pdf_max_2d": float(pdf2.max()),
            "max_abs_z": float(z.max()) if z.size else None, "bins": int(ok.sum()), "range": [lo, hi]}


def passed_steps(h, dN):
    """EM steps of the passed trajectories of a histogram result (N_mean is
    NaN when none passed)."""
    return h["N_mean"] * h["n_passed"] / dN if h["n_passed"] > 0 else 0.0


def fixed_sweep(fpt, ctx, stream, seed, rank, N_tail, m, As, steps_per_s, n=1 << 21):
    """Tail ESS per EM step of each constant amplitude A (one run of n
    trajectories each), the implied ESS rate at steps_per_s (the whole job's
    EM-step rate), and the best A."""
    rows = {}
    for k, A in enumerate(As):
        fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=seed, run_id=k, A=A, traj_offset=rank * n)], stream=stream)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        steps = passed_steps(h, m.dN) + h["n_capped"] * float(m.max_steps)
        ess = float(h["ess_tail"])
        rows[str(A)] = {"ess_tail": round(ess, 2), "em_steps": steps, "n_capped": int(h["n_capped"]),
                        "ess_tail_per_s": ess / steps * steps_per_s if steps > 0 else 0.0}
    best = max(rows, key=lambda a: rows[a]["ess_tail_per_s"])
    return {"n_traj_per_A": n, "em_steps_per_s": steps_per_s, "per_A": rows, "best_A": float(best),
            "best_ess_tail_per_s": rows[best]["ess_tail_per_s"]}


def window_leg(fpt, torch, shard, m, stream, seed, rank, N_tail, A, sm_count, sm_max, autotune=True):
    """The paper's production setting (Sec. 4.1): Bessel-matched noise indexed
    by the time since the start along the background, on for the whole
    background range [N_in, N_end] and off after it (classical completion):
    direct-sampling throughput and issue roofline of the noise-window stepper,
    and the tail ESS rate with the constant bias A."""
    nd = 1 << 22
    Nw = m.n_end - m.n_in
    out = {"table": f"Bessel, sigma = 1, 4096 points over N in [0, {Nw:.4f}]", "n_traj_per_run": nd}
    ctx = fpt.fpt_init_model([m], device=torch.cuda.current_device())
    fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL_N, 4096, 1.0, 0.0, Nw)
    if autotune:
        fpt.fpt_autotune(ctx, [fpt.run_desc(0, nd, seed=seed + 11, run_id=99)], fraction=0.25)
    d = lambda k, A_=0.0: fpt.run_desc(0, nd, seed=seed + 11, run_id=k, A=A_, traj_offset=rank * nd)
    fpt.fpt_run(ctx, [d(100)], stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, steps = [], 0.0
    for k in range(3):
        e0.record(stream)
        fpt.fpt_run(ctx, [d(k)], stream=stream)
        e1.record(stream)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        steps += passed_steps(h, m.dN)
    t = sum(ms) * 1e-3
    out["direct_traj_per_s"] = 3 * nd / t
    out["em_steps_per_s"] = steps / t
    rl = roofline(steps / 3, float(np.mean(ms)), sm_count, sm_max, None, INSTR_PER_STEP_NIDX)
    rl["kernel"] = "em_kernel<direct, smem table, noise window>"
    out["roofline"] = rl
    fpt.fpt_run(ctx, [d(50, A)], stream=stream)
    e0.record(stream)
    sw = sw2 = 0.0
    for k in range(3):
        fpt.fpt_run(ctx, [d(60 + k, A)], stream=stream)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        a, b = shard.tail_sums(h)
        sw += a
        sw2 += b
    e1.record(stream)
    torch.cuda.synchronize()
    out["fixed_bias"] = {"A": A, "ess_tail_per_s": shard.ess_of(sw, sw2) / (e0.elapsed_time(e1) * 1e-3),
                         "note": "the bias acts only inside the window; after it the classical completion "
                                 "rarely reaches N_12"}
    fpt.fpt_sync(ctx)
    ctx.close()
    return out


def bump_leg(fpt, torch, shard, stream, seed, rank, sm_count, sm_max, autotune=True):
    """Gaussian-bump model (Sec. 4.3), 4096-point Bessel table at sigma = 1:
    direct-sampling throughput of the stepper with the tabulated drift, and the
    classical-delta-N comparison -- Var(N) of the direct run against
    sigma_R^2 of linear theory (Eq. 2.18), and the eps2 of Eq. (2.20) fitted
    to the importance-sampled tail (A = 2) against eps2 at the end of the
    mode range."""
    m = W.BUMP_MODEL
    nd = 1 << 22
    out = {"model": "Gaussian bump, K=1.17e-3 m=0.5 width=1.59e-2 phi0=2.18812, V0 from P_R peak 5e-3",
           "n_traj_per_run": nd}
    t0 = time.perf_counter()
    c = fpt.fpt_classical_dn(m, 1.0, 129)
    out["classical_host_s"] = round(time.perf_counter() - t0, 3)
    ctx = fpt.fpt_init_model([m], device=torch.cuda.current_device())
    fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 4096, 1.0)
    if autotune:
        fpt.fpt_autotune(ctx, [fpt.run_desc(0, nd, seed=seed + 9, run_id=99)], fraction=0.25)
    d = lambda k, A=0.0: fpt.run_desc(0, nd, seed=seed + 9, run_id=k, A=A, traj_offset=rank * nd)
    fpt.fpt_run(ctx, [d(100)], stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, steps = [], 0.0
    for k in range(3):
        e0.record(stream)
        fpt.fpt_run(ctx, [d(k)], stream=stream)
        e1.record(stream)
        h = fpt.fpt_histogram(ctx, 0, 3.0, 5.0, 200, stream=stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        steps += passed_steps(h, m.dN)
    t = sum(ms) * 1e-3
    out["direct_traj_per_s"] = 3 * nd / t
    out["em_steps_per_s"] = steps / t
    rl = roofline(steps / 3, float(np.mean(ms)), sm_count, sm_max, None, INSTR_PER_STEP_BUMP)
    rl["kernel"] = "em_kernel<direct, smem table, drift table>"
    out["roofline"] = rl
    Nbuf = np.zeros(nd)
    fpt.fpt_run(ctx, [d(3)], [dict(N=Nbuf)], stream=stream)
    fpt.fpt_sync(ctx)
    varN = float(Nbuf.var())
    out["classical_dn"] = {"sigma_R2": c["sigma_R2"], "var_N": varN,
                           "var_N_se": varN * math.sqrt(2.0 / nd), "mean_N": float(Nbuf.mean()),
                           "eps2_end": c["eps2_end"]}
    Nm = float(Nbuf.mean())
    fpt.fpt_run(ctx, [d(7, 2.0)], stream=stream)
    hb = fpt.fpt_histogram(ctx, 0, 3.0, 6.0, 120, stream=stream)
    centres = 3.0 + (np.arange(120) + 0.5) * hb["db"]
    dN = centres - Nm
    sel = (dN > 2 * math.sqrt(c["sigma_R2"])) & (hb["count"] >= 50)
    if sel.sum() >= 5:
        f = fpt.fpt_fit_eps2(dN[sel], hb["pdf"][sel], hb["se_w"][sel], c["sigma_R2"], 0.0, 5.0)
        out["classical_dn"].update({"eps2_fit": f["eps2"], "fit_chi2_per_bin": f["chi2"] / f["bins"],
                                    "fit_bins": f["bins"], "fit_range_dN": [float(dN[sel].min()),
                                                                            float(dN[sel].max())]})
        gauss = fpt.fpt_classical_pdf(dN[sel], c["sigma_R2"], 0.0)
        out["classical_dn"]["tail_over_gaussian_max"] = float(np.max(hb["pdf"][sel] / gauss))
    fpt.fpt_sync(ctx)
    ctx.close()
    return out


def legs_once(fpt, torch, n=1 << 22, seed=17):
    """One direct launch (no bias, default launch shape) of each constant-bias
    stepper variant at the legs' sizes -- the 1-D stepper on the sudden-
    transition model's Bessel table, the full-rank 2-D stepper on its numerical
    table, the noise-window stepper on the time-indexed table, the bump stepper
    with its drift table -- for profiling them under ncu (one launch each, in
    this order, after one warm-up launch each); prints the EM steps and the
    CUDA-event time of each timed launch as one JSON line."""
    m = usr_model()
    cases = [("direct", m, lambda c: fpt.fpt_noise_table(c, 0, fpt.FPT_TABLE_BESSEL, 4096, 1.0)),
             ("noise_2d", m, lambda c: fpt.fpt_noise_table2(c, 0, fpt.FPT_TABLE_NUMERIC, 4096, 1.0)),
             ("window", m, lambda c: fpt.fpt_noise_table(c, 0, fpt.FPT_TABLE_BESSEL_N, 4096, 1.0, 0.0,
                                                        m.n_end - m.n_in)),
             ("bump", W.BUMP_MODEL, lambda c: fpt.fpt_noise_table(c, 0, fpt.FPT_TABLE_BESSEL, 4096, 1.0))]
    out = {}
    for name, mod, table in cases:
        with fpt.fpt_init_model([mod], device=torch.cuda.current_device()) as ctx:
            table(ctx)
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=seed + 1)], stream=stream)    # warm-up (graph capture)
            torch.cuda.synchronize()
            e0.record(stream)
            st = fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=seed)], stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            h = fpt.fpt_histogram(ctx, 0, 0.0, 100.0, 512, stream=stream)
            steps = passed_steps(h, mod.dN) + h["n_capped"] * float(mod.max_steps)
            ms = e0.elapsed_time(e1)
            out[name] = {"em_steps": steps, "ms": ms, "em_steps_per_s": steps / (ms * 1e-3), "status": int(st)}
    print(json.dumps({"legs_once": out, "n_traj": n}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--proposal", default="learned", choices=["learned", "fixed"])
    ap.add_argument("--n-traj", type=int, default=0, help="trajectories per step per GPU (0: proposal default)")
    ap.add_argument("--ref-traj", type=int, default=1 << 15, help="oracle trajectories per step")
    ap.add_argument("--cpu-traj", type=int, default=1 << 18, help="CPU-baseline sample size")
    ap.add_argument("--train-rounds", type=int, default=TRAIN["rounds"])
    ap.add_argument("--lam", type=float, default=TRAIN["lam"], help="tilt lambda of the training target")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e / constant-bias / direct legs")
    ap.add_argument("--no-2d", action="store_true", help="skip the full-rank (2-D) noise leg")
    ap.add_argument("--no-bump", action="store_true", help="skip the Gaussian-bump leg")
    ap.add_argument("--no-window", action="store_true", help="skip the noise-window leg")
    ap.add_argument("--no-far", action="store_true", help="skip the 1e-20 tail leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the eight-amplitude batched leg")
    ap.add_argument("--no-family", action="store_true", help="skip the 64-model batched leg")
    ap.add_argument("--pipeline", type=int, default=2, help="steps in flight (contexts / streams)")
    ap.add_argument("--net", default="", help="load a trained proposal (.npz of --save-net) instead of training")
    ap.add_argument("--save-net", default="", help="store the trained proposal (.npz)")
    ap.add_argument("--legs-once", action="store_true",
                    help="profiling aid: one direct launch of each constant-bias stepper variant, then exit")
    args = ap.parse_args()
    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    import __graft_entry__
    from paper_2410_13683_gb300 import fpt
    from paper_2410_13683_gb300 import shard
    from paper_2410_13683_gb300 import train as TR

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()
    if args.legs_once:
        return legs_once(fpt, torch)
    TRAIN["rounds"] = args.train_rounds
    TRAIN["lam"] = args.lam
    tail = load_tail()
    N_tail, A_fixed = tail["N_12"], tail["A"]
    m = usr_model()
    learned = args.proposal == "learned"
    n = args.n_traj or (1 << 22)
    seed = 20260
    dev = torch.cuda.current_device()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    ctx = fpt.fpt_init_model([m], device=dev)
    S_tab, T_tab = fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
    info = fpt.fpt_model_get_info(ctx, 0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    off = shard.shard_offset(n, rank)

    train_info = None
    prop = None
    if learned and args.net:
        prop = load_proposal(ctx, fpt, TR, args.net)
    elif learned:
        prop, train_s = train_proposal(ctx, fpt, TR, info, N_tail)
        if args.save_net and rank == 0:
            save_proposal(prop, args.save_net)
        h = prop.history
        train_info = {"rounds": len(h), "seconds": round(train_s, 2), "traj_per_round": TRAIN["n_traj"],
                      "lambda": TRAIN["lam"], "N_cut": N_tail, "final_loss": round(h[-1]["loss"], 3),
                      "first_loss": round(h[0]["loss"], 3), "segment": TRAIN["segment"],
                      "alpha_max": TRAIN["alpha_max"], "inputs": "(ln x, pi, N)",
                      "selection": {"val_traj": TRAIN["val_traj"] * TRAIN["val_runs"],
                                    "criterion": "held-out tail ESS per EM step",
                                    "kept_round": max(prop.selection, key=lambda v: v["ess_per_step"])["round"],
                                    "checkpoints": [[v["round"], round(v["ess_tail"]), float("%.4g" % v["ess_per_step"])]
                                                    for v in prop.selection]}}

    def desc(step, nn=n, offset=off):
        if learned:
            return prop.desc(0, nn, seed=seed, run_id=step, traj_offset=offset)
        return fpt.run_desc(0, nn, seed=seed, run_id=step, A=A_fixed, traj_offset=offset)

    if args.no_autotune:
        launch = fpt.fpt_get_launch(ctx)
    else:
        launch = fpt.fpt_autotune(ctx, [desc(10_000)], fraction=0.25)

    # Pipeline: P contexts on P streams, each step's launch issued before the
    # previous step's histogram is read back, so that the tail of one launch
    # (its longest trajectories, with most lanes idle) overlaps the next one.
    P = max(1, args.pipeline)
    ctxs, streams = [ctx], [stream]
    for _ in range(P - 1):
        c = fpt.fpt_init_model([m], device=dev)
        fpt.fpt_noise_table(c, 0, fpt.FPT_TABLE_BESSEL, W.USR_TABLE.n_points, W.USR_TABLE.sigma)
        fpt.fpt_set_launch(c, **{k: launch[k] for k in ("block", "blocks_per_sm", "check_steps", "use_graph")})
        ctxs.append(c)
        streams.append(torch.cuda.Stream())

    def issue(k, step, ev=None, d=None):
        c, st = ctxs[k % P], streams[k % P]
        if ev is not None:
            ev[0].record(st)
        fpt.fpt_run(c, [d or desc(step)], stream=st)
        if ev is not None:
            ev[1].record(st)

    def collect(k):
        c, st = ctxs[k % P], streams[k % P]
        h = fpt.fpt_histogram(c, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=st)
        sw, sw2 = shard.tail_sums(h)
        steps = passed_steps(h, m.dN) + h["n_capped"] * float(m.max_steps)
        return sw, sw2, steps

    def pipelined(K, step_of, ev=None, before=None, dfun=None, per_step=None):
        """K steps, up to P in flight; returns the summed tail sums and steps
        (and appends each step's (sum_T w, sum_T w^2) to per_step)."""
        tot = [0.0, 0.0, 0.0]
        for k in range(min(P - 1, K)):
            if before:
                before(k)
            issue(k, step_of(k), ev[k] if ev else None, dfun(step_of(k)) if dfun else None)
        for k in range(K):
            j = k + P - 1
            if j < K:
                if before:
                    before(j)
                issue(j, step_of(j), ev[j] if ev else None, dfun(step_of(j)) if dfun else None)
            r = collect(k)
            for i in range(3):
                tot[i] += r[i]
            if per_step is not None:
                per_step.append((r[0], r[1]))
        return tot

    def one_step(step, ev=None, d=None):
        issue(0, step, ev, d)
        return collect(0)

    pipelined(args.warmup, lambda k: 100_000 + k)

    clocks = Clocks(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    t_start.record(streams[0])
    for st in streams[1:]:
        st.wait_event(t_start)
    ess_steps = []
    sw_tot, sw2_tot, steps_tot = pipelined(args.steps, lambda k: k, run_ev, per_step=ess_steps)
    for st in streams[1:]:
        e = torch.cuda.Event()
        e.record(st)
        streams[0].wait_event(e)
    t_end.record(streams[0])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) * 1e-3
    run_ms = [a.elapsed_time(b) for a, b in run_ev]
    if dist:
        t = torch.tensor([elapsed], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    sw_tot, sw2_tot = shard.merge_shards(sw_tot, sw2_tot, off, n, world * n, dist, device="cuda")
    ess_total = shard.ess_of(sw_tot, sw2_tot)
    # spread of the pooled ESS over the timed steps (this rank's steps)
    spread = shard.ess_spread([a for a, _ in ess_steps], [b for _, b in ess_steps])
    n_total = float(n) * args.steps * world
    value = ess_total / elapsed

    extras = {}
    if not args.no_extras:
        # end to end through the public API with host buffers: the noise table
        # from pinned host memory, descriptors from the host, the histogram read
        # back to host memory, all on the host clock
        S_pin = torch.from_numpy(S_tab).pin_memory().numpy()
        T_pin = torch.from_numpy(T_tab).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def upload(k):
            fpt.fpt_noise_table(ctxs[k % P], 0, fpt.FPT_TABLE_USER, len(S_pin), 1.0, float("nan"),
                                float("nan"), S_pin, T_pin)

        # the timed steps' trajectories (same seed and run ids): the
        # difference from `value` is the host path alone
        sw_e, sw2_e, _ = pipelined(args.steps, lambda k: k, before=upload)
        torch.cuda.synchronize()
        e2e_t = time.perf_counter() - t0
        sw_e, sw2_e = shard.merge_shards(sw_e, sw2_e, off, n, world * n, dist, device="cuda")
        extras["e2e"] = {"value": shard.ess_of(sw_e, sw2_e) / e2e_t, "unit": UNIT,
                         "h2d_bytes_per_step": len(S_pin) * 16 + 128 + (fpt.FPT_MLP_BLOB_BYTES if learned else 0),
                         "d2h_bytes_per_step": (10 * 512 + 16) * 8}
        # the constant-bias comparison (the method without the learned part)
        nj = 1 << 22
        jd = lambda k: fpt.run_desc(0, nj, seed=seed + 2, run_id=k, A=A_fixed, traj_offset=rank * nj)
        pipelined(1, lambda k: 900, dfun=jd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        swj, sw2j, stj = pipelined(4, lambda k: k, dfun=jd)     # as pipelined as the learned steps
        torch.cuda.synchronize()
        fixed_t = time.perf_counter() - t0
        swj, sw2j = shard.merge_shards(swj, sw2j, rank * nj, nj, world * nj, dist, device="cuda")
        fixed_rate = shard.ess_of(swj, sw2j) / fixed_t
        extras["fixed_bias"] = {"A": A_fixed, "n_traj_per_step": nj, "ess_tail_per_s": fixed_rate,
                                "timing": "host clock over 4 pipelined steps"}
        # other constant amplitudes around A_fixed: tail ESS per EM step
        # on 2^21 trajectories each, priced at the A_fixed run's pipelined EM-step
        # rate (the constant-bias stepper's cost per step does not depend on A)
        extras["fixed_bias_sweep"] = fixed_sweep(fpt, ctx, stream, seed + 3, rank, N_tail, m,
                                                 FIXED_SWEEP, stj / fixed_t * world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # direct sampling on the same GPU: ESS_T = n * 1e-12 in expectation
        nd = 1 << 22
        fpt.fpt_run(ctx, [fpt.run_desc(0, nd, seed=seed + 1, run_id=0, traj_offset=rank * nd)], stream=stream)
        fpt.fpt_sync(ctx)
        e0.record(stream)
        for k in range(3):
            fpt.fpt_run(ctx, [fpt.run_desc(0, nd, seed=seed + 1, run_id=k + 1, traj_offset=rank * nd)],
                        stream=stream)
            fpt.fpt_histogram(ctx, 0, 0.0, 400.0, 512, N_tail=N_tail, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        direct_traj_s = 3 * nd / (e0.elapsed_time(e1) * 1e-3)
        extras["direct"] = {"traj_per_s": direct_traj_s * world, "ess_tail_per_s": direct_traj_s * TAIL_P * world}
        if not args.no_2d:
            sm_max_2d = measured_peaks().get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
            extras["noise_2d"] = noise_2d_leg(fpt, torch, shard, m, stream, seed, rank, N_tail, A_fixed,
                                              sm_count, sm_max_2d, autotune=not args.no_autotune)
        if not args.no_window:
            sm_max_w = measured_peaks().get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
            extras["noise_window"] = window_leg(fpt, torch, shard, m, stream, seed, rank, N_tail, A_fixed,
                                                sm_count, sm_max_w, autotune=not args.no_autotune)
        if not args.no_batch:
            sm_max_b8 = measured_peaks().get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
            extras["batched_biases"] = batched_bias_leg(fpt, torch, shard, m, stream, seed, rank, N_tail,
                                                        sm_count, sm_max_b8, autotune=not args.no_autotune)
        if learned and not args.no_family:
            sm_max_f = measured_peaks().get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
            extras["model_family"] = model_family_leg(fpt, torch, TR, prop, stream, seed, rank, sm_count,
                                                      sm_max_f, autotune=not args.no_autotune)
        if learned and not args.no_far and "N_20" in tail:
            far = far_tail_leg(fpt, torch, TR, shard, ctx, prop, m, tail, n, seed, rank, stream, dist, world)
            extras["far_tail_20"] = far
            # direct sampling reaches 1e-20 at traj/s x 1e-20 effective samples per second
            far["gain_vs_direct"] = far["ess_tail_per_s"] / (extras["direct"]["traj_per_s"] * 1e-20)
        if not args.no_bump:
            sm_max_b = measured_peaks().get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
            extras["bump"] = bump_leg(fpt, torch, shard, stream, seed, rank, sm_count, sm_max_b,
                                      autotune=not args.no_autotune)

    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
    traffic = None
    prof = os.path.join(ROOT, "profiles", "em_kernel_traffic.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("bytes_per_launch_scaled")
        except Exception:
            traffic = None
    mean_run_ms = float(np.mean(run_ms))
    # P launches are in flight: each launch's own events overlap its neighbours,
    # so the stepper's rate is taken over the timed region (launch interval =
    # elapsed / steps; the histograms take ~0.3% of it)
    interval_ms = 1e3 * elapsed / args.steps
    rl = roofline(steps_tot / args.steps, interval_ms if P > 1 else mean_run_ms, sm_count, sm_max, traffic,
                  INSTR_PER_STEP_MLP if learned else INSTR_PER_STEP)
    rl["launch_time"] = ("timed region / steps, %d launches in flight" % P) if P > 1 else "CUDA events per launch"
    if learned:
        rl["frac_incl_network"] = round(rl["frac"] * (INSTR_PER_STEP_MLP + INSTR_NETWORK_PER_STEP) /
                                        INSTR_PER_STEP_MLP, 4)
    pipes = pipe_fractions(steps_tot / elapsed, sm_count, sm_max)
    if pipes and learned:
        rl.update(pipes)
    if not learned:
        rl["kernel"] = "em_kernel<weighted, smem table>"

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "usr_learned_tail" if learned else "usr_fixed_bias_tail",
                       "model": USR_MODEL_TEXT,
                       "proposal": "learned MLP 3-64-64-2 (bf16)" if learned else f"constant A={A_fixed}",
                       "n_traj_per_step_per_gpu": n, "N_tail": N_tail,
                       "table_points": W.USR_TABLE.n_points, "dN": m.dN, "max_steps": m.max_steps,
                       "l2": "inputs are generated in-kernel; the 64 KB table and 12 KB weights stay in shared memory",
                       "launch": launch},
            "roofline": rl,
            "gpu_launches": 4 * args.steps,
            "clocks": clk,
            "ess_tail_total": ess_total,
            # each step's own tail ESS: with heavy-tailed weights a few paths
            # decide sum w^2, and the spread shows it
            "ess_tail_per_step": [round(shard.ess_of(a, b)) for a, b in ess_steps],
            # the rate's own uncertainty: bootstrap over the timed steps (95%) and
            # the delete-one-step jackknife error
            "value_ci": [value * spread["lo"], value * spread["hi"]] if spread["lo"] is not None else None,
            "value_rel_se": spread["rel_se"],
            # the estimate itself, beside the oracle's (FP64, constant bias): the
            # weights are exact, so a good proposal changes the error, not the value
            "p_tail": {"value": sw_tot / n_total, "rel_se": math.sqrt(max(0.0, 1.0 / ess_total - 1.0 / n_total))
                       if ess_total > 0 else None,
                       "oracle": tail["ccdf_at_N_12"], "oracle_rel_se": tail["rel_se_at_N_12"]},
            "em_steps_per_step": steps_tot / args.steps,
            "em_steps_per_s": steps_tot / elapsed, "pipeline": P,
            "em_launch_ms": mean_run_ms}
    if args.net:
        line["config"]["proposal"] += f" (loaded from {os.path.basename(args.net)}, not trained in this run)"
    if train_info:
        line["train"] = train_info
        # the training charged to this run: ESS of the timed steps over training + timed time
        line["value_incl_training"] = ess_total / (train_info["seconds"] + elapsed)
    line.update(extras)
    if "far_tail_20" in extras:
        f20 = extras["far_tail_20"]
        line["p_tail_20"] = f20["p_tail"]
        line["ess_tail_per_s_20"] = f20["ess_tail_per_s"]
    if "direct" in extras and extras["direct"]["ess_tail_per_s"] > 0:
        line["gain_vs_direct"] = value / extras["direct"]["ess_tail_per_s"]
    if "fixed_bias" in extras and extras["fixed_bias"]["ess_tail_per_s"] > 0:
        line["gain_vs_fixed_bias"] = value / extras["fixed_bias"]["ess_tail_per_s"]
    if "fixed_bias_sweep" in extras and extras["fixed_bias_sweep"]["best_ess_tail_per_s"] > 0:
        line["gain_vs_best_fixed_bias"] = value / extras["fixed_bias_sweep"]["best_ess_tail_per_s"]
        if "value_incl_training" in line:
            line["gain_vs_best_fixed_bias_incl_training"] = (line["value_incl_training"] /
                                                             extras["fixed_bias_sweep"]["best_ess_tail_per_s"])
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import tables as OT
        res = OT.resolve(m)
        tab = OT.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=os.cpu_count())
        e, dt, cores, nsteps = cpu_oracle_sample((m, res, tab), A_fixed, N_tail, args.cpu_traj)
        line["cpu_baseline"] = {"value": e / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_traj} trajectories of the same workload with the "
                                          f"constant-bias proposal A={A_fixed} ({nsteps} Euler-Maruyama "
                                          f"steps, {dt:.1f} s)"}
        # the same method on both sides: the GPU's constant-bias rate over the oracle's
        if "fixed_bias" in extras and e > 0:
            line["gpu_vs_oracle_same_proposal"] = extras["fixed_bias"]["ess_tail_per_s"] / (e / dt)
    for c in ctxs:
        fpt.fpt_sync(c)
        c.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
