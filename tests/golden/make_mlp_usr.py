"""Train the learned proposal with the FP64 oracle and store it as a fixture.

Writes tests/golden/mlp_usr_trained.json: the fp32 parameters of a
3 -> 64 -> 64 -> 2 SiLU network trained on the sudden-transition model in the
configuration the benchmark times -- inputs (ln x, pi, N) shifted and scaled,
alpha held for 128-step segments, |alpha| <= 8, ln x floored at 2^-14 x_in,
step cap 2^19 -- by the
log-variance loss towards the tilted target e^{lambda min(N, N_cut)} P
(lambda = 0.25, N_cut raised from 10 to N_12 = 152.5 e-folds), with Adam, 110
rounds of 1024 trajectories. Everything
here runs in oracle/: the trajectories and their segment records come from the
FP64 C stepper (oracle.stepper.run_segments, Philox seed 4004, run id = round),
the gradient from oracle.mlp.alpha_grad (bf16 rounding of the network's
operands, as deployed). The fixture is an input of the per-trajectory parity
test of the learned stepper; no value in it comes from the CUDA path.

    python tests/golden/make_mlp_usr.py [--rounds R] [--traj N]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time
from dataclasses import replace

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "mlp_usr_trained.json")
SEED = 4004
SEGMENT, ALPHA_MAX, LAM = 128, 8.0, 0.25

X_FLOOR_REL = 2.0 ** -14
_G = {}


def _init(m, res, tab):
    _G.update(m=m, res=res, tab=tab)


def _one(args):
    from oracle import stepper as S
    params, shift, scale, r, traj = args
    x_in = _G["res"].phi_in - _G["res"].phi_end
    mlp = S.MLPBias(params, segment=SEGMENT, in_shift=shift, in_scale=scale, alpha_max=ALPHA_MAX,
                    round_bf16=True, log_x=True, x_floor=x_in * X_FLOOR_REL)
    return S.run_segments(_G["m"], _G["res"], _G["tab"], mlp, seed=SEED, run_id=r, traj=traj, cap=1 << 13)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rounds", type=int, default=110)
    ap.add_argument("--traj", type=int, default=1024)
    ap.add_argument("--ncut-max", type=float, default=152.5)
    args = ap.parse_args()

    import workloads as W
    from oracle import mlp as OM
    from oracle import tables as T

    m = replace(W.USR_MODEL, max_steps=1 << 19)
    res = T.resolve(m)
    tab = T.bessel_table(m, res, W.USR_TABLE.n_points, W.USR_TABLE.sigma, processes=os.cpu_count())
    x_in = res.phi_in - res.phi_end
    shift = (math.log(x_in), 0.0, 0.0)
    scale = (0.2, 1.0 / abs(res.pi_in), 0.01)
    # the network's weights are kept fp32-representable, as the library stores them
    p = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in W.mlp_init(21, out_scale=0.0).items()}
    mom = {k: np.zeros_like(v) for k, v in p.items()}
    vel = {k: np.zeros_like(v) for k, v in p.items()}
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 3e-3
    hist = []
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count(), initializer=_init, initargs=(m, res, tab)) as pool:
        for r in range(args.rounds):
            N_cut = min(args.ncut_max, 10.0 * 1.3 ** r)
            trajs = pool.map(_one, [(p, shift, scale, r, j) for j in range(args.traj)], chunksize=8)
            N = np.array([t["nsteps"] for t in trajs]) * m.dN
            Y = np.array([t["logw"] for t in trajs]) + LAM * np.minimum(N, N_cut)
            n = len(trajs)
            coef = 2.0 / n * (Y - Y.mean())
            g = {k: np.zeros_like(v) for k, v in p.items()}
            for j, tr in enumerate(trajs):
                if len(tr["sum_xi"]) == 0:
                    continue
                s = OM.normalise(tr["state"], shift, scale)
                dal = coef[j] * (-math.sqrt(m.dN) * tr["sum_xi"])
                gj = OM.alpha_grad(p, s, tr["tan_theta"], ALPHA_MAX, dal, round_bf16=True)
                for k in g:
                    g[k] += gj[k]
            for k in p:
                mom[k] = b1 * mom[k] + (1 - b1) * g[k]
                vel[k] = b2 * vel[k] + (1 - b2) * g[k] ** 2
                upd = lr * (mom[k] / (1 - b1 ** (r + 1))) / (np.sqrt(vel[k] / (1 - b2 ** (r + 1))) + eps)
                p[k] = (p[k] - upd).astype(np.float32).astype(np.float64)
            al = np.concatenate([t["alpha"] for t in trajs if len(t["alpha"])])
            hist.append(dict(round=r, N_cut=N_cut, loss=float(np.var(Y)), mean_N=float(N.mean()),
                             max_N=float(N.max()), alpha_mean=float(al.mean()),
                             alpha_clamped=float(np.mean(np.abs(al) >= ALPHA_MAX))))
            print(f"round {r}: N_cut {N_cut:.1f} loss {hist[-1]['loss']:.3f} mean N {N.mean():.2f} "
                  f"max N {N.max():.1f} alpha mean {al.mean():.2f} clamped {hist[-1]['alpha_clamped']:.3f} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    out = {"about": "learned-proposal network trained by the FP64 oracle (tests/golden/make_mlp_usr.py); "
                    "log-variance loss towards the tilted target, Sec. 4.1 weights; inputs (ln x, pi, N)",
           "model": "sudden transition, V0=2e-10 a+=1e-3 a-=1e-6 phi*=1, 4096-point Bessel table sigma=1, "
                    "dN=1e-3, max_steps=2^19",
           "segment": SEGMENT, "alpha_max": ALPHA_MAX, "log_x": True, "x_floor": x_in * X_FLOOR_REL,
           "shift": list(shift),
           "scale": list(scale), "lambda": LAM, "rounds": args.rounds, "traj_per_round": args.traj,
           "seed": SEED, "history": hist,
           "params": {k: [float(x) for x in np.asarray(v, np.float32).ravel()] for k, v in p.items()},
           "shapes": {k: list(np.shape(v)) for k, v in p.items()}}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
