"""Training driver of the learned importance-sampling proposal.

Host orchestration only: every round calls fpt_mlp_train_round (generation
with segment records, loss coefficients, bf16 tensor-core backward, Adam and
re-packing all run in libfpt.so). Device memory comes from PyTorch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import fpt


@dataclass
class Proposal:
    """A trained proposal: fp32 master parameters, the packed bf16 blob and
    the input normalisation it was trained with."""
    params: object           # torch CUDA float32 tensor [FPT_MLP_PARAMS]
    blob: object             # torch CUDA uint8 tensor [FPT_MLP_BLOB_BYTES]
    shift: tuple
    scale: tuple
    segment: int
    alpha_max: float
    flags: int = 0
    x_floor: float = 0.0     # log-field input: ln max(x, x_floor)
    history: List[dict] = field(default_factory=list)
    selection: List[dict] = field(default_factory=list)

    def desc(self, model: int, n_traj: int, seed: int, run_id: int, traj_offset: int = 0):
        return fpt.run_desc(model, n_traj, seed=seed, run_id=run_id, traj_offset=traj_offset,
                            bias_kind=fpt.FPT_BIAS_MLP, mlp=self.blob, mlp_segment=self.segment,
                            mlp_shift=self.shift, mlp_scale=self.scale, alpha_max=self.alpha_max,
                            mlp_flags=self.flags, mlp_x_floor=self.x_floor)


def new_proposal(ctx, init_params: np.ndarray, shift, scale, segment: int = 64, alpha_max: float = 4.0,
                 flags: int = 0, x_floor: float = 0.0, device: str = "cuda"):
    import torch
    p = torch.tensor(np.asarray(init_params, np.float32), device=device)
    blob = torch.zeros(fpt.FPT_MLP_BLOB_BYTES, dtype=torch.uint8, device=device)
    fpt.fpt_mlp_pack(ctx, p, blob)
    if p.is_cuda:
        torch.cuda.synchronize()
    return Proposal(p, blob, tuple(float(v) for v in shift), tuple(float(v) for v in scale), segment,
                    alpha_max, flags, float(x_floor))


def train(ctx, prop: Proposal, model: int, rounds: int, n_traj: int, seed: int, lam: float,
          N_cut: Callable[[int], float], lr=3e-3, chunk: Optional[int] = None,
          clip: float = 0.0, log: Optional[Callable[[dict], None]] = None,
          first_round: int = 0) -> Proposal:
    """`rounds` Adam steps of the log-variance loss; round r draws n_traj
    fresh trajectories (Philox run id = r) from the current proposal. `lr`
    is a number or a function of the round."""
    import torch
    if not hasattr(prop, "_adam"):
        prop._adam = (torch.zeros_like(prop.params), torch.zeros_like(prop.params))
    m, v = prop._adam
    ch = chunk or n_traj
    for r in range(first_round, first_round + rounds):
        run = prop.desc(model, n_traj, seed=seed, run_id=r)
        lr_r = lr(r) if callable(lr) else lr
        while True:
            try:
                st = fpt.fpt_mlp_train_round(ctx, run, ch, lam, N_cut(r),
                                             dict(lr=lr_r, step=r + 1, clip=clip), prop.params, m, v, prop.blob)
                break
            except fpt.FptError as e:
                # more segment records than the record buffer holds: the round
                # left the parameters untouched, so it is redone in halves
                if e.status != fpt.FPT_E_NOMEM or ch <= 1024:
                    raise
                ch = (ch + 1) // 2
        st["chunk"] = ch
        st["round"] = r
        st["N_cut"] = N_cut(r)
        st["lr"] = lr_r
        prop.history.append(st)
        if log:
            log(st)
    return prop


def tail_ess(ctx, prop: Proposal, model: int, n_traj: int, seed: int, run_ids, N_tail: float,
             max_steps: int, dN: float, stream=None) -> dict:
    """Runs of the proposal on n_traj fresh trajectories per run id (one id
    or a list), pooled: the tail effective sample size (sum_T w)^2 / sum_T w^2
    over T = {N >= N_tail}, the tail probability estimate sum_T w / n, the EM
    steps taken and the tail ESS per step (the cost-aware figure of merit of a
    proposal). Pooling several runs catches more of the rare large weights
    that decide the ESS of a long production run."""
    ids = [run_ids] if isinstance(run_ids, int) else list(run_ids)
    sw = sw2 = steps = 0.0
    for rid in ids:
        run = prop.desc(model, n_traj, seed=seed, run_id=rid)
        fpt.fpt_run(ctx, [run], stream=stream)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 2.0 * N_tail, 256, N_tail=N_tail, stream=stream)
        if h["n_passed"] > 0:        # N_mean is NaN when no trajectory passed
            steps += h["N_mean"] * h["n_passed"] / dN
        steps += h["n_capped"] * float(max_steps)
        a = h["p_tail"] * h["n_total"]
        sw += a
        sw2 += a * a / h["ess_tail"] if h["ess_tail"] > 0 else 0.0
    ess = sw * sw / sw2 if sw2 > 0 else 0.0
    return {"ess_tail": ess, "p_tail": sw / (float(n_traj) * len(ids)), "steps": steps,
            "ess_per_step": ess / steps if steps > 0 else 0.0}


def train_select(ctx, prop: Proposal, model: int, rounds: int, checkpoints, val_traj: int, val_seed: int,
                 N_tail: float, max_steps: int, dN: float, val_runs: int = 1, **train_kw) -> Proposal:
    """train() for `rounds` rounds with model selection on held-out runs: at
    each round count in `checkpoints` (and at the end) the current proposal
    is run val_runs times on val_traj trajectories of Philox seed val_seed
    (run ids 0 .. val_runs-1, independent of the training runs when val_seed
    differs from the training seed), and the parameters with the most pooled
    tail ESS per EM step are kept and re-packed. Every checkpoint sees the
    same noise (common random numbers): a rare path with a large weight then
    weighs on all candidates alike instead of on whichever checkpoint drew
    it. The measurements go to prop.selection."""
    import torch
    if val_runs < 1:
        raise ValueError("val_runs must be at least 1")
    stops = sorted({int(c) for c in checkpoints if 0 < int(c) < rounds} | {rounds})
    best, best_params, done = -1.0, None, 0
    for c in stops:
        train(ctx, prop, model, rounds=c - done, first_round=done, **train_kw)
        done = c
        v = tail_ess(ctx, prop, model, val_traj, val_seed, list(range(val_runs)), N_tail, max_steps, dN)
        v["round"] = c
        prop.selection.append(v)
        if v["ess_per_step"] > best:
            best, best_params = v["ess_per_step"], prop.params.clone()
    if best_params is not None:
        prop.params.copy_(best_params)
        fpt.fpt_mlp_pack(ctx, prop.params, prop.blob)
        if prop.params.is_cuda:
            torch.cuda.synchronize()
    return prop


def new_proposals(ctx, init_params, shifts, scales, segment: int = 64, alpha_max: float = 4.0, flags: int = 0,
                  x_floors=None, device: str = "cuda"):
    """len(init_params) proposals whose parameters and packed blobs are the
    rows of two shared device tensors, as fpt_mlp_train_batch expects."""
    import torch
    n = len(init_params)
    P = torch.tensor(np.stack([np.asarray(v, np.float32) for v in init_params]), device=device)
    B = torch.zeros((n, fpt.FPT_MLP_BLOB_BYTES), dtype=torch.uint8, device=device)
    for k in range(n):
        fpt.fpt_mlp_pack(ctx, P[k], B[k])
    if P.is_cuda:
        torch.cuda.synchronize()
    fl = list(x_floors) if x_floors is not None else [0.0] * n
    props = [Proposal(P[k], B[k], tuple(float(v) for v in shifts[k]), tuple(float(v) for v in scales[k]), segment,
                      alpha_max, flags, float(fl[k])) for k in range(n)]
    return props, P, B


def train_batch(ctx, props, P, B, models, rounds: int, n_traj: int, seed: int, lam: float, N_cuts, lr=3e-3,
                clip: float = 0.0, first_round: int = 0, log: Optional[Callable[[list], None]] = None):
    """`rounds` Adam steps of every proposal at once (fpt_mlp_train_batch):
    proposal k trains on model models[k], n_traj fresh paths per round
    (Philox run id = round * len(props) + k). N_cuts: one N_cut per proposal,
    or a function of the round giving the list."""
    import torch
    if not hasattr(P, "_adam"):
        P._adam = (torch.zeros_like(P), torch.zeros_like(P))
    m, v = P._adam
    hist = []
    for r in range(first_round, first_round + rounds):
        runs = [props[k].desc(models[k], n_traj, seed=seed, run_id=r * len(props) + k) for k in range(len(props))]
        cuts = N_cuts(r) if callable(N_cuts) else N_cuts
        lr_r = lr(r) if callable(lr) else lr
        nn = n_traj
        while True:
            try:
                st = fpt.fpt_mlp_train_batch(ctx, runs, lam, cuts, dict(lr=lr_r, step=r + 1, clip=clip), P, m, v, B)
                break
            except fpt.FptError as e:
                # more segment records than the buffer holds: the round left the
                # parameters untouched, so it is redone on half the paths
                if e.status != fpt.FPT_E_NOMEM or nn <= 64:
                    raise
                nn //= 2
                runs = [props[k].desc(models[k], nn, seed=seed, run_id=r * len(props) + k)
                        for k in range(len(props))]
        for k, s in enumerate(st):
            s["round"] = r
            props[k].history.append(s)
        hist.append(st)
        if log:
            log(st)
    return hist


def save_checkpoint(prop: Proposal, path: str) -> None:
    """Everything a training run needs to resume: the fp32 parameters, the
    Adam moments, the input normalisation and the per-round history (the
    next round number is len(history))."""
    import json
    import torch
    m, v = getattr(prop, "_adam", (torch.zeros_like(prop.params), torch.zeros_like(prop.params)))
    np.savez(path, params=prop.params.detach().cpu().numpy(), adam_m=m.detach().cpu().numpy(),
             adam_v=v.detach().cpu().numpy(), shift=np.asarray(prop.shift), scale=np.asarray(prop.scale),
             segment=prop.segment, alpha_max=prop.alpha_max, flags=prop.flags, x_floor=prop.x_floor,
             history=json.dumps(prop.history))


def load_checkpoint(ctx, path: str, device: str = "cuda") -> Proposal:
    """A proposal saved by save_checkpoint, packed for ctx, with its Adam
    moments restored: train(..., first_round=len(prop.history)) continues the
    run as if it had not stopped (rounds are keyed by their number)."""
    import json
    import torch
    z = np.load(path)
    prop = new_proposal(ctx, z["params"], shift=tuple(z["shift"]), scale=tuple(z["scale"]),
                        segment=int(z["segment"]), alpha_max=float(z["alpha_max"]), flags=int(z["flags"]),
                        x_floor=float(z["x_floor"]), device=device)
    dev = prop.params.device
    prop._adam = (torch.tensor(z["adam_m"], device=dev), torch.tensor(z["adam_v"], device=dev))
    prop.history = json.loads(str(z["history"]))
    return prop


def save_batch_checkpoint(props, P, path: str) -> None:
    """The state of a batch training (train_batch): every proposal's fp32
    parameters (the rows of P), the shared Adam moments, each proposal's input
    normalisation and history (the next round number is len(history))."""
    import json
    import torch
    m, v = getattr(P, "_adam", (torch.zeros_like(P), torch.zeros_like(P)))
    meta = [dict(shift=list(q.shift), scale=list(q.scale), segment=q.segment, alpha_max=q.alpha_max, flags=q.flags,
                 x_floor=q.x_floor, history=q.history) for q in props]
    np.savez(path, params=P.detach().cpu().numpy(), adam_m=m.detach().cpu().numpy(),
             adam_v=v.detach().cpu().numpy(), meta=json.dumps(meta))


def load_batch_checkpoint(ctx, path: str, device: str = "cuda"):
    """(props, P, B) of a batch training saved by save_batch_checkpoint, packed
    for ctx, with the Adam moments restored: train_batch(..., first_round=
    len(props[0].history)) continues it as if it had not stopped."""
    import json
    import torch
    z = np.load(path)
    meta = json.loads(str(z["meta"]))
    q0 = meta[0]
    props, P, B = new_proposals(ctx, list(z["params"]), [q["shift"] for q in meta], [q["scale"] for q in meta],
                                segment=q0["segment"], alpha_max=q0["alpha_max"], flags=q0["flags"],
                                x_floors=[q["x_floor"] for q in meta], device=device)
    P._adam = (torch.tensor(z["adam_m"], device=P.device), torch.tensor(z["adam_v"], device=P.device))
    for q, mq in zip(props, meta):
        q.history = mq["history"]
    return props, P, B
