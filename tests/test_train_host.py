"""Host logic of the training driver on CPU, with the library calls faked:
a round whose segment records overflow the record buffer is redone in
halves (and the halved chunk is kept), other errors pass through, and the
held-out selection measures at the right rounds with distinct run ids and
keeps the best parameters; a checkpointed run resumes exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_13683_gb300 import fpt
from paper_2410_13683_gb300 import train as TR


def _prop():
    return TR.Proposal(params=torch.zeros(8), blob=torch.zeros(16, dtype=torch.uint8), shift=(0.0, 0.0, 0.0),
                       scale=(1.0, 1.0, 1.0), segment=64, alpha_max=4.0)


def _fake_round(limit, calls, status=fpt.FPT_E_NOMEM):
    def f(ctx, run, chunk, lam, N_cut, adam, params, m, v, blob, stream=None):
        calls.append(chunk)
        if chunk > limit:
            raise fpt.FptError(status, "segment records exceed the record buffer")
        params += 1.0          # one Adam step
        return {"loss": 1.0 / adam["step"]}
    return f


def test_overflowing_round_is_redone_in_halves(monkeypatch):
    calls = []
    monkeypatch.setattr(fpt, "fpt_mlp_train_round", _fake_round(3000, calls))
    prop = TR.train(None, _prop(), 0, rounds=3, n_traj=10000, seed=1, lam=0.5, N_cut=lambda r: 9.0,
                    lr=1e-3, chunk=10000)
    assert calls == [10000, 5000, 2500, 2500, 2500]
    assert [h["chunk"] for h in prop.history] == [2500] * 3
    assert [h["round"] for h in prop.history] == [0, 1, 2]
    assert float(prop.params[0]) == 3.0      # each round updated the parameters once


def test_other_errors_and_tiny_chunks_are_raised(monkeypatch):
    calls = []
    monkeypatch.setattr(fpt, "fpt_mlp_train_round", _fake_round(10, calls, status=fpt.FPT_E_CUDA))
    with pytest.raises(fpt.FptError):
        TR.train(None, _prop(), 0, rounds=1, n_traj=4096, seed=1, lam=0.5, N_cut=lambda r: 9.0, lr=1e-3)
    assert calls == [4096]
    calls.clear()
    monkeypatch.setattr(fpt, "fpt_mlp_train_round", _fake_round(10, calls))
    with pytest.raises(fpt.FptError):
        TR.train(None, _prop(), 0, rounds=1, n_traj=4096, seed=1, lam=0.5, N_cut=lambda r: 9.0, lr=1e-3)
    assert calls == [4096, 2048, 1024]


def test_selection_stops_run_ids_and_kept_parameters(monkeypatch):
    trained, measured, packed = [], [], []

    def fake_train(ctx, prop, model, rounds, first_round=0, **kw):
        trained.append((first_round, rounds))
        prop.params.fill_(float(first_round + rounds))     # parameters name the round count
        return prop

    score = {20: 1.0, 40: 3.0, 60: 2.0}

    def fake_ess(ctx, prop, model, n_traj, seed, run_ids, N_tail, max_steps, dN, stream=None):
        c = int(prop.params[0])
        measured.append((c, seed, list(run_ids)))
        return {"ess_tail": score[c] * 100, "p_tail": 1e-3, "steps": 100.0, "ess_per_step": score[c]}

    monkeypatch.setattr(TR, "train", fake_train)
    monkeypatch.setattr(TR, "tail_ess", fake_ess)
    monkeypatch.setattr(fpt, "fpt_mlp_pack", lambda ctx, p, b, stream=None: packed.append(float(p[0])))
    prop = TR.train_select(None, _prop(), 0, rounds=60, checkpoints=[40, 20, 20, 0, 75], val_traj=1024,
                           val_seed=7, N_tail=5.0, max_steps=1000, dN=1e-3, val_runs=3)
    assert trained == [(0, 20), (20, 20), (40, 20)]
    # common random numbers: every checkpoint runs on the same held-out trajectories
    assert measured == [(20, 7, [0, 1, 2]), (40, 7, [0, 1, 2]), (60, 7, [0, 1, 2])]
    assert [v["round"] for v in prop.selection] == [20, 40, 60]
    assert float(prop.params[0]) == 40.0 and packed == [40.0]
    with pytest.raises(ValueError):
        TR.train_select(None, _prop(), 0, rounds=10, checkpoints=[], val_traj=8, val_seed=1, N_tail=1.0,
                        max_steps=10, dN=1e-3, val_runs=0)


def test_batch_rounds_halve_on_overflow_and_number_runs(monkeypatch):
    """train_batch: proposal k of round r draws Philox run id r K + k on its
    model; a round whose records overflow is redone on half the paths (all
    runs alike) and the parameters step once per round; N_cuts may depend on
    the round."""
    calls = []

    def fake(ctx, runs, lam, cuts, adam, P, m, v, B, stream=None):
        calls.append(([r.n_traj for r in runs], [r.run_id for r in runs], [r.model for r in runs], list(cuts)))
        if runs[0].n_traj > 1000:
            raise fpt.FptError(fpt.FPT_E_NOMEM, "segment records exceed the record buffer")
        P += 1.0
        return [{"loss": 0.5} for _ in runs]

    monkeypatch.setattr(fpt, "fpt_mlp_train_batch", fake)
    P = torch.zeros((3, 8))
    B = torch.zeros((3, 16), dtype=torch.uint8)
    props = [TR.Proposal(params=P[k], blob=B[k], shift=(0.0, 0.0, 0.0), scale=(1.0, 1.0, 1.0), segment=64,
                         alpha_max=4.0) for k in range(3)]
    hist = TR.train_batch(None, props, P, B, [2, 0, 1], rounds=2, n_traj=4000, seed=5, lam=0.25,
                          N_cuts=lambda r: [10.0 + r, 20.0, 30.0], lr=1e-3)
    assert [c[0][0] for c in calls] == [4000, 2000, 1000, 4000, 2000, 1000]
    assert calls[0][1] == [0, 1, 2] and calls[3][1] == [3, 4, 5]
    assert calls[2][2] == [2, 0, 1]
    assert calls[2][3] == [10.0, 20.0, 30.0] and calls[5][3] == [11.0, 20.0, 30.0]
    assert float(P[0, 0]) == 2.0 and len(hist) == 2 and [h["round"] for h in props[1].history] == [0, 1]
    # other errors pass through
    monkeypatch.setattr(fpt, "fpt_mlp_train_batch",
                        lambda *a, **k: (_ for _ in ()).throw(fpt.FptError(fpt.FPT_E_CUDA, "launch failed")))
    with pytest.raises(fpt.FptError):
        TR.train_batch(None, props, P, B, [0, 0, 0], rounds=1, n_traj=100, seed=5, lam=0.25, N_cuts=[1.0] * 3)


def test_checkpoint_resume_equals_uninterrupted_training(monkeypatch, tmp_path):
    """Train 3 rounds, save, load into a fresh proposal and train 2 more: the
    parameters, Adam moments, run ids and history equal those of 5 rounds
    without the stop."""
    def fake(ctx, run, chunk, lam, N_cut, adam, params, m, v, blob, stream=None):
        g = torch.sin(params + float(run.run_id))          # a gradient that depends on the state and the round
        m.mul_(0.9).add_(0.1 * g)
        v.mul_(0.999).add_(0.001 * g * g)
        params.sub_(adam["lr"] * m / (v.sqrt() + 1e-8))
        return {"loss": float(params.sum()), "run_id": int(run.run_id)}

    monkeypatch.setattr(fpt, "fpt_mlp_train_round", fake)
    monkeypatch.setattr(fpt, "fpt_mlp_pack", lambda ctx, p, b, stream=None: None)

    def fresh():
        return TR.new_proposal(None, np.linspace(-1, 1, 8), shift=(0.5, 0.0, 0.0), scale=(0.2, 1.0, 0.01),
                               segment=128, alpha_max=8.0, flags=fpt.FPT_MLP_LOG_X, x_floor=1e-4,
                               device="cpu")

    kw = dict(model=0, n_traj=1024, seed=4, lam=0.25, N_cut=lambda r: 10.0 + r)
    ref = TR.train(None, fresh(), rounds=5, **kw)

    a = TR.train(None, fresh(), rounds=3, **kw)
    path = str(tmp_path / "ck.npz")
    TR.save_checkpoint(a, path)
    b = TR.load_checkpoint(None, path, device="cpu")
    assert (b.shift, b.scale, b.segment, b.alpha_max, b.flags, b.x_floor) == \
        (a.shift, a.scale, a.segment, a.alpha_max, a.flags, a.x_floor)
    assert torch.equal(b.params, a.params) and b.params.dtype == torch.float32
    assert all(torch.equal(x, y) for x, y in zip(b._adam, a._adam))
    TR.train(None, b, rounds=2, first_round=len(b.history), **kw)
    assert [h["run_id"] for h in b.history] == [0, 1, 2, 3, 4]
    assert [h["round"] for h in b.history] == [h["round"] for h in ref.history]
    assert torch.equal(b.params, ref.params)
    assert all(torch.equal(x, y) for x, y in zip(b._adam, ref._adam))


def test_batch_checkpoint_resume_equals_uninterrupted_training(monkeypatch, tmp_path):
    """A batch training (every proposal of a model family in one call per
    round) saved after 2 rounds and resumed for 2 more equals 4 rounds without
    the stop: parameters, shared Adam moments, run ids and histories."""
    def fake(ctx, runs, lam, cuts, adam, P, m, v, B, stream=None):
        ids = torch.tensor([float(r.run_id) for r in runs])[:, None]
        g = torch.cos(P * 0.7 + ids)
        m.mul_(0.9).add_(0.1 * g)
        v.mul_(0.999).add_(0.001 * g * g)
        P.sub_(adam["lr"] * m / (v.sqrt() + 1e-8))
        return [{"loss": float(P[k].sum()), "run_id": int(r.run_id)} for k, r in enumerate(runs)]

    monkeypatch.setattr(fpt, "fpt_mlp_train_batch", fake)
    monkeypatch.setattr(fpt, "fpt_mlp_pack", lambda ctx, p, b, stream=None: None)

    def fresh():
        return TR.new_proposals(None, [np.linspace(-1, 1, 8) * (k + 1) for k in range(3)],
                                [(0.1 * k, 0.0, 0.0) for k in range(3)], [(0.2, 1.0 + k, 0.01) for k in range(3)],
                                segment=128, alpha_max=8.0, flags=fpt.FPT_MLP_LOG_X,
                                x_floors=[1e-4 * (k + 1) for k in range(3)], device="cpu")

    kw = dict(models=[0, 1, 2], n_traj=512, seed=5, lam=0.25, N_cuts=[10.0, 20.0, 30.0])
    props_r, P_r, B_r = fresh()
    TR.train_batch(None, props_r, P_r, B_r, rounds=4, **kw)

    props_a, P_a, B_a = fresh()
    TR.train_batch(None, props_a, P_a, B_a, rounds=2, **kw)
    path = str(tmp_path / "batch.npz")
    TR.save_batch_checkpoint(props_a, P_a, path)
    props_b, P_b, B_b = TR.load_batch_checkpoint(None, path, device="cpu")
    assert [(q.shift, q.scale, q.x_floor) for q in props_b] == [(q.shift, q.scale, q.x_floor) for q in props_a]
    TR.train_batch(None, props_b, P_b, B_b, rounds=2, first_round=len(props_b[0].history), **kw)
    assert torch.equal(P_b, P_r)
    assert all(torch.equal(x, y) for x, y in zip(P_b._adam, P_r._adam))
    assert [h["run_id"] for h in props_b[1].history] == [h["run_id"] for h in props_r[1].history] == [1, 4, 7, 10]
