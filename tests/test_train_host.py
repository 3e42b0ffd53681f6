"""Host logic of the training driver on CPU, with the library calls faked:
a round whose segment records overflow the record buffer is redone in
halves (and the halved chunk is kept), other errors pass through, and the
held-out selection measures at the right rounds with distinct run ids and
keeps the best parameters."""
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
