"""GPU parity of the paper's production setting: noise indexed by the time
since the start along the classical background, switched off after a window,
then a classical completion (Sec. 4.1)."""
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


def test_window_brownian_parity(torch):
    m = W.BM.model
    S, T = np.full(16, W.BM_S), np.zeros(16)
    N_lo, N_hi = 0.25, 1.5
    n = 4096
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER_N, 16, 1.0, N_lo, N_hi, S, T)
        runs = [fpt.run_desc(0, n, seed=70, run_id=0), fpt.run_desc(0, n, seed=70, run_id=1, A=0.8)]
        st, g = gpu_run(ctx, runs, [n, n])
        assert st == fpt.FPT_OK
    res = OT.resolve(m)
    tab = OT.user_table_N(S, T, N_lo, N_hi)
    for r, A in enumerate([0.0, 0.8]):
        o = OS.run(m, res, tab, seed=70, run_id=r, n=n, A=A)
        o.phi_end_value = res.phi_end
        compare(g[r], o, res.phi_in - res.phi_end, f"window A={A}")
    # most paths finish classically after the window
    assert np.mean(g[0]["N"] > N_hi) > 0.9


def test_window_usr_parity(torch):
    """Sudden-transition model, Bessel-matched noise in global time over the
    whole background range (noise on until the background reaches phi_end),
    direct and biased runs in one launch."""
    m = W.USR_MODEL
    res = OT.resolve(m)
    Nw = m.n_end - m.n_in
    n_pts, n = 256, 4096
    with fpt.fpt_init_model([m]) as ctx:
        S, Sp = fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL_N, n_pts, 1.0, 0.0, Nw)
        runs = [fpt.run_desc(0, n, seed=71, run_id=0), fpt.run_desc(0, n, seed=71, run_id=1, A=1.0)]
        st, g = gpu_run(ctx, runs, [n, n])
        assert st == fpt.FPT_OK
    tab = OT.bessel_table_N(m, res, n_pts, 1.0, 0.0, Nw, processes=8)
    np.testing.assert_allclose(S, tab.S, rtol=1e-8)
    # After the window the completion is classical at the late slow-roll
    # velocity pi dN ~ 1e-9 per step, below tau = 1e-5 x_in = 2.5e-9: every
    # post-window passage is a near-tie, and a field difference of ~1e-10
    # (FP32 state vs FP64) moves it by at most one step. So each mismatch must
    # be a near-tie and at most one step off; their fraction is bounded only
    # loosely (25%): a window error would move the field by S xi ~ 4e-8 >> tau
    # and fail as a non-near-tie.
    for r, A in enumerate([0.0, 1.0]):
        o = OS.run(m, res, tab, seed=71, run_id=r, n=n, A=A)
        o.phi_end_value = res.phi_end
        mism, near = compare(g[r], o, res.phi_in - res.phi_end, f"usr window A={A}",
                             max_mismatch=0.25, max_step_diff=1)
        print(f"usr window A={A}: mismatch {mism:.4%}, near-ties {near:.4%}")


def test_learned_run_with_a_time_indexed_table_is_rejected(torch):
    """The learned-proposal steppers index every table by the field, so a call
    that carries an MLP run on a phi-indexed table and another run on a
    time-indexed (noise-window) table must be refused before any launch."""
    m = W.BM.model
    S, T = np.full(16, W.BM_S), np.zeros(16)
    with fpt.fpt_init_model([m, m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, -0.1, 0.2, S, T)
        fpt.fpt_noise_table(ctx, 1, fpt.FPT_TABLE_USER_N, 16, 1.0, 0.25, 1.5, S, T)
        blob = torch.zeros(fpt.FPT_MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
        fpt.fpt_mlp_pack(ctx, torch.zeros(fpt.FPT_MLP_PARAMS, device="cuda"), blob)
        mlp = fpt.run_desc(0, 256, seed=72, run_id=0, bias_kind=fpt.FPT_BIAS_MLP, mlp=blob, mlp_segment=64,
                           mlp_shift=(0.0, 0.0, 0.0), mlp_scale=(1.0, 1.0, 1.0), alpha_max=2.0)
        for other in (fpt.run_desc(1, 256, seed=72, run_id=1, A=0.5), fpt.run_desc(1, 256, seed=72, run_id=1)):
            with pytest.raises(fpt.FptError) as e:
                fpt.fpt_run(ctx, [mlp, other])
            assert e.value.status == fpt.FPT_E_INVALID and "phi-indexed" in str(e.value)
        # an empty MLP run still selects the learned stepper: refused as well
        empty = fpt.run_desc(0, 0, seed=72, run_id=0, bias_kind=fpt.FPT_BIAS_MLP, mlp=blob, mlp_segment=64,
                             mlp_shift=(0.0, 0.0, 0.0), mlp_scale=(1.0, 1.0, 1.0), alpha_max=2.0)
        with pytest.raises(fpt.FptError) as e:
            fpt.fpt_run(ctx, [empty, fpt.run_desc(1, 256, seed=72, run_id=1)])
        assert e.value.status == fpt.FPT_E_INVALID
        # the context stays usable
        assert fpt.fpt_run(ctx, [mlp]) == fpt.FPT_OK and fpt.fpt_sync(ctx) == fpt.FPT_OK
