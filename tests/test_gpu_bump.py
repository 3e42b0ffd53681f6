"""GPU parity on the Gaussian-bump model (Sec. 4.3): a smooth transition to
ultra-slow roll where the drift V'/V is the small difference of two large
terms (the stepper reads it from a cubic FP64-valued table) and the noise
angle tan(theta_n) = nu - 3/2 is far from zero, with 1-D and 2-D noise."""
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


@pytest.fixture(scope="module")
def bump():
    m = W.BUMP_MODEL
    res = OT.resolve(m)
    return m, res, OT.bessel_table(m, res, 129, 1.0, processes=8)


def test_bump_noise_off_is_classical(torch, bump):
    """Zero noise: the GPU's FP32 Euler path with the tabulated drift takes the
    same number of steps as the oracle's FP64 path."""
    m, res, _ = bump
    z = np.zeros(8)
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 8, 1.0, res.phi_end, res.phi_in, z, z)
        st, g = gpu_run(ctx, [fpt.run_desc(0, 64, seed=1)], [64])
        assert st == fpt.FPT_OK
    o = OS.run(m, res, OT.user_table(z, z, res.phi_end, res.phi_in), seed=1, run_id=0, n=64)
    assert np.all(g[0]["nsteps"] == o.nsteps)


def test_bump_parity(torch, bump):
    """Bessel-matched 1-D noise (t = nu - 3/2 ~ 0.25..0.38), direct and two
    constant biases in one launch, per trajectory against the oracle."""
    m, res, tab = bump
    n = 4096
    As = [0.0, 1.0, 3.0]
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, len(tab.S), 1.0, tab.phi_lo,
                            tab.phi_lo + tab.h * (len(tab.S) - 1), tab.S, tab.T)
        runs = [fpt.run_desc(0, n, seed=90, run_id=r, A=A) for r, A in enumerate(As)]
        st, g = gpu_run(ctx, runs, [n] * len(As))
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    for r, A in enumerate(As):
        o = OS.run(m, res, tab, seed=90, run_id=r, n=n, A=A)
        o.phi_end_value = res.phi_end
        mism, near = compare(g[r], o, res.phi_in - res.phi_end, f"bump A={A}")
        print(f"bump A={A}: mismatch {mism:.4%}, near-ties {near:.4%}")


def test_bump_library_table_parity(torch, bump):
    """The library's own Bessel table for the bump (host FP64 build) against the
    oracle's, and the run on it against the oracle's run on its own table."""
    m, res, _ = bump
    M, n = 65, 4096
    tab = OT.bessel_table(m, res, M, 1.0, processes=8)
    with fpt.fpt_init_model([m]) as ctx:
        S, Sp = fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, M, 1.0)
        np.testing.assert_allclose(S, tab.S, rtol=1e-8)
        np.testing.assert_allclose(Sp, tab.T, rtol=1e-8)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=91, A=2.0)], [n])
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    o = OS.run(m, res, tab, seed=91, run_id=0, n=n, A=2.0)
    o.phi_end_value = res.phi_end
    compare(g[0], o, res.phi_in - res.phi_end, "bump library table")


def test_bump_2d_parity(torch, bump):
    """Full-rank noise on the bump (numerical matching at sigma = 1)."""
    m, res, _ = bump
    tab = OT.numeric_table(m, res, 65, 1.0)
    n = 4096
    betas = [(0.0, 0.0), (1.0, 0.5)]
    with fpt.fpt_init_model([m]) as ctx:
        M = len(tab.Spp)
        fpt.fpt_noise_table2(ctx, 0, fpt.FPT_TABLE_USER2, M, 1.0, tab.phi_lo, tab.phi_lo + tab.h * (M - 1),
                             (tab.Spp, tab.Spq, tab.Sqq))
        runs = [fpt.run_desc(0, n, seed=92, run_id=r, A=b1, A2=b2) for r, (b1, b2) in enumerate(betas)]
        st, g = gpu_run(ctx, runs, [n, n])
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    for r, (b1, b2) in enumerate(betas):
        o = OS.run2(m, res, tab, seed=92, run_id=r, n=n, A=b1, A2=b2)
        o.phi_end_value = res.phi_end
        compare(g[r], o, res.phi_in - res.phi_end, f"bump 2-D beta=({b1},{b2})")


def test_bump_rules(torch):
    """The bump does not share a call with other potentials; no noise window."""
    with fpt.fpt_init_model([W.BUMP_MODEL, W.USR_MODEL]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 64, 1.0)
        fpt.fpt_noise_table(ctx, 1, fpt.FPT_TABLE_BESSEL, 64, 1.0)
        with pytest.raises(fpt.FptError):
            fpt.fpt_run(ctx, [fpt.run_desc(0, 64, seed=1), fpt.run_desc(1, 64, seed=1, run_id=1)])
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL_N, 64, 1.0, 0.0, 2.0)
        with pytest.raises(fpt.FptError):
            fpt.fpt_run(ctx, [fpt.run_desc(0, 64, seed=1)])
