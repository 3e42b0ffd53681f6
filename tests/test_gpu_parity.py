"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
trajectory by trajectory on identical Philox streams, and the histogram
kernels against the oracle's estimators."""
import math
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from oracle import estimators as E
from oracle import stepper as OS
from oracle import tables as OT
from paper_2410_13683_gb300 import fpt

from gpu_common import compare, gpu_run, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def oracle_traj(m, res, tab, seed, run_id, n, A=0.0, traj0=0):
    tr = OS.run(m, res, tab, seed=seed, run_id=run_id, n=n, A=A, traj0=traj0)
    tr.phi_end_value = res.phi_end
    return tr


def bm_table():
    return np.full(16, W.BM_S), np.zeros(16), -0.1, 0.2


def test_brownian_direct_and_biased(torch):
    wl = W.BM
    m = wl.model
    S, Tt, lo, hi = bm_table()
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        n = 8192
        runs = [fpt.run_desc(0, n, seed=wl.seed, run_id=0),
                fpt.run_desc(0, n, seed=wl.seed, run_id=1, A=0.7)]
        st, g = gpu_run(ctx, runs, [n, n])
        assert st == fpt.FPT_OK
    res = OT.resolve(m)
    tab = OT.user_table(S, Tt, lo, hi)
    for r, A in enumerate([0.0, 0.7]):
        o = oracle_traj(m, res, tab, wl.seed, r, n, A=A)
        compare(g[r], o, res.phi_in - res.phi_end, f"BM A={A}")
    assert np.all(g[0]["logw"] == 0.0)


def test_linear_slow_roll_workload(torch):
    """The slow-roll linear case at full size (16384 trajectories)."""
    wl = W.LINEAR
    m = wl.model
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_DESITTER, 4096, 1.0, wl.table.phi_lo, wl.table.phi_hi)
        st, g = gpu_run(ctx, [fpt.run_desc(0, wl.n_traj, seed=wl.seed, run_id=wl.run_id)], [wl.n_traj])
        assert st == fpt.FPT_OK
        h = fpt.fpt_histogram(ctx, 0, 4.0, 6.0, 64)
    res = OT.resolve(m)
    tab = OT.desitter_table(m, res, 4096, wl.table.phi_lo, wl.table.phi_hi)
    o = oracle_traj(m, res, tab, wl.seed, wl.run_id, wl.n_traj)
    mism, near = compare(g[0], o, res.phi_in - res.phi_end, "linear")
    N = g[0]["N"]
    se = N.std() / math.sqrt(len(N))
    assert abs(N.mean() - 5.0029) < 4 * se
    assert abs(N.var() - 0.04225) < 4 * 4.7e-4
    assert h["n_total"] == wl.n_traj and h["n_capped"] == 0
    assert h["N_mean"] == pytest.approx(N.mean(), rel=1e-12)


@pytest.fixture(scope="module")
def usr512():
    """The sudden-transition model with 512-point Bessel tables, built
    independently by the library (C++) and the oracle (SciPy)."""
    m = W.USR_MODEL
    res = OT.resolve(m)
    tab = OT.bessel_table(m, res, 512, 1.0, processes=8)
    return m, res, tab


def test_usr_direct_parity(torch, usr512):
    m, res, tab = usr512
    n = 8192
    with fpt.fpt_init_model([m]) as ctx:
        S, Sp = fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        np.testing.assert_allclose(S, tab.S, rtol=1e-8)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=2, run_id=0)], [n])
    o = oracle_traj(m, res, tab, 2, 0, n)
    mism, near = compare(g[0], o, res.phi_in - res.phi_end, "usr direct")
    print(f"usr direct: mismatch {mism:.4%}, near-ties {near:.4%}")


def test_usr_fixed_bias_batch_parity(torch, usr512):
    """Several bias amplitudes (and direct sampling) in one persistent launch,
    uneven lengths and capped trajectories included."""
    m, res, tab = usr512
    m = replace(m, max_steps=1 << 15)
    biases = [0.0, 0.5, 1.0, 2.0]
    n = 2048
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        runs = [fpt.run_desc(0, n, seed=3, run_id=i, A=A) for i, A in enumerate(biases)]
        st, g = gpu_run(ctx, runs, [n] * len(biases))
        assert st in (fpt.FPT_OK, fpt.FPT_W_CAPPED)
    for i, A in enumerate(biases):
        o = oracle_traj(m, res, tab, 3, i, n, A=A)
        compare(g[i], o, res.phi_in - res.phi_end, f"usr A={A}")
    assert (g[3]["status"] == fpt.FPT_TRAJ_CAPPED).any()
    assert st == fpt.FPT_W_CAPPED


def test_histogram_kernel_on_oracle_trajectories(torch, usr512):
    """K2 + finalize on the oracle's own trajectories equals the oracle's
    estimators: counts exactly, sums to FP64 rounding."""
    m, res, tab = usr512
    m = replace(m, max_steps=1 << 15)
    n = 1 << 14
    o = oracle_traj(m, res, tab, 5, 0, n, A=0.5)
    lo, hi, nb, tail = 2.0, 20.0, 96, 12.0
    h_or = E.histogram(o.nsteps, o.logw, o.status, m.dN, lo, hi, nb)
    with fpt.fpt_init_model([m]) as ctx:
        h = fpt.fpt_histogram_data(ctx, o.nsteps.astype(np.int32), o.logw, o.status, m.dN, lo, hi, nb, tail)
    assert np.array_equal(h["count"], h_or.count)
    nz = h_or.count > 0
    np.testing.assert_allclose(h["log_sum_w"][nz], h_or.log_sum_w[nz], rtol=0, atol=1e-12)
    np.testing.assert_allclose(h["log_sum_w2"][nz], h_or.log_sum_w2[nz], rtol=0, atol=1e-12)
    np.testing.assert_allclose(h["sum_lw"], h_or.sum_lw, rtol=1e-12, atol=1e-9)
    P, se = E.p_weighted(h_or)
    np.testing.assert_allclose(h["pdf"], P, rtol=1e-11)
    np.testing.assert_allclose(h["se_w"], se, rtol=1e-8, atol=1e-300)
    Pl, sel = E.p_lognormal(h_or)
    ok = np.isfinite(Pl)
    np.testing.assert_allclose(h["pdf_ln"][ok], Pl[ok], rtol=1e-9)
    np.testing.assert_allclose(h["se_ln"][ok], sel[ok], rtol=1e-7)
    Pj, sej = E.p_jackknife(h_or)
    np.testing.assert_allclose(h["se_jk"], sej, rtol=1e-7, atol=1e-300)
    assert h["n_under"] == h_or.n_under and h["n_over"] == h_or.n_over
    assert h["n_capped"] == h_or.n_capped and h["n_total"] == n
    e, p, k = E.tail_ess(o.nsteps, o.logw, o.status, m.dN, tail)
    assert h["n_tail"] == k
    assert h["ess_tail"] == pytest.approx(e, rel=1e-10)
    assert h["p_tail"] == pytest.approx(p, rel=1e-10)
    assert h["N_mean"] == pytest.approx(E.mean_N(o.nsteps, o.status, m.dN), rel=1e-12)
    assert h["N_mean_w"] == pytest.approx(E.mean_N(o.nsteps, o.status, m.dN, o.logw), rel=1e-10)


def test_histogram_of_gpu_run_matches_oracle_run(torch, usr512):
    """P(delta N) from a GPU importance-sampled run agrees bin by bin with the
    oracle's run of the same trajectories within 3 combined standard errors."""
    m, res, tab = usr512
    m = replace(m, max_steps=1 << 15)
    n = 1 << 14
    lo, hi, nb = 2.0, 20.0, 48
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=6, run_id=0, A=0.5)])
        h = fpt.fpt_histogram(ctx, 0, lo, hi, nb)
    o = oracle_traj(m, res, tab, 6, 0, n, A=0.5)
    h_or = E.histogram(o.nsteps, o.logw, o.status, m.dN, lo, hi, nb)
    P, se = E.p_weighted(h_or)
    ok = (h_or.count >= 10)
    assert ok.sum() > 10
    diff = np.abs(h["pdf"][ok] - P[ok])
    assert np.all(diff <= 3 * np.hypot(h["se_w"][ok], se[ok]) + 1e-300)


def test_launch_shape_and_split_invariance(torch, usr512):
    """Results depend only on (seed, trajectory, run): not on block size,
    refill interval, graph replay, or how the id range is split."""
    m, res, tab = usr512
    n = 3000
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        ref = None
        for block, check, graph in [(256, 32, True), (128, 4, False), (512, 64, True), (256, 8, True)]:
            fpt.fpt_set_launch(ctx, block=block, check_steps=check, use_graph=graph)
            for rep in range(2):        # second call replays the captured graph
                _, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=9, run_id=4, A=0.5)], [n])
                if ref is None:
                    ref = g[0]
                assert np.array_equal(g[0]["nsteps"], ref["nsteps"])
                assert np.array_equal(g[0]["logw"], ref["logw"])
        _, parts = gpu_run(ctx, [fpt.run_desc(0, 1000, seed=9, run_id=4, A=0.5, traj_offset=0),
                                 fpt.run_desc(0, 2000, seed=9, run_id=4, A=0.5, traj_offset=1000)],
                           [1000, 2000])
        assert np.array_equal(np.concatenate([parts[0]["nsteps"], parts[1]["nsteps"]]), ref["nsteps"])
        assert np.array_equal(np.concatenate([parts[0]["logw"], parts[1]["logw"]]), ref["logw"])


def test_graph_replay_takes_the_seed_and_the_current_table(torch):
    """A replayed graph runs with the call's Philox key and the model's
    current table constants: after a call of the same launch shape with
    another seed, or after a new table of the same size on another field
    range, the results are those of a fresh context without graphs."""
    m = W.BM.model
    n = 4096
    S = W.BM_S * np.linspace(0.5, 1.5, 16)
    cases = [(9, -0.1, 0.2), (10, -0.1, 0.2), (10, -0.2, 0.3), (9, -0.2, 0.3)]

    def run(ctx, seed):
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=seed, run_id=1, A=0.3)], [n])
        assert st == fpt.FPT_OK
        return g[0]

    fresh = []
    for seed, lo, hi in cases:
        with fpt.fpt_init_model([m]) as c:
            fpt.fpt_set_launch(c, use_graph=False)
            fpt.fpt_noise_table(c, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, np.zeros(16))
            fresh.append(run(c, seed))
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_set_launch(ctx, use_graph=True)
        table = None
        for (seed, lo, hi), want in zip(cases, fresh):
            if table != (lo, hi):
                fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, np.zeros(16))
                table = (lo, hi)
            for rep in range(2):
                g = run(ctx, seed)
                assert np.array_equal(g["nsteps"], want["nsteps"]), (seed, lo, hi, rep)
                assert np.array_equal(g["logw"], want["logw"]), (seed, lo, hi, rep)
    # the four cases differ from one another
    for i in range(len(cases)):
        for j in range(i):
            assert not np.array_equal(fresh[i]["nsteps"], fresh[j]["nsteps"])


def test_device_outputs_and_streams(torch, usr512):
    m, res, tab = usr512
    n = 4096
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_BESSEL, 512, 1.0)
        s = torch.cuda.Stream()
        dn = torch.zeros(n, dtype=torch.int32, device="cuda")
        dl = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = fpt.fpt_run(ctx, [fpt.run_desc(0, n, seed=2, run_id=0)], [dict(nsteps=dn, logw=dl)], stream=s)
        assert st == fpt.FPT_OK
        assert fpt.fpt_sync(ctx) == fpt.FPT_OK
        _, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=2, run_id=0)], [n])
        assert np.array_equal(dn.cpu().numpy(), g[0]["nsteps"])


def test_cap_warning_and_status(torch):
    wl = W.BM
    m = replace(wl.model, max_steps=100)
    S, Tt, lo, hi = bm_table()
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        st, g = gpu_run(ctx, [fpt.run_desc(0, 512, seed=1)], [512])
        assert st == fpt.FPT_W_CAPPED
        assert np.all(g[0]["status"] == fpt.FPT_TRAJ_CAPPED) and np.all(g[0]["nsteps"] == 100)
        h = fpt.fpt_histogram(ctx, 0, 0.0, 1.0, 8)
        assert h["n_capped"] == 512 and h["n_passed"] == 0


def test_deadline_aborts_and_context_recovers(torch):
    """A kernel deadline ends the launch early with FPT_E_TIMEOUT; no fault,
    and the same context runs normally afterwards."""
    wl = W.BM
    m = replace(wl.model, max_steps=1 << 24)
    S, Tt, lo, hi = np.full(16, 1e-9), np.zeros(16), -0.1, 0.2   # essentially never passes
    m = replace(m, mu=1e-9, pi_in=-1e-9)
    with fpt.fpt_init_model([m]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        fpt.fpt_set_launch(ctx, deadline_s=0.05)
        with pytest.raises(fpt.FptError) as e:
            gpu_run(ctx, [fpt.run_desc(0, 4096, seed=1)], [4096])
        assert e.value.status == fpt.FPT_E_TIMEOUT
        with pytest.raises(fpt.FptError) as e2:
            fpt.fpt_histogram(ctx, 0, 0.0, 1.0, 8)
        assert e2.value.status == fpt.FPT_E_STATE
        fpt.fpt_set_launch(ctx, deadline_s=0.0)
    m2 = wl.model
    with fpt.fpt_init_model([m2]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, np.full(16, W.BM_S), Tt)
        st, g = gpu_run(ctx, [fpt.run_desc(0, 1024, seed=1)], [1024])
        assert st == fpt.FPT_OK and np.all(g[0]["status"] == 0)


def test_invalid_runs_are_rejected_before_launch(torch):
    wl = W.BM
    S, Tt, lo, hi = bm_table()
    with fpt.fpt_init_model([wl.model]) as ctx:
        with pytest.raises(fpt.FptError) as e:
            fpt.fpt_run(ctx, [fpt.run_desc(0, 16, seed=1)])
        assert e.value.status == fpt.FPT_E_STATE          # no table yet
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        bad = [
            [fpt.run_desc(1, 16, seed=1)],
            [fpt.run_desc(0, 16, seed=1), fpt.run_desc(0, 16, seed=2)],
            [fpt.run_desc(0, 16, seed=1, traj_offset=(1 << 32) - 8)],
            [fpt.run_desc(0, 16, seed=1, A=float("inf"))],
        ]
        for runs in bad:
            with pytest.raises(fpt.FptError) as e:
                fpt.fpt_run(ctx, runs)
            assert e.value.status == fpt.FPT_E_INVALID
        with pytest.raises(fpt.FptError):
            fpt.fpt_histogram(ctx, 0, 1.0, 0.0, 8)


def test_capped_allocator_reports_nomem_and_context_recovers(torch):
    """The context's device allocations are counted; past its limit an
    allocation fails as an out-of-memory cudaMalloc would: FPT_E_NOMEM, the
    message names the limit, and the same context runs normally once the
    request fits -- with the same trajectories as an uncapped context."""
    wl = W.BM
    S, Tt, lo, hi = bm_table()
    n, small_n, spare = 1 << 20, 4096, 2 << 20
    with fpt.fpt_init_model([wl.model]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        used, cap = fpt.fpt_memory_in_use(ctx)
        assert used > 0 and cap == 0
        # 2^20 trajectories need ~21 MB of outputs; the 2^16-unit minimum fits in 1.4 MB
        fpt.fpt_set_memory_limit(ctx, used + spare)
        assert fpt.fpt_memory_in_use(ctx)[1] == used + spare
        with pytest.raises(fpt.FptError) as e:
            gpu_run(ctx, [fpt.run_desc(0, n, seed=3)], [n])
        assert e.value.status == fpt.FPT_E_NOMEM and "limit" in str(e.value)
        assert fpt.fpt_memory_in_use(ctx)[0] <= used + spare
        st, small = gpu_run(ctx, [fpt.run_desc(0, small_n, seed=3)], [small_n])
        assert st == fpt.FPT_OK
        assert fpt.fpt_memory_in_use(ctx)[0] <= used + spare
        with pytest.raises(fpt.FptError) as e:
            fpt.fpt_set_memory_limit(ctx, -1)
        assert e.value.status == fpt.FPT_E_INVALID
        fpt.fpt_set_memory_limit(ctx, 0)
        st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=3)], [n])
        assert st == fpt.FPT_OK
        assert fpt.fpt_memory_in_use(ctx)[0] > used + spare
    with fpt.fpt_init_model([wl.model]) as ref:
        fpt.fpt_noise_table(ref, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        st, r = gpu_run(ref, [fpt.run_desc(0, n, seed=3)], [n])
    for k in ("nsteps", "logw", "status"):
        assert np.array_equal(g[0][k], r[0][k])
        assert np.array_equal(small[0][k], r[0][k][:small_n])


def test_pooled_runs_equal_one_histogram_of_their_union(torch, tmp_path):
    """A sampling job of three runs (Philox run ids 0-2) pooled run by run
    (paper_2410_13683_gb300.accumulate), checkpointed after the second and
    resumed from the file, equals the library's histogram of the three runs'
    trajectories taken in one call."""
    from paper_2410_13683_gb300.accumulate import RunAccumulator
    wl = W.BM
    S, Tt, lo, hi = bm_table()
    n, A, N_lo, N_hi, nb, N_tail = 1 << 16, 0.7, 0.0, 12.0, 256, 5.5
    path = str(tmp_path / "job.npz")
    outs = []
    with fpt.fpt_init_model([wl.model]) as ctx:
        fpt.fpt_noise_table(ctx, 0, fpt.FPT_TABLE_USER, 16, 1.0, lo, hi, S, Tt)
        acc = RunAccumulator(seed=9, N_lo=N_lo, N_hi=N_hi, n_bins=nb, N_tail=N_tail)
        for r in range(3):
            st, g = gpu_run(ctx, [fpt.run_desc(0, n, seed=9, run_id=r, A=A)], [n])
            assert st == fpt.FPT_OK
            outs.append(g[0])
            acc.add(r, fpt.fpt_histogram(ctx, 0, N_lo, N_hi, nb, N_tail=N_tail))
            if r == 1:
                acc.save(path)
                acc = RunAccumulator.load(path)
        cat = {k: np.concatenate([o[k] for o in outs]) for k in ("nsteps", "logw", "status")}
        h = fpt.fpt_histogram_data(ctx, cat["nsteps"], cat["logw"], cat["status"], wl.model.dN, N_lo, N_hi, nb,
                                   N_tail=N_tail)
    est = acc.estimates()
    assert est["runs"] == 3 and est["n_total"] == h["n_total"] == 3 * n
    assert np.array_equal(est["count"], h["count"])
    np.testing.assert_allclose(est["pdf"], h["pdf"], rtol=1e-12)
    np.testing.assert_allclose(est["se_w"], h["se_w"], rtol=1e-8, atol=1e-12 * np.max(h["se_w"]))
    np.testing.assert_allclose(est["pdf_ln"], h["pdf_ln"], rtol=1e-11, equal_nan=True)
    np.testing.assert_allclose(est["se_ln"], h["se_ln"], rtol=1e-11, equal_nan=True)
    assert est["p_tail"] == pytest.approx(h["p_tail"], rel=1e-12)
    assert est["ess_tail"] == pytest.approx(h["ess_tail"], rel=1e-11)
