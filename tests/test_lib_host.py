"""CPU tests of libfpt.so: it builds, loads, exports every declared symbol,
and its host FP64 model resolution / table builder agree with the oracle."""
import ctypes as C
import math
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import tables as T
from paper_2410_13683_gb300 import build as B
from paper_2410_13683_gb300 import fpt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    fpt.load()


def declared_functions():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(fpt_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "fpt_run" in names and "fpt_histogram" in names and "fpt_noise_table" in names
    lib = C.CDLL(B.LIB)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fpt_[a-z0-9_]+)", out))
    assert set(names) <= exported
    # the binding declares exactly the header's functions
    assert set(fpt._SIGNATURES) == set(names)


def test_checked_build_compiles_and_loads():
    """The FPT_CHECKS debug build (device bounds checks on table indexes,
    trajectory indexes and histogram bins) compiles, loads beside the plain
    build and exports the same functions."""
    path = B.build(checks=True)
    assert path == B.LIB_CHECKS != B.LIB
    lib = C.CDLL(path)
    lib.fpt_version.restype = C.c_char_p
    assert b"FPT_CHECKS" in lib.fpt_version()
    assert b"FPT_CHECKS" not in fpt.load().fpt_version()
    for n in declared_functions():
        assert hasattr(lib, n), n


@pytest.mark.parametrize("wl", [W.LINEAR, W.BM])
def test_resolve_explicit_models(wl):
    info = fpt.fpt_resolve_model(wl.model)
    r = T.resolve(wl.model)
    assert info["phi_in"] == r.phi_in and info["phi_end"] == r.phi_end
    assert info["pi_in"] == pytest.approx(r.pi_in, rel=1e-15)
    assert math.isnan(info["N_T"])


def test_resolve_transition_rule_matches_oracle():
    info = fpt.fpt_resolve_model(W.USR_MODEL)
    r = T.resolve(W.USR_MODEL)
    assert abs(info["N_T"] - r.N_T) < 1e-9
    assert abs(info["phi_in"] - r.phi_in) < 1e-12
    assert abs(info["pi_in"] / r.pi_in - 1) < 1e-9
    assert abs(info["phi_end"] - r.phi_end) < 1e-12


def test_bessel_table_matches_oracle():
    m = W.USR_MODEL
    S, Sp = fpt.fpt_table_build(m, fpt.FPT_TABLE_BESSEL, 4096, 1.0)
    idx = [0, 1, 7, 300, 1500, 2048, 3333, 4000, 4094, 4095]
    tab = T.bessel_table(m, T.resolve(m), 4096, 1.0, indices=idx)
    np.testing.assert_allclose(S[idx], tab.S[idx], rtol=1e-8)
    np.testing.assert_allclose(Sp[idx], tab.T[idx], rtol=0, atol=1e-8 * float(np.max(tab.S[idx])))


def test_bessel_table_other_sigma_and_range():
    m = W.USR_MODEL
    r = T.resolve(m)
    lo, hi = r.phi_end + 1e-5, r.phi_in - 1e-5
    S, Sp = fpt.fpt_table_build(m, fpt.FPT_TABLE_BESSEL, 64, 0.5, lo, hi)
    tab = T.bessel_table(m, r, 64, 0.5, lo, hi, indices=[0, 31, 63])
    np.testing.assert_allclose(S[[0, 31, 63]], tab.S[[0, 31, 63]], rtol=1e-8)


def test_desitter_table_matches_oracle():
    wl = W.LINEAR
    S, Sp = fpt.fpt_table_build(wl.model, fpt.FPT_TABLE_DESITTER, 4096, 1.0, 0.0, 0.06)
    tab = T.desitter_table(wl.model, T.resolve(wl.model), 4096, 0.0, 0.06)
    np.testing.assert_allclose(S, tab.S, rtol=1e-14)
    assert np.all(Sp == 0)


@pytest.mark.parametrize("patch,msg", [
    (dict(V0=-1.0), "V0"),
    (dict(dN=0.0), "dN"),
    (dict(max_steps=0), "max_steps"),
    (dict(phi_in=-1.0), "phi_in > phi_end"),
    (dict(kind=7), "kind"),
])
def test_invalid_models_are_rejected(patch, msg):
    m = dict(W.LINEAR.model.__dict__)
    m.update(patch)
    with pytest.raises(fpt.FptError) as e:
        fpt.fpt_resolve_model(m)
    assert e.value.status == fpt.FPT_E_INVALID and msg in str(e.value)


def test_invalid_table_arguments():
    with pytest.raises(fpt.FptError) as e:
        fpt.fpt_table_build(W.LINEAR.model, fpt.FPT_TABLE_BESSEL, 16, 1.0)   # no transition rule
    assert e.value.status == fpt.FPT_E_INVALID
    with pytest.raises(fpt.FptError):
        fpt.fpt_table_build(W.USR_MODEL, fpt.FPT_TABLE_BESSEL, 1, 1.0)
    with pytest.raises(fpt.FptError):
        fpt.fpt_table_build(W.USR_MODEL, fpt.FPT_TABLE_BESSEL, 16, 0.0)


def test_context_needs_a_gpu_or_fails_loudly():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(fpt.FptError) as e:
        fpt.fpt_init_model([W.LINEAR.model])
    assert e.value.status == fpt.FPT_E_CUDA


def test_time_indexed_bessel_table_matches_oracle():
    """Noise along the classical background in global time (the paper's
    production setting): library vs oracle at sampled grid times."""
    m = W.USR_MODEL
    r = T.resolve(m)
    Nw = m.n_end - m.n_in
    S, Sp = fpt.fpt_table_build(m, fpt.FPT_TABLE_BESSEL_N, 512, 1.0, 0.0, Nw)
    idx = [0, 1, 100, 256, 510, 511]
    tab = T.bessel_table_N(m, r, 512, 1.0, 0.0, Nw, indices=idx)
    np.testing.assert_allclose(S[idx], tab.S[idx], rtol=1e-8)
    # the time-indexed table at time N equals the phi-indexed one at phi_bg(N_in + N)
    ph, _, _ = r.bg.state(r.N_in + Nw * 256 / 511)
    S_phi, _ = fpt.fpt_table_build(m, fpt.FPT_TABLE_BESSEL, 2, 1.0, ph, ph + 1e-9)
    assert S[256] == pytest.approx(S_phi[0], rel=1e-7)


def test_time_indexed_table_needs_a_window():
    with pytest.raises(fpt.FptError):
        fpt.fpt_table_build(W.USR_MODEL, fpt.FPT_TABLE_BESSEL_N, 64, 1.0)


@pytest.mark.parametrize("sigma,rtol", [(1.0, 1e-7), (0.1, 1e-5)])
def test_numeric_table_matches_oracle(sigma, rtol):
    """Full-rank table (Eq. 3.9, symmetric square root) of the host builder vs
    the oracle's numerical matching; at sigma = 0.1 Xi is squeezed
    (det / (Xi_pp Xi_qq) ~ 1e-5), so sqrt(det) carries the cancellation of
    the determinant and the tolerance is wider."""
    m = W.USR_MODEL
    M = 1024
    Spp, Spq, Sqq = fpt.fpt_table_build2(m, fpt.FPT_TABLE_NUMERIC, M, sigma)
    idx = [0, 1, 100, 511, 1000, 1023]
    tab = T.numeric_table(m, T.resolve(m), M, sigma, indices=idx)
    for got, ref in ((Spp, tab.Spp), (Spq, tab.Spq), (Sqq, tab.Sqq)):
        np.testing.assert_allclose(got[idx], ref[idx], rtol=rtol)


def test_numeric_table_arguments():
    with pytest.raises(fpt.FptError):
        fpt.fpt_table_build2(W.LINEAR.model, fpt.FPT_TABLE_NUMERIC, 16, 1.0)   # no transition rule
    with pytest.raises(fpt.FptError):
        fpt.fpt_table_build2(W.USR_MODEL, fpt.FPT_TABLE_USER2, 16, 1.0)       # user tables are not built
    with pytest.raises(fpt.FptError):
        fpt.fpt_table_build2(W.USR_MODEL, fpt.FPT_TABLE_NUMERIC, 16, 0.0)


def test_bump_model_resolution_and_tables_match_oracle():
    """Gaussian bump (Sec. 4.3): start/end from the ultra-slow-roll onset and the
    Bessel-matched and numerically matched tables, host builder vs oracle."""
    m = W.BUMP_MODEL
    info = fpt.fpt_resolve_model(m)
    r = T.resolve(m)
    assert abs(info["N_T"] - r.N_T) < 1e-8
    assert abs(info["phi_in"] - r.phi_in) < 1e-12 and abs(info["phi_end"] - r.phi_end) < 1e-12
    assert abs(info["pi_in"] / r.pi_in - 1) < 1e-8
    idx = [0, 511, 1023]
    S, Sp = fpt.fpt_table_build(m, fpt.FPT_TABLE_BESSEL, 1024, 1.0)
    tab = T.bessel_table(m, r, 1024, 1.0, indices=idx)
    np.testing.assert_allclose(S[idx], tab.S[idx], rtol=1e-8)
    np.testing.assert_allclose(Sp[idx], tab.T[idx], rtol=1e-8)
    Spp, Spq, Sqq = fpt.fpt_table_build2(m, fpt.FPT_TABLE_NUMERIC, 1024, 1.0)
    t2 = T.numeric_table(m, r, 1024, 1.0, indices=idx)
    for got, ref in ((Spp, t2.Spp), (Spq, t2.Spq), (Sqq, t2.Sqq)):
        np.testing.assert_allclose(got[idx], ref[idx], rtol=1e-7)


def test_bump_model_arguments():
    import dataclasses
    with pytest.raises(fpt.FptError):
        fpt.fpt_resolve_model(dataclasses.replace(W.BUMP_MODEL, bump_width=0.0))
    with pytest.raises(fpt.FptError) as e:
        fpt.fpt_resolve_model(dataclasses.replace(W.BUMP_MODEL, bg_phi0=2.19))   # starts past the bump: no USR onset
    assert "ultra-slow roll" in str(e.value)


def test_classical_dn_matches_oracle():
    """Eq. (2.18) over the simulated mode range and the power spectrum, host
    builder vs oracle, for the sudden transition and the bump."""
    from oracle import classical as C
    for m in (W.USR_MODEL, W.BUMP_MODEL):
        r = T.resolve(m)
        c = fpt.fpt_classical_dn(m, 1.0, 33)
        assert c["sigma_R2"] == pytest.approx(C.sigma_R2(m, r, 1.0, n_k=33), rel=1e-7)
        assert c["eps2_end"] == pytest.approx(C.eps2_at(m, r, r.N_end), rel=1e-7, abs=1e-9)
        Ns = np.array([r.N_in, 0.5 * (r.N_in + r.N_end), r.N_end])
        P = fpt.fpt_power_spectrum(m, 1.0, Ns)
        ref = [C.power_spectrum_at(m, r, N, 1.0, r.N_end + C.LATE) for N in Ns]
        np.testing.assert_allclose(P, ref, rtol=1e-7)


def test_classical_pdf_and_fit():
    """Eq. (2.20) against the oracle's restatement, and the eps2 fit recovering
    eps2 from exact PDF values."""
    from oracle import classical as C
    d = np.linspace(-0.3, 1.5, 40)
    for e2 in (0.0, 0.745, -1.2):
        np.testing.assert_allclose(fpt.fpt_classical_pdf(d, 0.0098, e2), C.pdf_constant_eps2(d, 0.0098, e2),
                                   rtol=1e-12)
    p = C.pdf_constant_eps2(d, 0.0098, 0.745)
    f = fpt.fpt_fit_eps2(d, p, 0.01 * p, 0.0098, 0.0, 3.0)
    assert f["eps2"] == pytest.approx(0.745, abs=1e-7) and f["chi2"] < 1e-9 and f["bins"] == 40
    with pytest.raises(fpt.FptError):
        fpt.fpt_classical_dn(W.LINEAR.model, 1.0, 33)       # no transition rule
    with pytest.raises(fpt.FptError):
        fpt.fpt_classical_dn(W.BUMP_MODEL, 1.0, 32)         # even n_k
