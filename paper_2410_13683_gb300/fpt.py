"""Thin ctypes binding of libfpt.so with the C ABI's names.

Argument marshalling only: every step of the sampler runs in the library's
CUDA kernels (and its host FP64 table builder). There is no CPU or PyTorch
fallback; if the library is missing or a call fails, an exception is raised.

Buffers may be torch tensors (host or CUDA), numpy arrays (host) or raw
integer addresses; streams may be ``torch.cuda.Stream`` objects, raw handles
or None (the context's private stream).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

NAN = float("nan")

FPT_OK, FPT_E_INVALID, FPT_E_CUDA, FPT_E_NOMEM, FPT_E_TIMEOUT, FPT_E_STATE = 0, 1, 2, 3, 4, 5
FPT_W_CAPPED = 100
FPT_POT_PWLINEAR, FPT_POT_EXP, FPT_POT_BUMP = 0, 1, 2
FPT_TABLE_DESITTER, FPT_TABLE_BESSEL, FPT_TABLE_USER, FPT_TABLE_BESSEL_N, FPT_TABLE_USER_N = 0, 1, 2, 3, 4
FPT_TABLE_NUMERIC, FPT_TABLE_USER2 = 5, 6
FPT_BIAS_NONE, FPT_BIAS_CONST, FPT_BIAS_MLP = 0, 1, 2
FPT_TRAJ_PASSED, FPT_TRAJ_CAPPED, FPT_TRAJ_ABORTED = 0, 1, 2
FPT_MLP_LOG_X = 1

_STATUS_NAMES = {0: "FPT_OK", 1: "FPT_E_INVALID", 2: "FPT_E_CUDA", 3: "FPT_E_NOMEM",
                 4: "FPT_E_TIMEOUT", 5: "FPT_E_STATE", 100: "FPT_W_CAPPED"}


class FptError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class fpt_model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("V0", C.c_double),
                ("a_plus", C.c_double), ("a_minus", C.c_double), ("phi_star", C.c_double),
                ("mu", C.c_double), ("phi_in", C.c_double), ("pi_in", C.c_double),
                ("phi_end", C.c_double), ("bg_phi0", C.c_double), ("n_in", C.c_double),
                ("n_end", C.c_double), ("dN", C.c_double), ("max_steps", C.c_int64),
                ("bump_K", C.c_double), ("bump_m", C.c_double), ("bump_width", C.c_double),
                ("bump_phi0", C.c_double)]


class fpt_model_info(C.Structure):
    _fields_ = [("phi_in", C.c_double), ("pi_in", C.c_double), ("phi_end", C.c_double),
                ("N_T", C.c_double)]


class fpt_run_desc(C.Structure):
    _fields_ = [("model", C.c_int32), ("bias_kind", C.c_int32), ("A", C.c_double),
                ("n_traj", C.c_int64), ("traj_offset", C.c_int64), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("mlp_segment", C.c_int32), ("mlp", C.c_void_p),
                ("mlp_shift", C.c_float * 3), ("mlp_scale", C.c_float * 3),
                ("alpha_max", C.c_float), ("mlp_flags", C.c_int32), ("A2", C.c_double),
                ("mlp_x_floor", C.c_float), ("pad_", C.c_int32)]


class fpt_classical(C.Structure):
    _fields_ = [("sigma_R2", C.c_double), ("eps2_in", C.c_double), ("eps2_end", C.c_double),
                ("N_in", C.c_double), ("N_end", C.c_double)]


class fpt_traj_out(C.Structure):
    _fields_ = [("N", C.c_void_p), ("logw", C.c_void_p), ("nsteps", C.c_void_p),
                ("status", C.c_void_p)]


class fpt_launch(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("check_steps", C.c_int32),
                ("use_graph", C.c_int32), ("deadline_s", C.c_double)]


class fpt_hist(C.Structure):
    _fields_ = [("count", C.c_void_p), ("log_sum_w", C.c_void_p), ("log_sum_w2", C.c_void_p),
                ("sum_lw", C.c_void_p), ("sum_lw2", C.c_void_p), ("pdf", C.c_void_p),
                ("se_w", C.c_void_p), ("pdf_ln", C.c_void_p), ("se_ln", C.c_void_p),
                ("se_jk", C.c_void_p), ("n_total", C.c_int64), ("n_passed", C.c_int64),
                ("n_under", C.c_int64), ("n_over", C.c_int64), ("n_capped", C.c_int64),
                ("n_tail", C.c_int64), ("N_mean", C.c_double), ("N_mean_w", C.c_double),
                ("ess_tail", C.c_double), ("p_tail", C.c_double), ("log_max_w", C.c_double)]


class fpt_adam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("clip", C.c_float), ("step", C.c_int32)]


class fpt_train_stats(C.Structure):
    _fields_ = [("loss", C.c_double), ("mean_Y", C.c_double), ("mean_N", C.c_double),
                ("n_traj", C.c_int64), ("n_records", C.c_int64), ("n_capped", C.c_int64),
                ("grad_norm", C.c_double)]


FPT_MLP_PARAMS = 4546
FPT_MLP_BLOB_BYTES = 11808


# Every function the header declares, with its ctypes signature.
_SIGNATURES = {
    "fpt_init_model": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(fpt_model), C.c_int32, C.c_int32]),
    "fpt_model_get_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(fpt_model_info)]),
    "fpt_noise_table": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                  C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "fpt_noise_table2": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                   C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "fpt_resolve_model": (C.c_int, [C.POINTER(fpt_model), C.POINTER(fpt_model_info)]),
    "fpt_table_build2": (C.c_int, [C.POINTER(fpt_model), C.c_int32, C.c_int32, C.c_double,
                                   C.c_double, C.c_double, C.c_void_p]),
    "fpt_table_build": (C.c_int, [C.POINTER(fpt_model), C.c_int32, C.c_int32, C.c_double,
                                  C.c_double, C.c_double, C.c_void_p, C.c_void_p]),
    "fpt_power_spectrum": (C.c_int, [C.POINTER(fpt_model), C.c_double, C.c_int32, C.c_void_p,
                                     C.c_double, C.c_void_p]),
    "fpt_classical_dn": (C.c_int, [C.POINTER(fpt_model), C.c_double, C.c_int32, C.c_double,
                                   C.POINTER(fpt_classical)]),
    "fpt_classical_pdf": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_void_p]),
    "fpt_fit_eps2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_double,
                               C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_int32)]),
    "fpt_set_launch": (C.c_int, [C.c_void_p, C.POINTER(fpt_launch)]),
    "fpt_get_launch": (C.c_int, [C.c_void_p, C.POINTER(fpt_launch)]),
    "fpt_autotune": (C.c_int, [C.c_void_p, C.POINTER(fpt_run_desc), C.c_int32, C.c_double,
                               C.POINTER(fpt_launch)]),
    "fpt_run": (C.c_int, [C.c_void_p, C.POINTER(fpt_run_desc), C.c_int32,
                          C.POINTER(fpt_traj_out), C.c_void_p]),
    "fpt_sync": (C.c_int, [C.c_void_p]),
    "fpt_histogram": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_int32,
                                C.c_double, C.POINTER(fpt_hist), C.c_void_p]),
    "fpt_histogram_data": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                     C.c_double, C.c_double, C.c_double, C.c_int32, C.c_double,
                                     C.POINTER(fpt_hist), C.c_void_p]),
    "fpt_mlp_pack": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fpt_mlp_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                               C.c_void_p, C.c_void_p, C.c_void_p]),
    "fpt_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                               C.c_float, C.c_void_p, C.c_void_p]),
    "fpt_mlp_grad2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                C.c_void_p, C.c_void_p]),
    "fpt_mlp_train_round": (C.c_int, [C.c_void_p, C.POINTER(fpt_run_desc), C.c_int64, C.c_double,
                                      C.c_double, C.POINTER(fpt_adam), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(fpt_train_stats), C.c_void_p]),
    "fpt_mlp_train_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p,
                                      C.POINTER(fpt_adam), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "fpt_run_records": (C.c_int, [C.c_void_p, C.POINTER(fpt_run_desc), C.c_int64, C.c_void_p,
                                  C.POINTER(C.c_int64), C.c_void_p]),
    "fpt_histogram_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                        C.c_double, C.c_double, C.c_int32, C.c_double, C.c_void_p,
                                        C.c_void_p]),
    "fpt_set_memory_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "fpt_memory_in_use": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "fpt_destroy": (None, [C.c_void_p]),
    "fpt_last_error": (C.c_char_p, [C.c_void_p]),
    "fpt_version": (C.c_char_p, []),
}

_LIB = None


def library_path() -> str:
    """libfpt.so, or the bounds-checked debug build libfpt_checks.so when the
    environment sets FPT_CHECKS=1 (built by build.build(checks=True))."""
    return _build.LIB_CHECKS if os.environ.get("FPT_CHECKS", "") == "1" else _build.LIB


def load(build_if_missing: bool = False):
    """Load libfpt.so (optionally building it first). Raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        _build.build(checks=os.environ.get("FPT_CHECKS", "") == "1")
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() first "
                           "(there is no fallback implementation)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, ctx=None):
    if status == FPT_OK or status == FPT_W_CAPPED:
        return status
    msg = load().fpt_last_error(ctx).decode(errors="replace")
    raise FptError(status, msg)


def _ptr(buf) -> Optional[int]:
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        return int(buf.data_ptr())
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be C-contiguous")
        return int(buf.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(buf)}")


CUDA_STREAM_LEGACY = 0x1      # cudaStreamLegacy: the legacy default stream


def _stream(stream) -> Optional[int]:
    """None -> the context's private stream; a torch stream (or handle) ->
    that stream. Handle 0 (torch's default stream) is the legacy default
    stream, which the ABI spells cudaStreamLegacy (NULL means "context")."""
    if stream is None:
        return None
    h = stream if isinstance(stream, int) else int(stream.cuda_stream)
    return h if h != 0 else CUDA_STREAM_LEGACY


def model_struct(m) -> fpt_model:
    """fpt_model from any object (or dict) with the header's field names."""
    get = (lambda k, d=NAN: m.get(k, d)) if isinstance(m, dict) else (lambda k, d=NAN: getattr(m, k, d))
    return fpt_model(kind=int(get("kind", 0)), pad=0, V0=get("V0"), a_plus=get("a_plus", 0.0),
                     a_minus=get("a_minus", 0.0), phi_star=get("phi_star", 0.0), mu=get("mu", 0.0),
                     phi_in=get("phi_in"), pi_in=get("pi_in"), phi_end=get("phi_end"),
                     bg_phi0=get("bg_phi0"), n_in=get("n_in"), n_end=get("n_end"), dN=get("dN"),
                     max_steps=int(get("max_steps", 1 << 20)), bump_K=get("bump_K", 0.0),
                     bump_m=get("bump_m", 0.0), bump_width=get("bump_width", 0.0),
                     bump_phi0=get("bump_phi0", 0.0))


class Context:
    """Owning handle of an fpt_ctx (destroyed on close() or garbage collection)."""

    def __init__(self, handle: int, n_models: int):
        self.handle = handle
        self.n_models = n_models

    def close(self):
        if self.handle:
            load().fpt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.handle)


def fpt_version() -> str:
    return load().fpt_version().decode()


def fpt_last_error(ctx: Optional[Context] = None) -> str:
    return load().fpt_last_error(ctx.handle if ctx else None).decode(errors="replace")


def fpt_init_model(models: Sequence, device: int = 0) -> Context:
    lib = load()
    arr = (fpt_model * len(models))(*[model_struct(m) for m in models])
    h = C.c_void_p()
    _check(lib.fpt_init_model(C.byref(h), arr, len(models), device))
    return Context(h.value, len(models))


def _info_dict(i: fpt_model_info) -> dict:
    return dict(phi_in=i.phi_in, pi_in=i.pi_in, phi_end=i.phi_end, N_T=i.N_T)


def fpt_model_get_info(ctx: Context, model: int) -> dict:
    i = fpt_model_info()
    _check(load().fpt_model_get_info(ctx.handle, model, C.byref(i)), ctx.handle)
    return _info_dict(i)


def fpt_resolve_model(model) -> dict:
    i = fpt_model_info()
    m = model_struct(model)
    _check(load().fpt_resolve_model(C.byref(m), C.byref(i)))
    return _info_dict(i)


def fpt_table_build(model, kind: int, n_points: int, sigma: float = 1.0, phi_lo: float = NAN,
                    phi_hi: float = NAN):
    S = np.zeros(n_points)
    T = np.zeros(n_points)
    m = model_struct(model)
    _check(load().fpt_table_build(C.byref(m), kind, n_points, sigma, phi_lo, phi_hi,
                                  _ptr(S), _ptr(T)))
    return S, T


def fpt_noise_table(ctx: Context, model: int, kind: int, n_points: int, sigma: float = 1.0,
                    phi_lo: float = NAN, phi_hi: float = NAN, user_S=None, user_Spi=None):
    S = np.zeros(n_points)
    T = np.zeros(n_points)
    uS = uT = None
    if kind in (FPT_TABLE_USER, FPT_TABLE_USER_N):
        uS = np.ascontiguousarray(user_S, dtype=np.float64)
        uT = np.ascontiguousarray(user_Spi, dtype=np.float64)
        if uS.shape != (n_points,) or uT.shape != (n_points,):
            raise ValueError("user tables must have n_points entries")
    _check(load().fpt_noise_table(ctx.handle, model, kind, n_points, sigma, phi_lo, phi_hi,
                                  _ptr(uS), _ptr(uT), _ptr(S), _ptr(T)), ctx.handle)
    return S, T


def fpt_table_build2(model, kind: int, n_points: int, sigma: float = 1.0, phi_lo: float = NAN,
                     phi_hi: float = NAN):
    """Full-rank table planes (S_phiphi, S_phipi, S_pipi), each n_points."""
    out = np.zeros(3 * n_points)
    m = model_struct(model)
    _check(load().fpt_table_build2(C.byref(m), kind, n_points, sigma, phi_lo, phi_hi, _ptr(out)))
    return out[:n_points], out[n_points:2 * n_points], out[2 * n_points:]


def fpt_noise_table2(ctx: Context, model: int, kind: int, n_points: int, sigma: float = 1.0,
                     phi_lo: float = NAN, phi_hi: float = NAN, user_S=None):
    """Full-rank (2-D) noise table; user_S = (S_phiphi, S_phipi, S_pipi) for USER2."""
    out = np.zeros(3 * n_points)
    uS = None
    if kind == FPT_TABLE_USER2:
        uS = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64) for v in user_S]))
        if uS.shape != (3 * n_points,):
            raise ValueError("user tables must have 3 planes of n_points entries")
    _check(load().fpt_noise_table2(ctx.handle, model, kind, n_points, sigma, phi_lo, phi_hi,
                                   _ptr(uS), _ptr(out)), ctx.handle)
    return out[:n_points], out[n_points:2 * n_points], out[2 * n_points:]


def fpt_power_spectrum(model, sigma: float, N_s, N_eval: float = NAN) -> np.ndarray:
    Ns = np.ascontiguousarray(N_s, dtype=np.float64)
    out = np.zeros(len(Ns))
    m = model_struct(model)
    _check(load().fpt_power_spectrum(C.byref(m), sigma, len(Ns), _ptr(Ns), N_eval, _ptr(out)))
    return out


def fpt_classical_dn(model, sigma: float = 1.0, n_k: int = 65, N_eval: float = NAN) -> dict:
    m = model_struct(model)
    o = fpt_classical()
    _check(load().fpt_classical_dn(C.byref(m), sigma, n_k, N_eval, C.byref(o)))
    return {k: getattr(o, k) for k, _ in fpt_classical._fields_}


def fpt_classical_pdf(dN, sigma_R2: float, eps2: float) -> np.ndarray:
    d = np.ascontiguousarray(dN, dtype=np.float64)
    out = np.zeros(len(d))
    _check(load().fpt_classical_pdf(_ptr(d), len(d), sigma_R2, eps2, _ptr(out)))
    return out


def fpt_fit_eps2(dN, pdf, se, sigma_R2: float, eps2_lo: float, eps2_hi: float) -> dict:
    d, p, e = (np.ascontiguousarray(v, dtype=np.float64) for v in (dN, pdf, se))
    eps2, chi2, used = C.c_double(), C.c_double(), C.c_int32()
    _check(load().fpt_fit_eps2(_ptr(d), _ptr(p), _ptr(e), len(d), sigma_R2, eps2_lo, eps2_hi,
                               C.byref(eps2), C.byref(chi2), C.byref(used)))
    return dict(eps2=eps2.value, chi2=chi2.value, bins=used.value)


def fpt_set_launch(ctx: Context, block: int = 0, blocks_per_sm: int = 0, check_steps: int = 0,
                   use_graph: bool = True, deadline_s: float = 0.0):
    l = fpt_launch(block=block, blocks_per_sm=blocks_per_sm, check_steps=check_steps,
                   use_graph=int(bool(use_graph)), deadline_s=deadline_s)
    _check(load().fpt_set_launch(ctx.handle, C.byref(l)), ctx.handle)


def fpt_get_launch(ctx: Context) -> dict:
    l = fpt_launch()
    _check(load().fpt_get_launch(ctx.handle, C.byref(l)), ctx.handle)
    return dict(block=l.block, blocks_per_sm=l.blocks_per_sm, check_steps=l.check_steps,
                use_graph=bool(l.use_graph), deadline_s=l.deadline_s)


def fpt_set_memory_limit(ctx: Context, max_bytes: int) -> None:
    """Cap the device memory the context may hold (0: no cap); allocations past
    it fail with FPT_E_NOMEM and leave the context usable."""
    _check(load().fpt_set_memory_limit(ctx.handle, int(max_bytes)), ctx.handle)


def fpt_memory_in_use(ctx: Context) -> tuple:
    """(bytes of device memory the context holds, its cap or 0)."""
    used, cap = C.c_int64(0), C.c_int64(0)
    _check(load().fpt_memory_in_use(ctx.handle, C.byref(used), C.byref(cap)), ctx.handle)
    return used.value, cap.value


def fpt_autotune(ctx: Context, runs: Sequence[fpt_run_desc], fraction: float = 0.25) -> dict:
    arr = (fpt_run_desc * len(runs))(*runs)
    l = fpt_launch()
    _check(load().fpt_autotune(ctx.handle, arr, len(runs), fraction, C.byref(l)), ctx.handle)
    return dict(block=l.block, blocks_per_sm=l.blocks_per_sm, check_steps=l.check_steps,
                use_graph=bool(l.use_graph), deadline_s=l.deadline_s)


def run_desc(model: int = 0, n_traj: int = 0, seed: int = 0, run_id: int = 0, A: float = 0.0,
             traj_offset: int = 0, bias_kind: Optional[int] = None, mlp=None, mlp_segment: int = 0,
             mlp_shift=(0.0, 0.0, 0.0), mlp_scale=(1.0, 1.0, 1.0), alpha_max: float = 0.0,
             mlp_flags: int = 0, A2: float = 0.0, mlp_x_floor: float = 0.0):
    if bias_kind is None:
        bias_kind = FPT_BIAS_MLP if mlp is not None else (
            FPT_BIAS_CONST if (A != 0.0 or A2 != 0.0) else FPT_BIAS_NONE)
    return fpt_run_desc(model=model, bias_kind=bias_kind, A=A, A2=A2, n_traj=n_traj,
                        traj_offset=traj_offset, seed=seed, run_id=run_id,
                        mlp_segment=mlp_segment, mlp=_ptr(mlp),
                        mlp_shift=(C.c_float * 3)(*mlp_shift), mlp_scale=(C.c_float * 3)(*mlp_scale),
                        alpha_max=alpha_max, mlp_flags=mlp_flags, mlp_x_floor=mlp_x_floor)


def fpt_run(ctx: Context, runs: Sequence[fpt_run_desc], out: Optional[Sequence[dict]] = None,
            stream=None) -> int:
    """Launch the runs; ``out`` is a list (one per run) of dicts with any of
    the keys N, logw, nsteps, status mapping to caller-owned buffers."""
    arr = (fpt_run_desc * len(runs))(*runs)
    outs = None
    if out is not None:
        if len(out) != len(runs):
            raise ValueError("one output dict per run")
        outs = (fpt_traj_out * len(runs))(*[
            fpt_traj_out(N=_ptr(o.get("N")), logw=_ptr(o.get("logw")),
                         nsteps=_ptr(o.get("nsteps")), status=_ptr(o.get("status")))
            for o in out])
    return _check(load().fpt_run(ctx.handle, arr, len(runs), outs, _stream(stream)), ctx.handle)


def fpt_sync(ctx: Context) -> int:
    return _check(load().fpt_sync(ctx.handle), ctx.handle)


HIST_ARRAYS = ("count", "log_sum_w", "log_sum_w2", "sum_lw", "sum_lw2", "pdf", "se_w", "pdf_ln",
               "se_ln", "se_jk")
HIST_SCALARS = ("n_total", "n_passed", "n_under", "n_over", "n_capped", "n_tail", "N_mean",
                "N_mean_w", "ess_tail", "p_tail", "log_max_w")


def fpt_histogram(ctx: Context, run: int, N_lo: float, N_hi: float, n_bins: int,
                  N_tail: float = NAN, stream=None) -> dict:
    arrs = {k: np.zeros(n_bins, np.int64 if k == "count" else np.float64) for k in HIST_ARRAYS}
    h = fpt_hist(**{k: _ptr(v) for k, v in arrs.items()})
    _check(load().fpt_histogram(ctx.handle, run, N_lo, N_hi, n_bins, N_tail, C.byref(h),
                                _stream(stream)), ctx.handle)
    res = dict(arrs)
    for k in HIST_SCALARS:
        res[k] = getattr(h, k)
    res["db"] = (N_hi - N_lo) / n_bins
    return res


def fpt_histogram_data(ctx: Context, nsteps, logw, status, dN: float, N_lo: float, N_hi: float,
                       n_bins: int, N_tail: float = NAN, stream=None) -> dict:
    """Histogram of caller-supplied per-trajectory arrays (host or device)."""
    if isinstance(nsteps, np.ndarray):
        nsteps = np.ascontiguousarray(nsteps, dtype=np.int32)
        logw = np.ascontiguousarray(logw, dtype=np.float64)
        status = np.ascontiguousarray(status, dtype=np.uint8)
    n = int(len(nsteps))
    arrs = {k: np.zeros(n_bins, np.int64 if k == "count" else np.float64) for k in HIST_ARRAYS}
    h = fpt_hist(**{k: _ptr(v) for k, v in arrs.items()})
    _check(load().fpt_histogram_data(ctx.handle, _ptr(nsteps), _ptr(logw), _ptr(status), n, dN,
                                     N_lo, N_hi, n_bins, N_tail, C.byref(h), _stream(stream)),
           ctx.handle)
    res = dict(arrs)
    for k in HIST_SCALARS:
        res[k] = getattr(h, k)
    res["db"] = (N_hi - N_lo) / n_bins
    return res


def fpt_mlp_pack(ctx: Context, params, blob, stream=None):
    """Pack fp32 parameters (host numpy/torch or device tensor) into the
    device weight blob (a CUDA tensor of >= FPT_MLP_BLOB_BYTES bytes)."""
    if isinstance(params, np.ndarray):
        params = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().fpt_mlp_pack(ctx.handle, _ptr(params), _ptr(blob), _stream(stream)), ctx.handle)


def fpt_mlp_eval(ctx: Context, blob, s, tan_t, alpha_max: float, stream=None):
    """alpha and raw outputs of the network at normalised inputs s (n x 3)."""
    s = np.ascontiguousarray(s, dtype=np.float32)
    t = np.ascontiguousarray(tan_t, dtype=np.float32)
    n = len(t)
    alpha = np.zeros(n, np.float32)
    o = np.zeros((n, 2), np.float32)
    _check(load().fpt_mlp_eval(ctx.handle, _ptr(blob), _ptr(s), _ptr(t), n, alpha_max, _ptr(alpha),
                               _ptr(o), _stream(stream)), ctx.handle)
    return alpha, o


def fpt_run_records(ctx: Context, run: fpt_run_desc, cap: int = 1 << 16, stream=None):
    """Segment records of one learned-proposal run, sorted by (unit, first
    step): dict of arrays in (n x 3), tan, raw, sum_xi, unit, n0."""
    rec = np.zeros((max(1, cap), 8), np.float32)
    n = C.c_int64(0)
    _check(load().fpt_run_records(ctx.handle, C.byref(run), cap, _ptr(rec), C.byref(n), _stream(stream)),
           ctx.handle)
    k = min(n.value, cap)
    rec = rec[:k]
    unit = rec[:, 6].view(np.uint32).astype(np.int64)
    n0 = rec[:, 7].view(np.int32).astype(np.int64)
    order = np.lexsort((n0, unit))
    rec, unit, n0 = rec[order], unit[order], n0[order]
    return {"in": rec[:, 0:3].astype(np.float64), "tan": rec[:, 3].astype(np.float64),
            "raw": rec[:, 4].astype(np.float64), "sum_xi": rec[:, 5].astype(np.float64),
            "unit": unit, "n0": n0, "n_records": n.value}


def fpt_mlp_grad(ctx: Context, params, s, tan_t, dalpha, alpha_max: float, stream=None):
    """sum_r dalpha_r d alpha(s_r, t_r)/d theta, canonical fp32 order."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.float32)
    t = np.ascontiguousarray(tan_t, dtype=np.float32)
    d = np.ascontiguousarray(dalpha, dtype=np.float32)
    g = np.zeros(FPT_MLP_PARAMS, np.float32)
    _check(load().fpt_mlp_grad(ctx.handle, _ptr(params), _ptr(s), _ptr(t), _ptr(d), len(t), alpha_max,
                               _ptr(g), _stream(stream)), ctx.handle)
    return g


def fpt_mlp_grad2(ctx: Context, params, s, dbeta, alpha_max: float, stream=None):
    """Gradient of sum(dbeta * beta(s)) for the 2-D bias beta = clamp(o)."""
    p = np.ascontiguousarray(params, np.float32) if isinstance(params, np.ndarray) else params
    sv = np.ascontiguousarray(s, np.float32)
    d = np.ascontiguousarray(dbeta, np.float32)
    g = np.zeros(FPT_MLP_PARAMS, np.float32)
    _check(load().fpt_mlp_grad2(ctx.handle, _ptr(p), _ptr(sv), _ptr(d), len(sv), alpha_max, _ptr(g),
                                _stream(stream)), ctx.handle)
    return g


def fpt_mlp_train_round(ctx: Context, run: fpt_run_desc, chunk: int, lam: float, N_cut: float,
                        adam: dict, params, adam_m, adam_v, blob, stream=None) -> dict:
    a = fpt_adam(lr=adam["lr"], beta1=adam.get("beta1", 0.9), beta2=adam.get("beta2", 0.999),
                 eps=adam.get("eps", 1e-8), clip=adam.get("clip", 0.0), step=adam["step"])
    st = fpt_train_stats()
    _check(load().fpt_mlp_train_round(ctx.handle, C.byref(run), chunk, lam, N_cut, C.byref(a),
                                      _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(blob), C.byref(st),
                                      _stream(stream)), ctx.handle)
    return {k: getattr(st, k) for k, _ in fpt_train_stats._fields_}


def fpt_mlp_train_batch(ctx: Context, runs: Sequence[fpt_run_desc], lam: float, N_cut, adam: dict, params,
                        adam_m, adam_v, blobs, stream=None) -> list:
    """One round for len(runs) proposals at once (run k on blob k, params row k)."""
    arr = (fpt_run_desc * len(runs))(*runs)
    cut = np.ascontiguousarray(N_cut, dtype=np.float64)
    if len(cut) != len(runs):
        raise ValueError("one N_cut per run")
    a = fpt_adam(lr=adam["lr"], beta1=adam.get("beta1", 0.9), beta2=adam.get("beta2", 0.999),
                 eps=adam.get("eps", 1e-8), clip=adam.get("clip", 0.0), step=adam["step"])
    st = (fpt_train_stats * len(runs))()
    _check(load().fpt_mlp_train_batch(ctx.handle, C.cast(arr, C.c_void_p), len(runs), lam, _ptr(cut), C.byref(a),
                                      _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(blobs), C.cast(st, C.c_void_p),
                                      _stream(stream)), ctx.handle)
    return [{k: getattr(x, k) for k, _ in fpt_train_stats._fields_} for x in st]


def canonical_params(p: dict) -> np.ndarray:
    """Flatten {W1, b1, W2, b2, W3, b3} into the canonical fp32 vector."""
    return np.concatenate([np.asarray(p[k], np.float64).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
                          ).astype(np.float32)


def params_dict(v) -> dict:
    v = np.asarray(v, np.float64)
    H = 64
    out, o = {}, 0
    for k, shape in (("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (2, H)), ("b3", (2,))):
        size = int(np.prod(shape))
        out[k] = v[o:o + size].reshape(shape)
        o += size
    return out


FPT_NOALLOC_MAX_BINS = 1024


def hist_out_doubles(n_bins: int) -> int:
    return 10 * n_bins + 16


def fpt_histogram_noalloc(nsteps, logw, status, dN: float, N_lo: float, N_hi: float, n_bins: int,
                          out, N_tail: float = NAN, stream=None) -> int:
    """Allocation-free histogram of device arrays into the device buffer
    `out` (hist_out_doubles(n_bins) doubles). Asynchronous on `stream`."""
    st = load().fpt_histogram_noalloc(_ptr(nsteps), _ptr(logw), _ptr(status), int(len(nsteps)), dN, N_lo,
                                      N_hi, n_bins, N_tail, _ptr(out), _stream(stream))
    return _check(st)


def unpack_hist(buf, n_bins: int) -> dict:
    """Split the packed histogram output into the fpt_histogram dict layout."""
    b = np.asarray(buf, dtype=np.float64)
    res = {}
    for i, k in enumerate(HIST_ARRAYS):
        v = b[i * n_bins:(i + 1) * n_bins]
        res[k] = v.astype(np.int64) if k == "count" else v.copy()
    sc = b[10 * n_bins:]
    for i, k in enumerate(HIST_SCALARS):
        res[k] = int(sc[i]) if k.startswith("n_") else float(sc[i])
    return res
