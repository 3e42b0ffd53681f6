"""ctypes binding of the FP64 C oracle stepper (oracle/fpt_oracle.c).

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fpt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, strict IEEE double)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32),
                ("V0", C.c_double), ("a_plus", C.c_double), ("a_minus", C.c_double),
                ("phi_star", C.c_double), ("mu", C.c_double),
                ("phi_in", C.c_double), ("pi_in", C.c_double), ("phi_end", C.c_double),
                ("dN", C.c_double), ("max_steps", C.c_int64),
                ("bump_K", C.c_double), ("bump_m", C.c_double), ("bump_w", C.c_double),
                ("bump_phi0", C.c_double)]


class _Table(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("phi_lo", C.c_double), ("h", C.c_double),
                ("S", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double)),
                ("n_indexed", C.c_int32), ("pad", C.c_int32)]


class _Bias(C.Structure):
    _fields_ = [("kind", C.c_int32), ("hidden", C.c_int32), ("A", C.c_double),
                ("segment", C.c_int64), ("alpha_max", C.c_double),
                ("round_bf16", C.c_int32), ("log_x", C.c_int32),
                ("W1", C.POINTER(C.c_double)), ("b1", C.POINTER(C.c_double)),
                ("W2", C.POINTER(C.c_double)), ("b2", C.POINTER(C.c_double)),
                ("W3", C.POINTER(C.c_double)), ("b3", C.POINTER(C.c_double)),
                ("in_shift", C.c_double * 3), ("in_scale", C.c_double * 3), ("x_floor", C.c_double)]


class _Table2(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("phi_lo", C.c_double), ("h", C.c_double),
                ("Spp", C.POINTER(C.c_double)), ("Spq", C.POINTER(C.c_double)),
                ("Sqq", C.POINTER(C.c_double))]


class _Seg2(C.Structure):
    _fields_ = [("cap", C.c_int64), ("n_seg", C.POINTER(C.c_int64)), ("state", C.POINTER(C.c_double)),
                ("beta", C.POINTER(C.c_double)), ("sum_xi", C.POINTER(C.c_double))]


class _Out(C.Structure):
    _fields_ = [("nsteps", C.POINTER(C.c_int64)), ("logw", C.POINTER(C.c_double)),
                ("status", C.POINTER(C.c_uint8)), ("phi_final", C.POINTER(C.c_double)),
                ("pi_final", C.POINTER(C.c_double)), ("xmin_pre", C.POINTER(C.c_double))]


class _Seg(C.Structure):
    _fields_ = [("cap", C.c_int64), ("n_seg", C.POINTER(C.c_int64)),
                ("state", C.POINTER(C.c_double)), ("tan_theta", C.POINTER(C.c_double)),
                ("alpha", C.POINTER(C.c_double)), ("sum_xi", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        _lib.oracle_normals4.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                         C.POINTER(C.c_double)]
        _lib.oracle_run.argtypes = [C.POINTER(_Model), C.POINTER(_Table), C.POINTER(_Bias),
                                    C.c_uint64, C.c_uint32, C.c_int64, C.c_int64, C.c_int,
                                    C.POINTER(_Out)]
        _lib.oracle_run.restype = C.c_int
        _lib.oracle_run_segments.argtypes = [C.POINTER(_Model), C.POINTER(_Table),
                                             C.POINTER(_Bias), C.c_uint64, C.c_uint32,
                                             C.c_int64, C.POINTER(C.c_int64),
                                             C.POINTER(C.c_double), C.POINTER(C.c_uint8),
                                             C.POINTER(_Seg)]
        _lib.oracle_run_segments.restype = C.c_int
        _lib.oracle_run2.argtypes = [C.POINTER(_Model), C.POINTER(_Table2), C.POINTER(_Bias),
                                     C.c_double, C.c_uint64, C.c_uint32, C.c_int64, C.c_int64,
                                     C.c_int, C.POINTER(_Out)]
        _lib.oracle_run2.restype = C.c_int
        _lib.oracle_run2_segments.argtypes = [C.POINTER(_Model), C.POINTER(_Table2), C.POINTER(_Bias),
                                              C.c_uint64, C.c_uint32, C.c_uint32, C.POINTER(C.c_int64),
                                              C.POINTER(C.c_double), C.POINTER(C.c_uint8), C.POINTER(_Seg2)]
        _lib.oracle_run2_segments.restype = C.c_int
        _lib.oracle_mlp_forward.argtypes = [C.POINTER(_Bias), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
        _lib.oracle_max_threads.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals4(seed: int, run_id: int, traj: int, block: int):
    z = (C.c_double * 4)()
    lib().oracle_normals4(seed, run_id, traj, block, z)
    return np.array(z[:])


@dataclass
class Trajectories:
    nsteps: np.ndarray
    logw: np.ndarray
    status: np.ndarray
    phi_final: np.ndarray
    pi_final: np.ndarray
    xmin_pre: np.ndarray
    dN: float

    @property
    def N(self):
        return self.nsteps * self.dN


def model_struct(m, phi_in, pi_in, phi_end) -> _Model:
    return _Model(kind=m.kind, pad=0, V0=m.V0, a_plus=m.a_plus, a_minus=m.a_minus,
                  phi_star=m.phi_star, mu=m.mu, phi_in=phi_in, pi_in=pi_in,
                  phi_end=phi_end, dN=m.dN, max_steps=m.max_steps,
                  bump_K=getattr(m, "bump_K", 0.0), bump_m=getattr(m, "bump_m", 0.0),
                  bump_w=getattr(m, "bump_width", 0.0), bump_phi0=getattr(m, "bump_phi0", 0.0))


class MLPBias:
    """FP64 MLP proposal parameters for the oracle (weights kept alive here).

    round_bf16: the network as bf16 tensor-core tiles hold it. The weight
    matrices W1, W2, W3 are rounded to bfloat16 here, once (biases stay as
    given), and the C forward rounds the inputs and hidden activations."""

    def __init__(self, params: dict, segment: int, in_shift, in_scale, alpha_max=20.0,
                 round_bf16=True, log_x=False, x_floor=0.0):
        from . import mlp as _mlp
        self.p = {k: np.ascontiguousarray(_mlp.bf16(v) if (round_bf16 and k.startswith("W")) else v,
                                          dtype=np.float64) for k, v in params.items()}
        self.segment = int(segment)
        self.in_shift = list(in_shift)
        self.in_scale = list(in_scale)
        self.alpha_max = float(alpha_max)
        self.round_bf16 = bool(round_bf16)
        self.log_x = bool(log_x)
        self.x_floor = float(x_floor)
        self.hidden = self.p["W1"].shape[0]

    def struct(self) -> _Bias:
        p = self.p
        return _Bias(kind=2, hidden=self.hidden, A=0.0, segment=self.segment,
                     alpha_max=self.alpha_max, round_bf16=int(self.round_bf16), log_x=int(self.log_x),
                     W1=_dp(p["W1"]), b1=_dp(p["b1"]), W2=_dp(p["W2"]), b2=_dp(p["b2"]),
                     W3=_dp(p["W3"]), b3=_dp(p["b3"]),
                     in_shift=(C.c_double * 3)(*self.in_shift),
                     in_scale=(C.c_double * 3)(*self.in_scale), x_floor=self.x_floor)


def bias_struct(A: float = 0.0, mlp: MLPBias | None = None) -> _Bias:
    if mlp is not None:
        return mlp.struct()
    z = (C.c_double * 3)(0.0, 0.0, 0.0)
    return _Bias(kind=1 if A != 0.0 else 0, hidden=0, A=float(A), segment=1, alpha_max=0.0,
                 round_bf16=0, log_x=0, in_shift=z, in_scale=z)


def run(m, resolved, table, seed: int, run_id: int, n: int, traj0: int = 0,
        A: float = 0.0, mlp: MLPBias | None = None, threads: int = 0) -> Trajectories:
    """FP64 trajectories traj0 .. traj0+n-1 of one run."""
    S = np.ascontiguousarray(table.S, dtype=np.float64)
    T = np.ascontiguousarray(table.T, dtype=np.float64)
    tab = _Table(n_points=len(S), phi_lo=table.phi_lo, h=table.h, S=_dp(S), T=_dp(T),
                 n_indexed=int(getattr(table, "n_indexed", False)), pad=0)
    ms = model_struct(m, resolved.phi_in, resolved.pi_in, resolved.phi_end)
    b = bias_struct(A, mlp)
    out = dict(nsteps=np.zeros(n, np.int64), logw=np.zeros(n), status=np.zeros(n, np.uint8),
               phi_final=np.zeros(n), pi_final=np.zeros(n), xmin_pre=np.zeros(n))
    o = _Out(nsteps=out["nsteps"].ctypes.data_as(C.POINTER(C.c_int64)),
             logw=_dp(out["logw"]), status=out["status"].ctypes.data_as(C.POINTER(C.c_uint8)),
             phi_final=_dp(out["phi_final"]), pi_final=_dp(out["pi_final"]),
             xmin_pre=_dp(out["xmin_pre"]))
    rc = lib().oracle_run(C.byref(ms), C.byref(tab), C.byref(b), seed, run_id, traj0, n,
                          threads, C.byref(o))
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    return Trajectories(dN=m.dN, **out)


def run_segments(m, resolved, table, mlp: MLPBias, seed: int, run_id: int, traj: int,
                 cap: int = 1 << 16):
    """One learned-bias trajectory with its per-segment records."""
    S = np.ascontiguousarray(table.S, dtype=np.float64)
    T = np.ascontiguousarray(table.T, dtype=np.float64)
    tab = _Table(n_points=len(S), phi_lo=table.phi_lo, h=table.h, S=_dp(S), T=_dp(T),
                 n_indexed=int(getattr(table, "n_indexed", False)), pad=0)
    ms = model_struct(m, resolved.phi_in, resolved.pi_in, resolved.phi_end)
    b = mlp.struct()
    n_seg = C.c_int64(0)
    state = np.zeros((cap, 3)); tt = np.zeros(cap); al = np.zeros(cap); sx = np.zeros(cap)
    seg = _Seg(cap=cap, n_seg=C.pointer(n_seg), state=_dp(state), tan_theta=_dp(tt),
               alpha=_dp(al), sum_xi=_dp(sx))
    ns = C.c_int64(0); lw = C.c_double(0.0); st = C.c_uint8(0)
    rc = lib().oracle_run_segments(C.byref(ms), C.byref(tab), C.byref(b), seed, run_id, traj,
                                   C.byref(ns), C.byref(lw), C.byref(st), C.byref(seg))
    if rc != 0:
        raise ValueError("oracle_run_segments rejected its arguments")
    k = n_seg.value
    return dict(nsteps=ns.value, logw=lw.value, status=st.value, state=state[:k],
                tan_theta=tt[:k], alpha=al[:k], sum_xi=sx[:k])


def mlp_forward_c(mlp: MLPBias, s):
    o = (C.c_double * 2)()
    sv = (C.c_double * 3)(*[float(v) for v in s])
    b = mlp.struct()
    lib().oracle_mlp_forward(C.byref(b), sv, o)
    return np.array(o[:])


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def run2(m, resolved, table2, seed: int, run_id: int, n: int, traj0: int = 0, A: float = 0.0,
         A2: float = 0.0, mlp: MLPBias | None = None, threads: int = 0) -> Trajectories:
    """FP64 trajectories with full-rank 2-D noise (NoiseTable2); the bias is
    B = S beta with beta = (A, A2), or the clamped MLP outputs."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (table2.Spp, table2.Spq, table2.Sqq)]
    tab = _Table2(n_points=len(arrs[0]), phi_lo=table2.phi_lo, h=table2.h, Spp=_dp(arrs[0]),
                  Spq=_dp(arrs[1]), Sqq=_dp(arrs[2]))
    ms = model_struct(m, resolved.phi_in, resolved.pi_in, resolved.phi_end)
    b = mlp.struct() if mlp is not None else bias_struct(A if (A != 0.0 or A2 != 0.0) else 0.0)
    if mlp is None and A == 0.0 and A2 != 0.0:
        b.kind = 1
    out = dict(nsteps=np.zeros(n, np.int64), logw=np.zeros(n), status=np.zeros(n, np.uint8),
               phi_final=np.zeros(n), pi_final=np.zeros(n), xmin_pre=np.zeros(n))
    o = _Out(nsteps=out["nsteps"].ctypes.data_as(C.POINTER(C.c_int64)),
             logw=_dp(out["logw"]), status=out["status"].ctypes.data_as(C.POINTER(C.c_uint8)),
             phi_final=_dp(out["phi_final"]), pi_final=_dp(out["pi_final"]),
             xmin_pre=_dp(out["xmin_pre"]))
    rc = lib().oracle_run2(C.byref(ms), C.byref(tab), C.byref(b), float(A2), seed, run_id, traj0, n,
                           threads, C.byref(o))
    if rc != 0:
        raise ValueError("oracle_run2 rejected its arguments")
    return Trajectories(dN=m.dN, **out)


def run2_segments(m, resolved, table2, mlp: MLPBias, seed: int, run_id: int, traj: int, cap: int = 1 << 16):
    """One learned-bias 2-D trajectory with its per-segment records (state,
    beta, sums of xi_1 and xi_2)."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (table2.Spp, table2.Spq, table2.Sqq)]
    tab = _Table2(n_points=len(arrs[0]), phi_lo=table2.phi_lo, h=table2.h, Spp=_dp(arrs[0]),
                  Spq=_dp(arrs[1]), Sqq=_dp(arrs[2]))
    ms = model_struct(m, resolved.phi_in, resolved.pi_in, resolved.phi_end)
    b = mlp.struct()
    n_seg = C.c_int64(0)
    state = np.zeros((cap, 3)); beta = np.zeros((cap, 2)); sx = np.zeros((cap, 2))
    seg = _Seg2(cap=cap, n_seg=C.pointer(n_seg), state=_dp(state), beta=_dp(beta), sum_xi=_dp(sx))
    ns = C.c_int64(0); lw = C.c_double(0.0); st = C.c_uint8(0)
    rc = lib().oracle_run2_segments(C.byref(ms), C.byref(tab), C.byref(b), seed, run_id, traj,
                                    C.byref(ns), C.byref(lw), C.byref(st), C.byref(seg))
    if rc != 0:
        raise ValueError("oracle_run2_segments rejected its arguments")
    k = n_seg.value
    return dict(nsteps=ns.value, logw=lw.value, status=st.value, state=state[:k], beta=beta[:k],
                sum_xi=sx[:k])
