"""FP64 CPU oracle for the AMYTISS abstraction + Bellman backup (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product path (paper_2005_06191_gb300)
never imports it, and it never imports the product path.

The arithmetic lives in amy_oracle.c (plain C, FP64, OpenMP over states); this
module only marshals arguments.  build_oracle() compiles it with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amy_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "amy_oracle_expr.c")]
_LIB = os.path.join(_HERE, "liboracle.so")

_SYS = {"affine": 0, "unicycle": 1, "expr": 2}
_SPEC = {"safety": 0, "reach": 1, "reach_avoid": 2}


def build_oracle(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max([os.path.getmtime(f) for f in _SRCS]
                                              + [os.path.getmtime(os.path.join(_HERE, "amy_oracle.h"))])):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
    subprocess.check_call(cmd, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("m", C.c_int32),
        ("x_lb", C.POINTER(C.c_double)), ("x_eta", C.POINTER(C.c_double)),
        ("x_count", C.POINTER(C.c_int32)), ("x_periodic", C.POINTER(C.c_uint8)),
        ("u_lb", C.POINTER(C.c_double)), ("u_eta", C.POINTER(C.c_double)),
        ("u_count", C.POINTER(C.c_int32)),
        ("sys_kind", C.c_int32), ("params", C.POINTER(C.c_double)), ("n_params", C.c_int64),
        ("sigma", C.POINTER(C.c_double)),
        ("gamma", C.c_double), ("window", C.POINTER(C.c_int32)),
        ("p", C.c_int32), ("w_lb", C.POINTER(C.c_double)), ("w_eta", C.POINTER(C.c_double)),
        ("w_count", C.POINTER(C.c_int32)),
        ("noise", C.c_int32), ("noise_p0", C.POINTER(C.c_double)), ("noise_p1", C.POINTER(C.c_double)),
        ("noise_p2", C.POINTER(C.c_double)), ("noise_p3", C.POINTER(C.c_double)),
        ("expr", C.c_void_p),
        ("noise_cdf", C.POINTER(C.c_double)),
    ]


_NOISE = {"gaussian": 0, "uniform": 1, "exponential": 2, "beta": 3, "mult_gaussian": 4, "user": 5}
USER_KNOTS = 1024


class _Spec(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("safe_lb", C.POINTER(C.c_double)), ("safe_ub", C.POINTER(C.c_double)),
        ("n_target", C.c_int32),
        ("target_lb", C.POINTER(C.c_double)), ("target_ub", C.POINTER(C.c_double)),
        ("n_avoid", C.c_int32),
        ("avoid_lb", C.POINTER(C.c_double)), ("avoid_ub", C.POINTER(C.c_double)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = C.CDLL(_LIB)
        P, S = C.POINTER(_Problem), C.POINTER(_Spec)
        lib.orc_grid_count.restype = C.c_int64
        lib.orc_grid_count.argtypes = [C.c_double, C.c_double, C.c_double]
        lib.orc_window_shape.argtypes = [P, C.c_void_p, C.c_void_p]
        lib.orc_mean.argtypes = [P, C.c_int64, C.c_int64, C.c_void_p]
        lib.orc_row.argtypes = [P, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
        lib.orc_spec_mask.argtypes = [P, S, C.c_void_p]
        lib.orc_backup_states.argtypes = [P, S, C.c_void_p, C.c_void_p, C.c_int64,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        lib.orc_action_values.argtypes = [P, C.c_void_p, C.c_int64, C.c_void_p]
        lib.orc_synthesize.argtypes = [P, S, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int]
        lib.orc_expr_compile.restype = C.c_void_p
        lib.orc_expr_compile.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_char_p, C.c_int]
        lib.orc_expr_free.argtypes = [C.c_void_p]
        lib.orc_expr_eval.restype = C.c_double
        lib.orc_expr_eval.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_expr_compile_pdf.restype = C.c_void_p
        lib.orc_expr_compile_pdf.argtypes = [C.c_void_p, C.c_int, C.c_char_p, C.c_int]
        lib.orc_gauss_legendre8.restype = C.c_double
        lib.orc_gauss_legendre8.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
        lib.orc_user_table.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p]
        lib.orc_user_cdf.restype = C.c_double
        lib.orc_user_cdf.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        lib.orc_philox4x64.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_simulate.argtypes = [P, S, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                     C.c_uint64, C.c_void_p]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _ExprOwner:
    def __init__(self, lib, h):
        self.lib, self.h = lib, h

    def __del__(self):
        self.lib.orc_expr_free(self.h)


class _Keep:
    """Owns the numpy buffers behind one ctypes struct."""

    def __init__(self):
        self.bufs = []

    def f64(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
        self.bufs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))

    def i32(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
        self.bufs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int32))

    def expr(self, lib, p):
        """Compiles a problem's mean expressions; freed with this object."""
        texts = [str(t).encode() for t in p.exprs]
        arr = (C.c_char_p * len(texts))(*texts)
        err = C.create_string_buffer(256)
        wc = list(getattr(p, "w_count", None) or [])
        h = lib.orc_expr_compile(arr, p.n, p.m, len(wc), int(np.asarray(p.params).size), err, 256)
        if not h:
            raise ValueError(f"expression: {err.value.decode()}")
        self.bufs.append(_ExprOwner(lib, h))
        return h

    def u8(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.uint8))
        self.bufs.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _problem(p, keep: _Keep) -> _Problem:
    s = _Problem()
    s.n, s.m = p.n, p.m
    s.x_lb, s.x_eta = keep.f64(p.x_lb), keep.f64(p.x_eta)
    s.x_count, s.x_periodic = keep.i32(p.x_count), keep.u8(p.x_periodic)
    s.u_lb, s.u_eta, s.u_count = keep.f64(p.u_lb), keep.f64(p.u_eta), keep.i32(p.u_count)
    s.sys_kind = _SYS[p.sys_kind]
    s.params = keep.f64(p.params)
    s.n_params = int(np.asarray(p.params).size)
    s.sigma = keep.f64(p.sigma)
    s.gamma = float(p.gamma)
    s.window = keep.i32(p.window) if p.window is not None else C.POINTER(C.c_int32)()
    wc = list(getattr(p, "w_count", None) or [])
    s.p = len(wc)
    if wc:
        s.w_lb, s.w_eta, s.w_count = keep.f64(p.w_lb), keep.f64(p.w_eta), keep.i32(wc)
    s.noise = _NOISE[getattr(p, "noise", "gaussian")]
    for i, arr in enumerate(list(getattr(p, "noise_params", None) or [])[:4]):
        setattr(s, f"noise_p{i}", keep.f64(arr))
    if p.sys_kind == "expr":
        s.expr = keep.expr(_load(), p)
    if getattr(p, "noise", "gaussian") == "user":
        s.noise_cdf = keep.f64(user_tables(p))
    return s


def _spec(p, sp, keep: _Keep) -> _Spec:
    n = p.n
    s = _Spec()
    s.kind = _SPEC[sp.kind]
    if sp.safe is not None:
        s.safe_lb, s.safe_ub = keep.f64(sp.safe[0]), keep.f64(sp.safe[1])
    else:
        s.safe_lb, s.safe_ub = keep.f64(np.full(n, -np.inf)), keep.f64(np.full(n, np.inf))
    s.n_target = len(sp.targets)
    s.target_lb = keep.f64(np.array([b[0] for b in sp.targets]).reshape(-1) if sp.targets else np.zeros(1))
    s.target_ub = keep.f64(np.array([b[1] for b in sp.targets]).reshape(-1) if sp.targets else np.zeros(1))
    s.n_avoid = len(sp.avoids)
    s.avoid_lb = keep.f64(np.array([b[0] for b in sp.avoids]).reshape(-1) if sp.avoids else np.zeros(1))
    s.avoid_ub = keep.f64(np.array([b[1] for b in sp.avoids]).reshape(-1) if sp.avoids else np.zeros(1))
    return s


def grid_count(lb: float, ub: float, eta: float) -> int:
    return int(_load().orc_grid_count(lb, ub, eta))


def window_shape(p):
    lib, keep = _load(), _Keep()
    W = np.zeros(p.n, np.int32)
    xs = np.zeros(p.n, np.float64)
    if lib.orc_window_shape(C.byref(_problem(p, keep)), W.ctypes.data, xs.ctypes.data) != 0:
        raise ValueError("invalid cutting window")
    return W, xs


def mean(p, x: int, u: int) -> np.ndarray:
    lib, keep = _load(), _Keep()
    mu = np.zeros(p.n, np.float64)
    if lib.orc_mean(C.byref(_problem(p, keep)), x, u, mu.ctypes.data) != 0:
        raise ValueError("bad system")
    return mu


def n_disturbances(p) -> int:
    wc = list(getattr(p, "w_count", None) or [])
    return int(np.prod(wc, dtype=np.int64)) if wc else 1


def row(p, x: int, u: int, w: int = 0):
    """(origin[n], probs[prod W]) of the transition row of (x, u[, w]), window C order."""
    lib, keep = _load(), _Keep()
    W, _ = window_shape(p)
    origin = np.zeros(p.n, np.int32)
    probs = np.zeros(int(np.prod(W, dtype=np.int64)), np.float64)
    pair = int(u) * n_disturbances(p) + int(w)
    if lib.orc_row(C.byref(_problem(p, keep)), x, pair, origin.ctypes.data, probs.ctypes.data) != 0:
        raise ValueError("orc_row failed")
    return origin, probs


def spec_mask(p, sp) -> np.ndarray:
    lib, keep = _load(), _Keep()
    mask = np.zeros(p.n_states, np.uint8)
    if lib.orc_spec_mask(C.byref(_problem(p, keep)), C.byref(_spec(p, sp, keep)), mask.ctypes.data) != 0:
        raise ValueError("invalid specification")
    return mask


def backup_states(p, sp, V_next, states: Sequence[int], nthreads: int = 0):
    """One Bellman backup at the listed states: (V, pi, gap)."""
    lib, keep = _load(), _Keep()
    Vn = np.ascontiguousarray(np.asarray(V_next, dtype=np.float64))
    assert Vn.size == p.n_states
    st = np.ascontiguousarray(np.asarray(states, dtype=np.int64))
    V = np.zeros(st.size, np.float64)
    pi = np.zeros(st.size, np.uint16)
    gap = np.zeros(st.size, np.float64)
    rc = lib.orc_backup_states(C.byref(_problem(p, keep)), C.byref(_spec(p, sp, keep)),
                               Vn.ctypes.data, st.ctypes.data, st.size,
                               V.ctypes.data, pi.ctypes.data, gap.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("orc_backup_states failed")
    return V, pi, gap


def action_values(p, V_next, x: int) -> np.ndarray:
    """Every input's value at state x (no masking): the window sum s_u, or
    with a disturbance grid min over w of s_{u,w}."""
    lib, keep = _load(), _Keep()
    Vn = np.ascontiguousarray(np.asarray(V_next, dtype=np.float64))
    out = np.zeros(p.n_inputs, np.float64)
    if lib.orc_action_values(C.byref(_problem(p, keep)), Vn.ctypes.data, int(x), out.ctypes.data) != 0:
        raise ValueError("orc_action_values failed")
    return out


def synthesize(p, sp, horizon: int, want_all: bool = False, nthreads: int = 0) -> dict:
    """Full synthesis: V0, pi[horizon][n_x], gap[horizon][n_x] (+ V_all when asked)."""
    lib, keep = _load(), _Keep()
    nx = p.n_states
    V = np.zeros(nx, np.float64)
    pi = np.zeros((horizon, nx), np.uint16)
    gap = np.zeros((horizon, nx), np.float64)
    V_all = np.zeros((horizon + 1, nx), np.float64) if want_all else None
    rc = lib.orc_synthesize(C.byref(_problem(p, keep)), C.byref(_spec(p, sp, keep)), int(horizon),
                            V.ctypes.data, pi.ctypes.data if horizon else None,
                            gap.ctypes.data if horizon else None,
                            V_all.ctypes.data if want_all else None, int(nthreads))
    if rc != 0:
        raise ValueError("orc_synthesize failed")
    out = {"V": V, "pi": pi, "gap": gap}
    if want_all:
        out["V_all"] = V_all
    return out


def philox4x64(counter, key) -> np.ndarray:
    """Philox4x64-10 of one 256-bit counter (4 words) under a 128-bit key (2 words)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    assert c.size == 4 and k.size == 2
    out = np.zeros(4, np.uint64)
    lib.orc_philox4x64(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def simulate(p, sp, horizon: int, policy, x0: Sequence[int], runs: int, seed: int) -> np.ndarray:
    """Closed-loop runs of the finite MDP under policy[horizon][n_x] from each
    initial state: the number of successful runs per state (Philox4x64-10
    draws at counter (run, step, draw // 4, 0), key (seed, 0))."""
    lib, keep = _load(), _Keep()
    pol = np.ascontiguousarray(np.asarray(policy, dtype=np.uint16))
    assert pol.size == horizon * p.n_states
    xs = np.ascontiguousarray(np.asarray(x0, dtype=np.int64))
    out = np.zeros(xs.size, np.int64)
    rc = lib.orc_simulate(C.byref(_problem(p, keep)), C.byref(_spec(p, sp, keep)), int(horizon),
                          pol.ctypes.data if horizon else None, xs.ctypes.data, xs.size, int(runs),
                          C.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), out.ctypes.data)
    if rc != 0:
        raise ValueError("orc_simulate failed")
    return out


def expr_eval(exprs, n: int, m: int, p: int, params, x, u, w) -> np.ndarray:
    """Every mean component of a text system at one point (x, u, w)."""
    lib = _load()
    texts = [str(t).encode() for t in exprs]
    arr = (C.c_char_p * len(texts))(*texts)
    err = C.create_string_buffer(256)
    prm = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
    h = lib.orc_expr_compile(arr, n, m, p, prm.size, err, 256)
    if not h:
        raise ValueError(f"expression: {err.value.decode()}")
    try:
        xs = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
        us = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1)) if m else np.zeros(1)
        ws = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1)) if p else np.zeros(1)
        pp = prm if prm.size else np.zeros(1)
        return np.array([lib.orc_expr_eval(h, d, xs.ctypes.data, us.ctypes.data, ws.ctypes.data, pp.ctypes.data)
                         for d in range(n)])
    finally:
        lib.orc_expr_free(h)


def _compile_pdf(lib, texts):
    enc = [str(t).encode() for t in texts]
    arr = (C.c_char_p * len(enc))(*enc)
    err = C.create_string_buffer(256)
    h = lib.orc_expr_compile_pdf(arr, len(enc), err, 256)
    if not h:
        raise ValueError(f"density: {err.value.decode()}")
    return h


def user_tables(p) -> np.ndarray:
    """The CDF tables of a problem's user densities (one block per dim)."""
    lib = _load()
    texts = list(p.noise_pdf or [])
    if len(texts) != p.n:
        raise ValueError(f"user noise needs {p.n} densities")
    lo, hi = p.noise_params[0], p.noise_params[1]
    h = _compile_pdf(lib, texts)
    try:
        out = np.zeros((p.n, 2 * (USER_KNOTS + 1)), np.float64)
        for d in range(p.n):
            if lib.orc_user_table(h, d, float(lo[d]), float(hi[d]), out[d].ctypes.data) != 0:
                raise ValueError(f"density {d}: not a density on [{lo[d]}, {hi[d]}]")
        return out.reshape(-1)
    finally:
        lib.orc_expr_free(h)


def gauss_legendre8(text: str, a: float, b: float) -> float:
    """The oracle's 8-point Gauss-Legendre integral of a density text over [a, b]."""
    lib = _load()
    h = _compile_pdf(lib, [text])
    try:
        return lib.orc_gauss_legendre8(h, 0, float(a), float(b))
    finally:
        lib.orc_expr_free(h)


def user_cdf(text: str, lo: float, hi: float, ts) -> np.ndarray:
    """The oracle's interpolated CDF of one user density at the points ts."""
    lib = _load()
    h = _compile_pdf(lib, [text])
    try:
        table = np.zeros(2 * (USER_KNOTS + 1), np.float64)
        if lib.orc_user_table(h, 0, float(lo), float(hi), table.ctypes.data) != 0:
            raise ValueError("not a density")
        return np.array([lib.orc_user_cdf(table.ctypes.data, float(lo), float(hi), float(t)) for t in ts])
    finally:
        lib.orc_expr_free(h)
