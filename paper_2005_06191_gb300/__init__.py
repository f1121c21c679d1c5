"""GB300 engine for the data-parallel hot path of AMYTISS (arxiv 2005.06191).

Thin Python binding over the C ABI of include/amy.h: the functions below carry
the C names and only marshal arguments; every step of the path (masks, row
construction, backup, max/argmax, batching, serving) runs in libamy.so's CUDA
kernels.  Device buffers may be torch CUDA tensors (data_ptr is passed through);
otherwise numpy arrays are used and the library copies to/from the device.

Problem and spec arguments are duck-typed: any object with the attributes of
workloads.Problem / workloads.Spec (grids, system kind and parameters, sigma,
gamma or window; spec kind and boxes) can be passed.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import _abi
from ._abi import STATUS_NAMES

TMODES = {"otf": 0, "stored_full": 1, "stored_factored": 2, "stored_separable": 3, "auto": 4}
PRECS = {"fp64": 0, "fp32": 1, "fp32_kahan": 2}
SYS_KINDS = {"affine": 0, "unicycle": 1, "expr": 2}
SPEC_KINDS = {"safety": 0, "reach": 1, "reach_avoid": 2}
VSTORES = {"native": 0, "bf16": 1, "u16": 2}
NOISE_KINDS = {"gaussian": 0, "uniform": 1, "exponential": 2, "beta": 3, "mult_gaussian": 4, "user": 5}
POLICY_NONE = 0xFFFF


class AmyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _lib():
    return _abi.load()


def _check(st: int):
    if st != 0:
        msg = _lib().amy_last_error()
        raise AmyError(st, msg.decode() if msg else "")


class _Keep:
    """Keeps the numpy buffers behind ctypes structs alive for one call."""

    def __init__(self):
        self.bufs = []

    def f64(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
        self.bufs.append(a)
        return a.ctypes.data_as(_abi.DP)

    def i32(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
        self.bufs.append(a)
        return a.ctypes.data_as(_abi.IP)

    def u8(self, v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.uint8))
        self.bufs.append(a)
        return a.ctypes.data_as(_abi.U8P)

    def obj(self, o):
        self.bufs.append(o)
        return o


def _grid(k: _Keep, lb, eta, count, periodic=None) -> _abi.amy_grid:
    g = _abi.amy_grid()
    g.n = len(count)
    g.lb, g.eta, g.count = k.f64(lb), k.f64(eta), k.i32(count)
    g.periodic = k.u8(periodic) if periodic is not None else _abi.U8P()
    return g


def _problem_structs(k: _Keep, p):
    sysd = _abi.amy_system()
    sysd.kind = SYS_KINDS[p.sys_kind]
    sysd.n, sysd.m = p.n, p.m
    sysd.params = k.f64(p.params)
    sysd.n_params = int(np.asarray(p.params).size)
    wc = list(getattr(p, "w_count", None) or [])
    if wc:
        sysd.disturb = C.pointer(k.obj(_grid(k, p.w_lb, p.w_eta, wc)))
    kind = getattr(p, "noise", "gaussian")
    if kind != "gaussian":
        nz = _abi.amy_noise()
        nz.kind = NOISE_KINDS[kind]
        for i, arr in enumerate(list(getattr(p, "noise_params", None) or [])[:4]):
            setattr(nz, f"p{i}", k.f64(arr))
        if kind == "user":
            texts = k.obj([str(t).encode() for t in (getattr(p, "noise_pdf", None) or [])])
            if len(texts) != p.n:
                raise ValueError(f"user noise needs {p.n} densities, got {len(texts)}")
            arr = k.obj((C.c_char_p * len(texts))(*texts))
            nz.pdf = C.cast(arr, C.POINTER(C.c_char_p))
        sysd.noise = C.pointer(k.obj(nz))
    if p.sys_kind == "expr":
        texts = k.obj([str(t).encode() for t in (p.exprs or [])])
        if len(texts) != p.n:
            raise ValueError(f"a text system needs {p.n} expressions, got {len(texts)}")
        arr = k.obj((C.c_char_p * len(texts))(*texts))
        sysd.expr = C.cast(arr, C.POINTER(C.c_char_p))
    states = _grid(k, p.x_lb, p.x_eta, p.x_count, p.x_periodic)
    inputs = _grid(k, p.u_lb, p.u_eta, p.u_count)
    cut = _abi.amy_cut()
    cut.gamma = float(p.gamma)
    cut.window = k.i32(p.window) if p.window is not None else _abi.IP()
    sigma = k.f64(p.sigma)
    return sysd, states, inputs, sigma, cut


def _box(k: _Keep, b) -> _abi.amy_box:
    x = _abi.amy_box()
    x.lb, x.ub = k.f64(b[0]), k.f64(b[1])
    return x


def _spec_struct(k: _Keep, sp) -> _abi.amy_spec:
    s = _abi.amy_spec()
    s.kind = SPEC_KINDS[sp.kind]
    if sp.safe is not None:
        s.safe = C.pointer(k.obj(_box(k, sp.safe)))
    nt, na = len(sp.targets), len(sp.avoids)
    if nt:
        arr = k.obj((_abi.amy_box * nt)(*[_box(k, b) for b in sp.targets]))
        s.target = C.cast(arr, C.POINTER(_abi.amy_box))
    if na:
        arr = k.obj((_abi.amy_box * na)(*[_box(k, b) for b in sp.avoids]))
        s.avoid = C.cast(arr, C.POINTER(_abi.amy_box))
    s.n_target, s.n_avoid = nt, na
    return s


def _is_cuda_tensor(t) -> bool:
    return hasattr(t, "is_cuda") and bool(t.is_cuda)


def _check_device_out(t, name: str, numel: int, dtypes) -> None:
    """Checks a caller's device buffer before its pointer goes to the library:
    a torch CUDA tensor on the current device, of one of `dtypes`,
    contiguous, with exactly `numel` entries (the kernels write that many)."""
    import torch
    if not _is_cuda_tensor(t):
        raise ValueError(f"{name} must be a torch CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}; expected one of {[str(d) for d in dtypes]}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} entries; expected {numel}")


def _policy_dtypes():
    import torch
    return tuple(d for d in (torch.int16, getattr(torch, "uint16", None)) if d is not None)


def _current_stream_ptr():
    """torch's current stream; its legacy default stream (handle 0) is passed
    as cudaStreamLegacy so that the library does not create its own stream."""
    import torch
    if torch.cuda.is_available():
        s = torch.cuda.current_stream().cuda_stream
        return C.c_void_p(s if s else 1)
    return C.c_void_p(0)


class AmyHandle:
    """Owns an amy_handle (device rows, V ping-pong, masks)."""

    def __init__(self, ptr: int, prec: str, n_states: int, n_inputs: int):
        self.ptr = C.c_void_p(ptr)
        self.prec = prec
        self.n_states = n_states
        self.n_inputs = n_inputs

    @property
    def out_dtype(self):
        return np.float64 if self.prec == "fp64" else np.float32

    def close(self):
        if self.ptr and self.ptr.value:
            _lib().amy_destroy(self.ptr)
            self.ptr = C.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def amy_grid_count(lb: float, ub: float, eta: float) -> int:
    return int(_lib().amy_grid_count(lb, ub, eta))


def amy_last_error() -> str:
    m = _lib().amy_last_error()
    return m.decode() if m else ""


def amy_build(problem, tmode: str = "otf", prec: str = "fp32", v_store: str = "native",
              device_mem_budget: int = 0, stream=None, use_graphs: bool = True,
              autotune: bool = False, launch_shape=None) -> AmyHandle:
    """amy_build: validate, derive the window and (stored modes) build T on the GPU.

    `stream` is a cudaStream_t as int; None uses torch's current stream.
    `autotune` times the backup's launch shapes at build and keeps the fastest;
    `launch_shape` = (input lanes, states per block, row tiles 1 / consecutive 2,
    box floats, dim-0 values per row tile) fixes them instead (0 entries = automatic)."""
    k = _Keep()
    sysd, states, inputs, sigma, cut = _problem_structs(k, problem)
    o = _abi.amy_opts()
    o.tmode, o.prec, o.v_store = TMODES[tmode], PRECS[prec], VSTORES[v_store]
    o.device_mem_budget = int(device_mem_budget)
    o.use_graphs = int(bool(use_graphs))
    o.autotune = int(bool(autotune))
    for i, v in enumerate(launch_shape or ()):
        o.launch_shape[i] = int(v)
    o.cuda_stream = C.c_void_p(stream) if stream is not None else _current_stream_ptr()
    out = C.c_void_p(0)
    _check(_lib().amy_build(C.byref(sysd), C.byref(states), C.byref(inputs), sigma, C.byref(cut),
                            C.byref(o), C.byref(out)))
    info = _abi.amy_info_t()
    _check(_lib().amy_info(out, C.byref(info)))
    return AmyHandle(out.value, prec, int(info.n_states), int(info.n_inputs))


def amy_info(h: AmyHandle) -> dict:
    info = _abi.amy_info_t()
    _check(_lib().amy_info(h.ptr, C.byref(info)))
    n = info.n
    return {
        "n_states": int(info.n_states), "n_inputs": int(info.n_inputs), "n": n,
        "window": [int(info.window[d]) for d in range(n)],
        "window_slots": int(info.window_slots), "window_sum": int(info.window_sum),
        "cut_half_width": [float(info.cut_half_width[d]) for d in range(n)],
        "device_bytes": int(info.device_bytes), "tmode": int(info.tmode), "prec": int(info.prec),
        "v_store": int(info.v_store), "input_lanes": int(info.input_lanes), "row_tiles": int(info.row_tiles), "block_states": int(info.block_states),
        "grouped_inputs": int(info.grouped_inputs), "backup_kernel": int(info.backup_kernel),
        "input_runs": int(info.input_runs), "inner_span": int(info.inner_span),
        "build_kernels": int(info.build_kernels), "tile_outer_rows": int(info.tile_outer_rows),
        "step_wait": int(info.step_wait), "backup_launch_kernels": int(info.backup_launch_kernels),
        "n_disturbances": int(info.n_disturbances),
    }


def amy_synthesize(h: AmyHandle, spec, horizon: int, V_out=None, policy_out=None,
                   policy_all_steps: bool = False, want_policy: bool = True):
    """amy_synthesize: `horizon` backups; returns (V_0, policy).

    With torch CUDA tensors for V_out (and policy_out) the outputs stay on the
    device (work enqueued on the handle's stream).  Otherwise the outputs are
    host arrays: the given numpy arrays (e.g. views of pinned memory, which
    the device writes at full copy speed) or new ones."""
    k = _Keep()
    s = _spec_struct(k, spec)
    nx = h.n_states
    if V_out is not None and _is_cuda_tensor(V_out):
        import torch
        _check_device_out(V_out, "V_out", nx, (torch.float64,) if h.prec == "fp64" else (torch.float32,))
        if policy_out is not None and horizon > 0:
            _check_device_out(policy_out, "policy_out", nx * (horizon if policy_all_steps else 1),
                              _policy_dtypes())
        vp = C.c_void_p(V_out.data_ptr())
        pp = C.c_void_p(policy_out.data_ptr()) if policy_out is not None else C.c_void_p(0)
        _check(_lib().amy_synthesize(h.ptr, C.byref(s), int(horizon), vp, pp, int(bool(policy_all_steps)), 1))
        return V_out, policy_out
    pshape = (horizon, nx) if policy_all_steps else (nx,)
    if V_out is not None:
        V = V_out
        if not (isinstance(V, np.ndarray) and V.dtype == h.out_dtype and V.size == nx and V.flags.c_contiguous):
            raise ValueError(f"V_out must be a contiguous {np.dtype(h.out_dtype)} array of {nx} values")
    else:
        V = np.zeros(nx, dtype=h.out_dtype)
    pi = None
    if policy_out is not None and horizon > 0:
        pi = policy_out
        if not (isinstance(pi, np.ndarray) and pi.dtype in (np.uint16, np.int16) and pi.size == int(np.prod(pshape))
                and pi.flags.c_contiguous):
            raise ValueError(f"policy_out must be a contiguous 16-bit array of shape {pshape}")
    elif want_policy and horizon > 0:
        pi = np.zeros(pshape, dtype=np.uint16)
    _check(_lib().amy_synthesize(h.ptr, C.byref(s), int(horizon), C.c_void_p(V.ctypes.data),
                                 C.c_void_p(pi.ctypes.data) if pi is not None else C.c_void_p(0),
                                 int(bool(policy_all_steps)), 0))
    return V, pi


def amy_backup_step(h: AmyHandle, spec, V_next, V_out=None, policy_out=None):
    """amy_backup_step: one backup from a caller-given V_{k+1}; returns (V_k, pi_k)."""
    k = _Keep()
    s = _spec_struct(k, spec)
    if _is_cuda_tensor(V_next):
        import torch
        fdt = (torch.float64,) if h.prec == "fp64" else (torch.float32,)
        _check_device_out(V_next, "V_next", h.n_states, fdt)
        _check_device_out(V_out, "V_out", h.n_states, fdt)
        if policy_out is not None:
            _check_device_out(policy_out, "policy_out", h.n_states, _policy_dtypes())
        _check(_lib().amy_backup_step(h.ptr, C.byref(s), C.c_void_p(V_next.data_ptr()),
                                      C.c_void_p(V_out.data_ptr()),
                                      C.c_void_p(policy_out.data_ptr()) if policy_out is not None else C.c_void_p(0),
                                      1))
        return V_out, policy_out
    Vn = np.ascontiguousarray(np.asarray(V_next, dtype=h.out_dtype))
    assert Vn.size == h.n_states
    V = np.zeros(h.n_states, dtype=h.out_dtype)
    pi = np.zeros(h.n_states, dtype=np.uint16)
    _check(_lib().amy_backup_step(h.ptr, C.byref(s), C.c_void_p(Vn.ctypes.data), C.c_void_p(V.ctypes.data),
                                  C.c_void_p(pi.ctypes.data), 0))
    return V, pi


def amy_query_rows(h: AmyHandle, xs, us):
    """amy_query_rows: (origins [count, n], probs [count, prod W]) as the engine computes them."""
    info = amy_info(h)
    x = np.ascontiguousarray(np.asarray(xs, dtype=np.int64))
    u = np.ascontiguousarray(np.asarray(us, dtype=np.int64))
    assert x.shape == u.shape
    org = np.zeros((x.size, info["n"]), dtype=np.int32)
    probs = np.zeros((x.size, info["window_slots"]), dtype=np.float64)
    _check(_lib().amy_query_rows(h.ptr, C.c_void_p(x.ctypes.data), C.c_void_p(u.ctypes.data), x.size,
                                 C.c_void_p(org.ctypes.data), C.c_void_p(probs.ctypes.data)))
    return org, probs


def amy_simulate(h: AmyHandle, spec, horizon: int, policy, x0, runs_per_x0: int, seed: int, out=None):
    """amy_simulate: closed-loop runs of the finite MDP under policy[horizon][n_states]
    from each initial state; returns the successful runs per state.

    With torch CUDA tensors for policy, x0 (int64) and out (int64) everything
    stays on the device; otherwise host arrays (a new int64 array is returned
    when out is None)."""
    k = _Keep()
    s = _spec_struct(k, spec)
    nx = h.n_states
    if _is_cuda_tensor(policy) or _is_cuda_tensor(x0) or _is_cuda_tensor(out):
        import torch
        if not _is_cuda_tensor(x0):
            raise ValueError("x0 must be a torch CUDA tensor when policy or out is one")
        if horizon > 0:
            _check_device_out(policy, "policy", nx * horizon, _policy_dtypes())
        _check_device_out(x0, "x0", x0.numel(), (torch.int64,))
        _check_device_out(out, "out", x0.numel(), (torch.int64,))
        pp = C.c_void_p(policy.data_ptr()) if horizon > 0 else C.c_void_p(0)
        _check(_lib().amy_simulate(h.ptr, C.byref(s), int(horizon), pp, C.c_void_p(x0.data_ptr()), x0.numel(),
                                   int(runs_per_x0), C.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF),
                                   C.c_void_p(out.data_ptr()), 1))
        return out
    xs = np.ascontiguousarray(np.asarray(x0, dtype=np.int64)).reshape(-1)
    pol = None
    if horizon > 0:
        pol = np.ascontiguousarray(np.asarray(policy))
        if pol.dtype not in (np.uint16, np.int16) or pol.size != nx * horizon:
            raise ValueError(f"policy must be a 16-bit array of shape ({horizon}, {nx})")
    res = out if out is not None else np.zeros(xs.size, dtype=np.int64)
    if not (isinstance(res, np.ndarray) and res.dtype == np.int64 and res.size == xs.size and res.flags.c_contiguous):
        raise ValueError(f"out must be a contiguous int64 array of {xs.size} values")
    _check(_lib().amy_simulate(h.ptr, C.byref(s), int(horizon),
                               C.c_void_p(pol.ctypes.data) if pol is not None else C.c_void_p(0),
                               C.c_void_p(xs.ctypes.data), xs.size, int(runs_per_x0),
                               C.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), C.c_void_p(res.ctypes.data), 0))
    return res


def amy_export_prism(h: AmyHandle, spec, horizon: int, path_prefix: str) -> int:
    """amy_export_prism: writes <prefix>.tra/.lab/.sta/.props (PRISM explicit
    MDP files of the handle's abstraction); returns the number of transitions."""
    k = _Keep()
    s = _spec_struct(k, spec)
    n = C.c_int64(0)
    _check(_lib().amy_export_prism(h.ptr, C.byref(s), int(horizon), os.fsencode(path_prefix), C.byref(n)))
    return int(n.value)


def amy_rebuild(h: AmyHandle, params=None) -> None:
    """amy_rebuild: rebuild the stored rows in place (optionally with new system parameters)."""
    if params is None:
        _check(_lib().amy_rebuild(h.ptr, C.c_void_p(0), 0))
        return
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    _check(_lib().amy_rebuild(h.ptr, C.c_void_p(p.ctypes.data), p.size))


def amy_set_profiling(h: AmyHandle, on: bool = True) -> None:
    _check(_lib().amy_set_profiling(h.ptr, int(bool(on))))


def amy_set_wait_limit(h: AmyHandle, polls: int = -1) -> None:
    """amy_set_wait_limit: polls before a wait between backups of the
    persistent kernel gives up (AMY_E_TIMEOUT); 0 gives up at once; -1
    restores the default."""
    _check(_lib().amy_set_wait_limit(h.ptr, int(polls)))


def amy_set_step_wait(h: AmyHandle, mode: int = 0) -> None:
    """amy_set_step_wait: 0 = the persistent kernel's blocks wait only for
    their neighbour tiles between backups, 1 = for every block."""
    _check(_lib().amy_set_step_wait(h.ptr, int(mode)))


def amy_set_plane(h: AmyHandle, on: int = 1, smem_bytes: int = 0) -> None:
    """amy_set_plane: 1 = the plane kernel (banded problems with tables,
    backup kernel 7) where it applies, in its tiled form (backup kernel 8)
    for planes of at least 256 states; 2 = the tiled form wherever it
    applies; 3 = never tiled; 0 = the per-state kernel.  smem_bytes caps the
    shared memory per block (0 = default)."""
    _check(_lib().amy_set_plane(h.ptr, int(on), int(smem_bytes)))


def amy_backup_work(h: AmyHandle, spec) -> dict:
    """amy_backup_work: the plane kernel's work in one backup for this spec
    (V values read from global memory, values read from the shared-memory
    partial box, second-stage rows); runs one untimed backup."""
    k = _Keep()
    s = _spec_struct(k, spec)
    a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _check(_lib().amy_backup_work(h.ptr, C.byref(s), C.byref(a), C.byref(b), C.byref(c)))
    return {"v_loads": a.value, "box_loads": b.value, "box_rows": c.value}


def amy_measure_l2() -> float:
    """amy_measure_l2: measured L2 read bandwidth (bytes/s) of the current device."""
    v = C.c_double(0.0)
    _check(_lib().amy_measure_l2(C.byref(v)))
    return v.value


def amy_kernel_times(h: AmyHandle) -> dict:
    """Summed CUDA-event durations (ms) and counts of backup / build kernels since
    the last call; backup_steps counts the backups those launches performed."""
    bms, bn, bs, cms, cn = C.c_double(0), C.c_int64(0), C.c_int64(0), C.c_double(0), C.c_int64(0)
    _check(_lib().amy_kernel_times(h.ptr, C.byref(bms), C.byref(bn), C.byref(bs), C.byref(cms), C.byref(cn)))
    return {"backup_ms": bms.value, "backup_launches": bn.value, "backup_steps": bs.value,
            "build_ms": cms.value, "build_launches": cn.value}


def amy_destroy(h: AmyHandle) -> None:
    h.close()


def amy_measure_lane_loads() -> dict:
    """amy_measure_lane_loads: measured lane-load ceilings (per second) of
    conflict-free shared-memory loads and L1-hitting global loads on the
    current device (roofline denominators)."""
    sh, gl = C.c_double(0.0), C.c_double(0.0)
    _check(_lib().amy_measure_lane_loads(C.byref(sh), C.byref(gl)))
    return {"shared": sh.value, "global_l1": gl.value}


def amy_measure_fma() -> dict:
    """amy_measure_fma: measured FP32 and FP64 fused multiply-add rates (FMAs
    per second over the whole device; roofline denominators)."""
    f32, f64 = C.c_double(0.0), C.c_double(0.0)
    _check(_lib().amy_measure_fma(C.byref(f32), C.byref(f64)))
    return {"fp32": f32.value, "fp64": f64.value}


def amy_measure_erfc() -> dict:
    """amy_measure_erfc: measured erfcf (FP32) and erfc (FP64) evaluation
    rates (per second over the whole device; the ceiling of mass tables formed
    on the fly)."""
    f32, f64 = C.c_double(0.0), C.c_double(0.0)
    _check(_lib().amy_measure_erfc(C.byref(f32), C.byref(f64)))
    return {"fp32": f32.value, "fp64": f64.value}


def amy_synthesize_noalloc(problem, spec, horizon: int, V_out, policy_out=None, prec: str = "fp32",
                           stream=None) -> None:
    """amy_synthesize_noalloc: on-the-fly synthesis whose intermediate device
    memory is the library's fixed scratch array (no allocation).  V_out
    (float32) and policy_out (16-bit, may be None) are torch CUDA tensors of
    n_states entries; the work is enqueued on `stream` (None: torch's current
    stream)."""
    import torch
    nx = int(np.prod(problem.x_count, dtype=np.int64))
    _check_device_out(V_out, "V_out", nx, (torch.float32,))
    if policy_out is not None:
        _check_device_out(policy_out, "policy_out", nx, _policy_dtypes())
    k = _Keep()
    sysd, states, inputs, sigma, cut = _problem_structs(k, problem)
    s = _spec_struct(k, spec)
    st = C.c_void_p(stream) if stream is not None else _current_stream_ptr()
    pp = C.c_void_p(policy_out.data_ptr()) if policy_out is not None else C.c_void_p(0)
    _check(_lib().amy_synthesize_noalloc(C.byref(sysd), C.byref(states), C.byref(inputs), sigma, C.byref(cut),
                                         PRECS[prec], C.byref(s), int(horizon), C.c_void_p(V_out.data_ptr()), pp,
                                         st))


from .serving import (AmyServer, amy_cancel, amy_poll, amy_result_free,  # noqa: E402
                      amy_server_create, amy_server_destroy, amy_server_graph_stats, amy_server_stats, amy_submit,
                      amy_wait)

__all__ = [
    "AmyError", "AmyHandle", "AmyServer", "amy_build", "amy_synthesize", "amy_backup_step",
    "amy_query_rows", "amy_simulate", "amy_export_prism", "amy_info", "amy_destroy", "amy_grid_count", "amy_last_error",
    "amy_rebuild", "amy_set_profiling", "amy_set_wait_limit", "amy_set_step_wait", "amy_set_plane", "amy_backup_work", "amy_measure_l2", "amy_kernel_times", "amy_synthesize_noalloc", "amy_measure_lane_loads", "amy_measure_fma", "amy_measure_erfc",
    "amy_server_create", "amy_submit", "amy_poll", "amy_wait", "amy_cancel", "amy_server_stats",
    "amy_server_graph_stats",
    "amy_server_destroy", "amy_result_free", "TMODES", "PRECS", "VSTORES", "POLICY_NONE",
]
