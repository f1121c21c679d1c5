"""Binding of the serving part of the C ABI (amy_server_create / amy_submit /
amy_poll / amy_wait / amy_cancel): argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi


def _pkg():
    from . import _check, _Keep, _problem_structs, _spec_struct, PRECS, VSTORES
    return _check, _Keep, _problem_structs, _spec_struct, PRECS, VSTORES


class AmyServer:
    def __init__(self, ptr: int):
        self.ptr = C.c_void_p(ptr)
        self._keep = {}

    def close(self):
        if self.ptr and self.ptr.value:
            _abi.load().amy_server_destroy(self.ptr)
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


def amy_server_create(device_mem_budget: int = 0, max_slots: int = 0, max_queue: int = 0,
                      batched: bool = True, use_graphs: bool = True, device: int = 0) -> AmyServer:
    _check = _pkg()[0]
    o = _abi.amy_server_opts()
    o.device_mem_budget, o.max_slots, o.max_queue = int(device_mem_budget), int(max_slots), int(max_queue)
    o.batched, o.use_graphs, o.device = int(bool(batched)), int(bool(use_graphs)), int(device)
    out = C.c_void_p(0)
    _check(_abi.load().amy_server_create(C.byref(o), C.byref(out)))
    return AmyServer(out.value)


def amy_submit(srv: AmyServer, workload) -> int:
    """Queue one request (a workloads.Workload-like object); returns its ticket."""
    _check, _Keep, _problem_structs, _spec_struct, PRECS, VSTORES = _pkg()
    k = _Keep()
    p = workload.problem
    sysd, states, inputs, sigma, cut = _problem_structs(k, p)
    r = _abi.amy_request()
    r.sys, r.states, r.inputs, r.sigma, r.cut = sysd, states, inputs, sigma, cut
    r.prec = PRECS[workload.precision]
    r.v_store = VSTORES[workload.v_store]
    r.spec = _spec_struct(k, workload.spec)
    r.horizon = int(workload.horizon)
    t = C.c_uint64(0)
    _check(_abi.load().amy_submit(srv.ptr, C.byref(r), C.byref(t)))
    return int(t.value)


def _take(res: _abi.amy_result) -> dict:
    n = int(res.n_states)
    out = {"status": int(res.status), "n_states": n, "submit_us": float(res.submit_us),
           "admit_us": float(res.admit_us), "finish_us": float(res.finish_us)}
    if res.V:
        out["V"] = np.ctypeslib.as_array(res.V, shape=(n,)).copy()
    if res.policy:
        out["policy"] = np.ctypeslib.as_array(res.policy, shape=(n,)).copy()
    _abi.load().amy_result_free(C.byref(res))
    return out


def amy_poll(srv: AmyServer, ticket: int):
    """Result dict, or None while not ready (AMY_E_NOT_READY)."""
    _check = _pkg()[0]
    res = _abi.amy_result()
    st = _abi.load().amy_poll(srv.ptr, C.c_uint64(ticket), C.byref(res))
    if st == 4:
        return None
    _check(st)
    return _take(res)


def amy_wait(srv: AmyServer, ticket: int, timeout_us: int = -1):
    _check = _pkg()[0]
    res = _abi.amy_result()
    st = _abi.load().amy_wait(srv.ptr, C.c_uint64(ticket), C.c_int64(timeout_us), C.byref(res))
    _check(st)
    return _take(res)


def amy_cancel(srv: AmyServer, ticket: int) -> None:
    _pkg()[0](_abi.load().amy_cancel(srv.ptr, C.c_uint64(ticket)))


def amy_server_stats(srv: AmyServer) -> dict:
    c, t, l = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    r = C.c_int32(0)
    _pkg()[0](_abi.load().amy_server_stats(srv.ptr, C.byref(c), C.byref(t), C.byref(l), C.byref(r)))
    return {"completed": c.value, "ticks": t.value, "launches": l.value, "resident": r.value}


def amy_server_graph_stats(srv: AmyServer) -> dict:
    """Tick graphs captured and replayed (servers created with use_graphs)."""
    c, r = C.c_int64(0), C.c_int64(0)
    _pkg()[0](_abi.load().amy_server_graph_stats(srv.ptr, C.byref(c), C.byref(r)))
    return {"captures": c.value, "replays": r.value}


def amy_result_free(res) -> None:
    _abi.load().amy_result_free(C.byref(res))


def amy_server_destroy(srv: AmyServer) -> None:
    srv.close()
