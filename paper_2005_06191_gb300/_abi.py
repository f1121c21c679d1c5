"""ctypes declarations mirroring include/amy.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamy.so")

AMY_OK = 0
STATUS_NAMES = {
    0: "AMY_OK", 1: "AMY_E_INVALID_ARG", 2: "AMY_E_OUT_OF_MEMORY", 3: "AMY_E_CUDA",
    4: "AMY_E_NOT_READY", 5: "AMY_E_TIMEOUT", 6: "AMY_E_QUEUE_FULL", 7: "AMY_E_CANCELLED",
    8: "AMY_E_UNSUPPORTED", 9: "AMY_E_NOT_FOUND",
}
MAX_DIMS = 8

DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int32)
U8P = C.POINTER(C.c_uint8)


class amy_grid(C.Structure):
    _fields_ = [("n", C.c_int32), ("lb", DP), ("eta", DP), ("count", IP), ("periodic", U8P)]


class amy_noise(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p0", DP), ("p1", DP), ("p2", DP), ("p3", DP),
                ("pdf", C.POINTER(C.c_char_p))]


class amy_system(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("params", DP),
                ("n_params", C.c_int64), ("disturb", C.POINTER(amy_grid)), ("noise", C.POINTER(amy_noise)),
                ("expr", C.POINTER(C.c_char_p))]


class amy_cut(C.Structure):
    _fields_ = [("gamma", C.c_double), ("window", IP)]


class amy_opts(C.Structure):
    _fields_ = [("tmode", C.c_int32), ("prec", C.c_int32), ("v_store", C.c_int32),
                ("device_mem_budget", C.c_int64), ("cuda_stream", C.c_void_p), ("use_graphs", C.c_int32),
                ("autotune", C.c_int32), ("launch_shape", C.c_int32 * 5)]


class amy_box(C.Structure):
    _fields_ = [("lb", DP), ("ub", DP)]


class amy_spec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("safe", C.POINTER(amy_box)), ("target", C.POINTER(amy_box)),
                ("n_target", C.c_int32), ("avoid", C.POINTER(amy_box)), ("n_avoid", C.c_int32)]


class amy_info_t(C.Structure):
    _fields_ = [("n_states", C.c_int64), ("n_inputs", C.c_int64), ("n", C.c_int32),
                ("window", C.c_int32 * MAX_DIMS), ("window_slots", C.c_int64),
                ("window_sum", C.c_int32), ("cut_half_width", C.c_double * MAX_DIMS),
                ("device_bytes", C.c_int64), ("tmode", C.c_int32), ("prec", C.c_int32),
                ("v_store", C.c_int32), ("input_lanes", C.c_int32), ("row_tiles", C.c_int32), ("block_states", C.c_int32),
                ("grouped_inputs", C.c_int32), ("backup_kernel", C.c_int32), ("input_runs", C.c_int32),
                ("inner_span", C.c_int32), ("build_kernels", C.c_int32),
                ("tile_outer_rows", C.c_int32), ("step_wait", C.c_int32),
                ("backup_launch_kernels", C.c_int32), ("n_disturbances", C.c_int32)]


class amy_server_opts(C.Structure):
    _fields_ = [("device_mem_budget", C.c_int64), ("max_slots", C.c_int32), ("max_queue", C.c_int32),
                ("batched", C.c_int32), ("use_graphs", C.c_int32), ("device", C.c_int32)]


class amy_request(C.Structure):
    _fields_ = [("sys", amy_system), ("states", amy_grid), ("inputs", amy_grid), ("sigma", DP),
                ("cut", amy_cut), ("prec", C.c_int32), ("v_store", C.c_int32), ("spec", amy_spec),
                ("horizon", C.c_int32)]


class amy_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_states", C.c_int64), ("V", C.POINTER(C.c_float)),
                ("policy", C.POINTER(C.c_uint16)), ("submit_us", C.c_double), ("admit_us", C.c_double),
                ("finish_us", C.c_double)]


# name -> (restype, argtypes)
PROTOTYPES = {
    "amy_grid_count": (C.c_int64, [C.c_double, C.c_double, C.c_double]),
    "amy_build": (C.c_int32, [C.POINTER(amy_system), C.POINTER(amy_grid), C.POINTER(amy_grid), DP,
                              C.POINTER(amy_cut), C.POINTER(amy_opts), C.POINTER(C.c_void_p)]),
    "amy_synthesize": (C.c_int32, [C.c_void_p, C.POINTER(amy_spec), C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_int32, C.c_int32]),
    "amy_backup_step": (C.c_int32, [C.c_void_p, C.POINTER(amy_spec), C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int32]),
    "amy_query_rows": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "amy_simulate": (C.c_int32, [C.c_void_p, C.POINTER(amy_spec), C.c_int32, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_int64, C.c_uint64, C.c_void_p, C.c_int32]),
    "amy_export_prism": (C.c_int32, [C.c_void_p, C.POINTER(amy_spec), C.c_int32, C.c_char_p,
                                     C.POINTER(C.c_int64)]),
    "amy_info": (C.c_int32, [C.c_void_p, C.POINTER(amy_info_t)]),
    "amy_rebuild": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64]),
    "amy_set_profiling": (C.c_int32, [C.c_void_p, C.c_int32]),
    "amy_set_wait_limit": (C.c_int32, [C.c_void_p, C.c_int32]),
    "amy_set_step_wait": (C.c_int32, [C.c_void_p, C.c_int32]),
    "amy_set_plane": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32]),
    "amy_backup_work": (C.c_int32, [C.c_void_p, C.POINTER(amy_spec), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)]),
    "amy_measure_l2": (C.c_int32, [DP]),
    "amy_kernel_times": (C.c_int32, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "amy_destroy": (None, [C.c_void_p]),
    "amy_last_error": (C.c_char_p, []),
    "amy_measure_lane_loads": (C.c_int32, [DP, DP]),
    "amy_measure_fma": (C.c_int32, [DP, DP]),
    "amy_measure_erfc": (C.c_int32, [DP, DP]),
    "amy_synthesize_noalloc": (C.c_int32, [C.POINTER(amy_system), C.POINTER(amy_grid), C.POINTER(amy_grid), DP,
                                           C.POINTER(amy_cut), C.c_int32, C.POINTER(amy_spec), C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "amy_server_create": (C.c_int32, [C.POINTER(amy_server_opts), C.POINTER(C.c_void_p)]),
    "amy_submit": (C.c_int32, [C.c_void_p, C.POINTER(amy_request), C.POINTER(C.c_uint64)]),
    "amy_poll": (C.c_int32, [C.c_void_p, C.c_uint64, C.POINTER(amy_result)]),
    "amy_wait": (C.c_int32, [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(amy_result)]),
    "amy_cancel": (C.c_int32, [C.c_void_p, C.c_uint64]),
    "amy_server_stats": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "amy_server_graph_stats": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "amy_server_destroy": (None, [C.c_void_p]),
    "amy_result_free": (None, [C.POINTER(amy_result)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libamy.so; fails loudly when the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2005_06191_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
