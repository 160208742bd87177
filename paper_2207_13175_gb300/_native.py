"""ctypes loader for ``libiod_gb300.so`` (the C ABI of include/iod.h).

There is no fallback: if the CUDA library is missing or fails to load, every entry
point raises.  Build it with ``python -m paper_2207_13175_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
# IOD_CHECK=1 selects the build with the swarm kernels' argument checks compiled in
LIB_PATH = os.path.join(_PKG, "libiod_gb300_check.so" if os.environ.get("IOD_CHECK") == "1"
                        else "libiod_gb300.so")
_lock = threading.Lock()
_lib = None


class Options(C.Structure):
    _fields_ = [("integrator", C.c_int), ("dt", C.c_double), ("rtol", C.c_double),
                ("atol", C.c_double), ("h0", C.c_double), ("max_steps", C.c_longlong),
                ("precision", C.c_int), ("cost_form", C.c_int), ("gbest_order", C.c_int),
                ("vmax_frac", C.c_double), ("use_range", C.c_int), ("sigma_range", C.c_double),
                ("record_trace", C.c_int), ("block_size", C.c_int),
                ("fp64_last_iters", C.c_int), ("moon_fp64_radius", C.c_double),
                ("tol_tau", C.c_double), ("tol_window", C.c_int), ("constriction", C.c_int),
                ("init_grid", C.c_int), ("init_cone", C.c_int), ("cone_rho_min", C.c_double),
                ("cone_rho_max", C.c_double), ("cone_sigmas", C.c_double),
                ("velocity_init", C.c_int), ("per_dim_random", C.c_int),
                ("threads_per_particle", C.c_int),
                ("dynamics", C.c_int), ("ecc", C.c_double), ("f0", C.c_double),
                ("schedule", C.c_int), ("refine_iters", C.c_int),
                ("shard_offset", C.c_int), ("shard_total", C.c_int), ("refine_gate", C.c_double)]


class Result(C.Structure):
    _fields_ = [("state", C.c_double * 6), ("cost", C.c_double), ("gbest_index", C.c_int),
                ("iters_done", C.c_int), ("rk_steps", C.c_longlong), ("fp64_steps", C.c_longlong),
                ("gcost_trace", C.POINTER(C.c_double)), ("gidx_trace", C.POINTER(C.c_int)),
                ("trace_capacity", C.c_int), ("schedule", C.c_int),
                ("pso_state", C.c_double * 6), ("pso_cost", C.c_double), ("refine_iters", C.c_int),
                ("fallback", C.c_int)]


class Request(C.Structure):
    _fields_ = [("mu", C.c_double), ("chief_state", C.POINTER(C.c_double)), ("n_obs", C.c_int),
                ("obs_times", C.POINTER(C.c_double)), ("obs_angles", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)), ("bounds", C.POINTER(C.c_double)),
                ("swarm_size", C.c_int), ("iters", C.c_int), ("w", C.c_double), ("c1", C.c_double),
                ("c2", C.c_double), ("seed", C.c_uint64)]


class BatchStats(C.Structure):
    _fields_ = [("resident", C.c_int), ("queued", C.c_int), ("finished", C.c_longlong),
                ("rounds", C.c_longlong), ("bytes_in_use", C.c_size_t),
                ("bytes_high_water", C.c_size_t), ("budget", C.c_size_t),
                ("deferred_admissions", C.c_longlong)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_P = C.c_void_p

SIGNATURES = {
    "iod_options_default": (C.c_int, [C.POINTER(Options)]),
    "iod_create": (C.c_int, [C.c_double, _D, C.c_int, _D, _D, _D, _D, C.POINTER(Options),
                             C.POINTER(_P)]),
    "iod_create_ranged": (C.c_int, [C.c_double, _D, C.c_int, _D, _D, _D, _D, _D,
                                    C.POINTER(Options), C.POINTER(_P)]),
    "iod_set_stream": (C.c_int, [_P, _P]),
    "iod_set_allocator": (C.c_int, [ALLOC_FN, RELEASE_FN, _P]),
    "iod_run": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64]),
    "iod_continue": (C.c_int, [_P, C.c_int]),
    "iod_result": (C.c_int, [_P, C.POINTER(Result)]),
    "iod_swarm_get": (C.c_int, [_P, _D, _D, _D, _D, _D, _D, _D, _I, _I]),
    "iod_swarm_set": (C.c_int, [_P, C.c_int, _D, _D, _D, _D, _D, C.c_double, C.c_int, C.c_int,
                                C.c_double, C.c_double, C.c_double, C.c_uint64]),
    "iod_gbest_get": (C.c_int, [_P, _D, _D, _I, _I]),
    "iod_gbest_set": (C.c_int, [_P, _D, C.c_double, C.c_int]),
    "iod_snapshot": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "iod_restore": (C.c_int, [_P, _P, C.c_size_t]),
    "iod_destroy": (None, [_P]),
    "iod_strerror": (C.c_char_p, [C.c_int]),
    "iod_last_error": (C.c_char_p, []),
    "iod_eval": (C.c_int, [_P, _P, C.c_int, _P]),
    "iod_propagate": (C.c_int, [_P, _P, C.c_int, _P]),
    "iod_chief_positions": (C.c_int, [_P, _D]),
    "iod_refine": (C.c_int, [_P, _D, C.c_int, C.c_int, _D, _D, _I]),
    "iod_bounds_from_chief": (C.c_int, [_D, C.c_double, C.c_double, C.c_double, C.c_double, _D]),
    "iod_simulate_obs": (C.c_int, [C.c_double, _D, _D, C.c_int, _D, C.c_double, C.c_double,
                                   C.c_double, _D, _D, _D]),
    "iod_simulate_obs_er3bp": (C.c_int, [C.c_double, C.c_double, C.c_double, _D, _D, C.c_int, _D,
                                         C.c_double, C.c_double, C.c_double, _D, _D, _D]),
    "iod_selftest_wait": (C.c_int, [C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "iod_selftest_fp64_issue": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "iod_score_noalloc": (C.c_int, [C.c_double, C.c_int, _P, C.c_double, C.c_double, C.c_double,
                                    _P, C.c_int, _P, _P, _P]),
    "iod_batch_create": (C.c_int, [C.POINTER(Options), C.c_size_t, C.c_int, C.POINTER(_P)]),
    "iod_batch_set_stream": (C.c_int, [_P, _P]),
    "iod_batch_set_block_sizes": (C.c_int, [_P, C.c_int, _I, _I]),
    "iod_batch_submit": (C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_longlong)]),
    "iod_batch_step": (C.c_int, [_P, C.c_int]),
    "iod_batch_run": (C.c_int, [_P, C.c_double]),
    "iod_batch_poll": (C.c_int, [_P, C.c_longlong, C.POINTER(Result)]),
    "iod_batch_times": (C.c_int, [_P, C.c_longlong, _D, _D, _D]),
    "iod_batch_cancel": (C.c_int, [_P, C.c_longlong]),
    "iod_batch_get_stats": (C.c_int, [_P, C.POINTER(BatchStats)]),
    "iod_batch_destroy": (None, [_P]),
    "iod_batch_set_step_sizes": (C.c_int, [_P, C.c_int, _I, _D]),
    "iod_batch_autotune_dt": (C.c_int, [_P, C.c_int, _I, C.POINTER(Request), C.c_int, _D, C.c_double,
                                        C.c_int, _D, _D]),
    "iod_batch_autotune": (C.c_int, [_P, C.c_int, _I, C.POINTER(Request), C.c_int, _I, C.c_int, _I, _D]),
}


class IodError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(what)


def lib() -> C.CDLL:
    """Load the CUDA library (once).  Raises if it is missing: no CPU path exists."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing; build it with `python -m paper_2207_13175_gb300.build`"
                    + (" --check" if LIB_PATH.endswith("_check.so") else ""))
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(code: int, call: str) -> None:
    if code != 0:
        L = lib()
        detail = L.iod_last_error().decode(errors="replace")
        raise IodError(code, f"{call}: {L.iod_strerror(code).decode()} ({detail})")
