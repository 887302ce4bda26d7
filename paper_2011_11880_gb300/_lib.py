"""ctypes declarations of the C ABI in include/pf.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpf.so")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
P = ctypes.POINTER

PF_OK = 0
PF_REDUCED = 0
PF_EXTENDED = 1
PF_STAGE_PHASOR = 1
PF_STAGE_FUSED = 2
ERRORS = {1: "PF_ERR_INVALID", 2: "PF_ERR_OOM", 3: "PF_ERR_CUDA", 4: "PF_ERR_TIMEOUT",
          5: "PF_ERR_UNSUPPORTED", 6: "PF_ERR_DEVICE"}


class PfSystem(ctypes.Structure):
    _fields_ = [
        ("n_bus", c_int32), ("n_branch", c_int32),
        ("br_from", P(c_int32)), ("br_to", P(c_int32)),
        ("br_r", P(c_double)), ("br_x", P(c_double)), ("br_b", P(c_double)),
        ("br_tap", P(c_double)), ("br_shift", P(c_double)),
        ("br_g_fr", P(c_double)), ("br_g_to", P(c_double)),
        ("br_status", P(ctypes.c_uint8)),
        ("n_load", c_int32), ("load_bus", P(c_int32)), ("load_p", P(c_double)), ("load_q", P(c_double)),
        ("n_pv", c_int32), ("pv_bus", P(c_int32)), ("pv_p", P(c_double)), ("pv_vset", P(c_double)),
        ("slack_bus", c_int32), ("slack_vset", c_double), ("slack_theta", c_double),
        ("n_shunt", c_int32), ("sh_bus", P(c_int32)), ("sh_g", P(c_double)), ("sh_b", P(c_double)),
    ]


class PfInstance(ctypes.Structure):
    _fields_ = [("grid", c_int32), ("outage", c_int32)]


class PfDims(ctypes.Structure):
    _fields_ = [
        ("formulation", c_int32), ("n_grids", c_int32), ("n_instances", c_int32), ("max_degree", c_int32),
        ("n_bus", c_int64), ("n_branch", c_int64), ("n_inc", c_int64), ("n_x", c_int64),
        ("n_f", c_int64), ("nnz", c_int64), ("n_bus_inst", c_int64), ("n_branch_inst", c_int64),
        ("n_gen_inst", c_int64),
    ]


class PfOverrides(ctypes.Structure):
    _fields_ = [("p_inj", c_void_p), ("q_inj", c_void_p), ("status", c_void_p),
                ("br_r", c_void_p), ("br_x", c_void_p), ("br_b", c_void_p), ("br_tap", c_void_p),
                ("gen_mode", c_void_p), ("gen_qlim", c_void_p)]


class PfGrads(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("p_inj", c_void_p), ("q_inj", c_void_p), ("br_r", c_void_p),
                ("br_x", c_void_p), ("br_b", c_void_p), ("br_tap", c_void_p)]


class PfTuning(ctypes.Structure):
    _fields_ = [("tile_inc", c_int32), ("ctas_per_sm", c_int32), ("split_rounds", c_int32),
                ("fuse_phasor", c_int32)]


class PfNewtonInfo(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("converged", c_int32), ("max_mismatch", ctypes.c_double),
                ("eval_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("update_ms", ctypes.c_double)]


# name -> (restype, argtypes); every symbol include/pf.h declares

SIGNATURES = {
    "pf_build": (c_int32, [P(PfSystem), c_int32, c_void_p, P(c_void_p)]),
    "pf_build_batch": (c_int32, [P(PfSystem), c_int32, P(PfInstance), c_int32, c_int32, c_void_p, P(c_void_p)]),
    "pf_destroy": (None, [c_void_p]),
    "pf_get_dims": (c_int32, [c_void_p, P(PfDims)]),
    "pf_offsets": (c_int32, [c_void_p, P(c_int64), P(c_int64), P(c_int64)]),
    "pf_pattern": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_int32)]),
    "pf_grid_sizes": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_int32), P(c_int32)]),
    "pf_incidence": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_int32), P(c_int32)]),
    "pf_contributions": (c_int32, [c_void_p, c_int32, P(c_int64), P(c_int32)]),
    "pf_residual": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_jacobian": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_residual_jacobian": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_eval": (c_int32, [c_void_p, c_void_p, P(PfOverrides), c_void_p, c_void_p, c_void_p]),
    "pf_eval_stage": (c_int32, [c_void_p, c_int32, c_void_p, P(PfOverrides), c_void_p, c_void_p, c_void_p]),
    "pf_residual_jacobian_static": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_residual_jacobian_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_vjp": (c_int32, [c_void_p, c_void_p, P(PfOverrides), c_void_p, c_int32, P(PfGrads), c_void_p]),
    "pf_newton": (c_int32, [c_void_p, c_void_p, ctypes.c_double, c_int32, c_void_p, P(PfNewtonInfo)]),
    "pf_newton_qlim": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_double,
                                 c_int32, c_int32, c_void_p, P(PfNewtonInfo), P(c_int32)]),
    "pf_set_newton_solver": (c_int32, [c_void_p, c_int32]),
    "pf_fdlf": (c_int32, [c_void_p, c_void_p, ctypes.c_double, c_int32, c_void_p, P(PfNewtonInfo)]),
    "pf_mismatch_norm": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_newton_update": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_get_tuning": (c_int32, [c_void_p, P(PfTuning)]),
    "pf_set_tuning": (c_int32, [c_void_p, P(PfTuning), c_void_p]),
    "pf_autotune": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, P(PfTuning)]),
    "pf_autotune_cache": (c_int32, [c_void_p, ctypes.c_char_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    P(PfTuning), P(c_int32)]),
    "pf_sincos": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "pf_voltage_records": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pf_fp64_peak": (c_int32, [c_int32, P(ctypes.c_double), P(ctypes.c_double), c_void_p]),
    "pf_error_string": (ctypes.c_char_p, [c_int32]),
    "pf_last_error": (ctypes.c_char_p, []),
    "pf_check_device": (c_int32, [c_void_p, c_void_p]),
}

_lib = None


class PFError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {message}")
        self.code = code


def load() -> ctypes.CDLL:
    """Loads the in-tree libpf.so.  Raises if it has not been built: there is
    no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not found: build it first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str) -> None:
    if code != PF_OK:
        msg = load().pf_last_error()
        raise PFError(code, where, msg.decode() if msg else "")
