"""ctypes binding of ``libspinsys.so`` -- argument marshalling only.

Every function here converts Python/numpy arguments to the C types of
``include/spinsys.h`` and calls the library; all arithmetic of the step runs in the CUDA
kernels.  There is no fallback: if the library cannot be loaded, import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspinsys.so")

SS_OK = 0
STATUS = {0: "SS_OK", 1: "SS_ERR_INVALID_ARG", 2: "SS_ERR_CUDA", 3: "SS_ERR_OOM", 4: "SS_ERR_TIMEOUT",
          5: "SS_ERR_NONFINITE", 6: "SS_ERR_STATE", 7: "SS_ERR_UNSUPPORTED"}
SS_FP64, SS_FP32_MIXED = 0, 1
SS_FLAG_CHECK_SYMMETRY, SS_FLAG_INIT_RANDOM = 1, 2
SS_EXEC_AUTO, SS_EXEC_KERNELS, SS_EXEC_GRAPH, SS_EXEC_PERSISTENT, SS_EXEC_SYSTEM_BLOCKS, SS_EXEC_CLUSTER = 0, 1, 2, 3, 4, 5

# Every entry point include/spinsys.h declares.
EXPORTS = (
    "spin_system_create", "spin_batch_create", "spin_system_destroy", "spin_system_set_stream", "set_field",
    "set_temperature", "set_temperature_batch", "set_temperature_schedule", "llg_heun_step", "get_spins",
    "get_spins_device", "get_magnetisation", "get_energy", "get_record", "set_spins", "set_step", "get_step",
    "spin_system_set_exec", "spin_system_set_launch", "spin_system_autotune", "spin_system_info",
    "spin_system_set_barrier_test", "spin_system_sync", "spin_system_time_kernels", "ss_debug_philox", "ss_debug_gaussians",
    "llg_heun_step_noalloc", "spin_system_set_draw_ahead", "spin_system_set_row_patterns", "spin_system_set_gaussian_pass", "spin_system_time_passes", "ss_debug_fp64_rate", "mc_step", "get_mc_stats", "set_demag", "llg_midpoint_step",
    "spin_system_set_exchange_rows", "spin_system_time_rows", "llg_semi_implicit_step",
    "ss_debug_fail_allocations", "ss_debug_live_bytes",
    "get_demag_field",
    "spin_slab_create", "spin_slab_info", "spin_slab_halo_runs", "get_state_device", "spin_system_heun_pass",
    "ss_last_error", "ss_status_string",
)


class SpinSysError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


class SSParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("pos", ctypes.c_void_p),
        ("mu_s", ctypes.c_void_p),
        ("k_u", ctypes.c_void_p),
        ("easy_axis", ctypes.c_void_p),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
        ("J", ctypes.c_void_p),
        ("K_neel", ctypes.c_void_p),
        ("S0", ctypes.c_void_p),
        ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("H_app", ctypes.c_double * 3),
        ("T", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("sys_id", ctypes.c_uint32),
        ("precision", ctypes.c_int),
        ("flags", ctypes.c_uint32),
        ("J_tensor", ctypes.c_void_p),
        ("k_c", ctypes.c_void_p),
    ]


class SSInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("num_systems", ctypes.c_int32),
        ("num_materials", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("exec", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("num_tiles", ctypes.c_int64),
        ("step", ctypes.c_int64),
        ("record_capacity", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("draw_ahead", ctypes.c_int32),
        ("exchange_rows", ctypes.c_int32),
        ("row_patterns", ctypes.c_int32),
        ("gaussian_pass", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SSSlabInfo(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_int64),
        ("hi", ctypes.c_int64),
        ("n_halo", ctypes.c_int64),
        ("num_runs", ctypes.c_int64),
        ("boundary_tiles", ctypes.c_int64),
        ("num_tiles", ctypes.c_int64),
        ("nslabs", ctypes.c_int32),
        ("slab", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libspinsys.so (built by ``paper_1310_6143_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("SPINSYS_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libspinsys.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (CUDA path is mandatory)")
    lib = ctypes.CDLL(path)
    P, I32, I64, U32, U64, D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                ctypes.c_double)
    sigs = {
        "spin_system_create": [P, P],
        "spin_batch_create": [P, I32, P],
        "spin_system_destroy": [P],
        "spin_system_set_stream": [P, P],
        "set_field": [P, I32, P],
        "set_temperature": [P, D],
        "set_temperature_batch": [P, P, I32],
        "set_temperature_schedule": [P, P, I64, I64],
        "llg_heun_step": [P, I64],
        "mc_step": [P, I64],
        "llg_midpoint_step": [P, I64, I32],
        "llg_semi_implicit_step": [P, I64],
        "ss_debug_fail_allocations": [I64],
        "get_mc_stats": [P, I32, P],
        "set_demag": [P, D, D, I32],
        "get_demag_field": [P, P],
        "get_spins": [P, P],
        "get_spins_device": [P, P, P, P],
        "get_magnetisation": [P, I32, P],
        "get_energy": [P, I32, P],
        "get_record": [P, I64, I64, P],
        "set_spins": [P, P],
        "set_step": [P, I64],
        "get_step": [P, P],
        "spin_system_set_exec": [P, ctypes.c_int],
        "spin_system_set_launch": [P, I32, I32],
        "spin_system_set_draw_ahead": [P, I32],
        "spin_system_set_row_patterns": [P, I32],
        "spin_system_set_gaussian_pass": [P, I32],
        "spin_system_time_passes": [P, I32, P],
        "spin_system_set_exchange_rows": [P, I32],
        "spin_system_time_rows": [P, I32, P],
        "spin_system_autotune": [P, I32, P],
        "spin_system_info": [P, P],
        "spin_system_set_barrier_test": [P, I32, I64],
        "spin_system_sync": [P],
        "spin_system_time_kernels": [P, I32, P],
        "ss_debug_philox": [P, P, I64, P],
        "ss_debug_gaussians": [U64, U32, U32, I64, I32, P],
        "ss_debug_fp64_rate": [I32, P],
        "spin_slab_create": [P, I32, I32, P],
        "spin_slab_info": [P, P],
        "spin_slab_halo_runs": [P, P, I64],
        "get_state_device": [P, I32, P, P, P],
        "spin_system_heun_pass": [P, I32, I64, I64],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ss_debug_live_bytes.argtypes = []
    lib.ss_debug_live_bytes.restype = ctypes.c_int64
    lib.ss_last_error.argtypes = [P]
    lib.ss_last_error.restype = ctypes.c_char_p
    lib.ss_status_string.argtypes = [ctypes.c_int]
    lib.ss_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int, handle=None) -> None:
    if status != SS_OK:
        msg = load().ss_last_error(handle)
        raise SpinSysError(status, msg.decode() if msg else "")


def ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)
