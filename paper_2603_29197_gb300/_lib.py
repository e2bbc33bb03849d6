"""ctypes view of the C ABI in include/qoco_gpu.h (argument marshalling only).

Every numerical step runs inside libqoco_gpu.so; this module only loads it and
declares its signatures.  Loading fails loudly when the library has not been
built — there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqoco_gpu.so")

# status codes
SOLVED, SOLVED_INACCURATE, MAX_ITER = 0, 1, 2
ERR_INVALID_DIMS, ERR_INVALID_CSC, ERR_INVALID_CONE, ERR_NONFINITE_DATA = -1, -2, -3, -4
ERR_NUMERICAL, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_NO_FACTOR = -5, -6, -7, -8, -9
ERR_INVALID_ARG, ERR_NOT_IMPLEMENTED, ERR_TOO_LARGE = -10, -11, -12
STATUS_NAMES = {
    0: "solved", 1: "solved_inaccurate", 2: "max_iter", -1: "invalid_dims", -2: "invalid_csc",
    -3: "invalid_cone", -4: "nonfinite_data", -5: "numerical", -6: "oom", -7: "cuda",
    -8: "device_timeout", -9: "no_factor", -10: "invalid_arg", -11: "not_implemented",
    -12: "too_large",
}
ORDER_AUTO, ORDER_AMD, ORDER_ND, ORDER_NATURAL = 0, 1, 2, 3


class CSC(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_cols", C.c_int), ("nnz", C.c_int),
                ("colptr", C.POINTER(C.c_int)), ("rowidx", C.POINTER(C.c_int)),
                ("val", C.POINTER(C.c_double))]


class Settings(C.Structure):
    _fields_ = [("abstol", C.c_double), ("reltol", C.c_double),
                ("abstol_inacc", C.c_double), ("reltol_inacc", C.c_double),
                ("max_iter", C.c_int), ("static_reg", C.c_double),
                ("dyn_reg_thresh", C.c_double), ("dyn_reg_value", C.c_double),
                ("max_refine", C.c_int), ("refine_tol", C.c_double),
                ("step_fraction", C.c_double), ("ordering", C.c_int), ("nd_leaf", C.c_int),
                ("wait_polls", C.c_int64), ("verbose", C.c_int), ("mixed_precision", C.c_int),
                ("mixed_reg", C.c_double),
                ("batch_schedule", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int),
                ("pobj", C.c_double), ("dobj", C.c_double), ("gap", C.c_double),
                ("pres", C.c_double), ("dres", C.c_double),
                ("setup_time_s", C.c_double), ("analysis_time_s", C.c_double),
                ("solve_time_s", C.c_double),
                ("kkt_dim", C.c_int64), ("kkt_nnz", C.c_int64), ("l_nnz", C.c_int64),
                ("front_entries", C.c_int64), ("factor_flops", C.c_double),
                ("n_supernodes", C.c_int), ("n_levels", C.c_int), ("max_front", C.c_int),
                ("ordering_used", C.c_int), ("refine_steps", C.c_int),
                ("last_backward_error", C.c_double), ("kernel_launches", C.c_int64),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
                ("large_fronts", C.c_int), ("fp32_factors", C.c_int), ("fp64_escalations", C.c_int),
                ("batch_schedule_used", C.c_int), ("krylov_steps", C.c_int),
                ("batch_warps", C.c_int), ("batch_thread_fronts", C.c_int),
                ("batch_warps_per_sm", C.c_int), ("fp32_floor_raises", C.c_int),
                ("message", C.c_char * 160)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "message"}
        d["message"] = self.message.decode(errors="replace")
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


PHASES = ("factor", "solve", "cone", "row")


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 4), ("calls", C.c_int64 * 4), ("launches", C.c_int64 * 4)]

    def as_dict(self):
        return {ph: dict(ms=self.ms[i], calls=self.calls[i], launches=self.launches[i])
                for i, ph in enumerate(PHASES)}


# every exported symbol with (restype, argtypes); tests check this list against the header
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)
SIGNATURES = {
    "qoco_gpu_default_settings": (None, [C.POINTER(Settings)]),
    "qoco_gpu_setup": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, C.c_int, C.POINTER(CSC), _DP,
                                 C.POINTER(CSC), _DP, C.POINTER(CSC), _DP, C.c_int, C.c_int, _IP,
                                 C.POINTER(Settings)]),
    "qoco_gpu_solve": (C.c_int, [_VP, _VP]),
    "qoco_gpu_get_solution": (C.c_int, [_VP, _DP, _DP, _DP, _DP, C.POINTER(Info)]),
    "qoco_gpu_solution_device": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP),
                                           C.POINTER(_VP)]),
    "qoco_gpu_get_info": (C.c_int, [_VP, C.POINTER(Info)]),
    "qoco_gpu_backward": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "qoco_gpu_copy_solution": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "qoco_gpu_setup_batch": (C.c_int, [C.POINTER(_VP), C.c_int, _IP, _IP, _IP, C.POINTER(CSC), C.POINTER(_DP),
                                       C.POINTER(CSC), C.POINTER(_DP), C.POINTER(CSC), C.POINTER(_DP), _IP, _IP,
                                       C.POINTER(_IP), C.POINTER(Settings)]),
    "qoco_gpu_batch_size": (C.c_int, [_VP]),
    "qoco_gpu_batch_offsets": (C.c_int, [_VP, _IP, _IP, _IP, _IP, _IP]),
    "qoco_gpu_batch_info": (C.c_int, [_VP, _IP, _IP, _DP, _DP, _DP]),
    "qoco_gpu_backward_info": (C.c_int, [_VP, _IP, _DP, _IP]),
    "qoco_gpu_update_data": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_int, _VP]),
    "qoco_gpu_cleanup": (C.c_int, [_VP]),
    "qoco_gpu_set_profiling": (C.c_int, [_VP, C.c_int]),
    "qoco_gpu_get_profile": (C.c_int, [_VP, C.POINTER(Profile)]),
    "qoco_gpu_kkt_factor_at": (C.c_int, [_VP, _VP, _VP, _VP]),
    "qoco_gpu_kkt_solve": (C.c_int, [_VP, _VP, _VP, _IP, _DP, _VP]),
    "qoco_gpu_get_kkt": (C.c_int, [_VP, C.POINTER(C.c_int64), _IP, _DP]),
    "qoco_gpu_get_factor_dense": (C.c_int, [_VP, _IP, _DP, _DP]),
    "qoco_gpu_get_pivot_reciprocals": (C.c_int, [_VP, _DP]),
    "qoco_gpu_selftest_wait_timeout": (C.c_int, [C.c_longlong, _VP]),
    "qoco_gpu_fp64_peaks": (C.c_int, [_DP, _DP, _VP]),
    "qoco_gpu_cones_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, _IP]),
    "qoco_gpu_cones_destroy": (C.c_int, [_VP]),
    "qoco_gpu_cone_nt_scaling": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "qoco_gpu_cone_product": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "qoco_gpu_cone_division": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "qoco_gpu_cone_max_step_scratch_bytes": (C.c_size_t, [_VP]),
    "qoco_gpu_cone_max_step": (C.c_int, [_VP, _VP, _VP, C.c_double, _VP, _VP, _VP]),
    "qoco_gpu_cone_max_step_noalloc": (C.c_int, [_VP, _VP, _VP, C.c_double, _VP, _VP]),
    "qoco_gpu_analyze": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(CSC), C.POINTER(CSC),
                                   C.POINTER(CSC), C.c_int, C.c_int, _IP, C.POINTER(Settings),
                                   C.POINTER(Info), _IP, _IP, _IP, _IP]),
    "qoco_gpu_analyze_batch": (C.c_int, [C.c_int, _IP, _IP, _IP, C.POINTER(CSC), C.POINTER(CSC),
                                         C.POINTER(CSC), _IP, _IP, C.POINTER(_IP), C.POINTER(Settings),
                                         C.POINTER(Info), _IP, _IP, _IP, _IP]),
}

_lib = None


def load(path: str | None = None):
    """Load libqoco_gpu.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built; run paper_2603_29197_gb300.build.build() "
                           "(the solver has no CPU fallback)")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
