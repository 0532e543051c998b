"""ctypes binding of the C ABI declared in include/fraclap.h.

Argument marshalling only: every step of the solver runs in
``libfraclap.so`` (built by ``paper_1802_03770_gb300.build``).  Loading fails
loudly if the library is missing; there is no CPU fallback.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfraclap.so")

FL_OK = 0
FL_INVALID_ARG = 1
FL_NOT_CONVERGED = 2
FL_BREAKDOWN = 3
FL_DEVICE_TIMEOUT = 4
FL_CUDA_ERROR = 5
FL_OOM = 6
STATUS_NAMES = {0: "FL_OK", 1: "FL_INVALID_ARG", 2: "FL_NOT_CONVERGED", 3: "FL_BREAKDOWN",
                4: "FL_DEVICE_TIMEOUT", 5: "FL_CUDA_ERROR", 6: "FL_OOM"}

FL_MODE_F64 = 0
FL_MODE_MIXED = 1
FL_MODE_LEARNED = 2
FL_PRECOND_FD = 0x00
FL_PRECOND_NONE = 0x10
FL_PRECOND_AUTO = 0x20
FL_PRECOND_SHIFTED = 0x30
FL_PRECOND_STENCIL = 0x40
FL_PRECOND_BOX = 0x50
FL_BATCH_PERSISTENT = 0x100


class FlOpts(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int)]


class FlSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FlPlanDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("fft_len", ctypes.c_int64 * 3),
                ("h", ctypes.c_double), ("alpha", ctypes.c_double), ("rho", ctypes.c_double),
                ("c_alpha_d", ctypes.c_double), ("lattice_zeta", ctypes.c_double),
                ("window_corr", ctypes.c_double), ("kernel0", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64)]


class FlKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int

# name -> (restype, argtypes); one entry per function of include/fraclap.h
SIGNATURES = {
    "fl_plan_create": (_I, [_I, ctypes.POINTER(ctypes.c_int64), _D, _D, _P,
                            ctypes.POINTER(FlOpts), ctypes.POINTER(_P)]),
    "fl_plan_destroy": (_I, [_P]),
    "fl_plan_describe": (_I, [_P, ctypes.POINTER(FlPlanDesc)]),
    "fl_apply": (_I, [_P, _P, _P]),
    "fl_apply_f32": (_I, [_P, _P, _P]),
    "fl_precond": (_I, [_P, _D, _D, _P, _P]),
    "fl_precond_f32": (_I, [_P, _D, _D, _P, _P]),
    "fl_precond_params": (_I, [_P, _I, _D, _D, _P, _P]),
    "fl_plan_set_tiles": (_I, [_P, _P]),
    "fl_plan_autotune": (_I, [_P, _P]),
    "fl_plan_set_row_shape": (_I, [_P, _I]),
    "fl_plan_row_shape": (_I, [_P]),
    "fl_solve_elliptic": (_I, [_P, _P, _P, _I, _D, _I, _I, ctypes.POINTER(FlSolveInfo)]),
    "fl_solve_elliptic_host": (_I, [_P, _P, _P, _D, _I, _I, ctypes.POINTER(FlSolveInfo)]),
    "fl_time_step": (_I, [_P, _D, _D, _P, _P, _P, _P, _D, _I, _I, ctypes.POINTER(FlSolveInfo)]),
    "fl_apply_f32_static": (_I, [_P, _P, _P]),
    "fl_solve_elliptic_batched": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P),
                                       ctypes.POINTER(_P), _D, _I, _I,
                                       ctypes.POINTER(FlSolveInfo)]),
    "fl_sync": (_I, [_P]),
    "fl_launch_count": (ctypes.c_longlong, []),
    "fl_check_grid_barrier": (_I, [_I]),
    "fl_profile_enable": (_I, [_P, _I]),
    "fl_profile_read": (_I, [_P, ctypes.POINTER(FlKernelStat), _I]),
    "fl_net_create": (_I, [_I, _I, ctypes.c_uint64, _P, ctypes.POINTER(_P)]),
    "fl_net_destroy": (_I, [_P]),
    "fl_net_num_params": (ctypes.c_longlong, [_P]),
    "fl_net_get_params": (_I, [_P, _P, _P]),
    "fl_net_set_params": (_I, [_P, _P]),
    "fl_net_forward": (_I, [_P, _P, _P]),
    "fl_net_loss_grad": (_I, [_P, _P, _P, _I, ctypes.POINTER(_D)]),
    "fl_net_train_step": (_I, [_P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(_D)]),
    "fl_net_save": (_I, [_P, ctypes.c_char_p]),
    "fl_net_load": (_I, [_P, ctypes.c_char_p]),
    "fl_plan_attach_net": (_I, [_P, _P]),
    "fl_net_set_tensor_cores": (_I, [_P, _I]),
    "fl_net_set_alpha_gate": (_I, [_P, ctypes.c_double, ctypes.c_double, _I, _P]),
    "fl_net_check": (_I, [_P]),
    "fl_net_training_pair": (_I, [_P, _P, _P, _P, _P, _P]),
    "fl_net_get_tensor": (_I, [_P, _I, _I, _P, ctypes.c_longlong]),
    "fl_last_error_string": (ctypes.c_char_p, []),
}

_lib = None


class FracLapError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = last_error() if _lib is not None else ""
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def load():
    """Load libfraclap.so (once) and declare its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -m paper_1802_03770_gb300.build` (there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def last_error():
    return load().fl_last_error_string().decode()


def check(status, where, allow=(FL_OK,)):
    if status not in allow:
        raise FracLapError(status, where)
    return status
