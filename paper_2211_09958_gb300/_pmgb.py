"""ctypes binding of libpmgb.so (include/pmgb.h), argument marshalling only.

Every call passes raw device pointers of torch CUDA tensors and the current
torch CUDA stream to the C ABI; all arithmetic of the method runs in the
library's kernels (and cuFFT).  There is no CPU fallback: if the shared
library is missing or fails to load, every entry point raises.
"""

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libpmgb.so")

PM_OK = 0
PM_ADJ_MU_ZERO = 1
ERRORS = {-1: "PM_EINVAL", -2: "PM_ENOMEM", -3: "PM_ECUDA", -4: "PM_ECUFFT", -5: "PM_ERANGE", -6: "PM_ESTATE"}
PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_ECUFFT, PM_ERANGE, PM_ESTATE = -1, -2, -3, -4, -5, -6

_c_double_p = ctypes.POINTER(ctypes.c_double)


class PmConfig(ctypes.Structure):
    _fields_ = [
        ("n_p", ctypes.c_int32),
        ("n_m", ctypes.c_int32),
        ("n_batch", ctypes.c_int32),
        ("n_steps", ctypes.c_int32),
        ("box", ctypes.c_double),
        ("a_init", ctypes.c_double),
        ("a_final", ctypes.c_double),
        ("h", ctypes.c_double),
        ("n_s", ctypes.c_double),
        ("omega_m", _c_double_p),
        ("sigma8", _c_double_p),
        ("solver", ctypes.c_int32),
    ]


SOLVER_SPECTRAL_GRADIENT, SOLVER_DECONVOLVE, SOLVER_LOG_A, SOLVER_TSC, SOLVER_GROWTH_EMULATOR = 1, 2, 4, 8, 16


_P = ctypes.c_void_p
_SIGNATURES = {
    "pm_create": (ctypes.c_int, [ctypes.POINTER(PmConfig), ctypes.POINTER(_P)]),
    "pm_destroy": (ctypes.c_int, [_P]),
    "pm_last_error": (ctypes.c_char_p, [_P]),
    "pm_set_stream": (ctypes.c_int, [_P, _P]),
    "pm_set_cosmology": (ctypes.c_int, [_P, _c_double_p, _c_double_p]),
    "pm_get_coefficients": (ctypes.c_int, [_P, _c_double_p, _c_double_p]),
    "pm_host_coefficients": (ctypes.c_int, [ctypes.POINTER(PmConfig), _c_double_p, _c_double_p, _c_double_p,
                                            _c_double_p]),
    "pm_init_lpt": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P, _P]),
    "pm_init_lpt_adjoint": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P, _P, _P, _c_double_p]),
    "pm_force": (ctypes.c_int, [_P, _P, _P]),
    "pm_kdk_step": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    "pm_integrate": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "pm_adjoint_integrate": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P, _c_double_p,
                                            ctypes.c_uint32]),
    "pm_density": (ctypes.c_int, [_P, _P, _P]),
    "pm_density_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "pm_mse_loss": (ctypes.c_int, [_P, _P, _P, _c_double_p, _P]),
    "pm_growth_emulate": (ctypes.c_int, [ctypes.c_double, ctypes.c_int32, _c_double_p, _c_double_p]),
    "pm_mse_loss_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _P, _P,
                                           _P, _P, _P]),
    "pm_mesh_rfft": (ctypes.c_int, [_P, _P, _P]),
    "pm_mesh_irfft": (ctypes.c_int, [_P, _P, _P]),
    "pm_power_spectrum": (ctypes.c_int, [_P, _P, _c_double_p, _c_double_p, _c_double_p]),
    "pm_launch_count": (ctypes.c_int64, [_P]),
    "pm_autotune": (ctypes.c_int, [_P, _P, _P]),
    "pm_set_tuning": (ctypes.c_int, [_P, _P]),
    "pm_get_tuning": (ctypes.c_int, [_P, _P]),
    "pm_nn_param_count": (ctypes.c_int, []),
    "pm_nn_set_params": (ctypes.c_int, [_P, _P]),
    "pm_nn_get_params": (ctypes.c_int, [_P, _P, _P]),
    "pm_nn_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "pm_nn_adam_step": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int64]),
    "pm_nn_predict": (ctypes.c_int, [_P, _P, ctypes.c_double, _P]),
    "pm_nn_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                        ctypes.c_int,
                                        _c_double_p]),
    "pm_use_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "pm_checkpoint_floats": (ctypes.c_int64, [_P, ctypes.c_int32]),
    "pm_set_checkpoints": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "pm_inject_wait_timeout": (ctypes.c_int, [_P, ctypes.c_int]),
    "pm_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "pm_profile_kinds": (ctypes.c_int, [_P]),
    "pm_profile_name": (ctypes.c_char_p, [_P, ctypes.c_int]),
    "pm_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), _c_double_p, ctypes.c_int]),
}

_lib = None


def library_path():
    return _LIB_PATH


def load():
    """Load libpmgb.so once; raises RuntimeError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libpmgb.so not built ({_LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(_c_double_p)


def make_config(n_p, n_m, box, omega_m, sigma8, n_steps, a_init=1.0 / 64, a_final=1.0, h=0.7, n_s=0.96, solver=0):
    om = np.ascontiguousarray(np.atleast_1d(omega_m), dtype=np.float64)
    s8 = np.ascontiguousarray(np.atleast_1d(sigma8), dtype=np.float64)
    if om.shape != s8.shape:
        raise ValueError("omega_m and sigma8 need the same length")
    cfg = PmConfig(n_p, n_m, len(om), n_steps, box, a_init, a_final, h, n_s, _dptr(om), _dptr(s8), int(solver))
    cfg._keep = (om, s8)
    return cfg


def host_coefficients(cfg):
    """Host-only FP64 tables of the library (no GPU needed)."""
    lib = load()
    b, n = cfg.n_batch, cfg.n_steps
    kdk = np.zeros((b, n, 3))
    dkdk = np.zeros((b, n, 3))
    lpt = np.zeros((b, 4))
    amp = np.zeros((b, 2))
    rc = lib.pm_host_coefficients(ctypes.byref(cfg), _dptr(kdk), _dptr(dkdk), _dptr(lpt), _dptr(amp))
    if rc != PM_OK:
        raise RuntimeError(f"pm_host_coefficients: {ERRORS.get(rc, rc)}: {lib.pm_last_error(None).decode()}")
    return kdk, dkdk, lpt, amp
