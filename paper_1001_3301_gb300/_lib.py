"""ctypes binding of ``librt_gb300.so`` (the C ABI in include/rt_irradiation.h).

Argument marshalling only: every step of the ray tracer runs in the library's CUDA
kernels. There is no fallback: if the library is missing or fails to load, the
import of this module raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "librt_gb300.so")

RT_OK = 0
RT_ERR_INVALID_ARG = -1
RT_ERR_NOT_CONFIGURED = -2
RT_ERR_CUDA = -3
RT_ERR_TIMEOUT = -4
RT_ERR_NONFINITE_INPUT = -5
RT_ERR_NO_MEMORY = -6

RT_KERNEL_TILE = 0
RT_KERNEL_RAY = 1
RT_KERNEL_RAY_CHUNKED = 2

RT_FP32_KAHAN = 0
RT_FP32_PLAIN = 1
RT_FP64 = 2
RT_MAX_NU = 128
RT_TABLE_NU = 0
RT_TABLE_NU_T_SEPARABLE = 1
RT_TABLE_NU_T = 2
RT_TABLE_NU_T_RANK2 = 3
RT_TABLE_NU_T_LOW_RANK = 4
RT_BATCH_MAX = 256

PRECISIONS = {"fp32_kahan": RT_FP32_KAHAN, "fp32_plain": RT_FP32_PLAIN, "fp64": RT_FP64}


class RtGridDesc(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("nphi", ctypes.c_int),
                ("r_if", ctypes.POINTER(ctypes.c_double)),
                ("theta_if", ctypes.POINTER(ctypes.c_double)),
                ("phi_if", ctypes.POINTER(ctypes.c_double)),
                ("precision", ctypes.c_int)]


class RtEnergy(ctypes.Structure):
    _fields_ = [("e_abs", ctypes.c_double), ("e_esc", ctypes.c_double),
                ("l_star", ctypes.c_double), ("rel_err", ctypes.c_double)]


RT_SUR_NPARAMS = 17793


class RtTrainCfg(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_longlong), ("batch", ctypes.c_int), ("steps", ctypes.c_int),
                ("lr", ctypes.c_float), ("seed", ctypes.c_ulonglong)]


class RtTrainStats(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_longlong), ("n_val", ctypes.c_longlong),
                ("mu", ctypes.c_double), ("sigma", ctypes.c_double), ("final_loss", ctypes.c_double),
                ("val_rms", ctypes.c_double), ("val_max", ctypes.c_double), ("train_ms", ctypes.c_double)]


class RtSurrogateStats(ctypes.Structure):
    _fields_ = [("n_dust", ctypes.c_longlong), ("n_fallback", ctypes.c_longlong),
                ("n_judged", ctypes.c_longlong), ("max_rel_err", ctypes.c_double),
                ("mean_rel_err", ctypes.c_double), ("e_abs", ctypes.c_double),
                ("e_esc", ctypes.c_double), ("rel_err", ctypes.c_double)]


class RtFldStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("passes", ctypes.c_int), ("rel_change", ctypes.c_double),
                ("levels", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "rt_create": (_I, [ctypes.POINTER(RtGridDesc), _P, ctypes.POINTER(_P)]),
    "rt_set_stream": (_I, [_P, _P]),
    "rt_set_opacity_table": (_I, [_P, _I, _DP, _DP, _D, _I]),
    "rt_set_star": (_I, [_P, _D, _D]),
    "rt_set_opacity_table_t": (_I, [_P, _I, _DP, _I, _DP, _DP, _D]),
    "rt_irradiate": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(RtEnergy)]),
    "rt_irradiate_host": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(RtEnergy)]),
    "rt_irradiate_host_async": (_I, [_P, _P, _P, _P, _P]),
    "rt_host_wait": (_I, [_P]),
    "rt_energy_last": (_I, [_P, ctypes.POINTER(RtEnergy)]),
    "rt_energy_reduce": (_I, [_P]),
    "rt_opacity_table_kind": (_I, [_P, ctypes.POINTER(_I)]),
    "rt_lut_build": (_I, [_P, ctypes.c_float]),
    "rt_irradiate_lut": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(RtEnergy), ctypes.POINTER(ctypes.c_uint)]),
    "rt_get_bins": (_I, [_P, _DP]),
    "rt_set_tuning": (_I, [_P, _I, _I, _I, _I]),
    "rt_get_tuning": (_I, [_P] + [ctypes.POINTER(_I)] * 4),
    "rt_list_tunings": (_I, [_P] + [ctypes.POINTER(_I)] * 4 + [_I]),
    "rt_autotune": (_I, [_P, _P, _P, _P, _P, _I]),
    "rt_destroy": (None, [_P]),
    "rt_last_error": (ctypes.c_char_p, [_P]),
    "rt_status_string": (ctypes.c_char_p, [_I]),
    "rt_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, ctypes.POINTER(_P)]),
    "rt_batch_run": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                          ctypes.POINTER(_P)]),
    "rt_batch_energy": (_I, [_P, ctypes.POINTER(RtEnergy)]),
    "rt_batch_autotune": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                               ctypes.POINTER(_P), _I]),
    "rt_batch_get_tuning": (_I, [_P] + [ctypes.POINTER(_I)] * 4),
    "rt_batch_set_tuning": (_I, [_P, _I, _I, _I, _I]),
    "rt_batch_last_error": (ctypes.c_char_p, [_P]),
    "rt_batch_destroy": (None, [_P]),
    "rt_irradiate_static": (_I, [ctypes.POINTER(RtGridDesc), _D, _D, _I, _DP, _DP, _D, _I,
                                 _P, _P, _P, _P, ctypes.POINTER(RtEnergy), _P]),
    "rt_probe_ex2": (_I, [_P, _P, ctypes.c_longlong, _P]),
    "rt_probe_alu_rates": (_I, [_DP, _DP, _DP]),
    "rt_planck_mean_opacity": (_I, [_P, _D, _DP]),
    "rt_dust_temperature": (_I, [_P, _P, _P, _P]),
    "rt_rosseland_mean_opacity": (_I, [_P, _D, _DP]),
    "rt_fld_step": (_I, [_P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _I, _P]),
    "rt_surrogate_train": (_I, [_P, ctypes.POINTER(RtTrainCfg), ctypes.POINTER(_P), ctypes.POINTER(_P), _I,
                                ctypes.POINTER(RtTrainStats)]),
    "rt_irradiate_surrogate": (_I, [_P, _P, _P, _P, _P, ctypes.c_float, _I, ctypes.POINTER(RtSurrogateStats)]),
    "rt_surrogate_set_params": (_I, [_P, ctypes.POINTER(ctypes.c_float), _D, _D]),
    "rt_surrogate_get_params": (_I, [_P, ctypes.POINTER(ctypes.c_float), _DP, _DP]),
    "rt_surrogate_grad": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _I,
                               ctypes.POINTER(ctypes.c_float), _DP]),
    "rt_surrogate_eval": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(ctypes.c_float)]),
    "rt_surrogate_loss_history": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    "rt_surrogate_trust_map": (_I, [_P, ctypes.c_float, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_float)]),
    "rt_surrogate_save": (_I, [_P, ctypes.c_char_p]),
    "rt_surrogate_load": (_I, [_P, ctypes.c_char_p]),
    "rt_probe_tanh": (_I, [_P, _P, ctypes.c_longlong, _I, _P]),
    "rt_probe_umma": (_I, [_P, _P, _I, _P, _P]),
    "rt_probe_tensor_rates": (_I, [_DP, _DP, _DP, _DP, _DP, _DP]),
}


class RtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


def status_string(status: int) -> str:
    return lib.rt_status_string(int(status)).decode()


def last_error(ctx) -> str:
    return lib.rt_last_error(ctx).decode()


def check(status: int, ctx=None):
    if status != RT_OK:
        raise RtError(status, last_error(ctx))
    return status
