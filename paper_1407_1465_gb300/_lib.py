"""ctypes binding of librsagpu.so: the C ABI of include/rsa_gb300.h, same names.

Argument marshalling only.  The library must have been built (``build.build()``);
loading fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librsagpu.so")

RSA_OK = 0
RSA_ERR_ARG = -1
RSA_ERR_KEY = -2
RSA_ERR_RANGE = -3
RSA_ERR_NOMEM = -4
RSA_ERR_CUDA = -5
RSA_ERR_TIMEOUT = -6
RSA_ERR_UNSUPPORTED = -7
RSA_ERR_VERIFY = -8

RSA_EXP_PUBLIC = 0
RSA_EXP_PRIVATE_CRT = 1
RSA_EXP_PRIVATE_PLAIN = 2
RSA_TUNE_RAGGED = 3          # rsa_set_tuning / rsa_get_tuning: the ragged-batch kernels
RSA_GCD_AUTO, RSA_GCD_SCAN, RSA_GCD_TREE = 0, 1, 2   # rsa_batch_gcd_ex methods

STATUS_NAMES = {
    0: "RSA_OK", -1: "RSA_ERR_ARG", -2: "RSA_ERR_KEY", -3: "RSA_ERR_RANGE", -4: "RSA_ERR_NOMEM",
    -5: "RSA_ERR_CUDA", -6: "RSA_ERR_TIMEOUT", -7: "RSA_ERR_UNSUPPORTED", -8: "RSA_ERR_VERIFY",
}


class RsaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


class rsa_tuning(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("variant", ctypes.c_int32), ("threads_per_op", ctypes.c_int32),
                ("window_big", ctypes.c_int32), ("window_tc", ctypes.c_int32), ("tc_min_ops", ctypes.c_int32)]


class rsa_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("ops", ctypes.c_uint64), ("bytes_resident", ctypes.c_uint64)]


class rsa_server_cfg(ctypes.Structure):
    _fields_ = [("max_inflight_batches", ctypes.c_int32), ("batch_window_us", ctypes.c_int32),
                ("max_batch_ops", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_uint64)]


RSA_SERVER_MIX_SIZES = 1


class rsa_request(ctypes.Structure):
    _fields_ = [("key_id", ctypes.c_int32), ("exp_sel", ctypes.c_int32), ("count", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("msgs", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("arrive_ns", ctypes.c_uint64)]


class rsa_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("ops_completed", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("span_s", ctypes.c_double)]


# (name, restype, argtypes) for every function declared in include/rsa_gb300.h
_P = ctypes.c_void_p
_U32P = ctypes.POINTER(ctypes.c_uint32)
_I32P = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = [
    ("rsa_ctx_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t]),
    ("rsa_ctx_destroy", ctypes.c_int, [_P]),
    ("rsa_keyload", ctypes.c_int, [_P, ctypes.c_uint32, _P, _P, ctypes.c_uint32, _P, _P, _P, _I32P]),
    ("rsa_key_record", ctypes.c_int, [ctypes.c_uint32, _P, _P, ctypes.c_uint32, _P, _P, _P, _P,
                                      ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    ("rsa_tc_operand_image", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("rsa_tc_round_operand_image", ctypes.c_int, [ctypes.c_uint32, _P, _P, ctypes.c_size_t]),
    ("rsa_keyunload", ctypes.c_int, [_P, ctypes.c_int32]),
    ("rsa_key_info", ctypes.c_int, [_P, ctypes.c_int32, _U32P, _I32P, _I32P]),
    ("rsa_modexp_key", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_modexp_batch", ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, _P, _P, _P, _P, _P]),
    ("rsa_sign_key", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_mr_batch", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, ctypes.c_uint32, _P, _P, _P]),
    ("rsa_batch_gcd", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_batch_gcd_host", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_batch_gcd_plan", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P]),
    ("rsa_batch_gcd_ex", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P, _P, ctypes.c_int, _P]),
    ("rsa_batch_gcd_method", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P]),
    ("rsa_batch_gcd_tree_bytes", ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, _P]),
    ("rsa_verify_key", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_modexp_key_host", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_modexp_batch_host", ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, _P, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_crt_decrypt_noalloc", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint64, _P, _P, _P, _P]),
    ("rsa_server_start", ctypes.c_int, [_P, ctypes.POINTER(rsa_server_cfg)]),
    ("rsa_server_submit", ctypes.c_int, [_P, ctypes.POINTER(rsa_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("rsa_server_submit_many", ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, ctypes.POINTER(ctypes.c_uint32)]),
    ("rsa_server_clock", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    ("rsa_server_poll", ctypes.c_int, [_P, ctypes.c_uint64, _I32P]),
    ("rsa_server_drain", ctypes.c_int, [_P, ctypes.c_int32]),
    ("rsa_server_get_stats", ctypes.c_int, [_P, ctypes.POINTER(rsa_server_stats), ctypes.c_int32]),
    ("rsa_server_stop", ctypes.c_int, [_P]),
    ("rsa_sync", ctypes.c_int, [_P, _P]),
    ("rsa_last_error", ctypes.c_char_p, []),
    ("rsa_set_tuning", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_int32, ctypes.POINTER(rsa_tuning)]),
    ("rsa_get_tuning", ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_int32, ctypes.POINTER(rsa_tuning)]),
    ("rsa_get_stats", ctypes.c_int, [_P, ctypes.POINTER(rsa_stats)]),
    ("rsa_autotune", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_char_p,
                                    ctypes.POINTER(rsa_tuning), ctypes.POINTER(ctypes.c_double)]),
    ("rsa_autotune_batch", ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, _P, _P, _P,
                                          ctypes.POINTER(rsa_tuning), ctypes.POINTER(ctypes.c_double)]),
    ("rsa_products_per_op", ctypes.c_double, [ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_int32]),
    ("rsa_imad_probe", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
]

_lock = threading.Lock()
_lib = None


def lib(path: str = LIB_PATH):
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError("librsagpu.so is not built (expected at %s); run "
                                   "`python -m paper_1407_1465_gb300.build`" % path)
            handle = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(handle, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def last_error() -> str:
    return (lib().rsa_last_error() or b"").decode()


def check(rc: int) -> int:
    if rc != RSA_OK:
        raise RsaError(rc, last_error())
    return rc
