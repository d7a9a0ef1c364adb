"""ctypes binding of libaat_gb300.so (include/aat.h, include/aat_testing.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaat_gb300.so")

AAT_OK = 0
AAT_EINVAL = -1
AAT_ENOTPRIME = -2
AAT_ERANGE = -3
AAT_ENOMEM = -4
AAT_ECUDA = -5
AAT_ETIMEOUT = -6
AAT_EUNSUPPORTED = -7

AAT_IN_BALANCED = 1 << 0
AAT_ZERO_UPPER = 1 << 1
AAT_LEAF_TC = 0 << 4
AAT_LEAF_SIMT = 1 << 4
AAT_LEAF_I8 = 2 << 4
AAT_LEAF_F64 = 3 << 4
AAT_DIGITS_PLAIN = 1 << 12
AAT_WINOGRAD = 1 << 13
AAT_LOW_MEMORY = 1 << 14
AAT_C_FP32 = 0 << 16
AAT_C_BF16X3 = 1 << 16
AAT_C_BF16 = 2 << 16


def AAT_LEVELS(l: int) -> int:
    return ((l + 1) & 0xF) << 8


#: every symbol include/aat.h and include/aat_testing.h declare
EXPORTS = [
    "aat_modp", "aat_modp_ex", "aat_syrk_modp", "aah_quat_modp", "aat_modp_host", "aat_modp_host_d2h_bytes", "aat_gemm_modp",
    "aat_gemm_modp_noalloc", "aat_tune_modp", "aat_tune_lookup", "aat_tune_save", "aat_tune_load",
    "aat_tune_clear",
    "aat_workspace_size", "aat_set_workspace_limit",
    "aat_last_error", "aat_device_status", "aat_shutdown", "aat_version",
    "aat_profile_begin", "aat_profile_end", "aah_complex", "aah_complex_ex", "aat_complex_2m",
    "aat_complex", "aat_complex_ex", "aat_plan_create", "aat_plan_execute", "aat_plan_info",
    "aat_plan_destroy",
    "aatx_is_prime", "aatx_sqrt_mod", "aatx_sos", "aatx_y_params", "aatx_digit_spec",
    "aatx_plan_stats", "aatx_leaf_groups", "aatx_sblocks", "aatx_split", "aatx_leaf", "aatx_postadd",
    "aatx_set_alloc_limit", "aatx_workspace_reserve", "aatx_wait_probe", "aatx_mma_peak",
]


AAT_KIND_MODP = 0
AAT_KIND_AAH = 1
AAT_KIND_AAT_C = 2


class Problem(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("A", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("k", ctypes.c_int64),
        ("lda", ctypes.c_int64),
        ("ldc", ctypes.c_int64),
        ("p", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
    ]


class Tune(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32),
        ("form", ctypes.c_int32),
        ("plain_digits", ctypes.c_int32),
        ("winograd", ctypes.c_int32),
        ("ms", ctypes.c_double),
        ("ms_default", ctypes.c_double),
    ]

    def as_dict(self):
        return dict(levels=int(self.levels), form=int(self.form),
                    plain_digits=int(self.plain_digits), winograd=int(self.winograd),
                    ms=float(self.ms),
                    ms_default=float(self.ms_default))


class AatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("aat error %d: %s" % (code, msg))
        self.code = code


class PlanStats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("n_pad", ctypes.c_int64),
        ("k_pad", ctypes.c_int64),
        ("recursive_products", ctypes.c_int64),
        ("general_products", ctypes.c_int64),
        ("syrk_leaves", ctypes.c_int64),
        ("block_additions", ctypes.c_int64),
        ("half_additions", ctypes.c_int64),
        ("ring_macs", ctypes.c_double),
        ("workspace_bytes", ctypes.c_size_t),
    ]


#: kernel classes of aat_profile_t
K_CLASSES = ["sblocks", "split", "leaf_tc", "leaf_simt", "postadd", "add_low", "copy", "leaf_f32",
             "leaf_mma", "winograd"]


class Profile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64 * 10),
        ("ms", ctypes.c_double * 10),
        ("work", ctypes.c_double * 10),
    ]

    def as_dict(self):
        out = {}
        for i, name in enumerate(K_CLASSES):
            if self.launches[i]:
                out[name] = dict(launches=int(self.launches[i]), ms=float(self.ms[i]),
                                 work=float(self.work[i]))
        return out


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libaat_gb300.so is not built; run paper_2101_01025_gb300.build.build() "
                "(nvcc, sm_103a).  There is no CPU fallback.")
        L = ctypes.CDLL(LIB_PATH)
        i64, u32, i32, vp, u64 = (ctypes.c_int64, ctypes.c_uint32, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_uint64)
        L.aat_modp.argtypes = [vp, i64, i64, u32, vp, vp]
        L.aat_modp_ex.argtypes = [vp, i64, i64, i64, u32, vp, i64, u32, vp]
        L.aat_modp_host.argtypes = [vp, i64, i64, u32, vp, u32]
        L.aat_syrk_modp.argtypes = [u32, vp, i64, i64, i64, u32, vp, i64, u32, u32, vp]
        L.aah_quat_modp.argtypes = [vp, vp, vp, vp, i64, i64, i64, u32, vp, vp, vp, vp, i64, u32,
                                    vp]
        L.aat_modp_host_d2h_bytes.argtypes = [i64, u32]
        L.aat_modp_host_d2h_bytes.restype = i64
        L.aat_gemm_modp.argtypes = [vp, i64, vp, i64, i64, i64, i64, u32, vp, i64, u32, vp]
        L.aat_gemm_modp_noalloc.argtypes = [vp, i64, vp, i64, i64, i64, i64, u32, vp, i64, vp]
        L.aat_tune_modp.argtypes = [i64, i64, u32, u32, i32, vp, ctypes.POINTER(Tune)]
        L.aat_tune_lookup.argtypes = [i64, i64, u32, ctypes.POINTER(Tune)]
        L.aat_tune_save.argtypes = [ctypes.c_char_p]
        L.aat_tune_load.argtypes = [ctypes.c_char_p]
        L.aat_tune_clear.restype = None
        L.aat_workspace_size.argtypes = [i64, i64, u32, u32]
        L.aat_workspace_size.restype = ctypes.c_size_t
        L.aat_set_workspace_limit.argtypes = [ctypes.c_size_t]
        L.aat_set_workspace_limit.restype = None
        L.aat_last_error.restype = ctypes.c_char_p
        L.aat_device_status.argtypes = [i32]
        L.aat_shutdown.restype = None
        L.aat_profile_end.argtypes = [ctypes.POINTER(Profile)]
        L.aah_complex.argtypes = [vp, i64, i64, vp, vp]
        L.aah_complex_ex.argtypes = [vp, i64, i64, i64, vp, i64, u32, vp]
        L.aat_complex_2m.argtypes = [vp, i64, i64, i64, vp, i64, u32, vp]
        L.aat_complex.argtypes = [vp, i64, i64, vp, vp]
        L.aat_plan_create.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(vp)]
        L.aat_plan_execute.argtypes = [vp, vp]
        L.aat_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_size_t)]
        L.aat_plan_destroy.argtypes = [vp]
        L.aat_plan_destroy.restype = None
        L.aat_complex_ex.argtypes = [vp, i64, i64, i64, vp, i64, u32, vp]
        L.aatx_is_prime.argtypes = [u64]
        L.aatx_sqrt_mod.argtypes = [i64, u64]
        L.aatx_sqrt_mod.restype = i64
        L.aatx_sos.argtypes = [i64, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.aatx_y_params.argtypes = [u32, ctypes.POINTER(i32), ctypes.POINTER(u32),
                                    ctypes.POINTER(u32)]
        L.aatx_digit_spec.argtypes = [u32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.aatx_plan_stats.argtypes = [i64, i64, u32, u32, ctypes.POINTER(PlanStats)]
        L.aatx_leaf_groups.argtypes = [u32, i64, u32, i32, vp, i32, ctypes.POINTER(i32)]
        L.aatx_sblocks.argtypes = [vp, i64, i64, i64, u32, vp, vp, vp, vp, i64, vp]
        L.aatx_split.argtypes = [vp, i64, i64, i64, u32, vp, vp]
        L.aatx_leaf.argtypes = [vp, i64, vp, i64, i64, i64, i64, u32, vp, i64, i32, i32, u32,
                                i32, vp]
        L.aatx_postadd.argtypes = [vp, i64, i64, u32, vp]
        L.aatx_set_alloc_limit.argtypes = [ctypes.c_size_t]
        L.aatx_set_alloc_limit.restype = None
        L.aatx_workspace_reserve.argtypes = [ctypes.c_size_t]
        L.aatx_wait_probe.argtypes = [i32, i64, vp]
        L.aatx_mma_peak.argtypes = [i32, i64, i32, vp, ctypes.POINTER(ctypes.c_double), vp]
        _lib = L
        return L


def last_error() -> str:
    return lib().aat_last_error().decode()


def check(rc: int) -> None:
    if rc != AAT_OK:
        raise AatError(rc, last_error())
