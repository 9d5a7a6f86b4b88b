"""ctypes view of libmtp_gb300.so (declarations mirror include/mtp.h).

Loading fails loudly: there is no pure-Python or CPU path behind these calls.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmtp_gb300.so")

MTP_OK = 0
MTP_STATUS_BREAK = 1
STATUS_NAMES = {
    1: "MTP_STATUS_BREAK", -1: "MTP_ERR_ARG", -2: "MTP_ERR_CUDA", -3: "MTP_ERR_OOM",
    -4: "MTP_ERR_NEIGHBOR_OVERFLOW", -5: "MTP_ERR_NONFINITE", -6: "MTP_ERR_TIMEOUT", -7: "MTP_ERR_UNSUPPORTED",
    -8: "MTP_ERR_STALE_LIST",
}
MTP_FP64 = 0
MTP_MIXED = 1
MTP_GRADE_TENSOR = 0
MTP_GRADE_FP64 = 1
MTP_ERR_STALE_LIST = -8


class MtpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


class ParamsDesc(ctypes.Structure):
    _fields_ = [
        ("level", ctypes.c_int32),
        ("n_species", ctypes.c_int32),
        ("n_q", ctypes.c_int32),
        ("r_min", ctypes.c_double),
        ("r_cut", ctypes.c_double),
        ("species_energy", ctypes.POINTER(ctypes.c_double)),
        ("radial", ctypes.POINTER(ctypes.c_double)),
        ("xi", ctypes.POINTER(ctypes.c_double)),
        ("m", ctypes.c_int64),
    ]


_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_P_I32 = ctypes.POINTER(ctypes.c_int32)
_P_I64 = ctypes.POINTER(ctypes.c_int64)
_P_D = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "mtp_basis_info": (ctypes.c_int, [_I32, _P_I32, _P_I32, _P_I32, _P_I32]),
    "mtp_basis_table": (ctypes.c_int, [_I32, _I32, _P_I64, _P_I64]),
    "mtp_load_params": (ctypes.c_int, [ctypes.POINTER(ParamsDesc), ctypes.POINTER(_VP)]),
    "mtp_free": (None, [_VP]),
    "mtp_param_count": (ctypes.c_int, [_VP, _P_I64]),
    "mtp_set_theta": (ctypes.c_int, [_VP, _VP, _VP]),
    "mtp_build_neighbors": (ctypes.c_int, [_VP, _VP, _I64, _P_D, _P_I32, ctypes.POINTER(_VP), _VP]),
    "mtp_nlist_info": (ctypes.c_int, [_VP, _P_I64, _P_I64]),
    "mtp_nlist_copy": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "mtp_free_nlist": (None, [_VP]),
    "mtp_compute_efv": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _P_D, _I32, _I64, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mtp_compute_efv_tangent": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _P_D, _I32, _VP, _VP, _VP, _VP]),
    "mtp_compute_grade": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _P_D, _VP, _VP, ctypes.c_double, ctypes.c_double,
                                         _I64, _I32, _VP, _VP, _P_D, _P_D, _P_I64, _P_I64, _VP]),
    "mtp_grade_tc_selftest": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "mtp_batch_create": (ctypes.c_int, [_VP, _I32, _P_I64, _P_D, _P_I32, _VP, _I32, ctypes.POINTER(_VP), _VP]),
    "mtp_batch_nlist": (ctypes.c_int, [_VP, ctypes.POINTER(_VP)]),
    "mtp_compute_batch": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mtp_batch_tune": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _I32, _P_I32, _VP, _VP, _VP, _VP, _VP]),
    "mtp_batch_free": (None, [_VP]),
    "mtp_compute_efv_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _P_D, _I64, _VP, _VP, _VP, _VP, _VP]),
    "mtp_compute_basis_rows": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _P_D, _VP, _VP]),
    "mtp_maxvol": (ctypes.c_int, [_VP, _I64, _I32, _P_I32, ctypes.c_double, _I32, _VP, _P_I32, _VP]),
    "mtp_md_create": (ctypes.c_int, [_VP, _VP, _I64, _P_D, _P_I32, ctypes.c_double, ctypes.POINTER(_VP), _VP]),
    "mtp_md_rebuild": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "mtp_md_nlist": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), _VP]),
    "mtp_md_status": (ctypes.c_int, [_VP, _P_I64, _P_I64, _VP]),
    "mtp_md_run": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _P_D, ctypes.c_double, _I32, _I32, _I32, _VP, _VP, _VP,
                                  _VP]),
    "mtp_md_free": (None, [_VP]),
    "mtp_md_set_grade": (ctypes.c_int, [_VP, _VP, _VP, _I32, ctypes.c_double, ctypes.c_double, _I32, _VP]),
    "mtp_md_set_barostat": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "mtp_md_info": (ctypes.c_int, [_VP, _P_I64, _P_I64, _P_D, _P_I64, _P_D, _P_D]),
    "mtp_device_status": (ctypes.c_int, [_VP, _VP]),
    "mtp_last_error": (ctypes.c_char_p, []),
    "mtp_probe_fma": (ctypes.c_int, [_I32, _I64, _I32, _P_D, _P_D]),
    "mtp_set_wait_limit": (ctypes.c_int, [_I64]),
    "mtp_set_efv_variant": (ctypes.c_int, [_VP, _I32]),
    "mtp_efv_tune": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _P_D, _I32, _P_I32, ctypes.POINTER(ctypes.c_float),
                                    _VP]),
    "mtp_grade_rows": (ctypes.c_int, [_VP, _I64, _I64, _VP, _I32, _VP, ctypes.c_double, ctypes.c_double, _VP, _VP,
                                      _P_D, _P_I64, _VP]),
}

_lib = None


def load():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmtp_gb300.so is not built (%s); run __graft_entry__.build() or "
                          "python paper_2510_00193_gb300/build.py" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int) -> int:
    if code < 0:
        msg = load().mtp_last_error()
        raise MtpError(code, msg.decode() if msg else "")
    return code
