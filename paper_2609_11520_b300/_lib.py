"""ctypes loader of libfio_b300.so (the C ABI of include/fio.h).

The library is the only compute path: if it is missing this module raises at
import time instead of falling back to anything else.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfio_b300.so")

FIO_OK, FIO_EINVAL, FIO_ENOMEM, FIO_ECUDA, FIO_ENOTHPD, FIO_ERANK, FIO_ETIMEOUT, FIO_EBUSY = range(8)
STATUS_NAMES = ["FIO_OK", "FIO_EINVAL", "FIO_ENOMEM", "FIO_ECUDA", "FIO_ENOTHPD", "FIO_ERANK",
                "FIO_ETIMEOUT", "FIO_EBUSY"]
PHASE_KINDS = {"dft": 0, "cabs": 1, "elliptic2d": 2, "cabs8": 3, "iso2d": 4}
AMP_KINDS = {"one": 0, "bumps": 1, "hankel": 2}
SAMPLER_NORMAL, SAMPLER_DENSE = 0, 1


class FioError(RuntimeError):
    def __init__(self, status, msg):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


class Phase(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("s", ctypes.c_double)]


class Amp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("m", ctypes.c_int), ("sigma2", ctypes.c_double),
                ("centers", ctypes.POINTER(ctypes.c_double))]


class Sampler(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("bf", ctypes.c_void_p), ("dense", ctypes.c_void_p),
                ("ld", ctypes.c_int64)]


P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int
PP = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "bf_build": (I32, [ctypes.POINTER(Phase), I32, I32, I32, P, PP]),
    "bf_apply": (I32, [P, P, P, I64, I32, I32, P]),
    "bf_build_amp": (I32, [ctypes.POINTER(Phase), ctypes.POINTER(Amp), I32, I32, I32, P, PP]),
    "bf_info": (I32, [P, ctypes.POINTER(I64)]),
    "bf_set_path": (I32, [P, I32]),
    "bf_set_precision": (I32, [P, I32]),
    "bf_apply_noalloc": (I32, [P, P, P, I64, I32, I32, P]),
    "bf_free": (None, [P]),
    "bf_entries": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), I32, P, ctypes.POINTER(ctypes.c_double)]),
    "bf_entry_error": (I32, [ctypes.POINTER(Phase), ctypes.POINTER(Amp), I32, I32, I32, ctypes.POINTER(I64),
                             ctypes.POINTER(I64), I32, P, ctypes.POINTER(ctypes.c_double)]),
    "bf_build_tol": (I32, [ctypes.POINTER(Phase), ctypes.POINTER(Amp), I32, I32, ctypes.c_double, ctypes.POINTER(I64),
                           ctypes.POINTER(I64), I32, P, PP, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double)]),
    "hss_build_from_samples": (I32, [ctypes.POINTER(Sampler), I64, I32, I32, ctypes.c_double, ctypes.c_uint64,
                                     P, PP]),
    "hss_from_generators": (I32, [I64, I32, ctypes.POINTER(I32), P, P, P, P, PP]),
    "hss_info": (I32, [P, ctypes.POINTER(I64), I32, ctypes.POINTER(I64)]),
    "hss_matvec": (I32, [P, P, P, I64, I32, P]),
    "hss_ulv_factor": (I32, [P, P]),
    "hss_solve": (I32, [P, P, P, I64, I32, P]),
    "hss_set_solve_path": (I32, [P, I32]),
    "fio_solve": (I32, [P, P, P, P, I64, I32, I32, P]),
    "hss_free": (None, [P]),
    "fio_batch_create": (I32, [ctypes.POINTER(P), ctypes.POINTER(P), I32, PP]),
    "fio_batch_set_mode": (I32, [P, I32]),
    "fio_batch_solve": (I32, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I32), P]),
    "fio_batch_autotune": (I32, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I32), I32, P,
                                 ctypes.c_char_p, I64]),
    "fio_batch_free": (None, [P]),
    "fio_last_error": (ctypes.c_char_p, []),
    "fio_device_status": (I32, []),
    "fio_selftest_wait_timeout": (I32, [P]),
    "fio_pcg": (I32, [P, P, P, P, I64, I32, ctypes.c_double, I32, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double),
                      P]),
    "fio_profile_enable": (I32, [I32]),
    "fio_set_large_node": (I32, [I32]),
    "fio_set_large_node_count": (I32, [I32]),
    "fio_profile_report": (I32, [ctypes.c_char_p, I64]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python paper_2609_11520_b300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def check(status):
    if status != FIO_OK:
        raise FioError(status, lib.fio_last_error().decode(errors="replace"))
