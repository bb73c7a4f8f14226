"""ctypes binding of libmg_cpu.so, the SIMD CPU build of the helicity-shared
program (include/mg_cpu.h): argument marshalling only, host numpy arrays.

A CPU baseline beside the GPU kernels (the paper's vectorised C++ build,
Sec. 4), not a fallback: the GPU binding (mg.py) never calls it.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None
PRECISIONS = {"fp64": 0, "fp32": 1}


class Params(ctypes.Structure):
    _fields_ = [("mz", ctypes.c_double), ("wz", ctypes.c_double), ("alpha_inv", ctypes.c_double),
                ("sw2", ctypes.c_double), ("mt", ctypes.c_double), ("wt", ctypes.c_double),
                ("alpha_s", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build_cpu()
            if not os.path.exists(path):
                raise RuntimeError("libmg_cpu.so was not built")
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            L.mgc_lanes.argtypes = [ctypes.c_int]
            L.mgc_sigmakin.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ip, ctypes.c_int, ctypes.POINTER(Params),
                                       dp, ctypes.c_int]
            _lib = L
    return _lib


def lanes(precision="fp32") -> int:
    return int(lib().mgc_lanes(PRECISIONS[precision]))


def sigmakin(proc: int, mom: np.ndarray, mask: np.ndarray, precision="fp32", params: dict | None = None,
             nthreads: int | None = None) -> np.ndarray:
    """mom (npar, 4, nevt) float64, mask (nhel,) int32 -> me (nevt,) float64, on the host cores."""
    from .inputs import SM_PARAMS
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    mask = np.ascontiguousarray(mask, dtype=np.int32)
    p = dict(SM_PARAMS)
    p.update(params or {})
    prm = Params(**{k: float(p[k]) for k, _ in Params._fields_})
    nevt = mom.shape[2]
    me = np.zeros(nevt)
    rc = lib().mgc_sigmakin(proc, nevt, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), PRECISIONS[precision],
                            ctypes.byref(prm), me.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("mgc_sigmakin failed with status %d" % rc)
    return me
