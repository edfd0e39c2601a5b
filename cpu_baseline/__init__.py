"""All-core OpenMP CPU baseline of aprod 1 / aprod 2 (benchmark context only).

A multi-threaded CPU implementation written independently of the oracle and
of the CUDA library; the benchmark times it on every host core beside the
single-core oracle. Not used by the library or the tests' parity checks.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_omp.c")
_SO = os.path.join(_HERE, "_build", "libgsr_omp.so")
_lib = None


def build(force=False):
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-march=native", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        args = [i64, i64, i64, i64, i32] + [p] * 6
        lib.gsr_omp_aprod1.argtypes = args
        lib.gsr_omp_aprod1.restype = None
        lib.gsr_omp_aprod2.argtypes = args
        lib.gsr_omp_aprod2.restype = ctypes.c_int
        lib.gsr_omp_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads():
    return int(_load().gsr_omp_threads())


def _args(sys):
    arr = [np.ascontiguousarray(sys["vals"], dtype=np.float64),
           np.ascontiguousarray(sys["astro_off"], dtype=np.int64),
           np.ascontiguousarray(sys["att_off"], dtype=np.int64),
           np.ascontiguousarray(sys["instr"], dtype=np.int32)]
    dims = (int(sys["n_rows"]), int(sys["n_stars"]), int(sys["n_knots"]), int(sys["n_instr"]),
            int(sys["n_glob"]))
    return dims, arr


def aprod1(sys, x, y):
    """y += A x on all host cores (y float64, contiguous, in place)."""
    dims, arr = _args(sys)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert y.dtype == np.float64 and y.flags.c_contiguous and y.shape == (dims[0],)
    _load().gsr_omp_aprod1(*dims, *[a.ctypes.data for a in arr], x.ctypes.data, y.ctypes.data)
    return y


def aprod2(sys, y, x):
    """x += A^T y on all host cores (x float64, contiguous, in place)."""
    dims, arr = _args(sys)
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    if _load().gsr_omp_aprod2(*dims, *[a.ctypes.data for a in arr], y.ctypes.data,
                              x.ctypes.data) != 0:
        raise MemoryError("gsr_omp_aprod2: allocation failed")
    return x
