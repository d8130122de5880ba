"""ctypes wrapper of ``paper_cpu_force.c``: the paper's mixed-precision force
loop (Sec. 3.2-3.3: double-precision relative positions, single-precision
pair arithmetic with a Newton-refined reciprocal square root, acceleration
and potential summed in double, jerk in single, two i against four j per
vector) on the host CPU.

A CPU baseline for the benchmark, beside the plain FP64 oracle; not part of
the GPU path.  Arrays are numpy float64, C-contiguous, positions and
velocities (n, 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paper_cpu_force.c")
_LIB_PATH = os.path.join(_HERE, "libpaper_cpu_force.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile with gcc: -O3, portable vector extensions (no -march), OpenMP."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-fPIC", "-shared", "-std=gnu11", "-fopenmp",
           "-Wno-psabi", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32, P = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.pcf_layout_bytes.argtypes = [i64]
        lib.pcf_layout_bytes.restype = i64
        lib.pcf_pack.argtypes = [i64, P, P, P, P]
        lib.pcf_pack.restype = None
        lib.pcf_force.argtypes = [i64, P, d, d, i64, P, P, P, P, i32]
        lib.pcf_force.restype = i32
        lib.pcf_has_openmp.argtypes = []
        lib.pcf_has_openmp.restype = i32
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Layout:
    """The packed j layout of one particle set (pcf_pack)."""

    def __init__(self, m, r, v):
        lib = _load()
        self.m = np.ascontiguousarray(m, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        self.n = len(self.m)
        self.work = np.empty(lib.pcf_layout_bytes(self.n) // 8 + 1, dtype=np.float64)
        lib.pcf_pack(self.n, _ptr(self.m), _ptr(r), _ptr(v), _ptr(self.work))

    def force(self, eps, idx=None, G=1.0, nthreads=None):
        """(acc, jerk, pot) of the particles idx (all if None)."""
        lib = _load()
        idx = np.arange(self.n, dtype=np.int32) if idx is None \
            else np.ascontiguousarray(idx, dtype=np.int32)
        k = len(idx)
        acc = np.empty((k, 3))
        jerk = np.empty((k, 3))
        pot = np.empty(k)
        nt = nthreads or os.cpu_count() or 1
        st = lib.pcf_force(self.n, _ptr(self.work), float(eps), float(G), k, _ptr(idx),
                           _ptr(acc), _ptr(jerk), _ptr(pot), int(nt))
        if st != 0:
            raise ValueError("active index out of range")
        return acc, jerk, pot


def force(m, r, v, eps, idx=None, G=1.0, nthreads=None):
    return Layout(m, r, v).force(eps, idx, G, nthreads)


def has_openmp() -> bool:
    return bool(_load().pcf_has_openmp())
