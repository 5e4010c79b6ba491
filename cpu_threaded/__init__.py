"""ctypes binding of the threaded CPU baseline (``ebe_omp.cpp``).

An OpenMP implementation of the same explicit EBE step with a colour-parallel
element loop, in FP64 or FP32, timed by ``bench.py`` on the host's cores as a
comparison point.  It is neither the product (the GPU library) nor the oracle.
Compiled with ``g++ -O3 -fopenmp`` into ``cpu_threaded/libebe_omp.so`` on first
use, or by ``build()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebe_omp.cpp")
_LIB = os.path.join(_HERE, "libebe_omp.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the baseline if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.ebe_cpu_create.restype = ctypes.c_void_p
        lib.ebe_cpu_create.argtypes = [_dp, _i64, _ip, _i64, _ip, _dp, ctypes.c_int32, _ip, _i64,
                                       _dp, _dp, _dp, _ip, _i64, _dp, _dp, ctypes.c_int,
                                       ctypes.c_int]
        lib.ebe_cpu_step.argtypes = [ctypes.c_void_p, _i64, ctypes.c_double]
        lib.ebe_cpu_temperature.argtypes = [ctypes.c_void_p, _dp]
        lib.ebe_cpu_energy.argtypes = [ctypes.c_void_p, _dp]
        lib.ebe_cpu_info.argtypes = [ctypes.c_void_p, _ip]
        lib.ebe_cpu_destroy.argtypes = [ctypes.c_void_p]
        _lib = lib
        return lib


def _p(a, t):
    return a.ctypes.data_as(t)


class ThreadedBaseline:
    """One problem (``meshgen.Problem``) on the threaded CPU baseline."""

    def __init__(self, p, precision: str = "fp64", threads: int = 0):
        if precision not in ("fp64", "fp32"):
            raise ValueError(precision)
        lib = _load()
        self._keep = [
            np.ascontiguousarray(p.xyz, np.float64), np.ascontiguousarray(p.tets, np.int32),
            np.ascontiguousarray(p.mat, np.int32), np.ascontiguousarray(p.materials, np.float64),
            np.ascontiguousarray(p.faces, np.int32).reshape(-1, 3),
            np.ascontiguousarray(p.h, np.float64), np.ascontiguousarray(p.t_inf, np.float64),
            np.ascontiguousarray(p.q, np.float64),
            np.ascontiguousarray(p.dir_nodes, np.int32), np.ascontiguousarray(p.dir_T, np.float64),
            np.ascontiguousarray(p.T0, np.float64)]
        xyz, tets, mat, mats, faces, h, ti, q, dn, dT, T0 = self._keep
        self.n_nodes = xyz.shape[0]
        self.n_tets = tets.shape[0]
        self.h = lib.ebe_cpu_create(
            _p(xyz, _dp), self.n_nodes, _p(tets, _ip), self.n_tets, _p(mat, _ip), _p(mats, _dp),
            mats.shape[0], _p(faces, _ip), faces.shape[0], _p(h, _dp), _p(ti, _dp), _p(q, _dp),
            _p(dn, _ip), dn.shape[0], _p(dT, _dp), _p(T0, _dp), int(precision == "fp32"),
            int(threads))
        if not self.h:
            raise ValueError("threaded baseline: invalid problem")
        self._lib = lib

    def step(self, n: int, dt: float) -> None:
        self._lib.ebe_cpu_step(self.h, int(n), float(dt))

    def temperature(self) -> np.ndarray:
        T = np.empty(self.n_nodes, np.float64)
        self._lib.ebe_cpu_temperature(self.h, _p(T, _dp))
        return T

    def energy(self) -> float:
        out = np.zeros(1, np.float64)
        self._lib.ebe_cpu_energy(self.h, _p(out, _dp))
        return float(out[0])

    def info(self) -> dict:
        out = np.zeros(3, np.int32)
        self._lib.ebe_cpu_info(self.h, _p(out, _ip))
        return {"threads": int(out[0]), "colours": int(out[1]), "face_colours": int(out[2])}

    def close(self) -> None:
        if getattr(self, "h", None):
            self._lib.ebe_cpu_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()
