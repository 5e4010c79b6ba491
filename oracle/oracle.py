"""ctypes binding of ``fem_oracle.c`` (test infrastructure only).

The C file is compiled with plain ``gcc -O2 -ffp-contract=off`` (no fused
multiply-add contraction, so x86 and Arm hosts round identically) into
``oracle/liboracle.so`` on first use, or by ``build()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_create.restype = ctypes.c_void_p
        lib.oracle_create.argtypes = [
            _i64, _dp, _i64, _ip, _ip, ctypes.c_int32, _dp, _i64, _ip, _dp, _dp, _dp,
            _i64, _ip, _dp, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_destroy.argtypes = [ctypes.c_void_p]
        lib.oracle_set_temperature.argtypes = [ctypes.c_void_p, _dp]
        lib.oracle_step.argtypes = [ctypes.c_void_p, _i64, ctypes.c_double]
        lib.oracle_energy.argtypes = [ctypes.c_void_p, _dp]
        lib.oracle_residual.restype = ctypes.c_double
        lib.oracle_residual.argtypes = [ctypes.c_void_p, _dp, _dp]
        lib.oracle_residual_part.restype = ctypes.c_double
        lib.oracle_residual_part.argtypes = [ctypes.c_void_p, _dp, _dp, _ip, _ip,
                                             ctypes.c_int32]
        lib.oracle_temperatures.argtypes = [ctypes.c_void_p, _dp]
        lib.oracle_stable_dt.restype = ctypes.c_double
        lib.oracle_stable_dt.argtypes = [ctypes.c_void_p]
        lib.oracle_get_E.argtypes = [ctypes.c_void_p, _dp]
        lib.oracle_set_E.argtypes = [ctypes.c_void_p, _dp]
        lib.oracle_get_lumped.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        lib.oracle_get_element.argtypes = [ctypes.c_void_p, _i64, _ip, _dp, _dp]
        lib.oracle_step_count.restype = _i64
        lib.oracle_step_count.argtypes = [ctypes.c_void_p]
        lib.oracle_time.restype = ctypes.c_double
        lib.oracle_time.argtypes = [ctypes.c_void_p]
        for name in ("oracle_E_from_T", "oracle_T_from_E"):
            f = getattr(lib, name)
            f.restype = ctypes.c_double
            f.argtypes = [ctypes.c_double] * 5
        lib.oracle_liquid_fraction.restype = ctypes.c_double
        lib.oracle_liquid_fraction.argtypes = [ctypes.c_double] * 3
        lib.oracle_tet_matrix.restype = ctypes.c_int
        lib.oracle_tet_matrix.argtypes = [_dp, ctypes.c_double, _dp, _dp]
        lib.oracle_set_interface.restype = ctypes.c_int
        lib.oracle_set_interface.argtypes = [ctypes.c_void_p, _i64, _ip, _dp, _i64, _ip, _dp]
        lib.oracle_set_conductivity.restype = ctypes.c_int
        lib.oracle_set_conductivity.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _dp, _dp]
        lib.oracle_conductivity.restype = ctypes.c_double
        lib.oracle_conductivity.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double]
        lib.oracle_set_formulation.restype = ctypes.c_int
        lib.oracle_set_formulation.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_apparent_cp.restype = ctypes.c_double
        lib.oracle_apparent_cp.argtypes = [ctypes.c_void_p, _i64, _dp]
        lib.oracle_interface_sister.restype = _i64
        lib.oracle_interface_sister.argtypes = [ctypes.c_void_p, _i64]
        _lib = lib
        return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


def E_from_T(T, C, Lc, Ts, Tl) -> float:
    return _load().oracle_E_from_T(T, C, Lc, Ts, Tl)


def T_from_E(E, C, Lc, Ts, Tl) -> float:
    return _load().oracle_T_from_E(E, C, Lc, Ts, Tl)


def liquid_fraction(T, Ts, Tl) -> float:
    return _load().oracle_liquid_fraction(T, Ts, Tl)


def tet_matrix(x4: np.ndarray, k: float):
    """Dense K^e (4x4) and signed volume of one tet with corners x4 [4,3]."""
    x = _d(np.asarray(x4).reshape(12))
    K = np.zeros(16)
    v = ctypes.c_double()
    st = _load().oracle_tet_matrix(_pd(x), k, _pd(K), ctypes.byref(v))
    if st != 0:
        raise ValueError("degenerate tet")
    return K.reshape(4, 4), v.value


class OracleProblem:
    """One problem held by the C oracle: set-up, stepping and read-back."""

    def __init__(self, prob, *, faces=True, dirichlet=True):
        lib = _load()
        self._lib = lib
        self.n_nodes = int(prob.xyz.shape[0])
        xyz, tets, mat, mats = _d(prob.xyz), _i(prob.tets), _i(prob.mat), _d(prob.materials)
        if faces and prob.faces.shape[0] > 0:
            fc, fh, ft, fq = _i(prob.faces), _d(prob.h), _d(prob.t_inf), _d(prob.q)
            nf = fc.shape[0]
        else:
            fc, fh, ft, fq = _i(np.zeros((1, 3))), _d(np.zeros(1)), _d(np.zeros(1)), _d(np.zeros(1))
            nf = 0
        if dirichlet and prob.dir_nodes.shape[0] > 0:
            dn, dT = _i(prob.dir_nodes), _d(prob.dir_T)
            nd = dn.shape[0]
        else:
            dn, dT, nd = _i(np.zeros(1)), _d(np.zeros(1)), 0
        st = ctypes.c_int()
        self._h = lib.oracle_create(
            self.n_nodes, _pd(xyz), tets.shape[0], _pi(tets), _pi(mat), mats.shape[0],
            _pd(mats), nf, _pi(fc), _pd(fh), _pd(ft), _pd(fq), nd, _pi(dn), _pd(dT),
            ctypes.byref(st))
        if not self._h:
            raise ValueError(f"oracle_create failed with status {st.value}")
        self._keep = (xyz, tets, mat, mats, fc, fh, ft, fq, dn, dT)
        for mt, Tk, kk in getattr(prob, "k_tables", ()):
            self.set_conductivity(mt, Tk, kk)
        ia = getattr(prob, "iface_a", None)
        if faces and ia is not None and ia.shape[0] > 0:
            a, ha = _i(prob.iface_a), _d(prob.h_ia)
            b, hb = _i(prob.iface_b), _d(prob.h_ib)
            rc = lib.oracle_set_interface(self._h, a.shape[0], _pi(a), _pd(ha), b.shape[0],
                                          _pi(b), _pd(hb))
            if rc != 0:
                raise ValueError(f"oracle_set_interface failed with status {rc}")
            self.n_interface = a.shape[0] + b.shape[0]
        else:
            self.n_interface = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    def set_temperature(self, T0) -> None:
        T0 = _d(T0)
        self._lib.oracle_set_temperature(self._h, _pd(T0))

    def step(self, n: int, dt: float) -> None:
        self._lib.oracle_step(self._h, int(n), float(dt))

    def temperature(self) -> np.ndarray:
        T = np.zeros(self.n_nodes)
        self._lib.oracle_temperatures(self._h, _pd(T))
        return T

    def enthalpy(self) -> np.ndarray:
        E = np.zeros(self.n_nodes)
        self._lib.oracle_get_E(self._h, _pd(E))
        return E

    def set_enthalpy(self, E) -> None:
        E = _d(E)
        self._lib.oracle_set_E(self._h, _pd(E))

    def energy(self) -> np.ndarray:
        out = np.zeros(4)
        self._lib.oracle_energy(self._h, _pd(out))
        return out

    def residual(self, T, elem_part=None, face_part=None, part: int = 0):
        """(R = F - K T, heat entering through the faces per unit time)."""
        T = _d(T)
        R = np.zeros(self.n_nodes)
        if elem_part is None:
            q = self._lib.oracle_residual(self._h, _pd(T), _pd(R))
        else:
            ep, fp = _i(elem_part), _i(face_part)
            q = self._lib.oracle_residual_part(self._h, _pd(T), _pd(R), _pi(ep), _pi(fp),
                                               int(part))
        return R, q

    def set_conductivity(self, mt: int, T, k) -> None:
        """Piecewise-linear k(T) table for material mt (evaluated at the
        element's mean temperature); an empty table restores constant k."""
        T, k = _d(T), _d(k)
        rc = self._lib.oracle_set_conductivity(self._h, int(mt), T.shape[0], _pd(T), _pd(k))
        if rc != 0:
            raise ValueError(f"oracle_set_conductivity failed with status {rc}")
        self._keep = self._keep + (T, k)

    def set_formulation(self, form: int) -> None:
        """0: enthalpy (Eq. 5); 1: apparent heat capacity by Lemmon's method
        (Eqs. 6-7) with T as the unknown (positive-width phase-change ranges
        only).  The current state carries over."""
        rc = self._lib.oracle_set_formulation(self._h, int(form))
        if rc != 0:
            raise ValueError(f"oracle_set_formulation failed with status {rc}")

    def apparent_cp(self, e: int, T) -> float:
        T = _d(T)
        return self._lib.oracle_apparent_cp(self._h, int(e), _pd(T))

    def conductivity(self, mt: int, T: float) -> float:
        return self._lib.oracle_conductivity(self._h, int(mt), float(T))

    def interface_sisters(self) -> np.ndarray:
        """Sister of every interface face (side-A faces first, then side B),
        as an index into that combined list."""
        return np.array([self._lib.oracle_interface_sister(self._h, f)
                         for f in range(self.n_interface)], np.int64)

    def stable_dt(self) -> float:
        return self._lib.oracle_stable_dt(self._h)

    def lumped(self):
        C, m, Lc = np.zeros(self.n_nodes), np.zeros(self.n_nodes), np.zeros(self.n_nodes)
        self._lib.oracle_get_lumped(self._h, _pd(C), _pd(m), _pd(Lc))
        return C, m, Lc

    def element(self, e: int):
        nodes = np.zeros(4, np.int32)
        K = np.zeros(16)
        v = ctypes.c_double()
        self._lib.oracle_get_element(self._h, int(e), _pi(nodes), _pd(K), ctypes.byref(v))
        return nodes, K.reshape(4, 4), v.value

    @property
    def step_count(self) -> int:
        return int(self._lib.oracle_step_count(self._h))

    @property
    def time(self) -> float:
        return float(self._lib.oracle_time(self._h))
