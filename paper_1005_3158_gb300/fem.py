"""Thin ctypes binding of libfem (include/fem.h).

Argument marshalling only: every computation of the step runs in the CUDA
kernels of ``libfem.so``.  The module-level functions carry the C names; the
``Mesh`` class wraps one handle.  Importing this module loads the library
and raises if it has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FEM_CHECKED=1 selects the checked build (device-side bounds checks on every
# indexed access; build it with build.build(checked=True))
LIB_PATH = os.path.join(_HERE, "libfem_checked.so" if os.environ.get("FEM_CHECKED") == "1"
                        else "libfem.so")

FEM_OK, FEM_EINVAL, FEM_ENOMEM, FEM_ECUDA, FEM_ESTATE, FEM_EUNSTABLE, FEM_ETIMEOUT = range(7)
FEM_ENTHALPY, FEM_APPARENT_CAPACITY = 0, 1
FORMULATIONS = {"enthalpy": FEM_ENTHALPY, "apparent": FEM_APPARENT_CAPACITY}
FEM_FP64, FEM_FP32 = 0, 1
FEM_VARIANT_BLOCK, FEM_VARIANT_ATOMIC, FEM_VARIANT_COLORED = 0, 1, 2
STATUS_NAMES = {0: "FEM_OK", 1: "FEM_EINVAL", 2: "FEM_ENOMEM", 3: "FEM_ECUDA", 4: "FEM_ESTATE",
                5: "FEM_EUNSTABLE", 6: "FEM_ETIMEOUT"}
VARIANTS = {"block": FEM_VARIANT_BLOCK, "atomic": FEM_VARIANT_ATOMIC,
            "colored": FEM_VARIANT_COLORED}
PRECISIONS = {"fp64": FEM_FP64, "f64": FEM_FP64, "fp32": FEM_FP32, "f32": FEM_FP32}

# names declared in include/fem.h
ABI_SYMBOLS = (
    "fem_mesh_create", "fem_mesh_create_ex", "fem_set_materials", "fem_set_boundary",
    "fem_set_interface", "fem_set_conductivity",
    "fem_set_dirichlet", "fem_set_temperature", "fem_stable_dt", "fem_step", "fem_step_profile",
    "fem_get_temperature", "fem_get_enthalpy", "fem_get_energy", "fem_set_stream",
    "fem_get_state", "fem_set_state", "fem_mesh_info", "fem_rcm_order", "fem_plan_array",
    "fem_last_error", "fem_mesh_destroy", "fem_energy_sums_noalloc", "fem_batch_create",
    "fem_instance_stable_dt", "fem_set_instance_dt", "fem_advance", "fem_get_instance_times",
    "fem_get_instance_energy", "fem_set_allocator", "fem_autotune", "fem_set_state_async",
    "fem_get_temperature_async", "fem_sync", "fem_set_state_async_f32",
    "fem_get_temperature_async_f32",
    "fem_surrogate_create", "fem_surrogate_info", "fem_surrogate_order",
    "fem_surrogate_set_params", "fem_surrogate_get_params", "fem_surrogate_read_state",
    "fem_surrogate_accumulate", "fem_surrogate_apply",
    "fem_surrogate_write_state", "fem_surrogate_predict", "fem_surrogate_train_step",
    "fem_surrogate_advance", "fem_surrogate_solve", "fem_surrogate_profile", "fem_surrogate_debug",
    "fem_surrogate_destroy",
)
FEM_SG_N_PARAMS = 30177


class FemMaterial(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("c", ctypes.c_double), ("k", ctypes.c_double),
                ("latent", ctypes.c_double), ("T_solidus", ctypes.c_double),
                ("T_liquidus", ctypes.c_double)]


class FemOptions(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block_elems", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("formulation", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class FemInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_nodes", "n_tets", "n_faces", "n_blocks", "n_interior_nodes", "n_shared_nodes",
        "n_shared_copies", "n_sched_rounds", "n_colors", "bandwidth_input",
        "bandwidth_internal", "max_block_elems", "device_bytes")] + [
        (n, ctypes.c_int32) for n in ("precision", "variant", "threads", "reorder",
                                      "ctas_per_sm", "smem_per_cta", "n_instances",
                                      "n_interface_faces")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class FemError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
            f"g.build()\"` (the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    i64 = ctypes.c_int64
    sig = {
        "fem_mesh_create": [dp, i64, ip, i64, ip, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)],
        "fem_mesh_create_ex": [dp, i64, ip, i64, ip, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(FemOptions), ctypes.POINTER(P)],
        "fem_set_materials": [P, ctypes.POINTER(FemMaterial), ctypes.c_int32],
        "fem_set_boundary": [P, ip, i64, dp, dp, dp],
        "fem_set_dirichlet": [P, ip, i64, dp],
        "fem_set_interface": [P, ip, i64, dp, ip, i64, dp],
        "fem_set_conductivity": [P, ctypes.c_int32, ctypes.c_int32, dp, dp],
        "fem_set_temperature": [P, dp],
        "fem_stable_dt": [P, dp],
        "fem_step": [P, i64, ctypes.c_double],
        "fem_step_profile": [P, i64, ctypes.c_double, dp, ctypes.c_int32,
                             ctypes.POINTER(ctypes.c_int32)],
        "fem_get_temperature": [P, P],
        "fem_get_enthalpy": [P, P],
        "fem_get_energy": [P, dp],
        "fem_set_stream": [P, P],
        "fem_get_state": [P, P, ctypes.POINTER(i64), dp],
        "fem_set_state": [P, P, i64, ctypes.c_double],
        "fem_mesh_info": [P, ctypes.POINTER(FemInfo)],
        "fem_rcm_order": [i64, ip, i64, ip, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "fem_plan_array": [P, ctypes.c_int32, ctypes.POINTER(P), ctypes.POINTER(i64)],
        "fem_energy_sums_noalloc": [ctypes.c_int, P, P, P, P, P, i64, P, P],
        "fem_batch_create": [ctypes.POINTER(P), ctypes.c_int32, ctypes.POINTER(P)],
        "fem_set_allocator": [P, P, P, P],
        "fem_instance_stable_dt": [P, dp],
        "fem_set_instance_dt": [P, dp],
        "fem_advance": [P, ctypes.c_double],
        "fem_get_instance_times": [P, dp, ctypes.POINTER(i64)],
        "fem_get_instance_energy": [P, ctypes.c_int32, dp],
        "fem_autotune": [P, ip, ip, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ip, dp],
        "fem_set_state_async": [P, P, i64, ctypes.c_double],
        "fem_get_temperature_async": [P, P],
        "fem_set_state_async_f32": [P, P, i64, ctypes.c_double],
        "fem_get_temperature_async_f32": [P, P],
        "fem_sync": [P],
        "fem_surrogate_create": [P, ctypes.c_double, ctypes.POINTER(P)],
        "fem_surrogate_info": [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "fem_surrogate_order": [P, ip],
        "fem_surrogate_set_params": [P, P, i64],
        "fem_surrogate_get_params": [P, P, i64],
        "fem_surrogate_read_state": [P, P],
        "fem_surrogate_write_state": [P, P],
        "fem_surrogate_predict": [P, P, P],
        "fem_surrogate_train_step": [P, P, P, ctypes.c_float, dp],
        "fem_surrogate_accumulate": [P, P, P, dp],
        "fem_surrogate_apply": [P, ctypes.c_float],
        "fem_surrogate_advance": [P, i64],
        "fem_surrogate_solve": [P, i64, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(i64), dp],
        "fem_surrogate_profile": [P, i64, dp],
        "fem_surrogate_debug": [P, ctypes.c_int32, ctypes.c_int32, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fem_last_error.restype = ctypes.c_char_p
    lib.fem_last_error.argtypes = []
    lib.fem_mesh_destroy.restype = None
    lib.fem_mesh_destroy.argtypes = [P]
    lib.fem_surrogate_destroy.restype = None
    lib.fem_surrogate_destroy.argtypes = [P]
    return lib


_lib = _load()


def lib():
    return _lib


def _check(st):
    if st != FEM_OK:
        raise FemError(st, _lib.fem_last_error().decode())


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _host_ptr(buf, n, writable, f32=False):
    """Pointer to a host buffer of n doubles (n floats with f32): a numpy
    array or a (pinned) torch CPU tensor.  Returns (pointer, keep-alive)."""
    want = "float32" if f32 else "float64"
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.dtype(want) or not buf.flags["C_CONTIGUOUS"] or buf.size < n:
            raise ValueError(f"host buffer must be a C-contiguous {want} array of size >= n_nodes")
        if writable and not buf.flags["WRITEABLE"]:
            raise ValueError("output buffer is read-only")
        return ctypes.c_void_p(buf.ctypes.data), buf
    # torch tensor (duck-typed so the binding does not import torch)
    if getattr(buf, "device", None) is not None and str(buf.device) != "cpu":
        raise ValueError("host buffer expected (got a device tensor)")
    if str(buf.dtype) != "torch." + want or not buf.is_contiguous() or buf.numel() < n:
        raise ValueError(f"host tensor must be contiguous {want} of size >= n_nodes")
    return ctypes.c_void_p(buf.data_ptr()), buf


def _is_f32(buf):
    return str(getattr(buf, "dtype", "")) in ("float32", "torch.float32")


# ---------------------------------------------------------------------------
# Module-level functions with the C names
# ---------------------------------------------------------------------------

def fem_mesh_create(xyz, tets, mat_id, prec=FEM_FP64, reorder=0, options=None):
    xyz, tets, mat_id = _d(xyz), _i(tets), _i(mat_id)
    h = ctypes.c_void_p()
    opt = None
    if options is not None:
        opt = FemOptions()
        opt.variant = int(options.get("variant", 0))
        opt.block_elems = int(options.get("block_elems", 0))
        opt.threads = int(options.get("threads", 0))
        opt.formulation = int(options.get("formulation", 0))
    if opt is None:
        st = _lib.fem_mesh_create(_pd(xyz), xyz.shape[0], _pi(tets), tets.shape[0], _pi(mat_id),
                                  prec, reorder, ctypes.byref(h))
    else:
        st = _lib.fem_mesh_create_ex(_pd(xyz), xyz.shape[0], _pi(tets), tets.shape[0],
                                     _pi(mat_id), prec, reorder, ctypes.byref(opt),
                                     ctypes.byref(h))
    _check(st)
    return h


def fem_set_materials(h, materials):
    mats = np.asarray(materials, dtype=np.float64).reshape(-1, 6)
    arr = (FemMaterial * len(mats))(*[FemMaterial(*row) for row in mats])
    _check(_lib.fem_set_materials(h, arr, len(mats)))


def fem_set_boundary(h, faces, hcoef, t_inf, q=None):
    faces = _i(np.asarray(faces).reshape(-1, 3))
    hcoef, t_inf = _d(hcoef), _d(t_inf)
    qq = _d(q) if q is not None else None
    _check(_lib.fem_set_boundary(h, _pi(faces), faces.shape[0], _pd(hcoef), _pd(t_inf),
                                 _pd(qq) if qq is not None else None))


def fem_set_dirichlet(h, nodes, T):
    nodes, T = _i(nodes), _d(T)
    _check(_lib.fem_set_dirichlet(h, _pi(nodes), nodes.shape[0], _pd(T)))


def fem_set_interface(h, faces_a, h_a, faces_b, h_b):
    fa_, fb_ = _i(faces_a).reshape(-1, 3), _i(faces_b).reshape(-1, 3)
    ha, hb = _d(h_a), _d(h_b)
    _check(_lib.fem_set_interface(h, _pi(fa_), fa_.shape[0], _pd(ha), _pi(fb_), fb_.shape[0],
                                  _pd(hb)))


def fem_set_conductivity(h, mat, T, k):
    T, k = _d(T), _d(k)
    _check(_lib.fem_set_conductivity(h, int(mat), T.shape[0], _pd(T), _pd(k)))


def fem_set_temperature(h, T0):
    T0 = _d(T0)
    _check(_lib.fem_set_temperature(h, _pd(T0)))


def fem_stable_dt(h):
    dt = ctypes.c_double()
    _check(_lib.fem_stable_dt(h, ctypes.byref(dt)))
    return dt.value


def fem_step(h, n_steps, dt):
    _check(_lib.fem_step(h, int(n_steps), float(dt)))


def fem_step_profile(h, n_steps, dt):
    """Run n_steps timing each kernel; returns the summed ms per kernel."""
    ms = np.zeros(8)
    n = ctypes.c_int32()
    _check(_lib.fem_step_profile(h, int(n_steps), float(dt), _pd(ms), 8, ctypes.byref(n)))
    return ms[:n.value].copy()


def fem_autotune(h, block_elems, threads=None, steps=20, dt=None):
    """Time each candidate partition (block_elems[i], threads[i]) and keep
    the fastest; returns (best index, ms per step of every candidate).
    dt defaults to 0.9 x the stable step."""
    if dt is None:
        dt = 0.9 * fem_stable_dt(h)
    be = np.ascontiguousarray(block_elems, np.int32)
    th = None if threads is None else np.ascontiguousarray(threads, np.int32)
    if th is not None and th.shape != be.shape:
        raise ValueError("block_elems and threads differ in length")
    ms = np.zeros(be.shape[0])
    best = ctypes.c_int32(-1)
    _check(_lib.fem_autotune(h, _pi(be), None if th is None else _pi(th), be.shape[0], int(steps),
                             float(dt), ctypes.byref(best), _pd(ms)))
    return best.value, ms


def fem_get_temperature(h, n_nodes, out=None):
    out = np.empty(n_nodes) if out is None else out
    p, _keep = _host_ptr(out, n_nodes, True)
    _check(_lib.fem_get_temperature(h, p))
    return out


def fem_get_enthalpy(h, n_nodes, out=None):
    out = np.empty(n_nodes) if out is None else out
    p, _keep = _host_ptr(out, n_nodes, True)
    _check(_lib.fem_get_enthalpy(h, p))
    return out


def fem_get_energy(h):
    out = np.zeros(4)
    _check(_lib.fem_get_energy(h, _pd(out)))
    return out


def fem_set_stream(h, stream):
    _check(_lib.fem_set_stream(h, ctypes.c_void_p(int(stream) if stream else 0)))


def fem_get_state(h, n_nodes, out=None):
    out = np.empty(n_nodes) if out is None else out
    p, _keep = _host_ptr(out, n_nodes, True)
    step = ctypes.c_int64()
    t = ctypes.c_double()
    _check(_lib.fem_get_state(h, p, ctypes.byref(step), ctypes.byref(t)))
    return out, step.value, t.value


def fem_set_state(h, n_nodes, E, step=0, t=0.0):
    p, _keep = _host_ptr(E, n_nodes, False)
    _check(_lib.fem_set_state(h, p, int(step), float(t)))


def fem_set_state_async(h, n_nodes, E, step=0, t=0.0):
    """Enqueue a state upload (see fem.h); E (float64, or float32 for the
    _f32 call) must stay alive and unchanged until fem_sync.  Returns the
    buffer to keep alive."""
    f32 = _is_f32(E)
    p, keep = _host_ptr(E, n_nodes, False, f32)
    fn = _lib.fem_set_state_async_f32 if f32 else _lib.fem_set_state_async
    _check(fn(h, p, int(step), float(t)))
    return keep


def fem_get_temperature_async(h, n_nodes, out):
    """Enqueue T(E) and its copy into `out` (float64, or float32 for the
    _f32 call; valid after fem_sync).  Returns the buffer to keep alive."""
    f32 = _is_f32(out)
    p, keep = _host_ptr(out, n_nodes, True, f32)
    fn = _lib.fem_get_temperature_async_f32 if f32 else _lib.fem_get_temperature_async
    _check(fn(h, p))
    return keep


def fem_sync(h):
    _check(_lib.fem_sync(h))


def fem_mesh_info(h):
    info = FemInfo()
    _check(_lib.fem_mesh_info(h, ctypes.byref(info)))
    return info.as_dict()


def fem_rcm_order(n_nodes, tets):
    tets = _i(tets)
    perm = np.empty(n_nodes, np.int32)
    b0, b1 = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.fem_rcm_order(n_nodes, _pi(tets), tets.shape[0], _pi(perm), ctypes.byref(b0),
                              ctypes.byref(b1)))
    return perm, b0.value, b1.value


_PLAN_TYPES = {0: np.int32, 1: np.int32, 2: np.int32, 3: np.int32, 4: np.int32, 5: np.int32,
               6: np.int32, 7: np.int32, 8: np.uint16, 9: np.int32, 10: np.int32, 11: np.int32,
               12: np.int32, 13: np.int32, 14: np.int32, 15: np.int32}
PLAN_ARRAYS = {"node_new": 0, "blocks": 1, "elem_order": 2, "face_order": 3, "copy_node": 4,
               "sh_ptr": 5, "sh_copy": 6, "grp": 7, "sched": 8, "elem_nodes": 9,
               "face_nodes": 10, "copy_pos": 11, "block_inst": 12, "inst_block_start": 13,
               "inst_order": 14, "if_sister": 15}


def fem_plan_array(h, which):
    w = PLAN_ARRAYS[which] if isinstance(which, str) else int(which)
    p = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(_lib.fem_plan_array(h, w, ctypes.byref(p), ctypes.byref(n)))
    dt = np.dtype(_PLAN_TYPES[w])
    if n.value == 0:
        return np.zeros(0, dt)
    buf = (ctypes.c_char * (n.value * dt.itemsize)).from_address(p.value)
    return np.frombuffer(buf, dtype=dt).copy()


def fem_energy_sums_noalloc(prec, E, C, Lc, phase, ranges, n_nodes, out, stream=0):
    """Device-pointer call (integers from e.g. ``tensor.data_ptr()``); see
    include/fem.h.  Allocates nothing; asynchronous on ``stream``."""
    _check(_lib.fem_energy_sums_noalloc(
        int(prec), ctypes.c_void_p(E), ctypes.c_void_p(C), ctypes.c_void_p(Lc),
        ctypes.c_void_p(phase), ctypes.c_void_p(ranges), int(n_nodes), ctypes.c_void_p(out),
        ctypes.c_void_p(int(stream) if stream else 0)))


def fem_batch_create(parts):
    arr = (ctypes.c_void_p * len(parts))(*[p for p in parts])
    out = ctypes.c_void_p()
    _check(_lib.fem_batch_create(arr, len(parts), ctypes.byref(out)))
    return out


def fem_instance_stable_dt(h, n_inst):
    out = np.zeros(n_inst)
    _check(_lib.fem_instance_stable_dt(h, _pd(out)))
    return out


def fem_set_instance_dt(h, dt):
    dt = _d(dt)
    _check(_lib.fem_set_instance_dt(h, _pd(dt)))


def fem_advance(h, t_end):
    _check(_lib.fem_advance(h, float(t_end)))


def fem_get_instance_times(h, n_inst):
    t = np.zeros(n_inst)
    n = np.zeros(n_inst, np.int64)
    _check(_lib.fem_get_instance_times(h, _pd(t), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return t, n


def fem_get_instance_energy(h, inst):
    out = np.zeros(4)
    _check(_lib.fem_get_instance_energy(h, int(inst), _pd(out)))
    return out


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def torch_allocator():
    """(alloc, free) callbacks over PyTorch's CUDA caching allocator, for
    fem_set_allocator; keep them referenced while the mesh lives."""
    import torch

    def alloc(n, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(n))
        except RuntimeError:   # out of memory: the library reports FEM_ENOMEM
            return None

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


def fem_set_allocator(h, alloc_cb=None, free_cb=None):
    _check(_lib.fem_set_allocator(h, ctypes.cast(alloc_cb, ctypes.c_void_p) if alloc_cb else None,
                                  ctypes.cast(free_cb, ctypes.c_void_p) if free_cb else None, None))


def fem_last_error():
    return _lib.fem_last_error().decode()


def fem_mesh_destroy(h):
    _lib.fem_mesh_destroy(h)


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class Mesh:
    """One libfem mesh handle built from a ``meshgen.Problem``-like object."""

    def __init__(self, prob, precision="fp64", reorder=1, variant="block", block_elems=0,
                 threads=0, faces=True, dirichlet=True, set_temperature=True,
                 formulation="enthalpy", allocator=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        form = FORMULATIONS[formulation] if isinstance(formulation, str) else int(formulation)
        self.n_nodes = int(prob.xyz.shape[0])
        self.n_tets = int(prob.tets.shape[0])
        self._inflight = []   # host buffers of asynchronous calls, until sync()
        self.h = fem_mesh_create(prob.xyz, prob.tets, prob.mat, prec, reorder,
                                 {"variant": var, "block_elems": block_elems, "threads": threads,
                                  "formulation": form})
        self._alloc_cbs = None
        try:
            if allocator == "torch":   # device memory from PyTorch's caching allocator
                self._alloc_cbs = torch_allocator()
                fem_set_allocator(self.h, *self._alloc_cbs)
            fem_set_materials(self.h, prob.materials)
            if faces and prob.faces.shape[0] > 0:
                fem_set_boundary(self.h, prob.faces, prob.h, prob.t_inf, prob.q)
            if dirichlet and prob.dir_nodes.shape[0] > 0:
                fem_set_dirichlet(self.h, prob.dir_nodes, prob.dir_T)
            for mt, Tk, kk in getattr(prob, "k_tables", ()):
                fem_set_conductivity(self.h, mt, Tk, kk)
            ia = getattr(prob, "iface_a", None)
            if faces and ia is not None and ia.shape[0] > 0:
                fem_set_interface(self.h, prob.iface_a, prob.h_ia, prob.iface_b, prob.h_ib)
            if set_temperature:
                fem_set_temperature(self.h, prob.T0)
        except Exception:
            fem_mesh_destroy(self.h)
            self.h = None
            raise

    def close(self):
        if self.h:
            fem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stable_dt(self):
        return fem_stable_dt(self.h)

    def step(self, n, dt):
        fem_step(self.h, n, dt)

    def step_profile(self, n, dt):
        return fem_step_profile(self.h, n, dt)

    def autotune(self, block_elems, threads=None, steps=20, dt=None):
        return fem_autotune(self.h, block_elems, threads, steps, dt)

    def set_temperature(self, T0):
        fem_set_temperature(self.h, T0)

    def temperature(self, out=None):
        return fem_get_temperature(self.h, self.n_nodes, out)

    def enthalpy(self, out=None):
        return fem_get_enthalpy(self.h, self.n_nodes, out)

    def energy(self):
        return fem_get_energy(self.h)

    def state(self, out=None):
        return fem_get_state(self.h, self.n_nodes, out)

    def set_state(self, E, step=0, t=0.0):
        fem_set_state(self.h, self.n_nodes, E, step, t)

    def set_stream(self, stream):
        fem_set_stream(self.h, stream)

    def set_state_async(self, E, step=0, t=0.0):
        self._inflight.append(fem_set_state_async(self.h, self.n_nodes, E, step, t))

    def temperature_async(self, out):
        self._inflight.append(fem_get_temperature_async(self.h, self.n_nodes, out))
        return out

    def sync(self):
        try:
            fem_sync(self.h)
        finally:
            self._inflight.clear()

    def info(self):
        return fem_mesh_info(self.h)

    def plan(self, which):
        return fem_plan_array(self.h, which)


class Batch(Mesh):
    """A batch of independent meshes (fem_batch_create) built from several
    ``meshgen.Problem``-like objects; the parts are released once copied."""

    def __init__(self, probs, precision="fp32", reorder=1, block_elems=0, threads=0,
                 formulation="enthalpy", allocator=None):
        parts = []
        self._inflight = []
        try:
            for p in probs:
                parts.append(Mesh(p, precision, reorder=reorder, variant="block",
                                  block_elems=block_elems, threads=threads,
                                  formulation=formulation))
            self.h = fem_batch_create([q.h for q in parts])
            self._alloc_cbs = None
            if allocator == "torch":
                self._alloc_cbs = torch_allocator()
                fem_set_allocator(self.h, *self._alloc_cbs)
        finally:
            for q in parts:
                q.close()
        self.n_inst = len(parts)
        self.node_start = np.cumsum([0] + [int(p.xyz.shape[0]) for p in probs])
        self.n_nodes = int(self.node_start[-1])
        self.n_tets = int(sum(int(p.tets.shape[0]) for p in probs))

    def instance_stable_dt(self):
        return fem_instance_stable_dt(self.h, self.n_inst)

    def set_instance_dt(self, dt):
        fem_set_instance_dt(self.h, dt)

    def advance(self, t_end):
        fem_advance(self.h, t_end)

    def instance_times(self):
        return fem_get_instance_times(self.h, self.n_inst)

    def instance_energy(self, i):
        return fem_get_instance_energy(self.h, i)

    def instance_temperature(self, i, T=None):
        T = self.temperature() if T is None else T
        return T[self.node_start[i]:self.node_start[i + 1]]


# ---------------------------------------------------------------------------
# Learned surrogate (fem_surrogate_*): device arrays are passed as pointers
# (e.g. torch.Tensor.data_ptr()), FP32, in the surrogate's node order.
# ---------------------------------------------------------------------------

def _dptr(buf):
    return ctypes.c_void_p(buf if isinstance(buf, int) else buf.data_ptr())


class Surrogate:
    """One surrogate on a Mesh or Batch (fem_surrogate_create).  dt: the
    mesh's explicit step (ignored for a batch)."""

    def __init__(self, mesh, dt=0.0):
        h = ctypes.c_void_p()
        _check(_lib.fem_surrogate_create(mesh.h, float(dt), ctypes.byref(h)))
        self.h = h
        self.mesh = mesh
        n, e, q = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.fem_surrogate_info(self.h, ctypes.byref(n), ctypes.byref(e), ctypes.byref(q)))
        self.n_nodes, self.n_edges, self.n_params = n.value, e.value, q.value

    def close(self):
        if getattr(self, "h", None):
            _lib.fem_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def order(self):
        out = np.zeros(self.n_nodes, np.int32)
        _check(_lib.fem_surrogate_order(self.h, _pi(out)))
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        _check(_lib.fem_surrogate_set_params(self.h, ctypes.c_void_p(th.ctypes.data), th.size))

    def params(self):
        th = np.zeros(self.n_params, np.float32)
        _check(_lib.fem_surrogate_get_params(self.h, ctypes.c_void_p(th.ctypes.data), th.size))
        return th

    def read_state(self, E_dev):
        _check(_lib.fem_surrogate_read_state(self.h, _dptr(E_dev)))

    def write_state(self, E_dev):
        _check(_lib.fem_surrogate_write_state(self.h, _dptr(E_dev)))

    def predict(self, E_in, E_out):
        _check(_lib.fem_surrogate_predict(self.h, _dptr(E_in), _dptr(E_out)))

    def train_step(self, E_in, E_star, lr, want_loss=True):
        loss = ctypes.c_double(float("nan"))
        _check(_lib.fem_surrogate_train_step(self.h, _dptr(E_in), _dptr(E_star), float(lr),
                                             ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def accumulate(self, E_in, E_star, want_loss=False):
        loss = ctypes.c_double(float("nan"))
        _check(_lib.fem_surrogate_accumulate(self.h, _dptr(E_in), _dptr(E_star),
                                             ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def apply(self, lr):
        _check(_lib.fem_surrogate_apply(self.h, float(lr)))

    def advance(self, n_macro):
        _check(_lib.fem_surrogate_advance(self.h, int(n_macro)))

    def solve(self, n_macro, judge_every, tol_K):
        """Hybrid stepping (fem_surrogate_solve): returns (macro steps by the
        surrogate, by the solver, failed judgements, largest judged
        difference in K)."""
        st = (ctypes.c_int64 * 3)()
        err = ctypes.c_double(0.0)
        _check(_lib.fem_surrogate_solve(self.h, int(n_macro), int(judge_every), float(tol_K),
                                        st, ctypes.byref(err)))
        return int(st[0]), int(st[1]), int(st[2]), float(err.value)

    def profile(self, n_macro):
        """Summed device ms of each forward kernel over n_macro passes
        (fem_surrogate_profile)."""
        out = np.zeros(5)
        _check(_lib.fem_surrogate_profile(self.h, int(n_macro), _pd(out)))
        return out

    def debug(self, which, layer=0):
        n = self.n_nodes
        shapes = {0: (np.uint16, (n, 16)), 1: (np.uint16, (n, 64)), 2: (np.uint16, (n, 32)),
                  3: (np.uint16, (n, 32)), 4: (np.uint16, (n, 64)), 5: (np.float32, (n, 64)),
                  6: (np.float32, (n,)), 7: (np.float32, (self.n_params,)),
                  8: (np.float32, (n, 5))}
        if which == 9:
            buf = np.zeros(n + 1 + 2 * self.n_edges, np.int32)
            _check(_lib.fem_surrogate_debug(self.h, 9, 0, ctypes.c_void_p(buf.ctypes.data)))
            rowptr, col = buf[:n + 1], buf[n + 1:n + 1 + self.n_edges]
            w = buf[n + 1 + self.n_edges:].view(np.float32)
            return rowptr, col, w
        dt, shape = shapes[which]
        out = np.zeros(shape, dt)
        _check(_lib.fem_surrogate_debug(self.h, int(which), int(layer), ctypes.c_void_p(out.ctypes.data)))
        if dt == np.uint16:
            out = (out.astype(np.uint32) << 16).view(np.float32)
        return out
