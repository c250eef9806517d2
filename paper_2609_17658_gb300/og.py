"""Thin ctypes binding of the C-ABI in include/og.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of its own: arrays are checked for dtype/shape/contiguity, their
pointers are passed through, and a negative status raises OGError with the
library's message.  Host arrays are numpy; device arrays are torch CUDA
tensors (the OG_DEVICE_PTRS flag is then set for the call).

The shared library must have been built (``paper_2609_17658_gb300.build``);
a missing library raises immediately -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

OG_OK = 0
OG_PENDING = 1
OG_ERR_ARG = -1
OG_ERR_OOM = -2
OG_ERR_CUDA = -3
OG_ERR_TIMEOUT = -4
OG_ERR_BUDGET = -5
OG_ERR_OVERFLOW = -6
OG_ERR_STATE = -7
OG_ERR_CANCELLED = -8

OG_OPEN_BH = 0
OG_OPEN_REL = 1
OG_DEVICE_PTRS = 1
OG_DEBUG_DUMP_LISTS = 2

(OG_F_SKEY, OG_F_PERM, OG_F_SPOS, OG_F_LEVEL, OG_F_NBEG, OG_F_NEND, OG_F_PARENT, OG_F_CBEG,
 OG_F_CCNT, OG_F_CHILD, OG_F_MASS, OG_F_COM, OG_F_NEXTNODE, OG_F_SIBLING, OG_F_PNEXT,
 OG_F_GBEG, OG_F_GEND, OG_F_GBOX, OG_F_LISTS, OG_F_EXTENT, OG_F_MSUM) = range(21)


class OGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"og status {status}: {msg}")
        self.status = status


class og_params(C.Structure):
    _fields_ = [("box", C.c_double), ("G", C.c_double), ("eps", C.c_double),
                ("r_s", C.c_double), ("rcut_over_rs", C.c_double), ("theta", C.c_double),
                ("alpha", C.c_double), ("theta_first_pass", C.c_double),
                ("opening", C.c_int32), ("leaf_max", C.c_int32), ("group_max", C.c_int32),
                ("flags", C.c_int32), ("walk_warps", C.c_int32), ("walk_chunk", C.c_int32)]


class og_tree_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nodes", C.c_int64), ("children", C.c_int64),
                ("groups", C.c_int64), ("list_entries", C.c_int64),
                ("interactions", C.c_int64), ("interactions_last_pass", C.c_int64),
                ("ms_build", C.c_double), ("ms_force", C.c_double), ("ms_walk", C.c_double),
                ("group_max", C.c_int32), ("walk_warps", C.c_int32), ("walk_chunk", C.c_int32),
                ("pad", C.c_int32), ("ms_pm", C.c_double), ("ms_sph", C.c_double)]


class og_box(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("mass", C.c_void_p), ("n", C.c_int64),
                ("params", og_params), ("a_old", C.c_void_p), ("acc", C.c_void_p),
                ("n_pp", C.c_void_p), ("n_pn", C.c_void_p)]


class og_batch_info(C.Structure):
    _fields_ = [("boxes", C.c_int64), ("particles", C.c_int64), ("groups", C.c_int64),
                ("interactions", C.c_int64), ("ms_total", C.c_double), ("ms_build", C.c_double),
                ("ms_walk", C.c_double)]


class og_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p), ("mass", C.c_void_p),
                ("params", og_params), ("nsteps", C.c_int32), ("dt_kick", C.c_double),
                ("dt_drift", C.c_double), ("acc_out", C.c_void_p), ("pos_out", C.c_void_p)]


class og_result(C.Structure):
    _fields_ = [("n", C.c_int64), ("steps", C.c_int64), ("rebuilds", C.c_int64),
                ("refits", C.c_int64), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libog.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_2609_17658_gb300.build)")
        L = C.CDLL(path)
        P, i64, sz = C.c_void_p, C.c_int64, C.c_size_t
        L.og_create.argtypes = [C.POINTER(P), C.c_int, sz]
        L.og_destroy.argtypes = [P]
        L.og_set_stream.argtypes = [P, P]
        L.og_params_default.argtypes = [C.POINTER(og_params)]
        L.og_tree_build.argtypes = [P, P, P, i64, C.POINTER(og_params), C.POINTER(P)]
        L.og_tree_refit.argtypes = [P, P]
        L.og_tree_force.argtypes = [P, P, P, P, P]
        L.og_tree_info_get.argtypes = [P, C.POINTER(og_tree_info)]
        L.og_tree_export.argtypes = [P, C.c_int, P, sz]
        L.og_tree_free.argtypes = [P]
        L.og_last_error.restype = C.c_char_p
        L.og_kernel_launches.restype = C.c_int64
        L.og_device_code_version.argtypes = [C.POINTER(C.c_int32)]
        L.og_device_code_version.restype = C.c_int
        L.og_debug_fail_allocations.argtypes = [C.c_int32, C.c_int32]
        L.og_debug_fail_allocations.restype = C.c_int
        L.og_debug_scan_wait_timeout.argtypes = [P, i64]
        L.og_debug_scan_wait_timeout.restype = C.c_int
        L.og_serve_cancel.argtypes = [P, C.c_uint64]
        L.og_serve_cancel.restype = C.c_int
        L.og_sort_keys_noalloc.argtypes = [P, P, P, i64, P]
        L.og_batch_force.argtypes = [P, i64, C.POINTER(og_box), C.POINTER(og_batch_info)]
        L.og_batch_force.restype = C.c_int
        L.og_serve_submit.argtypes = [P, C.POINTER(og_request), C.POINTER(C.c_uint64)]
        L.og_serve_submit.restype = C.c_int
        L.og_serve_poll.argtypes = [P, C.c_uint64, C.POINTER(og_result), C.c_int]
        L.og_serve_poll.restype = C.c_int
        L.og_serve_request_bytes.argtypes = [i64]
        L.og_serve_request_bytes.restype = C.c_size_t
        L.og_sort_keys_noalloc.restype = C.c_int
        L.og_tree_force_pot.argtypes = [P, P, P, P, P, P]
        L.og_tree_force_f64.argtypes = [P, P, P, P, P]
        L.og_tree_force_f64.restype = C.c_int
        L.og_tree_pm_force.argtypes = [P, C.c_int32, P]
        L.og_tree_pm_force.restype = C.c_int
        L.og_tree_sph_density.argtypes = [P, P, P, P]
        L.og_tree_sph_density.restype = C.c_int
        L.og_tree_sph_smoothing.argtypes = [P, C.c_double, C.c_double, C.c_int32, P, P, P,
                                            C.POINTER(C.c_int32)]
        L.og_tree_sph_smoothing.restype = C.c_int
        L.og_tree_force_pot.restype = C.c_int
        L.og_kdk_run.argtypes = [P, i64, P, P, P, C.POINTER(og_params), C.POINTER(og_kdk_params), P, P,
                                 C.POINTER(og_kdk_stats)]
        L.og_kdk_run.restype = C.c_int
        L.og_tree_force_active.argtypes = [P, P, P, P, P, P, C.POINTER(C.c_int64)]
        L.og_tree_force_active.restype = C.c_int
        L.og_tune_group_max.argtypes = [P, P, P, i64, C.POINTER(og_params), C.POINTER(C.c_int32)]
        L.og_tune_walk.argtypes = [P, P, P, i64, C.POINTER(og_params), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.og_tune_save.argtypes = [P, C.c_char_p]
        L.og_tune_load.argtypes = [P, C.c_char_p]
        L.og_measure_fp32_peak.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        for name in ("og_tune_group_max", "og_tune_walk", "og_tune_save", "og_tune_load",
                     "og_measure_fp32_peak"):
            getattr(L, name).restype = C.c_int
        for name in ("og_create", "og_destroy", "og_set_stream", "og_params_default",
                     "og_tree_build", "og_tree_refit", "og_tree_force", "og_tree_info_get",
                     "og_tree_export", "og_tree_free"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def og_last_error() -> str:
    return lib().og_last_error().decode(errors="replace")


def og_kernel_launches() -> int:
    return int(lib().og_kernel_launches())


def og_debug_fail_allocations(count: int, skip: int = 0) -> None:
    """Let the library's next ``skip`` device allocations through and make
    the ``count`` after them fail (tests of error handling; see
    include/og.h).  count = 0 clears it."""
    _check(lib().og_debug_fail_allocations(int(skip), int(count)))


def og_debug_scan_wait_timeout(ctx, n: int) -> None:
    """Run the one-kernel scan with its first tile never taken, so that a
    bounded wait runs out (tests of error handling; see include/og.h); raises
    OGError with OG_ERR_TIMEOUT."""
    _check(lib().og_debug_scan_wait_timeout(ctx, int(n)))


def og_serve_cancel(ctx, ticket: int) -> None:
    """Cancel a queued or running served request (see include/og.h)."""
    _check(lib().og_serve_cancel(ctx, C.c_uint64(ticket)))


def og_device_code_version() -> int:
    """Compute capability of the device code the current GPU runs (103: sm_103a)."""
    v = C.c_int32()
    _check(lib().og_device_code_version(C.byref(v)))
    return int(v.value)


def _check(st: int):
    if st < 0:
        raise OGError(st, og_last_error())
    return st


def params_from_dict(p: dict, flags: int = 0) -> og_params:
    q = og_params()
    _check(lib().og_params_default(C.byref(q)))
    for k in ("box", "G", "eps", "r_s", "rcut_over_rs", "theta", "alpha", "theta_first_pass"):
        if k in p:
            setattr(q, k, float(p[k]))
    for k in ("opening", "leaf_max", "group_max", "flags", "walk_warps", "walk_chunk"):
        if k in p:
            setattr(q, k, int(p[k]))
    q.flags = int(q.flags) | int(flags)
    return q


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _host_ptr(a: np.ndarray, dtype, shape_tail=()):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    if shape_tail and a.shape[1:] != shape_tail:
        raise ValueError(f"expected shape (N, {shape_tail})")
    return a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t, dtype_name: str):
    """Device address of a contiguous CUDA tensor on the current device.  A CPU
    tensor, or one on another GPU, is rejected here: its address would reach
    the kernels as if it were this device's memory."""
    if not _is_torch_cuda(t):
        raise TypeError(f"expected a CUDA tensor of {dtype_name}, got a host object")
    if str(t.dtype) != f"torch.{dtype_name}" or not t.is_contiguous():
        raise TypeError(f"expected a contiguous CUDA tensor of {dtype_name}")
    import torch
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError(f"tensor on cuda:{t.device.index}, but the current device is cuda:{cur}")
    return C.c_void_p(t.data_ptr())


# ---- C entry points -------------------------------------------------------

def og_create(device: int = 0, hbm_budget_bytes: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().og_create(C.byref(h), int(device), int(hbm_budget_bytes)))
    return h


def og_destroy(ctx) -> None:
    _check(lib().og_destroy(ctx))


def og_set_stream(ctx, stream_handle: int | None) -> None:
    """Order the context's work on a CUDA stream handle (e.g. torch's cuda_stream)."""
    _check(lib().og_set_stream(ctx, C.c_void_p(stream_handle) if stream_handle else None))


def _inputs(pos, mass, params: dict):
    dev = _is_torch_cuda(pos)
    if dev:
        pp, mp = _dev_ptr(pos, "float64"), _dev_ptr(mass, "float64")
    else:
        pp, mp = _host_ptr(pos, np.float64, (3,)), _host_ptr(mass, np.float64)
    n = int(pos.shape[0])
    if int(mass.shape[0]) != n:
        raise ValueError("mass and pos lengths differ")
    prm = params_from_dict(params, OG_DEVICE_PTRS if dev else 0)
    if not dev:
        prm.flags = int(prm.flags) & ~OG_DEVICE_PTRS
    return pp, mp, n, prm


def og_tree_build(ctx, pos, mass, params: dict) -> C.c_void_p:
    """pos: float64 [N,3], mass: float64 [N] (numpy host or torch CUDA)."""
    pp, mp, n, prm = _inputs(pos, mass, params)
    h = C.c_void_p()
    _check(lib().og_tree_build(ctx, pp, mp, n, C.byref(prm), C.byref(h)))
    return h


def og_tune_group_max(ctx, pos, mass, params: dict) -> int:
    """The measured group size for inputs of this kind (see include/og.h)."""
    pp, mp, n, prm = _inputs(pos, mass, params)
    g = C.c_int32()
    _check(lib().og_tune_group_max(ctx, pp, mp, n, C.byref(prm), C.byref(g)))
    return int(g.value)


def og_tune_walk(ctx, pos, mass, params: dict) -> dict:
    """The measured group size and walk launch shape for inputs of this kind."""
    pp, mp, n, prm = _inputs(pos, mass, params)
    g, w, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().og_tune_walk(ctx, pp, mp, n, C.byref(prm), C.byref(g), C.byref(w), C.byref(c)))
    return {"group_max": int(g.value), "walk_warps": int(w.value), "walk_chunk": int(c.value)}


def og_tune_save(ctx, path: str) -> None:
    _check(lib().og_tune_save(ctx, os.fsencode(path)))


def og_tune_load(ctx, path: str) -> None:
    _check(lib().og_tune_load(ctx, os.fsencode(path)))


def og_measure_fp32_peak(ctx) -> dict:
    """Measured FP32 FMA and f32x2 FMA rates of the device, TFLOP/s."""
    f1, f2 = C.c_double(0.0), C.c_double(0.0)
    _check(lib().og_measure_fp32_peak(ctx, C.byref(f1), C.byref(f2)))
    return {"fma": f1.value, "fma2": f2.value}


def og_tree_force(tree, acc, a_old=None, n_pp=None, n_pn=None) -> None:
    """Fill acc (float32 [N,3]) and optionally n_pp, n_pn (uint32 [N] / int32 CUDA)."""
    if _is_torch_cuda(acc):
        ap = _dev_ptr(acc, "float32")
        op = None if a_old is None else _dev_ptr(a_old, "float32")
        pp = None if n_pp is None else _dev_ptr(n_pp, "int32")
        np_ = None if n_pn is None else _dev_ptr(n_pn, "int32")
    else:
        ap = _host_ptr(acc, np.float32, (3,))
        op = None if a_old is None else _host_ptr(a_old, np.float32, (3,))
        pp = None if n_pp is None else _host_ptr(n_pp, np.uint32)
        np_ = None if n_pn is None else _host_ptr(n_pn, np.uint32)
    _check(lib().og_tree_force(tree, op, ap, pp, np_))


def og_tree_pm_force(tree, mesh: int, acc) -> None:
    """Long-range particle-mesh acceleration, acc float32 [N,3] (caller order)."""
    ap = _dev_ptr(acc, "float32") if _is_torch_cuda(acc) else _host_ptr(acc, np.float32, (3,))
    _check(lib().og_tree_pm_force(tree, int(mesh), ap))


def og_tree_sph_density(tree, h, rho, n_ngb=None) -> None:
    """SPH density at the smoothing lengths h float32 [N]: rho float32 [N], n_ngb uint32 [N]."""
    if _is_torch_cuda(rho):
        hp = _dev_ptr(h, "float32")
        rp = _dev_ptr(rho, "float32")
        cp = None if n_ngb is None else _dev_ptr(n_ngb, "int32")
    else:
        hp = _host_ptr(h, np.float32)
        rp = _host_ptr(rho, np.float32)
        cp = None if n_ngb is None else _host_ptr(n_ngb, np.uint32)
    _check(lib().og_tree_sph_density(tree, hp, rp, cp))


def og_tree_sph_smoothing(tree, n_target: float, tol: float, max_iter: int, h, rho, n_ngb=None) -> int:
    """Smoothing lengths from (4 pi / 3) h^3 rho = N m, h float32 [N] in/out; returns the iterations."""
    if _is_torch_cuda(rho):
        hp = _dev_ptr(h, "float32")
        rp = _dev_ptr(rho, "float32")
        cp = None if n_ngb is None else _dev_ptr(n_ngb, "int32")
    else:
        hp = _host_ptr(h, np.float32)
        rp = _host_ptr(rho, np.float32)
        cp = None if n_ngb is None else _host_ptr(n_ngb, np.uint32)
    it = C.c_int32(0)
    _check(lib().og_tree_sph_smoothing(tree, float(n_target), float(tol), int(max_iter), hp, rp, cp,
                                       C.byref(it)))
    return int(it.value)


def og_tree_force_f64(tree, acc, a_old=None, n_pp=None, n_pn=None) -> None:
    """og_tree_force with acc float64 [N,3] (scaled to G M / L^2 in FP64)."""
    if _is_torch_cuda(acc):
        ap = _dev_ptr(acc, "float64")
        op = None if a_old is None else _dev_ptr(a_old, "float32")
        pp = None if n_pp is None else _dev_ptr(n_pp, "int32")
        np_ = None if n_pn is None else _dev_ptr(n_pn, "int32")
    else:
        ap = _host_ptr(acc, np.float64, (3,))
        op = None if a_old is None else _host_ptr(a_old, np.float32, (3,))
        pp = None if n_pp is None else _host_ptr(n_pp, np.uint32)
        np_ = None if n_pn is None else _host_ptr(n_pn, np.uint32)
    _check(lib().og_tree_force_f64(tree, op, ap, pp, np_))


def og_tree_force_pot(tree, acc, pot, a_old=None, n_pp=None, n_pn=None) -> None:
    """og_tree_force plus the short-range potential (pot: float32 [N])."""
    if _is_torch_cuda(acc):
        ap, pp_ = _dev_ptr(acc, "float32"), _dev_ptr(pot, "float32")
        op = None if a_old is None else _dev_ptr(a_old, "float32")
        cp = None if n_pp is None else _dev_ptr(n_pp, "int32")
        np_ = None if n_pn is None else _dev_ptr(n_pn, "int32")
    else:
        ap, pp_ = _host_ptr(acc, np.float32, (3,)), _host_ptr(pot, np.float32)
        op = None if a_old is None else _host_ptr(a_old, np.float32, (3,))
        cp = None if n_pp is None else _host_ptr(n_pp, np.uint32)
        np_ = None if n_pn is None else _host_ptr(n_pn, np.uint32)
    _check(lib().og_tree_force_pot(tree, op, ap, pp_, cp, np_))


def og_tree_force_active(tree, active, acc, a_old=None, n_pp=None, n_pn=None) -> int:
    """Forces on the active particles only (active: uint8 [N], nonzero = active);
    the other entries of acc / n_pp / n_pn are left as they were.  Returns the
    number of groups walked."""
    g = C.c_int64(0)
    if _is_torch_cuda(acc):
        act = _dev_ptr(active, "uint8")
        ap = _dev_ptr(acc, "float32")
        op = None if a_old is None else _dev_ptr(a_old, "float32")
        pp = None if n_pp is None else _dev_ptr(n_pp, "int32")
        np_ = None if n_pn is None else _dev_ptr(n_pn, "int32")
    else:
        act = _host_ptr(active, np.uint8)
        ap = _host_ptr(acc, np.float32, (3,))
        op = None if a_old is None else _host_ptr(a_old, np.float32, (3,))
        pp = None if n_pp is None else _host_ptr(n_pp, np.uint32)
        np_ = None if n_pn is None else _host_ptr(n_pn, np.uint32)
    _check(lib().og_tree_force_active(tree, act, op, ap, pp, np_, C.byref(g)))
    return int(g.value)


class og_kdk_params(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("eta", C.c_double), ("max_bin", C.c_int32),
                ("nsteps", C.c_int32), ("rebuild_every", C.c_int32), ("pad", C.c_int32)]


class og_kdk_stats(C.Structure):
    _fields_ = [("ticks", C.c_int64), ("forces", C.c_int64), ("groups_walked", C.c_int64),
                ("interactions", C.c_int64), ("rebuilds", C.c_int64), ("refits", C.c_int64),
                ("ms", C.c_double)]


def og_kdk_run(ctx, pos, vel, mass, params: dict, dt_max: float, eta: float = 0.05,
               max_bin: int = 6, nsteps: int = 1, rebuild_every: int = 1):
    """Integrate (host numpy arrays; pos and vel are updated in place).
    Returns (acc float32 [N,3], bins int32 [N], stats dict)."""
    n = int(pos.shape[0])
    pp = _host_ptr(pos, np.float64, (3,))
    vp = _host_ptr(vel, np.float64, (3,))
    mp = _host_ptr(mass, np.float64)
    prm = params_from_dict(params, 0)
    prm.flags = int(prm.flags) & ~OG_DEVICE_PTRS
    kp = og_kdk_params(dt_max=float(dt_max), eta=float(eta), max_bin=int(max_bin),
                       nsteps=int(nsteps), rebuild_every=int(rebuild_every))
    acc = np.zeros((n, 3), np.float32)
    bins = np.zeros(n, np.int32)
    st = og_kdk_stats()
    _check(lib().og_kdk_run(ctx, n, pp, vp, mp, C.byref(prm), C.byref(kp),
                            acc.ctypes.data_as(C.c_void_p), bins.ctypes.data_as(C.c_void_p),
                            C.byref(st)))
    return acc, bins, {k: getattr(st, k) for k, _ in og_kdk_stats._fields_}


def og_tree_info_get(tree) -> dict:
    info = og_tree_info()
    _check(lib().og_tree_info_get(tree, C.byref(info)))
    return {k: getattr(info, k) for k, _ in og_tree_info._fields_}


_FIELD_SPEC = {
    OG_F_SKEY: ("n", np.uint64, ()), OG_F_PERM: ("n", np.uint32, ()),
    OG_F_SPOS: ("n", np.uint32, "3n"), OG_F_LEVEL: ("nodes", np.uint8, ()),
    OG_F_NBEG: ("nodes", np.uint32, ()), OG_F_NEND: ("nodes", np.uint32, ()),
    OG_F_PARENT: ("nodes", np.int32, ()), OG_F_CBEG: ("nodes", np.uint32, ()),
    OG_F_CCNT: ("nodes", np.uint32, ()), OG_F_CHILD: ("children", np.uint32, ()),
    OG_F_MASS: ("nodes", np.float64, ()), OG_F_COM: ("nodes", np.uint32, (3,)),
    OG_F_NEXTNODE: ("nodes", np.int32, ()), OG_F_SIBLING: ("nodes", np.int32, ()),
    OG_F_PNEXT: ("n", np.int32, ()), OG_F_GBEG: ("groups", np.uint32, ()),
    OG_F_GEND: ("groups", np.uint32, ()), OG_F_GBOX: ("groups", np.uint32, (6,)),
    OG_F_LISTS: ("list_entries", np.uint32, (2,)),
    OG_F_EXTENT: ("nodes", np.uint32, "2x3"),
    OG_F_MSUM: ("nodes", np.float64, (3,)),
}


def og_tree_export(tree, field: int) -> np.ndarray:
    info = og_tree_info_get(tree)
    key, dt, tail = _FIELD_SPEC[field]
    cnt = int(info[key])
    if tail == "3n":
        out = np.zeros((3, cnt), dtype=dt)
    elif tail == "2x3":
        out = np.zeros((2, cnt, 3), dtype=dt)
    else:
        out = np.zeros((cnt,) + tuple(tail), dtype=dt)
    _check(lib().og_tree_export(tree, int(field), out.ctypes.data_as(C.c_void_p), out.nbytes))
    return out


def og_batch_force(ctx, boxes) -> dict:
    """Many independent boxes in one call.  ``boxes``: sequence of dicts with
    keys pos (float64 [n,3]), mass (float64 [n]), params (dict), acc (float32
    [n,3] out) and optionally a_old (float32 [n,3]), n_pp, n_pn (uint32 [n]
    out); numpy host arrays or torch CUDA tensors (all boxes alike)."""
    nb = len(boxes)
    arr = (og_box * nb)()
    dev = _is_torch_cuda(boxes[0]["pos"])
    for k, b in enumerate(boxes):
        x = arr[k]
        if dev:
            x.pos = _dev_ptr(b["pos"], "float64").value
            x.mass = _dev_ptr(b["mass"], "float64").value
            x.acc = _dev_ptr(b["acc"], "float32").value
            x.a_old = _dev_ptr(b["a_old"], "float32").value if b.get("a_old") is not None else None
            x.n_pp = _dev_ptr(b["n_pp"], "int32").value if b.get("n_pp") is not None else None
            x.n_pn = _dev_ptr(b["n_pn"], "int32").value if b.get("n_pn") is not None else None
        else:
            x.pos = _host_ptr(b["pos"], np.float64, (3,)).value
            x.mass = _host_ptr(b["mass"], np.float64).value
            x.acc = _host_ptr(b["acc"], np.float32, (3,)).value
            x.a_old = _host_ptr(b["a_old"], np.float32, (3,)).value if b.get("a_old") is not None else None
            x.n_pp = _host_ptr(b["n_pp"], np.uint32).value if b.get("n_pp") is not None else None
            x.n_pn = _host_ptr(b["n_pn"], np.uint32).value if b.get("n_pn") is not None else None
        x.n = int(b["pos"].shape[0])
        prm = params_from_dict(b["params"], OG_DEVICE_PTRS if dev else 0)
        if not dev:
            prm.flags = int(prm.flags) & ~OG_DEVICE_PTRS
        x.params = prm
    info = og_batch_info()
    _check(lib().og_batch_force(ctx, nb, arr, C.byref(info)))
    return {k: getattr(info, k) for k, _ in og_batch_info._fields_}


def og_serve_submit(ctx, pos, vel, mass, params: dict, nsteps: int = 8, dt_kick: float = 1e-5,
                    dt_drift: float = 1.0, acc_out=None, pos_out=None) -> int:
    """Queue a served request (host numpy arrays; acc_out float32 [n,3] and
    pos_out float64 [n,3] are filled when the request completes and must stay
    alive until og_serve_poll returns it).  Returns the ticket."""
    r = og_request()
    r.n = int(pos.shape[0])
    r.pos = _host_ptr(pos, np.float64, (3,)).value
    r.vel = _host_ptr(vel, np.float64, (3,)).value
    r.mass = _host_ptr(mass, np.float64).value
    prm = params_from_dict(params)
    prm.flags = int(prm.flags) & ~OG_DEVICE_PTRS
    r.params = prm
    r.nsteps = int(nsteps)
    r.dt_kick = float(dt_kick)
    r.dt_drift = float(dt_drift)
    r.acc_out = _host_ptr(acc_out, np.float32, (3,)).value if acc_out is not None else None
    r.pos_out = _host_ptr(pos_out, np.float64, (3,)).value if pos_out is not None else None
    t = C.c_uint64()
    _check(lib().og_serve_submit(ctx, C.byref(r), C.byref(t)))
    return int(t.value)


def og_serve_request_bytes(n: int) -> int:
    return int(lib().og_serve_request_bytes(int(n)))


def og_serve_poll(ctx, ticket: int, timeout_ms: int = -1):
    """(status, result dict or None): OG_OK with the result, or OG_PENDING."""
    res = og_result()
    st = lib().og_serve_poll(ctx, C.c_uint64(ticket), C.byref(res), int(timeout_ms))
    if st == OG_PENDING:
        return st, None
    _check(st)
    return st, {k: getattr(res, k) for k, _ in og_result._fields_}


OG_NOALLOC_MAX_N = 1048576


def og_sort_keys_noalloc(keys_in, keys_out, perm_out, stream_handle: int | None = None) -> None:
    """Sort device keys without any device allocation (see include/og.h).
    keys_in, keys_out: CUDA int64 tensors holding the uint64 key bits;
    perm_out: CUDA int32 tensor.  Queued on ``stream_handle`` (None: default
    stream); synchronise before reading the outputs."""
    n = int(keys_in.shape[0])
    if int(keys_out.shape[0]) != n or int(perm_out.shape[0]) != n:
        raise ValueError("keys_in, keys_out and perm_out lengths differ")
    _check(lib().og_sort_keys_noalloc(_dev_ptr(keys_in, "int64"), _dev_ptr(keys_out, "int64"),
                                      _dev_ptr(perm_out, "int32"), n,
                                      C.c_void_p(stream_handle) if stream_handle else None))


def og_tree_free(tree) -> None:
    _check(lib().og_tree_free(tree))


def og_tree_refit(tree, pos) -> None:
    pp = _dev_ptr(pos, "float64") if _is_torch_cuda(pos) else _host_ptr(pos, np.float64, (3,))
    _check(lib().og_tree_refit(tree, pp))


# ---- convenience wrappers -------------------------------------------------

class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.h = og_create(device, hbm_budget_bytes)
        self._trees = weakref.WeakSet()

    def close(self):
        if self.h is not None:
            for t in list(self._trees):      # a tree must not outlive its context
                t.free()
            og_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree:
    """One system's device-resident tree (og_tree_build / og_tree_force)."""

    def __init__(self, ctx: Context, pos, mass, params: dict):
        self.ctx = ctx
        self.n = int(pos.shape[0])
        self.h = og_tree_build(ctx.h, pos, mass, params)
        ctx._trees.add(self)

    def force(self, a_old=None, counts: bool = True):
        acc = np.zeros((self.n, 3), dtype=np.float32)
        npp = np.zeros(self.n, dtype=np.uint32) if counts else None
        npn = np.zeros(self.n, dtype=np.uint32) if counts else None
        ao = None if a_old is None else np.ascontiguousarray(a_old, dtype=np.float32)
        og_tree_force(self.h, acc, ao, npp, npn)
        return acc, npp, npn

    def pm_force(self, mesh: int):
        """Long-range particle-mesh acceleration float32 [N,3] (og_tree_pm_force)."""
        acc = np.zeros((self.n, 3), dtype=np.float32)
        og_tree_pm_force(self.h, mesh, acc)
        return acc

    def sph_density(self, h):
        """(rho float32 [N], n_ngb uint32 [N]) at the smoothing lengths h (og_tree_sph_density)."""
        rho = np.zeros(self.n, dtype=np.float32)
        cnt = np.zeros(self.n, dtype=np.uint32)
        og_tree_sph_density(self.h, np.ascontiguousarray(h, dtype=np.float32), rho, cnt)
        return rho, cnt

    def sph_smoothing(self, h0, n_target=32.0, tol=0.01, max_iter=100):
        """(h, rho, n_ngb, iterations) of og_tree_sph_smoothing from the guesses h0."""
        h = np.ascontiguousarray(h0, dtype=np.float32).copy()
        rho = np.zeros(self.n, dtype=np.float32)
        cnt = np.zeros(self.n, dtype=np.uint32)
        it = og_tree_sph_smoothing(self.h, n_target, tol, max_iter, h, rho, cnt)
        return h, rho, cnt, it

    def force_pot(self, a_old=None):
        """(acc, n_pp, n_pn, pot) of one force call with the potential output."""
        acc = np.zeros((self.n, 3), dtype=np.float32)
        pot = np.zeros(self.n, dtype=np.float32)
        npp = np.zeros(self.n, dtype=np.uint32)
        npn = np.zeros(self.n, dtype=np.uint32)
        ao = None if a_old is None else np.ascontiguousarray(a_old, dtype=np.float32)
        og_tree_force_pot(self.h, acc, pot, ao, npp, npn)
        return acc, npp, npn, pot

    def refit(self, pos) -> None:
        og_tree_refit(self.h, np.ascontiguousarray(pos, dtype=np.float64) if not _is_torch_cuda(pos) else pos)

    def info(self) -> dict:
        return og_tree_info_get(self.h)

    def export(self, field: int) -> np.ndarray:
        return og_tree_export(self.h, field)

    def free(self):
        if self.h is not None:
            if self.ctx.h is not None:       # else og_destroy has freed it already
                og_tree_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
