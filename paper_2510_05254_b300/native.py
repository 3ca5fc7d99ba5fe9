"""Python binding of libndg (include/ndg.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name; a non-zero status raises
``NdgError`` carrying ndg_last_error().  All computation happens in libndg's CUDA kernels; if
the library cannot be loaded (or built from csrc/ with nvcc), importing this module's functions
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libndg.so")

NDG_OK, NDG_EINVAL, NDG_ENOMEM, NDG_ECUDA, NDG_ENONFINITE, NDG_EAGAIN, NDG_ETIMEOUT, NDG_ESTATE = range(8)
NDG_ADVECTION, NDG_ISO_EULER = 0, 1
NDG_FLUX_UPWIND, NDG_FLUX_LLF = 0, 1
NDG_RK3, NDG_RK4, NDG_RK6 = 3, 4, 6
NDG_F64, NDG_F32, NDG_F64_FF = 0, 1, 2
NDG_LAYOUT_ELEMENT, NDG_LAYOUT_GRID = 0, 1
NDG_KERNEL_AUTO, NDG_KERNEL_LINE, NDG_KERNEL_LINE_VAR = 0, 1, 2
NDG_MASS_LUMPED, NDG_MASS_EXACT = 0, 1
STATUS_NAMES = {0: "NDG_OK", 1: "NDG_EINVAL", 2: "NDG_ENOMEM", 3: "NDG_ECUDA", 4: "NDG_ENONFINITE",
                5: "NDG_EAGAIN", 6: "NDG_ETIMEOUT", 7: "NDG_ESTATE"}


class NdgError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ndg_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("elems", ctypes.c_int * 3),
                ("equation", ctypes.c_int), ("flux", ctypes.c_int), ("dtype", ctypes.c_int),
                ("length", ctypes.c_double * 3), ("velocity", ctypes.c_double * 3),
                ("sound_speed", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("elems_per_block", ctypes.c_int), ("device", ctypes.c_int), ("kernel", ctypes.c_int),
                ("mass", ctypes.c_int)]


class ndg_norms_t(ctypes.Structure):
    _fields_ = [("l2", ctypes.c_double), ("linf", ctypes.c_double), ("integral", ctypes.c_double * 4),
                ("max_speed", ctypes.c_double), ("t", ctypes.c_double), ("steps", ctypes.c_int64),
                ("nonfinite", ctypes.c_int64)]


class ndg_info_t(ctypes.Structure):
    _fields_ = [("nvar", ctypes.c_int), ("nodes_per_elem", ctypes.c_int), ("nelem", ctypes.c_int64),
                ("ndof", ctypes.c_int64), ("state_bytes", ctypes.c_size_t),
                ("device_bytes", ctypes.c_size_t), ("elems_per_block", ctypes.c_int), ("kernel", ctypes.c_int)]


class ndg_solve_stats_t(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("t", ctypes.c_double), ("steps", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.c_void_p
_SIGS = {
    "ndg_config_init": [ctypes.POINTER(ndg_config)],
    "ndg_create": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                   ctypes.POINTER(_P)],
    "ndg_create_ex": [ctypes.POINTER(ndg_config), ctypes.POINTER(_P)],
    "ndg_destroy": [_P],
    "ndg_set_state": [_P, _P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int],
    "ndg_get_state": [_P, _P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int],
    "ndg_step": [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int],
    "ndg_step_split": [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int],
    "ndg_norms": [_P, _P, ctypes.c_int, ctypes.POINTER(ndg_norms_t)],
    "ndg_stable_dt": [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
    "ndg_norms_noalloc": [ctypes.POINTER(ndg_config), _P, _P, ctypes.c_int, _P, _P],
    "ndg_debug_stall_copies": [ctypes.c_int],
    "ndg_node_coords": [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t],
    "ndg_info": [_P, ctypes.POINTER(ndg_info_t)],
    "ndg_lgl": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "ndg_stream": [_P],
    "ndg_synchronize": [_P],
    "ndg_last_error": [],
    "ndg_set_allocator": [ALLOC_FN, FREE_FN, _P],
    "ndg_autotune": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
    "ndg_batch_create": [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)],
    "ndg_batch_step": [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int],
    "ndg_batch_destroy": [_P],
    "ndg_partition_create": [ctypes.POINTER(ndg_config), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_P)],
    "ndg_partition_set_state": [_P, _P, ctypes.c_size_t, ctypes.c_int],
    "ndg_partition_get_state": [_P, _P, ctypes.c_size_t, ctypes.c_int],
    "ndg_partition_step": [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int],
    "ndg_partition_norms": [_P, ctypes.POINTER(ndg_norms_t)],
    "ndg_partition_info": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "ndg_partition_destroy": [_P],
    "ndg_pool_create": [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_P)],
    "ndg_pool_submit": [_P, ctypes.POINTER(ndg_config), _P, ctypes.c_size_t, ctypes.c_int, ctypes.c_double,
                        ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)],
    "ndg_pool_poll": [_P, ctypes.c_uint64, _P, ctypes.c_size_t, ctypes.POINTER(ndg_solve_stats_t),
                      ctypes.c_double],
    "ndg_pool_status": [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t),
                        ctypes.POINTER(ctypes.c_size_t)],
    "ndg_pool_destroy": [_P],
}
_RESTYPES = {"ndg_last_error": ctypes.c_char_p, "ndg_stream": _P}

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libndg.so (building it with nvcc when absent).  Raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                if not build_if_missing:
                    raise OSError(f"{LIB_PATH} is missing")
                from . import build as _build
                _build.build()
            lib = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(lib, name, None)
                if fn is None:
                    continue
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, ctypes.c_int)
            _lib = lib
    return _lib


def exported_symbols():
    return [name for name in _SIGS if getattr(load(), name, None) is not None]


def _call(name, *args):
    fn = getattr(load(), name)
    rc = fn(*args)
    if rc != NDG_OK:
        raise NdgError(rc, name, ndg_last_error())
    return rc


def ndg_last_error() -> str:
    return load().ndg_last_error().decode()


def ndg_config_init() -> ndg_config:
    cfg = ndg_config()
    _call("ndg_config_init", ctypes.byref(cfg))
    return cfg


def ndg_create(dim, degree, elems, equation, flux) -> int:
    h = _P()
    e = (ctypes.c_int * 3)(*(list(elems) + [1] * (3 - len(elems))))
    _call("ndg_create", dim, degree, e, equation, flux, ctypes.byref(h))
    return h.value


def ndg_create_ex(cfg: ndg_config) -> int:
    h = _P()
    _call("ndg_create_ex", ctypes.byref(cfg), ctypes.byref(h))
    return h.value


def ndg_destroy(ctx) -> None:
    _call("ndg_destroy", ctx)


def ndg_set_state(ctx, ptr: int, nbytes: int, on_device: bool, layout: int = NDG_LAYOUT_ELEMENT) -> None:
    _call("ndg_set_state", ctx, ptr, nbytes, int(on_device), layout)


def ndg_get_state(ctx, ptr: int, nbytes: int, on_device: bool, layout: int = NDG_LAYOUT_ELEMENT) -> None:
    _call("ndg_get_state", ctx, ptr, nbytes, int(on_device), layout)


def ndg_step(ctx, dt: float, nsteps: int, rk: int = NDG_RK4) -> None:
    _call("ndg_step", ctx, float(dt), int(nsteps), int(rk))


def ndg_step_split(ctx, dt: float, nsteps: int, rk: int = NDG_RK4) -> None:
    """ndg_step with every stage in split form (volume / surface / update kernels): verification."""
    _call("ndg_step_split", ctx, float(dt), int(nsteps), int(rk))


def ndg_norms(ctx, ref_ptr=None, ref_on_device: bool = False, allow_nonfinite: bool = False) -> ndg_norms_t:
    out = ndg_norms_t()
    rc = load().ndg_norms(ctx, ref_ptr, int(ref_on_device), ctypes.byref(out))
    if rc != NDG_OK and not (allow_nonfinite and rc == NDG_ENONFINITE):
        raise NdgError(rc, "ndg_norms", ndg_last_error())
    return out


def ndg_norms_noalloc(cfg: ndg_config, u_ptr: int, ref_ptr, nblocks: int, out_ptr: int, stream: int = 0) -> None:
    """Norms into a caller-owned device buffer of 8 doubles, with no allocation by the library."""
    _call("ndg_norms_noalloc", ctypes.byref(cfg), u_ptr, ref_ptr, int(nblocks), out_ptr, stream)


def ndg_stable_dt(ctx, cfl: float) -> float:
    dt = ctypes.c_double()
    _call("ndg_stable_dt", ctx, float(cfl), ctypes.byref(dt))
    return dt.value


def ndg_node_coords(ctx, out_ptr: int, count: int) -> None:
    _call("ndg_node_coords", ctx, ctypes.cast(out_ptr, ctypes.POINTER(ctypes.c_double)), count)


def ndg_info(ctx) -> ndg_info_t:
    out = ndg_info_t()
    _call("ndg_info", ctx, ctypes.byref(out))
    return out


def ndg_lgl(degree: int):
    """(xi, w) as lists of degree+1 floats."""
    xi = (ctypes.c_double * (degree + 1))()
    w = (ctypes.c_double * (degree + 1))()
    _call("ndg_lgl", degree, xi, w)
    return list(xi), list(w)


def ndg_stream(ctx) -> int:
    return load().ndg_stream(ctx) or 0


def ndg_synchronize(ctx) -> None:
    _call("ndg_synchronize", ctx)


def ndg_debug_stall_copies(polls: int) -> None:
    """Test hook: work lists uploaded from now on make bulk-copy waits run out after `polls`
    polls (0 restores normal operation)."""
    _call("ndg_debug_stall_copies", int(polls))


_alloc_keep = []


def ndg_set_allocator(alloc, free, user=None) -> None:
    """alloc(bytes, user, stream) -> int device pointer; free(ptr, user, stream).  None, None resets."""
    if alloc is None:
        _call("ndg_set_allocator", ALLOC_FN(), FREE_FN(), None)
        _alloc_keep.clear()
        return
    a, f = ALLOC_FN(alloc), FREE_FN(free)
    _alloc_keep[:] = [a, f]
    _call("ndg_set_allocator", a, f, user)


def ndg_autotune(ctx, rk: int = NDG_RK4):
    best = ctypes.c_int()
    ms = ctypes.c_double()
    _call("ndg_autotune", ctx, rk, ctypes.byref(best), ctypes.byref(ms))
    return best.value, ms.value


def ndg_batch_create(ctxs) -> int:
    arr = (_P * len(ctxs))(*ctxs)
    h = _P()
    _call("ndg_batch_create", arr, len(ctxs), ctypes.byref(h))
    return h.value


def ndg_batch_step(batch, dts, nsteps: int, rk: int = NDG_RK4) -> None:
    arr = (ctypes.c_double * len(dts))(*dts)
    _call("ndg_batch_step", batch, arr, int(nsteps), int(rk))


def ndg_batch_destroy(batch) -> None:
    _call("ndg_batch_destroy", batch)


def ndg_partition_create(cfg: ndg_config, parts) -> int:
    h = _P()
    arr = (ctypes.c_int * 3)(*(list(parts) + [1] * (3 - len(parts))))
    _call("ndg_partition_create", ctypes.byref(cfg), arr, ctypes.byref(h))
    return h.value


def ndg_partition_set_state(part, ptr: int, nbytes: int, on_device: bool) -> None:
    _call("ndg_partition_set_state", part, ptr, nbytes, int(on_device))


def ndg_partition_get_state(part, ptr: int, nbytes: int, on_device: bool) -> None:
    _call("ndg_partition_get_state", part, ptr, nbytes, int(on_device))


def ndg_partition_step(part, dt: float, nsteps: int, rk: int = NDG_RK4) -> None:
    _call("ndg_partition_step", part, float(dt), int(nsteps), int(rk))


def ndg_partition_norms(part) -> ndg_norms_t:
    out = ndg_norms_t()
    _call("ndg_partition_norms", part, ctypes.byref(out))
    return out


def ndg_partition_info(part, index: int):
    o = (ctypes.c_int * 3)()
    e = (ctypes.c_int * 3)()
    _call("ndg_partition_info", part, index, o, e)
    return list(o), list(e)


def ndg_partition_destroy(part) -> None:
    _call("ndg_partition_destroy", part)


def ndg_pool_create(budget_bytes: int, device: int = 0) -> int:
    h = _P()
    _call("ndg_pool_create", int(budget_bytes), int(device), ctypes.byref(h))
    return h.value


def ndg_pool_submit(pool, cfg: ndg_config, u0_ptr: int, nbytes: int, rk: int, dt: float, nsteps: int) -> int:
    t = ctypes.c_uint64()
    _call("ndg_pool_submit", pool, ctypes.byref(cfg), u0_ptr, nbytes, rk, float(dt), int(nsteps), ctypes.byref(t))
    return t.value


def ndg_pool_poll(pool, ticket: int, result_ptr, nbytes: int, timeout_s: float):
    """Returns (status, stats): status NDG_OK, NDG_EAGAIN or NDG_ETIMEOUT; other codes raise."""
    st = ndg_solve_stats_t()
    rc = load().ndg_pool_poll(pool, ticket, result_ptr, nbytes, ctypes.byref(st), float(timeout_s))
    if rc not in (NDG_OK, NDG_EAGAIN, NDG_ETIMEOUT):
        raise NdgError(rc, "ndg_pool_poll", ndg_last_error())
    return rc, st


def ndg_pool_status(pool):
    q, r, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    b, pk = ctypes.c_size_t(), ctypes.c_size_t()
    _call("ndg_pool_status", pool, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f), ctypes.byref(b),
          ctypes.byref(pk))
    return {"queued": q.value, "running": r.value, "finished": f.value, "bytes_in_use": b.value,
            "peak_bytes": pk.value}


def ndg_pool_destroy(pool) -> None:
    _call("ndg_pool_destroy", pool)
