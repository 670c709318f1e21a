"""ctypes binding of libgs (include/gs.h), one Python function per C entry point.

Argument marshalling only: every step of the Gray-Scott path runs in the CUDA
kernels of libgs.so.  Host buffers are numpy arrays (or CPU torch tensors);
device buffers and streams are integers or torch objects (PyTorch supplies
device memory and streams).  A non-zero status raises GsError carrying the
library's message.  The library must be built first
(``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gs.h")

GS_F32, GS_F64 = 0, 1
GS_U, GS_V = 0, 1
GS_OK, GS_EINVAL, GS_ENOMEM, GS_ECUDA, GS_ETIMEOUT, GS_ESTATE, GS_EIO = 0, -1, -2, -3, -4, -5, -6
GS_KERNEL_AUTO, GS_KERNEL_NAIVE, GS_KERNEL_ZMARCH, GS_KERNEL_TBLOCK = 0, 1, 2, 3
GS_MAX_L = 1625  # largest edge (the noise hash counts cells in 32 bits)
STATUS_NAMES = {0: "GS_OK", -1: "GS_EINVAL", -2: "GS_ENOMEM", -3: "GS_ECUDA", -4: "GS_ETIMEOUT",
                -5: "GS_ESTATE", -6: "GS_EIO"}


class GsError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_d = ctypes.c_double
_sz = ctypes.c_size_t
_pp = ctypes.POINTER(ctypes.c_void_p)

# argtypes of every entry point (restype int unless listed in _RESTYPES)
_SIGS = {
    "gs_create": [_i, _d, _d, _d, _d, _d, _d, _u64, _i, _pp],
    "gs_create_on": [_i, _d, _d, _d, _d, _d, _d, _u64, _i, _vp, _vp, _vp, _vp, _vp, _pp],
    "gs_set_stream": [_vp, _vp],
    "gs_init": [_vp],
    "gs_step": [_vp, _i64],
    "gs_read": [_vp, _i, _vp, _sz],
    "gs_write": [_vp, _i, _vp, _sz],
    "gs_device_ptr": [_vp, _i, _pp],
    "gs_get_step": [_vp, ctypes.POINTER(_i64)],
    "gs_set_step": [_vp, _i64],
    "gs_set_plan": [_vp, _i, _i, _i, _i, _i],
    "gs_get_plan": [_vp] + [ctypes.POINTER(_i)] * 5,
    "gs_get_plan_full": [_vp, _vp],
    "gs_sync": [_vp],
    "gs_set_plan_full": [_vp, _vp],
    "gs_autotune": [_vp, _i, _vp, _i, ctypes.POINTER(_i), _vp],
    "gs_batch_autotune": [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(_i)],
    "gs_read_async": [_vp, _i, _vp, _sz],
    "gs_write_async": [_vp, _i, _vp, _sz],
    "gs_autotune_cached": [_vp, _i, ctypes.c_char_p, _vp, ctypes.POINTER(_i)],
    "gs_set_fault": [_vp, _i, _u64],
    "gs_launch_count": [_vp, ctypes.POINTER(_i64)],
    "gs_destroy": [_vp],
    "gs_last_error": [],
    "gs_noise_field": [_u64, _i64, _i64, _i, _vp, _vp],
    "gs_set_boundary": [_vp, _i],
    "gs_set_arith": [_vp, _i],
    "gs_get_arith": [_vp, ctypes.POINTER(_i)],
    "gs_get_boundary": [_vp, ctypes.POINTER(_i)],
    "gs_single_create": [_i, _d, _d, _i, _i, ctypes.POINTER(_vp)],
    "gs_single_set_stream": [_vp, _vp],
    "gs_single_write": [_vp, _vp, ctypes.c_size_t],
    "gs_single_read": [_vp, _vp, ctypes.c_size_t],
    "gs_single_step": [_vp, _i64],
    "gs_single_info": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "gs_single_sync": [_vp],
    "gs_single_destroy": [_vp],
    "gs_stats": [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_i64)],
    "gs_slice": [_vp, _i, _i, _i, _vp, ctypes.c_size_t],
    "gs_snap_open": [_vp, ctypes.c_char_p, ctypes.POINTER(_vp)],
    "gs_snap_write": [_vp],
    "gs_snap_flush": [_vp],
    "gs_snap_info": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_d)],
    "gs_snap_close": [_vp],
    "gs_checkpoint_save": [_vp, ctypes.c_char_p],
    "gs_checkpoint_load": [_vp, ctypes.c_char_p],
    "gs_batch_create": [_i, _vp, _vp, _vp, _d, _d, _d, _d, _u64, _i, _pp],
    "gs_batch_set_stream": [_vp, _vp],
    "gs_batch_init": [_vp],
    "gs_batch_step": [_vp, _i64],
    "gs_batch_step_sequential": [_vp, _i64],
    "gs_batch_read": [_vp, _i, _i, _vp, _sz],
    "gs_batch_write": [_vp, _i, _i, _vp, _sz],
    "gs_batch_get_step": [_vp, ctypes.POINTER(_i64)],
    "gs_batch_set_step": [_vp, _i64],
    "gs_batch_sync": [_vp],
    "gs_batch_set_fault": [_vp, _i, _u64],
    "gs_batch_set_plan": [_vp, _i, _i],
    "gs_batch_set_depth": [_vp, _i],
    "gs_batch_info": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                      ctypes.POINTER(_i64), ctypes.POINTER(_i)],
    "gs_batch_destroy": [_vp],
    "gs_get_stream": [_vp, _pp],
    "gs_sim_shape": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "gs_surr_param_count": [ctypes.POINTER(_sz)],
    "gs_surr_create": [_pp],
    "gs_surr_set_stream": [_vp, _vp],
    "gs_surr_set_params": [_vp, _vp, _sz],
    "gs_surr_get_params": [_vp, _vp, _sz],
    "gs_surr_get_grads": [_vp, _vp, _sz],
    "gs_surr_trace_grads": [_vp, _vp, _sz],
    "gs_surr_save": [_vp, ctypes.c_char_p],
    "gs_surr_load": [_vp, ctypes.c_char_p],
    "gs_surr_get_train_output": [_vp, _vp, _vp, _sz],
    "gs_surr_forward": [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
    "gs_surr_grad": [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d)],
    "gs_surr_adam": [_vp, _d, _d, _d, _d],
    "gs_surr_train_step": [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _d, ctypes.POINTER(_d)],
    "gs_surr_diff": [_vp, _vp, _vp, _i64, ctypes.POINTER(_d), ctypes.POINTER(_d)],
    "gs_surr_run": [_vp, _vp, _d, _d, _i64, _i, _d, _vp],
    "gs_surr_set_backend": [_vp, _i],
    "gs_surr_sync": [_vp],
    "gs_surr_launch_count": [_vp, ctypes.POINTER(_i64)],
    "gs_surr_destroy": [_vp],
    "gs_batch_step_noalloc": [_i, _vp, _vp, _vp, _d, _d, _d, _d, _u64, _i, _vp, _i64, _i, _i64, _vp],
    "gs_measure_fp64_fma": [_vp, ctypes.POINTER(_d)],
    "gs_set_alloc_guard": [_sz],
    "gs_batch_guard_check": [_vp, ctypes.POINTER(_i64)],
    "gs_surr_guard_check": [_vp, ctypes.POINTER(_i64)],
    "gs_slab_create_on": [_i, _i, _i, _i, _d, _d, _d, _d, _d, _d, _u64, _i, _vp, _vp, _vp, _vp, _pp],
    "gs_slab_set_stream": [_vp, _vp],
    "gs_slab_init": [_vp],
    "gs_slab_pass": [_vp],
    "gs_slab_state": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i)],
    "gs_slab_set_state": [_vp, _i64, _i],
    "gs_slab_exchange": [_vp, _i],
    "gs_slab_sync": [_vp],
    "gs_slab_launch_count": [_vp, ctypes.POINTER(_i64)],
    "gs_slab_destroy": [_vp],
}
_RESTYPES = {"gs_last_error": ctypes.c_char_p}


def lib():
    """Load libgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library with "
                               "__graft_entry__.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, ctypes.c_int)
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Names of the functions include/gs.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int, func: str):
    if rc != GS_OK:
        raise GsError(rc, func, lib().gs_last_error().decode())


def _ptr(x) -> int | None:
    """Address of a device/host buffer given as int, torch tensor or numpy array."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int | None:
    if s is None or isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _dtype_code(dtype) -> int:
    if dtype in (GS_F32, "f32", "float32", np.float32):
        return GS_F32
    if dtype in (GS_F64, "f64", "float64", np.float64):
        return GS_F64
    raise ValueError(f"dtype {dtype!r} must be f32 or f64")


def np_dtype(code: int):
    return np.float32 if code == GS_F32 else np.float64


# ---------------------------------------------------------------------------
# Entry points
# ---------------------------------------------------------------------------
def gs_last_error() -> str:
    return lib().gs_last_error().decode()


def gs_create(L, Du, Dv, F, k, dt, noise, seed, dtype):
    out = ctypes.c_void_p()
    _check(lib().gs_create(L, Du, Dv, F, k, dt, noise, seed, _dtype_code(dtype), ctypes.byref(out)),
           "gs_create")
    return out.value


def gs_create_on(L, Du, Dv, F, k, dt, noise, seed, dtype, u0, v0, u1, v1, stream=None):
    out = ctypes.c_void_p()
    _check(lib().gs_create_on(L, Du, Dv, F, k, dt, noise, seed, _dtype_code(dtype), _ptr(u0), _ptr(v0),
                              _ptr(u1), _ptr(v1), _stream(stream), ctypes.byref(out)), "gs_create_on")
    return out.value


def gs_set_stream(sim, stream):
    _check(lib().gs_set_stream(sim, _stream(stream)), "gs_set_stream")


def gs_init(sim):
    _check(lib().gs_init(sim), "gs_init")


def gs_step(sim, n: int):
    _check(lib().gs_step(sim, int(n)), "gs_step")


def gs_read(sim, field: int, dst):
    """Copy a field into the host buffer dst (numpy array / CPU tensor of L^3 elements)."""
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(lib().gs_read(sim, field, _ptr(dst), nbytes), "gs_read")
    return dst


def gs_write(sim, field: int, src):
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    if isinstance(src, np.ndarray):
        assert src.flags["C_CONTIGUOUS"]
    _check(lib().gs_write(sim, field, _ptr(src), nbytes), "gs_write")


def gs_device_ptr(sim, field: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().gs_device_ptr(sim, field, ctypes.byref(p)), "gs_device_ptr")
    return p.value


def gs_get_step(sim) -> int:
    t = _i64()
    _check(lib().gs_get_step(sim, ctypes.byref(t)), "gs_get_step")
    return t.value


def gs_set_step(sim, t: int):
    _check(lib().gs_set_step(sim, int(t)), "gs_set_step")


def gs_set_plan(sim, kernel: int, tile_x=0, tile_y=0, tile_z=0, depth=0):
    _check(lib().gs_set_plan(sim, kernel, tile_x, tile_y, tile_z, depth), "gs_set_plan")


def gs_get_plan(sim) -> dict:
    v = [_i() for _ in range(5)]
    _check(lib().gs_get_plan(sim, *[ctypes.byref(x) for x in v]), "gs_get_plan")
    return dict(zip(("kernel", "tile_x", "tile_y", "tile_z", "depth"), (x.value for x in v)))


class GsPlan(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("depth", ctypes.c_int), ("stages", ctypes.c_int),
                ("us_per_step", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def gs_set_plan_full(sim, plan: dict):
    p = GsPlan(**{k: plan[k] for k in ("kernel", "tile_x", "tile_y", "tile_z", "depth", "stages")
                  if k in plan})
    _check(lib().gs_set_plan_full(sim, ctypes.byref(p)), "gs_set_plan_full")


def gs_get_plan_full(sim) -> dict:
    p = GsPlan()
    _check(lib().gs_get_plan_full(sim, ctypes.byref(p)), "gs_get_plan_full")
    return p.as_dict()


def gs_autotune(sim, steps_per_trial: int = 12, max_results: int = 256):
    """Run the native autotuner; returns (best plan, list of trials) as dicts."""
    res = (GsPlan * max_results)()
    n = _i()
    best = GsPlan()
    _check(lib().gs_autotune(sim, steps_per_trial, res, max_results, ctypes.byref(n), ctypes.byref(best)),
           "gs_autotune")
    return best.as_dict(), [res[i].as_dict() for i in range(min(n.value, max_results))]


def gs_autotune_cached(sim, path: str, steps_per_trial: int = 12):
    """Autotune through the plan cache file `path`; returns (best plan dict, hit)."""
    best = GsPlan()
    hit = _i()
    _check(lib().gs_autotune_cached(sim, steps_per_trial, os.fsencode(path), ctypes.byref(best), ctypes.byref(hit)),
           "gs_autotune_cached")
    return best.as_dict(), bool(hit.value)


def gs_batch_autotune(b, steps_per_trial: int = 20) -> dict:
    """Tune the batched launch's z-chunk, ring depth and temporal-blocking
    depth; returns the kept plan."""
    tz, st, us, d = _i(), _i(), ctypes.c_double(), _i()
    _check(lib().gs_batch_autotune(b, steps_per_trial, ctypes.byref(tz), ctypes.byref(st), ctypes.byref(us),
                                   ctypes.byref(d)), "gs_batch_autotune")
    return {"tile_z": tz.value, "stages": st.value, "depth": d.value, "us_per_step": us.value}


def gs_read_async(sim, field: int, dst):
    """Enqueue a copy of a field into the host buffer dst (page-locked for
    overlap); dst is valid once the object's stream has passed it."""
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(lib().gs_read_async(sim, field, _ptr(dst), nbytes), "gs_read_async")
    return dst


def gs_write_async(sim, field: int, src):
    """Enqueue a copy of the host buffer src into a field (src must stay
    unchanged until the object's stream has passed the copy)."""
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    _check(lib().gs_write_async(sim, field, _ptr(src), nbytes), "gs_write_async")


def gs_sync(sim):
    _check(lib().gs_sync(sim), "gs_sync")


def gs_set_fault(sim, mode: int, timeout_ns: int = 2_000_000_000):
    _check(lib().gs_set_fault(sim, mode, timeout_ns), "gs_set_fault")


def gs_launch_count(sim) -> int:
    c = _i64()
    _check(lib().gs_launch_count(sim, ctypes.byref(c)), "gs_launch_count")
    return c.value


def gs_destroy(sim):
    _check(lib().gs_destroy(sim), "gs_destroy")


def gs_noise_field(seed, t, n, dtype, dev_out, stream=None):
    _check(lib().gs_noise_field(seed, t, n, _dtype_code(dtype), _ptr(dev_out), _stream(stream)),
           "gs_noise_field")


GS_BOUNDARY_PERIODIC, GS_BOUNDARY_HELD = 0, 1
GS_ARITH_IEEE, GS_ARITH_DS, GS_ARITH_FX, GS_ARITH_FXF = 0, 1, 2, 3


def gs_set_arith(sim, arith: int):
    _check(lib().gs_set_arith(sim, arith), "gs_set_arith")


def gs_get_arith(sim) -> int:
    a = _i()
    _check(lib().gs_get_arith(sim, ctypes.byref(a)), "gs_get_arith")
    return a.value


def gs_set_boundary(sim, boundary: int):
    _check(lib().gs_set_boundary(sim, boundary), "gs_set_boundary")


def gs_get_boundary(sim) -> int:
    b = _i()
    _check(lib().gs_get_boundary(sim, ctypes.byref(b)), "gs_get_boundary")
    return b.value


def gs_single_create(L: int, D: float, dt: float, dtype, boundary: int = 0):
    out = ctypes.c_void_p()
    _check(lib().gs_single_create(L, D, dt, _dtype_code(dtype), boundary, ctypes.byref(out)), "gs_single_create")
    return out.value


def gs_single_set_stream(h, stream=None):
    _check(lib().gs_single_set_stream(h, _stream(stream)), "gs_single_set_stream")


def gs_single_write(h, src: np.ndarray):
    _check(lib().gs_single_write(h, src.ctypes.data_as(_vp), src.nbytes), "gs_single_write")


def gs_single_read(h, dst: np.ndarray):
    _check(lib().gs_single_read(h, dst.ctypes.data_as(_vp), dst.nbytes), "gs_single_read")


def gs_single_step(h, n: int):
    _check(lib().gs_single_step(h, n), "gs_single_step")


def gs_single_info(h) -> dict:
    z, st, la = _i(), _i64(), _i64()
    _check(lib().gs_single_info(h, ctypes.byref(z), ctypes.byref(st), ctypes.byref(la)), "gs_single_info")
    return {"zmarch": bool(z.value), "steps": st.value, "launches": la.value}


def gs_single_sync(h):
    _check(lib().gs_single_sync(h), "gs_single_sync")


def gs_single_destroy(h):
    _check(lib().gs_single_destroy(h), "gs_single_destroy")


def gs_stats(sim, field: int) -> dict:
    """min, max, mean, rms and the NaN count of a field of the current state."""
    out = (_d * 4)()
    nan = _i64()
    _check(lib().gs_stats(sim, field, out, ctypes.byref(nan)), "gs_stats")
    return {"min": out[0], "max": out[1], "mean": out[2], "rms": out[3], "nan": nan.value}


def gs_slice(sim, field: int, axis: int, index: int, dst: np.ndarray):
    """Fill dst (an L x L array of the simulation's dtype) with one plane."""
    _check(lib().gs_slice(sim, field, axis, index, dst.ctypes.data_as(_vp), dst.nbytes), "gs_slice")


def gs_snap_open(sim, path: str):
    out = ctypes.c_void_p()
    _check(lib().gs_snap_open(sim, os.fsencode(path), ctypes.byref(out)), "gs_snap_open")
    return out.value


def gs_snap_write(snap):
    _check(lib().gs_snap_write(snap), "gs_snap_write")


def gs_snap_flush(snap):
    _check(lib().gs_snap_flush(snap), "gs_snap_flush")


def gs_snap_info(snap) -> dict:
    n, b = _i64(), _d()
    _check(lib().gs_snap_info(snap, ctypes.byref(n), ctypes.byref(b)), "gs_snap_info")
    return {"records": n.value, "bytes": b.value}


def gs_snap_close(snap):
    _check(lib().gs_snap_close(snap), "gs_snap_close")


def gs_checkpoint_save(sim, path: str):
    _check(lib().gs_checkpoint_save(sim, os.fsencode(path)), "gs_checkpoint_save")


def gs_checkpoint_load(sim, path: str):
    _check(lib().gs_checkpoint_load(sim, os.fsencode(path)), "gs_checkpoint_load")


def gs_batch_create(L, F, k, Du, Dv, dt, noise, seed, dtype):
    n = len(L)
    La = (ctypes.c_int * n)(*[int(x) for x in L])
    Fa = (ctypes.c_double * n)(*[float(x) for x in F])
    ka = (ctypes.c_double * n)(*[float(x) for x in k])
    out = ctypes.c_void_p()
    _check(lib().gs_batch_create(n, La, Fa, ka, Du, Dv, dt, noise, seed, _dtype_code(dtype),
                                 ctypes.byref(out)), "gs_batch_create")
    return out.value


def gs_batch_set_stream(b, stream):
    _check(lib().gs_batch_set_stream(b, _stream(stream)), "gs_batch_set_stream")


def gs_batch_init(b):
    _check(lib().gs_batch_init(b), "gs_batch_init")


def gs_batch_step(b, n: int):
    _check(lib().gs_batch_step(b, int(n)), "gs_batch_step")


def gs_batch_step_sequential(b, n: int):
    _check(lib().gs_batch_step_sequential(b, int(n)), "gs_batch_step_sequential")


def gs_batch_read(b, i: int, field: int, dst):
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(lib().gs_batch_read(b, i, field, _ptr(dst), nbytes), "gs_batch_read")
    return dst


def gs_batch_write(b, i: int, field: int, src):
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    _check(lib().gs_batch_write(b, i, field, _ptr(src), nbytes), "gs_batch_write")


def gs_batch_get_step(b) -> int:
    t = _i64()
    _check(lib().gs_batch_get_step(b, ctypes.byref(t)), "gs_batch_get_step")
    return t.value


def gs_batch_set_step(b, t: int):
    _check(lib().gs_batch_set_step(b, int(t)), "gs_batch_set_step")


def gs_batch_sync(b):
    _check(lib().gs_batch_sync(b), "gs_batch_sync")


def gs_batch_set_fault(b, mode: int, timeout_ns: int = 2_000_000_000):
    _check(lib().gs_batch_set_fault(b, mode, timeout_ns), "gs_batch_set_fault")


def gs_batch_set_plan(b, tile_z: int, stages: int):
    _check(lib().gs_batch_set_plan(b, tile_z, stages), "gs_batch_set_plan")


def gs_batch_set_depth(b, depth: int):
    _check(lib().gs_batch_set_depth(b, depth), "gs_batch_set_depth")


def gs_batch_info(b) -> dict:
    g, it, co, la, d = _i(), _i(), _i(), _i64(), _i()
    _check(lib().gs_batch_info(b, ctypes.byref(g), ctypes.byref(it), ctypes.byref(co), ctypes.byref(la),
                               ctypes.byref(d)), "gs_batch_info")
    return {"grid": g.value, "items": it.value, "cooperative": bool(co.value), "launches": la.value,
            "depth": d.value}


def gs_batch_destroy(b):
    _check(lib().gs_batch_destroy(b), "gs_batch_destroy")


def gs_batch_step_noalloc(L, F, k, Du, Dv, dt, noise, seed, dtype, arena, t, cur, nsteps, stream=None):
    """Allocation-free batched step on a caller-owned arena (see include/gs.h)."""
    n = len(L)
    La = (ctypes.c_int * n)(*[int(x) for x in L])
    Fa = (ctypes.c_double * n)(*[float(x) for x in F])
    ka = (ctypes.c_double * n)(*[float(x) for x in k])
    _check(lib().gs_batch_step_noalloc(n, La, Fa, ka, Du, Dv, dt, noise, seed, _dtype_code(dtype),
                                       _ptr(arena), int(t), int(cur), int(nsteps), _stream(stream)),
           "gs_batch_step_noalloc")


def noalloc_arena_offsets(L, dtype) -> tuple[list, int]:
    """Element offsets (u0, v0, u1, v1) of each instance in an allocation-free arena,
    and the arena's total length in elements."""
    esz = 4 if _dtype_code(dtype) == GS_F32 else 8
    align = 256 // esz
    off, out = 0, []
    for x in L:
        cells = int(x) ** 3
        o = []
        for _ in range(4):
            o.append(off)
            off += (cells + align - 1) // align * align
        out.append(o)
    return out, off


def gs_get_stream(sim) -> int:
    p = ctypes.c_void_p()
    _check(lib().gs_get_stream(sim, ctypes.byref(p)), "gs_get_stream")
    return p.value or 0


def gs_sim_shape(sim):
    L, dt = _i(), _i()
    _check(lib().gs_sim_shape(sim, ctypes.byref(L), ctypes.byref(dt)), "gs_sim_shape")
    return L.value, dt.value


# ---------------------------------------------------------------------------
# Learned surrogate
# ---------------------------------------------------------------------------
class GsSurrReport(ctypes.Structure):
    _fields_ = [("surrogate_applications", ctypes.c_int64), ("surrogate_steps", ctypes.c_int64),
                ("stencil_steps", ctypes.c_int64), ("checks", ctypes.c_int64), ("fallbacks", ctypes.c_int64),
                ("max_check_error", ctypes.c_double), ("last_check_error", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def _f64_array(x):
    x = [float(v) for v in x]
    return (ctypes.c_double * len(x))(*x)


def gs_surr_param_count() -> int:
    n = _sz()
    _check(lib().gs_surr_param_count(ctypes.byref(n)), "gs_surr_param_count")
    return n.value


def gs_surr_create():
    out = ctypes.c_void_p()
    _check(lib().gs_surr_create(ctypes.byref(out)), "gs_surr_create")
    return out.value


def gs_surr_set_stream(s, stream):
    _check(lib().gs_surr_set_stream(s, _stream(stream)), "gs_surr_set_stream")


def gs_surr_set_params(s, flat: np.ndarray):
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    _check(lib().gs_surr_set_params(s, flat.ctypes.data, flat.size), "gs_surr_set_params")


def gs_surr_get_params(s) -> np.ndarray:
    out = np.empty(gs_surr_param_count(), dtype=np.float32)
    _check(lib().gs_surr_get_params(s, out.ctypes.data, out.size), "gs_surr_get_params")
    return out


def gs_surr_get_grads(s) -> np.ndarray:
    out = np.empty(gs_surr_param_count(), dtype=np.float32)
    _check(lib().gs_surr_get_grads(s, out.ctypes.data, out.size), "gs_surr_get_grads")
    return out


def gs_surr_save(s, path: str):
    _check(lib().gs_surr_save(s, os.fsencode(path)), "gs_surr_save")


def gs_surr_load(s, path: str):
    _check(lib().gs_surr_load(s, os.fsencode(path)), "gs_surr_load")


def gs_surr_trace_grads(s, dh, count: int = 0):
    """dh: a float32 CUDA tensor of 5 * N * L^3 * 32 elements, or None (off)."""
    _check(lib().gs_surr_trace_grads(s, _ptr(dh) if dh is not None else None,
                                     int(count) if dh is not None else 0), "gs_surr_trace_grads")


def gs_surr_get_train_output(s, u_out, v_out, cells: int):
    _check(lib().gs_surr_get_train_output(s, _ptr(u_out), _ptr(v_out), int(cells)), "gs_surr_get_train_output")


def gs_surr_forward(s, N, L, u, v, F, k, u_out, v_out):
    _check(lib().gs_surr_forward(s, N, L, _ptr(u), _ptr(v), _f64_array(F), _f64_array(k), _ptr(u_out),
                                 _ptr(v_out)), "gs_surr_forward")


def gs_surr_grad(s, N, L, u, v, F, k, u_tgt, v_tgt) -> float:
    loss = _d()
    _check(lib().gs_surr_grad(s, N, L, _ptr(u), _ptr(v), _f64_array(F), _f64_array(k), _ptr(u_tgt),
                              _ptr(v_tgt), ctypes.byref(loss)), "gs_surr_grad")
    return loss.value


def gs_surr_adam(s, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib().gs_surr_adam(s, lr, beta1, beta2, eps), "gs_surr_adam")


def gs_surr_train_step(s, N, L, u, v, F, k, u_tgt, v_tgt, lr) -> float:
    loss = _d()
    _check(lib().gs_surr_train_step(s, N, L, _ptr(u), _ptr(v), _f64_array(F), _f64_array(k), _ptr(u_tgt),
                                    _ptr(v_tgt), lr, ctypes.byref(loss)), "gs_surr_train_step")
    return loss.value


def gs_surr_diff(s, a, b, n):
    mx, rms = _d(), _d()
    _check(lib().gs_surr_diff(s, _ptr(a), _ptr(b), int(n), ctypes.byref(mx), ctypes.byref(rms)), "gs_surr_diff")
    return mx.value, rms.value


def gs_surr_run(s, sim, F, k, nsteps, check_every=64, tol=0.05) -> dict:
    rep = GsSurrReport()
    _check(lib().gs_surr_run(s, sim, F, k, int(nsteps), int(check_every), tol, ctypes.byref(rep)), "gs_surr_run")
    return rep.as_dict()


GS_SURR_AUTO, GS_SURR_MMA, GS_SURR_TCGEN05 = 0, 1, 2


def gs_surr_set_backend(s, backend: int):
    _check(lib().gs_surr_set_backend(s, backend), "gs_surr_set_backend")


def gs_surr_sync(s):
    _check(lib().gs_surr_sync(s), "gs_surr_sync")


def gs_surr_launch_count(s) -> int:
    c = _i64()
    _check(lib().gs_surr_launch_count(s, ctypes.byref(c)), "gs_surr_launch_count")
    return c.value


def gs_surr_destroy(s):
    _check(lib().gs_surr_destroy(s), "gs_surr_destroy")


SURR_CHANNELS = (4, 32, 32, 32, 32, 32, 2)


def surr_flatten(params) -> np.ndarray:
    """[(w [27, cin, cout], b [cout]), ...] -> the flat FP32 layout of gs_surr_set_params."""
    return np.concatenate([np.concatenate([np.asarray(w, dtype=np.float32).ravel(),
                                           np.asarray(b, dtype=np.float32).ravel()]) for w, b in params])


def surr_unflatten(flat) -> list:
    out, o = [], 0
    for l in range(6):
        cin, cout = SURR_CHANNELS[l], SURR_CHANNELS[l + 1]
        nw = 27 * cin * cout
        out.append((np.asarray(flat[o:o + nw], dtype=np.float64).reshape(27, cin, cout),
                    np.asarray(flat[o + nw:o + nw + cout], dtype=np.float64)))
        o += nw + cout
    return out


class Surrogate:
    """The 16-step surrogate network with its FP32 master parameters on the GPU."""

    def __init__(self, params=None, stream=None):
        import torch
        self.handle = gs_surr_create()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        gs_surr_set_stream(self.handle, self.stream)
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        flat = params if isinstance(params, np.ndarray) else surr_flatten(params)
        gs_surr_set_params(self.handle, flat)

    def params(self):
        return surr_unflatten(gs_surr_get_params(self.handle))

    def grads(self):
        return surr_unflatten(gs_surr_get_grads(self.handle))

    def save(self, path: str):
        gs_surr_save(self.handle, path)

    def load(self, path: str):
        gs_surr_load(self.handle, path)

    def forward(self, u, v, F, k):
        """u, v: torch float32 CUDA tensors [N, L, L, L]; returns predicted (u, v) after 16 steps."""
        import torch
        N, L = u.shape[0], u.shape[1]
        uo, vo = torch.empty_like(u), torch.empty_like(v)
        gs_surr_forward(self.handle, N, L, u, v, F, k, uo, vo)
        return uo, vo

    def grad(self, u, v, F, k, ut, vt) -> float:
        return gs_surr_grad(self.handle, u.shape[0], u.shape[1], u, v, F, k, ut, vt)

    def train_step(self, u, v, F, k, ut, vt, lr) -> float:
        return gs_surr_train_step(self.handle, u.shape[0], u.shape[1], u, v, F, k, ut, vt, lr)

    def run(self, sim, F, k, nsteps, check_every=64, tol=0.05) -> dict:
        return gs_surr_run(self.handle, sim.handle, F, k, nsteps, check_every, tol)

    def close(self):
        if self.handle:
            gs_surr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_set_alloc_guard(nbytes: int):
    _check(lib().gs_set_alloc_guard(int(nbytes)), "gs_set_alloc_guard")


def gs_batch_guard_check(b) -> int:
    n = _i64()
    _check(lib().gs_batch_guard_check(b, ctypes.byref(n)), "gs_batch_guard_check")
    return n.value


def gs_surr_guard_check(s) -> int:
    n = _i64()
    _check(lib().gs_surr_guard_check(s, ctypes.byref(n)), "gs_surr_guard_check")
    return n.value


def gs_measure_fp64_fma(stream=None) -> float:
    """FP64 fused multiply-adds per second of this GPU (measured)."""
    r = _d()
    _check(lib().gs_measure_fp64_fma(_stream(stream), ctypes.byref(r)), "gs_measure_fp64_fma")
    return r.value


# ---------------------------------------------------------------------------
# z-slab decomposition (gs_slab_*)
# ---------------------------------------------------------------------------
def slab_bounds(L: int, nslabs: int) -> list:
    """(z0, nz) of nslabs z-slabs of an L^3 grid, as even as possible."""
    return [(L * i // nslabs, L * (i + 1) // nslabs - L * i // nslabs) for i in range(nslabs)]


class GrayScottSlab:
    """One z-slab (global planes z0 .. z0+nz-1) of a periodic L^3 grid with
    `depth` ghost planes on each side; its four buffers are torch tensors
    [nz + 2 depth, L, L] on the current CUDA device."""

    def __init__(self, L, z0, nz, depth, Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0, noise=0.0, seed=0,
                 dtype="f32", stream=None, device=None):
        import torch
        self.L, self.z0, self.nz, self.depth = int(L), int(z0), int(nz), int(depth)
        self.dtype = _dtype_code(dtype)
        tdt = torch.float32 if self.dtype == GS_F32 else torch.float64
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        planes = self.nz + 2 * self.depth
        self._bufs = [torch.empty((planes, L, L), dtype=tdt, device=dev) for _ in range(4)]
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        out = ctypes.c_void_p()
        _check(lib().gs_slab_create_on(self.L, self.z0, self.nz, self.depth, Du, Dv, F, k, dt, noise, seed,
                                       self.dtype, *(_ptr(b) for b in self._bufs), ctypes.byref(out)),
               "gs_slab_create_on")
        self.handle = out.value
        _check(lib().gs_slab_set_stream(self.handle, _stream(self.stream)), "gs_slab_set_stream")

    def init(self):
        _check(lib().gs_slab_init(self.handle), "gs_slab_init")

    def run_pass(self):
        """`depth` steps; the ghosts must hold the neighbours' planes at the current step."""
        _check(lib().gs_slab_pass(self.handle), "gs_slab_pass")

    def state(self):
        t, cur = _i64(), _i()
        _check(lib().gs_slab_state(self.handle, ctypes.byref(t), ctypes.byref(cur)), "gs_slab_state")
        return t.value, cur.value

    @property
    def t(self) -> int:
        return self.state()[0]

    def fields(self, cur=None):
        """(u, v) tensors of buffer set cur (default: the current one), all planes."""
        c = self.state()[1] if cur is None else cur
        return self._bufs[2 * c], self._bufs[2 * c + 1]

    def halo_views(self):
        """Per field, the four plane ranges a transport moves in one exchange
        (views of the current set): send_lo / send_hi = the D interior planes
        next to the low / high face, recv_lo / recv_hi = the ghost planes."""
        D, nz = self.depth, self.nz
        out = []
        for f in self.fields():
            out.append({"send_lo": f[D:2 * D], "send_hi": f[nz:nz + D],
                        "recv_lo": f[0:D], "recv_hi": f[nz + D:nz + 2 * D]})
        return out

    def read(self):
        """Interior planes of u and v as numpy arrays [nz, L, L]."""
        self.sync()
        u, v = self.fields()
        D = self.depth
        return u[D:D + self.nz].cpu().numpy(), v[D:D + self.nz].cpu().numpy()

    def sync(self):
        _check(lib().gs_slab_sync(self.handle), "gs_slab_sync")

    def launches(self) -> int:
        c = _i64()
        _check(lib().gs_slab_launch_count(self.handle, ctypes.byref(c)), "gs_slab_launch_count")
        return c.value

    def close(self):
        if self.handle:
            lib().gs_slab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def slab_exchange(slabs):
    """The halo exchange among the slabs of one grid in this process (z order,
    periodic), by device-to-device copies on each slab's stream."""
    arr = (ctypes.c_void_p * len(slabs))(*[s.handle for s in slabs])
    _check(lib().gs_slab_exchange(arr, len(slabs)), "gs_slab_exchange")


def slab_exchange_dist(views, group=None):
    """The same exchange between ranks, one slab per rank in z order
    (periodic), over torch.distributed point-to-point messages (NCCL for
    device tensors, gloo for host tensors).  `views` is halo_views() of this
    rank's slab (or the same dictionaries over host arrays).  Each rank sends
    its low interior planes to the rank below (its high ghosts) and its high
    interior planes to the rank above (its low ghosts); with one rank the
    copies stay local.  The tags tell the two faces apart when both
    neighbours are the same rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        for v in views:
            v["recv_hi"].copy_(v["send_lo"])
            v["recv_lo"].copy_(v["send_hi"])
        return
    rank = dist.get_rank(group)
    lo, hi = (rank - 1) % world, (rank + 1) % world
    ops = []
    for f, v in enumerate(views):
        ops += [dist.P2POp(dist.isend, v["send_lo"].contiguous(), lo, group, tag=2 * f),
                dist.P2POp(dist.irecv, v["recv_hi"], hi, group, tag=2 * f),
                dist.P2POp(dist.isend, v["send_hi"].contiguous(), hi, group, tag=2 * f + 1),
                dist.P2POp(dist.irecv, v["recv_lo"], lo, group, tag=2 * f + 1)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()


class GrayScottBatch:
    """Many independent grids (edges L[i], feed F[i], kill k[i]) on the current device."""

    def __init__(self, L, F, k, Du=0.2, Dv=0.1, dt=1.0, noise=0.0, seed=0, dtype="f32", stream=None):
        import torch
        self.L = [int(x) for x in L]
        self.dtype = _dtype_code(dtype)
        self.handle = gs_batch_create(self.L, F, k, Du, Dv, dt, noise, seed, self.dtype)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        gs_batch_set_stream(self.handle, self.stream)

    def step(self, n: int):
        gs_batch_step(self.handle, n)

    def step_sequential(self, n: int):
        gs_batch_step_sequential(self.handle, n)

    def init(self):
        gs_batch_init(self.handle)

    @property
    def t(self) -> int:
        return gs_batch_get_step(self.handle)

    @t.setter
    def t(self, value: int):
        gs_batch_set_step(self.handle, value)

    def read(self, i: int):
        L = self.L[i]
        u = np.empty((L, L, L), dtype=np_dtype(self.dtype))
        v = np.empty_like(u)
        gs_batch_read(self.handle, i, GS_U, u)
        gs_batch_read(self.handle, i, GS_V, v)
        return u, v

    def write(self, i: int, u, v):
        gs_batch_write(self.handle, i, GS_U, np.ascontiguousarray(u, dtype=np_dtype(self.dtype)))
        gs_batch_write(self.handle, i, GS_V, np.ascontiguousarray(v, dtype=np_dtype(self.dtype)))

    def sync(self):
        gs_batch_sync(self.handle)

    def set_depth(self, depth: int):
        """Temporal-blocking depth of the persistent launch (1 = one step per pass)."""
        gs_batch_set_depth(self.handle, depth)

    def autotune(self, steps_per_trial: int = 20) -> dict:
        """Pick the batched launch's z-chunk, ring depth and temporal-blocking depth (state left unchanged)."""
        return gs_batch_autotune(self.handle, steps_per_trial)

    @property
    def info(self) -> dict:
        return gs_batch_info(self.handle)

    def close(self):
        if self.handle:
            gs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Convenience owner of one simulation whose fields live in PyTorch tensors.
# ---------------------------------------------------------------------------
class GrayScott:
    """One periodic L^3 Gray-Scott grid on the current CUDA device.

    The four field buffers are torch tensors (PyTorch's allocator); the stream
    is torch's current stream at construction.  All compute runs in libgs.
    """

    def __init__(self, L, Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0, noise=0.0, seed=0, dtype="f32",
                 device=None, stream=None):
        import torch
        self.L = int(L)
        self.dtype = _dtype_code(dtype)
        tdt = torch.float32 if self.dtype == GS_F32 else torch.float64
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._bufs = [torch.empty((L, L, L), dtype=tdt, device=dev) for _ in range(4)]
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.handle = gs_create_on(self.L, Du, Dv, F, k, dt, noise, seed, self.dtype, *self._bufs,
                                   stream=self.stream)

    def step(self, n: int):
        gs_step(self.handle, n)

    def init(self):
        gs_init(self.handle)

    def set_plan(self, kernel, tile_x=0, tile_y=0, tile_z=0, depth=0):
        gs_set_plan(self.handle, kernel, tile_x, tile_y, tile_z, depth)

    @property
    def arith(self) -> int:
        """GS_ARITH_IEEE, GS_ARITH_DS (FP64 fields in double-single arithmetic),
        GS_ARITH_FX (FP64 fields in 64-bit fixed-point arithmetic) or
        GS_ARITH_FXF (FP64 fields in 32-bit fixed point with a float remainder)."""
        return gs_get_arith(self.handle)

    @arith.setter
    def arith(self, value: int):
        gs_set_arith(self.handle, value)

    @property
    def boundary(self) -> int:
        return gs_get_boundary(self.handle)

    @boundary.setter
    def boundary(self, value: int):
        gs_set_boundary(self.handle, value)

    @property
    def plan(self) -> dict:
        """Every field of the current plan (gs_get_plan_full)."""
        return gs_get_plan_full(self.handle)

    def autotune(self, steps_per_trial: int = 12):
        """Pick the fastest plan for this grid (state is left unchanged)."""
        return gs_autotune(self.handle, steps_per_trial)

    def autotune_cached(self, path: str, steps_per_trial: int = 12):
        """Autotune once per device / grid configuration, remembered in the
        plan cache file `path`; returns (plan, hit)."""
        return gs_autotune_cached(self.handle, path, steps_per_trial)

    @property
    def t(self) -> int:
        return gs_get_step(self.handle)

    @t.setter
    def t(self, value: int):
        gs_set_step(self.handle, value)

    def read(self):
        """(u, v) of the current state as numpy arrays shaped [L, L, L] ([z, y, x])."""
        u = np.empty((self.L,) * 3, dtype=np_dtype(self.dtype))
        v = np.empty_like(u)
        gs_read(self.handle, GS_U, u)
        gs_read(self.handle, GS_V, v)
        return u, v

    def write(self, u, v):
        gs_write(self.handle, GS_U, np.ascontiguousarray(u, dtype=np_dtype(self.dtype)))
        gs_write(self.handle, GS_V, np.ascontiguousarray(v, dtype=np_dtype(self.dtype)))

    def tensors(self):
        """Device tensors (u, v) of the current state (valid until the next step)."""
        pu = gs_device_ptr(self.handle, GS_U)
        pv = gs_device_ptr(self.handle, GS_V)
        by = {b.data_ptr(): b for b in self._bufs}
        return by[pu], by[pv]

    def sync(self):
        gs_sync(self.handle)

    def stats(self, field: int = 0) -> dict:
        """min / max / mean / rms (and NaN count) of U (field 0) or V (field 1)."""
        return gs_stats(self.handle, field)

    def slice(self, field: int = 0, axis: int = 2, index=None):
        """One plane of a field as an L x L numpy array (default: the centre z plane)."""
        out = np.empty((self.L, self.L), dtype=np_dtype(self.dtype))
        gs_slice(self.handle, field, axis, self.L // 2 if index is None else index, out)
        return out

    def checkpoint(self, path: str):
        gs_checkpoint_save(self.handle, path)

    def restore(self, path: str):
        gs_checkpoint_load(self.handle, path)

    def snapshots(self, path: str) -> "SnapshotWriter":
        """A writer appending (step, U, V) records to `path` while the run goes on."""
        return SnapshotWriter(self, path)

    def close(self):
        if self.handle:
            gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SnapshotWriter:
    """Context manager over gs_snap_*: `write()` enqueues the current state."""

    def __init__(self, sim: GrayScott, path: str):
        self.sim = sim
        self.path = path
        self.handle = gs_snap_open(sim.handle, path)

    def write(self):
        gs_snap_write(self.handle)

    def flush(self):
        gs_snap_flush(self.handle)

    def info(self) -> dict:
        return gs_snap_info(self.handle)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            gs_snap_close(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


class SingleField:
    """One field f' = f + dt (D lap f) (the paper's "1-variable no random"
    kernel) on the current CUDA device, stepped on torch's current stream."""

    def __init__(self, L: int, D: float = 0.2, dt: float = 1.0, dtype: str = "f32",
                 boundary: int = GS_BOUNDARY_PERIODIC):
        import torch
        self.L, self.dtype = L, _dtype_code(dtype)
        self.handle = gs_single_create(L, D, dt, dtype, boundary)
        gs_single_set_stream(self.handle, torch.cuda.current_stream().cuda_stream)

    def write(self, f):
        gs_single_write(self.handle, np.ascontiguousarray(f, dtype=np_dtype(self.dtype)))

    def read(self):
        out = np.empty((self.L,) * 3, dtype=np_dtype(self.dtype))
        gs_single_read(self.handle, out)
        return out

    def step(self, n: int = 1):
        gs_single_step(self.handle, n)

    @property
    def info(self) -> dict:
        return gs_single_info(self.handle)

    def sync(self):
        gs_single_sync(self.handle)

    def close(self):
        if self.handle:
            gs_single_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

