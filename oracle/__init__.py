"""Gray-Scott CPU oracle — TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU restatement of the method, written from the paper (Eq. 1-3,
Section 3.1-3.2) and from the published definitions it cites, used only by
``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The product package never imports this module; it shares no
code with the CUDA path.

The arithmetic lives in ``gs_oracle.c`` (compiled with contraction off);
this module compiles it, loads it with ctypes and composes the surrogate
network (not in the paper) from its convolution primitives in numpy.

Pins (tests/test_oracle_pins.py): fixed point, octahedral symmetry, sine-mode
closed form, numpy brute force on tiny grids, light cone, translation
equivariance, conservation, MurmurHash3 vectors, exact noise distribution,
FFT convolution, adjoint identity, finite differences.  Adam and the MSE loss
below are pinned by hand-derived closed forms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile gs_oracle.c into liboracle.so (gcc, FP contraction off)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_fmix32.argtypes = [ctypes.c_uint32]
        lib.oracle_fmix32.restype = ctypes.c_uint32
        lib.oracle_noise_r.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32]
        lib.oracle_noise_r.restype = ctypes.c_double
        lib.oracle_noise_field.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, dp]
        lib.oracle_init.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_step.argtypes = [ctypes.c_int, dp, dp] + [ctypes.c_double] * 6 + [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_step.restype = ctypes.c_int
        lib.oracle_step_held.argtypes = [ctypes.c_int, dp, dp] + [ctypes.c_double] * 6 + [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_step_held.restype = ctypes.c_int
        lib.oracle_diffuse.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int64]
        lib.oracle_diffuse.restype = ctypes.c_int
        lib.oracle_window.argtypes = [ctypes.c_int] * 5 + [dp, dp] + [ctypes.c_double] * 6 + [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, dp, dp]
        lib.oracle_window.restype = ctypes.c_int
        lib.oracle_conv3d_fwd.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp, dp]
        lib.oracle_conv3d_bwd_data.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp]
        lib.oracle_conv3d_bwd_weight.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp, dp]
        lib.oracle_bf16_round.argtypes = [ctypes.c_int64, dp, dp]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> int:
    """Set the OpenMP thread count used by the oracle loops; returns the count in use."""
    return _load().oracle_set_threads(int(n))


# --------------------------------------------------------------------------
# Noise r (Eq. 1a), counter-based: see gs_oracle.c for the definition.
# --------------------------------------------------------------------------
def fmix32(h: int) -> int:
    return int(_load().oracle_fmix32(h & 0xFFFFFFFF))


def noise_r(seed: int, t: int, c: int) -> float:
    return float(_load().oracle_noise_r(seed, t, c))


def noise_field(seed: int, t: int, n: int) -> np.ndarray:
    r = np.empty(n, dtype=np.float64)
    _load().oracle_noise_field(seed, t, n, _dp(r))
    return r


# --------------------------------------------------------------------------
# Simulation (Eq. 1-3, periodic wrap).
# --------------------------------------------------------------------------
def init(L: int) -> tuple[np.ndarray, np.ndarray]:
    """Centred-cube initial state, arrays shaped [L, L, L] indexed [z, y, x]."""
    u = np.empty((L, L, L), dtype=np.float64)
    v = np.empty((L, L, L), dtype=np.float64)
    _load().oracle_init(L, _dp(u), _dp(v))
    return u, v


def step(u: np.ndarray, v: np.ndarray, nsteps: int, *, Du: float, Dv: float, F: float,
         k: float, dt: float, noise: float, seed: int, t0: int = 0):
    """Return (u, v) after ``nsteps`` forward-Euler steps starting at step index t0."""
    L = u.shape[0]
    assert u.shape == (L, L, L) and v.shape == (L, L, L)
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    vv = np.ascontiguousarray(v, dtype=np.float64).copy()
    rc = _load().oracle_step(L, _dp(uu), _dp(vv), Du, Dv, F, k, dt, noise, seed, t0, nsteps)
    if rc != 0:
        raise RuntimeError(f"oracle_step failed with status {rc}")
    return uu, vv


def step_held(u: np.ndarray, v: np.ndarray, nsteps: int, *, Du: float, Dv: float, F: float,
              k: float, dt: float, noise: float, seed: int, t0: int = 0):
    """As step(), with the paper's kernel's outer layer held (cells on the first or
    last layer of any axis keep their values; interior cells never wrap)."""
    L = u.shape[0]
    assert u.shape == (L, L, L) and v.shape == (L, L, L)
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    vv = np.ascontiguousarray(v, dtype=np.float64).copy()
    rc = _load().oracle_step_held(L, _dp(uu), _dp(vv), Du, Dv, F, k, dt, noise, seed, t0, nsteps)
    if rc != 0:
        raise RuntimeError(f"oracle_step_held failed with status {rc}")
    return uu, vv


def diffuse(f: np.ndarray, nsteps: int, *, D: float, dt: float, held: bool = False):
    """One field, f' = f + dt (D lap f) ("1-variable, no random"), periodic or with
    the outer layer held."""
    L = f.shape[0]
    assert f.shape == (L, L, L)
    ff = np.ascontiguousarray(f, dtype=np.float64).copy()
    rc = _load().oracle_diffuse(L, _dp(ff), D, dt, 1 if held else 0, nsteps)
    if rc != 0:
        raise RuntimeError(f"oracle_diffuse failed with status {rc}")
    return ff


def window(L: int, center, m: int, nsteps: int, *, Du, Dv, F, k, dt, noise, seed, t0=0,
           u0=None, v0=None):
    """(u, v) after nsteps on the (2m+1)^3 cells centred at center=(x, y, z) of an
    L^3 periodic grid that starts from the centred cube (or from full u0, v0),
    computed from the light cone only.  Arrays shaped [2m+1]*3 ([z, y, x])."""
    side = 2 * m + 1
    uo = np.empty((side, side, side))
    vo = np.empty((side, side, side))
    pu = pv = None
    if u0 is not None:
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        pu, pv = _dp(u0), _dp(v0)
    cx, cy, cz = center
    rc = _load().oracle_window(L, cx, cy, cz, m, pu, pv, Du, Dv, F, k, dt, noise, seed, t0, nsteps,
                               _dp(uo), _dp(vo))
    if rc != 0:
        raise RuntimeError(f"oracle_window failed with status {rc}")
    return uo, vo


# --------------------------------------------------------------------------
# Surrogate primitives (not in the paper): circular 3x3x3 conv, channels-last.
# x: [N, L, L, L, Cin]   w: [27, Cin, Cout]   b: [Cout]
# --------------------------------------------------------------------------
def conv3d_fwd(x: np.ndarray, w: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    N, L, _, _, Cin = x.shape
    Cout = w.shape[2]
    assert w.shape == (27, Cin, Cout)
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    y = np.empty((N, L, L, L, Cout), dtype=np.float64)
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    _load().oracle_conv3d_fwd(N, L, Cin, Cout, _dp(x), _dp(w),
                              None if bb is None else _dp(bb), _dp(y))
    return y


def conv3d_bwd_data(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    N, L, _, _, Cout = dy.shape
    Cin = w.shape[1]
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    dx = np.empty((N, L, L, L, Cin), dtype=np.float64)
    _load().oracle_conv3d_bwd_data(N, L, Cin, Cout, _dp(dy), _dp(w), _dp(dx))
    return dx


def conv3d_bwd_weight(x: np.ndarray, dy: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    N, L, _, _, Cin = x.shape
    Cout = dy.shape[4]
    x = np.ascontiguousarray(x, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    dw = np.empty((27, Cin, Cout), dtype=np.float64)
    db = np.empty(Cout, dtype=np.float64)
    _load().oracle_conv3d_bwd_weight(N, L, Cin, Cout, _dp(x), _dp(dy), _dp(dw), _dp(db))
    return dw, db


def bf16_round(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty_like(a)
    _load().oracle_bf16_round(a.size, _dp(a), _dp(out))
    return out


# --------------------------------------------------------------------------
# Surrogate network (not in the paper), FP64 with optional bf16 emulation at
# the points where the GPU path stores bf16 values.
#   x0 = (u - 1, v, F*FK_SCALE, k*FK_SCALE)                   [N, L, L, L, 4]
#        (u - 1 is zero on the u = 1 background, so bfloat16 keeps small
#        deviations at full relative precision)
#   h1 = relu(conv1(x0))                                      4 -> 32
#   h_l = h_{l-1} + relu(conv_l(h_{l-1})),  l = 2..5          32 -> 32
#   d  = conv6(h5)                                            32 -> 2
#   out = (u, v) + d          (state after K = 16 stencil steps)
# --------------------------------------------------------------------------
FK_SCALE = 20.0
CHANNELS = (4, 32, 32, 32, 32, 32, 2)


def _q(a, emulate):
    return bf16_round(a) if emulate else a


def surrogate_forward(params, u, v, F, k, *, emulate_bf16: bool = False):
    """params: list of 6 (w, b) pairs.  u, v: [N, L, L, L]; F, k: [N].

    Returns (out [N, L, L, L, 2], cache) where cache holds what the backward
    pass needs.  With emulate_bf16 the input, weights and hidden activations
    are rounded to bfloat16 where the GPU stores them in that format.
    """
    N, L = u.shape[0], u.shape[1]
    x0 = np.empty((N, L, L, L, 4), dtype=np.float64)
    x0[..., 0] = np.asarray(u, dtype=np.float64) - 1.0
    x0[..., 1] = v
    x0[..., 2] = (np.asarray(F, dtype=np.float64) * FK_SCALE)[:, None, None, None]
    x0[..., 3] = (np.asarray(k, dtype=np.float64) * FK_SCALE)[:, None, None, None]
    x0 = _q(x0, emulate_bf16)
    ws = [_q(w, emulate_bf16) for (w, _) in params]
    hs = [x0]
    zs = []
    z = conv3d_fwd(x0, ws[0], params[0][1])
    zs.append(z)
    h = _q(np.maximum(z, 0.0), emulate_bf16)
    hs.append(h)
    for l in range(1, 5):
        z = conv3d_fwd(h, ws[l], params[l][1])
        zs.append(z)
        h = _q(h + np.maximum(z, 0.0), emulate_bf16)
        hs.append(h)
    d = conv3d_fwd(h, ws[5], params[5][1])
    out = np.stack([u, v], axis=-1).astype(np.float64) + d
    return out, {"hs": hs, "zs": zs, "ws": ws}


def mse_loss(out: np.ndarray, target: np.ndarray) -> tuple[float, np.ndarray]:
    """Mean squared error over every element and its gradient w.r.t. out."""
    diff = out - target
    n = diff.size
    return float(np.sum(diff * diff) / n), 2.0 * diff / n


def surrogate_backward(cache, dout: np.ndarray, *, emulate_bf16: bool = False, return_dh: bool = False):
    """Gradients of the loss w.r.t. each layer's (w, b), given dL/dout.

    Chain rule through the network of surrogate_forward: for the residual
    layers h_{l+1} = h_l + relu(z_l), dL/dh_l = dL/dh_{l+1} + conv_l^T(dz_l)
    with dz_l = dL/dh_{l+1} * [z_l > 0].  With emulate_bf16 the values the
    GPU stores in bfloat16 are rounded where it rounds them: dL/dout (its
    storage has the first layer's 16-channel format) and every residual-path
    sum dL/dh_l; dz_l, a masked copy of a stored dL/dh_{l+1}, is then
    bfloat16 already.  With return_dh the list [dL/dh_1, ..., dL/dh_5] is
    returned as well.
    """
    hs, zs, ws = cache["hs"], cache["zs"], cache["ws"]
    grads = [None] * 6
    dhs = [None] * 6
    dout = _q(dout, emulate_bf16)
    dw, db = conv3d_bwd_weight(hs[5], dout)
    grads[5] = (dw, db)
    dh = _q(conv3d_bwd_data(dout, ws[5]), emulate_bf16)
    dhs[5] = dh
    for l in range(4, 0, -1):
        dz = dh * (zs[l] > 0.0)
        dw, db = conv3d_bwd_weight(hs[l], dz)
        grads[l] = (dw, db)
        dh = _q(dh + conv3d_bwd_data(dz, ws[l]), emulate_bf16)
        dhs[l] = dh
    dz = dh * (zs[0] > 0.0)
    dw, db = conv3d_bwd_weight(hs[0], dz)
    grads[0] = (dw, db)
    if return_dh:
        return grads, dhs[1:]
    return grads


def adam_update(p, g, m, v, t, *, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015, Algorithm 1), returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
