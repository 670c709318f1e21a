"""Seeded synthetic inputs shared by the GPU path's tests/benchmarks and the oracle.

This module holds no Gray-Scott arithmetic: it only draws random numbers
(numpy's PCG64, seeded) in the shapes the workloads use.  Both sides receive
the same arrays from here; neither side's results feed back into it.

Workloads (the paper's own runs are synthetic too: Listing 1's provenance
record gives Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1, noise=0.1):
  * plain grids    L in {64, 512, 1024}, centred-cube start (made on each side)
  * random grids   u, v ~ U[lo, hi) for tiny or odd L in parity tests
  * batch          256 instances, L_i uniform on {32, 48, 64, 96, 128},
                   F_i ~ U[0.01, 0.06], k_i ~ U[0.04, 0.07]
  * surrogate      He-uniform initial weights for the 6-layer conv network;
                   for gradient parity, sparse dyadic weights and fields on a
                   coarse grid (few significant bits), so that every sum the
                   network forms is exact in FP32 as in FP64
"""
from __future__ import annotations

import numpy as np

PAPER_PARAMS = dict(Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0)
BATCH_SIZES = (32, 48, 64, 96, 128)


def random_fields(L: int, seed: int, lo: float = 0.0, hi: float = 1.0):
    """u, v ~ U[lo, hi) as float64 arrays shaped [L, L, L] ([z, y, x])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(lo, hi, size=(L, L, L))
    v = rng.uniform(lo, hi, size=(L, L, L))
    return u, v


def batch_instances(n: int = 256, seed: int = 0, sizes=BATCH_SIZES):
    """Per-instance (L_i, F_i, k_i) for the batched workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ls = rng.choice(np.asarray(sizes, dtype=np.int64), size=n)
    Fs = rng.uniform(0.01, 0.06, size=n)
    ks = rng.uniform(0.04, 0.07, size=n)
    return [int(x) for x in Ls], [float(x) for x in Fs], [float(x) for x in ks]


def surrogate_init_params(seed: int = 0, channels=(4, 32, 32, 32, 32, 32, 2),
                          last_scale: float = 0.0):
    """He-uniform weights [27, Cin, Cout] and zero biases for each layer.

    The last layer is scaled by last_scale: 0 (the default) makes an untrained
    network exactly the identity map of its residual output ("no change").
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    nl = len(channels) - 1
    for l in range(nl):
        cin, cout = channels[l], channels[l + 1]
        bound = np.sqrt(6.0 / (27 * cin))
        if l == nl - 1:
            bound *= last_scale
        w = rng.uniform(-bound, bound, size=(27, cin, cout))
        b = np.zeros(cout)
        params.append((w, b))
    return params


def random_tensor(shape, seed: int, lo: float = -1.0, hi: float = 1.0):
    """Uniform float64 tensor of the given shape (conv parity inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def dyadic_fields(shape, seed: int, step: float = 1.0 / 16, lo: float = 0.0, hi: float = 1.0):
    """Float64 array of the given shape with values k * step in [lo, hi] (step a power of two)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(round((hi - lo) / step))
    return lo + step * rng.integers(0, n + 1, size=shape).astype(np.float64)


def surrogate_dyadic_params(seed: int = 0, channels=(4, 32, 32, 32, 32, 32, 2),
                            wstep: float = 0.25, density=(0.3, 0.02, 0.02, 0.02, 0.02, 0.005),
                            bstep: float = 1.0 / 64, bmax: int = 8):
    """Sparse weights on a dyadic grid: each entry is 0, or +-wstep, +-2 wstep
    with probability density[l]; biases are integers in [-bmax, bmax] times
    bstep.  Values with so few significant bits keep the network's sums
    exactly representable (in FP32 as in FP64) over several layers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for l in range(len(channels) - 1):
        cin, cout = channels[l], channels[l + 1]
        on = rng.uniform(size=(27, cin, cout)) < density[l]
        mag = rng.integers(1, 3, size=(27, cin, cout)) * rng.choice([-1.0, 1.0], size=(27, cin, cout))
        w = np.where(on, mag * wstep, 0.0)
        b = bstep * rng.integers(-bmax, bmax + 1, size=cout).astype(np.float64)
        params.append((w, b))
    return params
