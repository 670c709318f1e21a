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
  * surrogate      He-uniform initial weights for the 6-layer conv network
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
