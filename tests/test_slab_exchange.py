"""The z-slab halo exchange across ranks (slab_exchange_dist) on gloo CPU
ranks: every ghost plane must end up holding the neighbouring rank's
interior plane of the same global index (periodic in z)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2309_10292_gb300 import gs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, L, depth, bounds, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        glob = [torch.from_numpy(rng.uniform(size=(L, L, L))) for _ in range(2)]  # u, v on every rank
        z0, nz = bounds[rank]
        planes = nz + 2 * depth
        views, local = [], []
        for g in glob:
            f = torch.full((planes, L, L), float("nan"), dtype=torch.float64)
            f[depth:depth + nz] = g[z0:z0 + nz]
            local.append(f)
            views.append({"send_lo": f[depth:2 * depth], "send_hi": f[nz:nz + depth],
                          "recv_lo": f[0:depth], "recv_hi": f[nz + depth:nz + 2 * depth]})
        gs.slab_exchange_dist(views)
        ok = True
        for f, g in zip(local, glob):
            want = g[[(z0 - depth + zl) % L for zl in range(planes)]]
            ok &= bool(torch.equal(f, want))
        q.put((rank, ok))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,L,depth", [(2, 8, 1), (2, 9, 3), (3, 10, 2)])
def test_slab_halo_exchange_across_gloo_ranks(world, L, depth):
    bounds = gs.slab_bounds(L, world)
    assert all(nz >= depth for _, nz in bounds)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, L, depth, bounds, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(res[r] for r in range(world)), res
