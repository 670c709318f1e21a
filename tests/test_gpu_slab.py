"""z-slab decomposition (Section 3.3's domain decomposition, cut along z):
slabs of one grid, advanced `depth` steps per pass between halo exchanges,
must reproduce the single-grid run bit for bit, noise included."""
import numpy as np
import pytest

from paper_2309_10292_gb300 import gs
from tests.gpu_util import PAPER, need_cuda

pytestmark = pytest.mark.gpu


def _run_slabs(L, nslabs, depth, passes, dtype, noise=0.1, seed=9, bounds=None, streams=False):
    torch = need_cuda()
    bounds = bounds or gs.slab_bounds(L, nslabs)
    sts = [torch.cuda.Stream() if streams else None for _ in bounds]
    slabs = [gs.GrayScottSlab(L, z0, nz, depth, noise=noise, seed=seed, dtype=dtype, stream=st, **PAPER)
             for (z0, nz), st in zip(bounds, sts)]
    for s in slabs:
        s.init()
    for _ in range(passes):
        for s in slabs:
            s.run_pass()
        gs.slab_exchange(slabs)
    out = [s.read() for s in slabs]
    ts = [s.t for s in slabs]
    for s in slabs:
        s.close()
    return bounds, out, ts


@pytest.mark.parametrize("nslabs,depth", [(2, 1), (2, 3), (3, 2), (4, 1), (4, 3), (1, 2)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_slabs_equal_single_grid(nslabs, depth, dtype):
    L, passes = 30, 3  # uneven slabs (30 planes over 4 slabs: 7, 8, 7, 8)
    bounds, out, ts = _run_slabs(L, nslabs, depth, passes, dtype)
    assert ts == [passes * depth] * nslabs
    ref = gs.GrayScott(L, noise=0.1, seed=9, dtype=dtype, **PAPER)
    ref.step(passes * depth)
    ur, vr = ref.read()
    ref.close()
    for (z0, nz), (u, v) in zip(bounds, out):
        np.testing.assert_array_equal(u, ur[z0:z0 + nz])
        np.testing.assert_array_equal(v, vr[z0:z0 + nz])


def test_slabs_on_separate_streams_and_thin_slabs():
    # one stream per slab (the exchange orders them by events), and slabs as
    # thin as the halo (nz = depth)
    L, depth = 24, 3
    bounds = [(0, 3), (3, 3), (6, 9), (15, 6), (21, 3)]
    b, out, ts = _run_slabs(L, len(bounds), depth, 4, "f32", bounds=bounds, streams=True)
    ref = gs.GrayScott(L, noise=0.1, seed=9, dtype="f32", **PAPER)
    ref.step(4 * depth)
    ur, vr = ref.read()
    ref.close()
    for (z0, nz), (u, v) in zip(bounds, out):
        np.testing.assert_array_equal(u, ur[z0:z0 + nz])
        np.testing.assert_array_equal(v, vr[z0:z0 + nz])


def test_distributed_transport_in_one_process_equals_native_exchange():
    # slab_exchange_dist with a single rank keeps its copies local: one slab
    # covering the grid, exchanged through the host-side schedule
    torch = need_cuda()
    L, depth = 16, 2
    s = gs.GrayScottSlab(L, 0, L, depth, noise=0.1, seed=9, **PAPER)
    s.init()
    for _ in range(3):
        s.run_pass()
        torch.cuda.synchronize()
        gs.slab_exchange_dist(s.halo_views())
    u, v = s.read()
    s.close()
    ref = gs.GrayScott(L, noise=0.1, seed=9, **PAPER)
    ref.step(3 * depth)
    ur, vr = ref.read()
    ref.close()
    np.testing.assert_array_equal(u, ur)
    np.testing.assert_array_equal(v, vr)


def test_slab_argument_errors():
    torch = need_cuda()
    with pytest.raises(gs.GsError) as e:
        gs.GrayScottSlab(16, 0, 2, 3)  # nz < depth
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError):
        gs.GrayScottSlab(16, 16, 4, 1)  # z0 outside the grid
    a = gs.GrayScottSlab(16, 0, 8, 1)
    b = gs.GrayScottSlab(16, 9, 7, 1)  # does not start where a ends
    with pytest.raises(gs.GsError) as e:
        gs.slab_exchange([a, b])
    assert "starts" in str(e.value)
    a.close()
    b.close()
