"""GPU tests of the temporally blocked form of the batched launch.

At depth D the persistent kernel advances every instance D steps per pass
over HBM (full-row tiles, a y halo recomputed level by level); a run of n
steps is n // D blocked passes plus n % D single steps.  Every instance must
still evolve bit for bit as with one step per pass (which the batch tests
tie to single grids and the oracle), and match the FP64 oracle itself.
"""
import numpy as np
import pytest

import oracle
from paper_2309_10292_gb300 import gs
from tests.gpu_util import maxabs, need_cuda

pytestmark = pytest.mark.gpu

BASE = dict(Du=0.2, Dv=0.1, dt=1.0)
# edges with 1 to 32 groups a row; L = 4 and 8 wrap the y and z halos more
# than once at the larger depths
LS = [32, 48, 8, 20, 64, 4, 96, 128, 12]


def make(Ls, noise, seed=9, depth=1, plan=None):
    need_cuda()
    F = list(np.linspace(0.015, 0.055, len(Ls)))
    k = list(np.linspace(0.065, 0.045, len(Ls)))
    b = gs.GrayScottBatch(Ls, F, k, noise=noise, seed=seed, dtype="f32", **BASE)
    if plan:
        gs.gs_batch_set_plan(b.handle, *plan)
    if depth > 1:
        b.set_depth(depth)
    return b, F, k


def assert_same(a, b, n):
    for i in range(n):
        ua, va = a.read(i)
        ub, vb = b.read(i)
        np.testing.assert_array_equal(ub, ua)
        np.testing.assert_array_equal(vb, va)


@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("noise", [0.0, 0.1])
def test_blocked_batch_bitwise_equal_to_single_steps(depth, noise):
    # 7 steps: whole passes plus a remainder on the single-step kernel, then
    # 2 * depth more steps replaying whole passes only
    ref, _, _ = make(LS, noise)
    b, _, _ = make(LS, noise, depth=depth)
    for n in (7, 2 * depth):
        ref.step(n)
        b.step(n)
        assert b.t == ref.t
        assert_same(ref, b, len(LS))
    info = b.info
    assert info["depth"] == depth and info["grid"] > 0 and info["items"] > 0
    ref.close()
    b.close()


@pytest.mark.parametrize("tz", [5, 16, 64])
def test_blocked_batch_z_chunks(tz):
    # z-chunks that do not divide L (ragged last chunk) and that exceed it
    ref, _, _ = make(LS, 0.1)
    b, _, _ = make(LS, 0.1, depth=3, plan=(tz, 4))
    ref.step(9)
    b.step(9)
    assert_same(ref, b, len(LS))
    ref.close()
    b.close()


def test_blocked_batch_matches_oracle():
    b, F, k = make(LS, 0.1, depth=3)
    b.step(12)
    for i, L in enumerate(LS):
        u0, v0 = oracle.init(L)
        uo, vo = oracle.step(u0, v0, 12, F=F[i], k=k[i], noise=0.1, seed=9 + i, **BASE)
        ub, vb = b.read(i)
        assert maxabs(ub, uo) <= 1e-4 and maxabs(vb, vo) <= 1e-4, (i, L)
    b.close()


def test_blocked_batch_largest_edge_and_limits():
    # L = 256 has 64 groups a row: one tile of 4 rows at D = 2, of 2 rows at
    # D = 3, none at D = 4
    Ls = [256, 32]
    ref, _, _ = make(Ls, 0.1)
    ref.step(6)
    for depth in (2, 3):
        b, _, _ = make(Ls, 0.1, depth=depth)
        b.step(6)
        assert_same(ref, b, len(Ls))
        b.close()
    b, _, _ = make(Ls, 0.1)
    with pytest.raises(gs.GsError) as e:
        b.set_depth(4)
    assert e.value.status == gs.GS_EINVAL
    for bad in (0, 5):
        with pytest.raises(gs.GsError):
            b.set_depth(bad)
    assert b.info["depth"] == 1
    b.step(6)  # still usable at depth 1 after the rejected depths
    assert_same(ref, b, len(Ls))
    b.close()
    ref.close()
    f64 = gs.GrayScottBatch([8, 16], [0.02, 0.03], [0.05, 0.06], dtype="f64", **BASE)
    with pytest.raises(gs.GsError) as e:
        f64.set_depth(2)
    assert e.value.status == gs.GS_EINVAL
    f64.close()


def test_blocked_batch_barrier_timeout_reported():
    # CTA 0 never arrives at the grid barrier after the first pass: the other
    # CTAs' bounded waits expire, GS_ETIMEOUT is reported, and the batch runs
    # correctly afterwards
    b, F, k = make(LS, 0.0, depth=2)
    gs.gs_batch_set_fault(b.handle, 2, 2_000_000)
    b.step(4)
    with pytest.raises(gs.GsError) as e:
        b.sync()
    assert e.value.status == gs.GS_ETIMEOUT
    gs.gs_batch_set_fault(b.handle, 0, 2_000_000_000)
    b.init()
    b.step(4)
    u, v = b.read(1)
    u0, v0 = oracle.init(LS[1])
    uo, vo = oracle.step(u0, v0, 4, F=F[1], k=k[1], noise=0.0, seed=9 + 1, **BASE)
    assert maxabs(u, uo) <= 1e-4 and maxabs(v, vo) <= 1e-4
    b.close()


def test_blocked_batch_autotune_depth_axis():
    Ls = [16, 32, 48, 64]
    a, _, _ = make(Ls, 0.0)
    ref, _, _ = make(Ls, 0.0)
    a.step(5)
    ref.step(5)
    before = [a.read(i) for i in range(len(Ls))]
    plan = a.autotune(steps_per_trial=4)
    assert plan["depth"] in (1, 2, 3, 4) and plan["tile_z"] in (16, 32, 64, 128) and plan["us_per_step"] > 0
    assert plan["depth"] > 1 or plan["tile_z"] <= 64
    assert a.info["depth"] == plan["depth"]
    assert a.t == 5
    for i in range(len(Ls)):
        np.testing.assert_array_equal(a.read(i)[0], before[i][0])
        np.testing.assert_array_equal(a.read(i)[1], before[i][1])
    a.step(11)
    ref.step(11)
    assert_same(ref, a, len(Ls))
    a.close()
    ref.close()
