"""GPU tests of the batched persistent launch (many grids of different sizes).

Each instance must evolve bit for bit as a single-grid simulation with its
own (L_i, F_i, k_i) and seed + i, whether stepped by the persistent graph
launch or by per-instance launches, and must match the FP64 oracle within
the stated tolerances.
"""
import numpy as np
import pytest

import oracle
from paper_2309_10292_gb300 import gs, inputs
from tests.gpu_util import maxabs, need_cuda

pytestmark = pytest.mark.gpu

BASE = dict(Du=0.2, Dv=0.1, dt=1.0)
TOL = {"f64": 1e-10, "f32": 1e-4}


def small_batch(dtype, noise=0.1, seed=5):
    need_cuda()
    v = 4 if dtype == "f32" else 2
    Ls = [8, 16, 32, 48, 12 if v == 4 else 6, 64, 24, 4 if v == 4 else 2, 96, 128]
    F = list(np.linspace(0.01, 0.06, len(Ls)))
    k = list(np.linspace(0.07, 0.04, len(Ls)))
    b = gs.GrayScottBatch(Ls, F, k, noise=noise, seed=seed, dtype=dtype, **BASE)
    return b, Ls, F, k


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_matches_single_grids_bitwise(dtype):
    b, Ls, F, k = small_batch(dtype)
    b.step(25)
    assert b.t == 25
    for i, L in enumerate(Ls):
        s = gs.GrayScott(L, F=F[i], k=k[i], noise=0.1, seed=5 + i, dtype=dtype, **BASE)
        s.step(25)
        us, vs = s.read()
        ub, vb = b.read(i)
        np.testing.assert_array_equal(ub, us)
        np.testing.assert_array_equal(vb, vs)
        s.close()
    b.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_matches_oracle(dtype):
    b, Ls, F, k = small_batch(dtype)
    b.step(30)
    for i, L in enumerate(Ls):
        u0, v0 = oracle.init(L)
        uo, vo = oracle.step(u0, v0, 30, F=F[i], k=k[i], noise=0.1, seed=5 + i, **BASE)
        ub, vb = b.read(i)
        assert maxabs(ub, uo) <= TOL[dtype] and maxabs(vb, vo) <= TOL[dtype], (i, L)
    b.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_persistent_sequential_and_graph_reuse(dtype):
    # 7 persistent + 5 per-instance + 7 persistent (graph replay) == 19 persistent
    a, Ls, F, k = small_batch(dtype)
    a.step(19)
    b, _, _, _ = small_batch(dtype)
    b.step(7)
    b.step_sequential(5)
    b.step(7)
    assert b.t == 19
    info = b.info
    assert info["grid"] > 0 and info["items"] > 0
    for i in range(len(Ls)):
        ua, va = a.read(i)
        ub, vb = b.read(i)
        np.testing.assert_array_equal(ua, ub)
        np.testing.assert_array_equal(va, vb)
    a.close()
    b.close()


def test_batch_random_state_resume():
    # write a random state into some instances, resume at step 11
    b, Ls, F, k = small_batch("f64", seed=9)
    states = {}
    for i in (0, 3, 5):
        u0, v0 = inputs.random_fields(Ls[i], seed=40 + i)
        b.write(i, u0, v0)
        states[i] = (u0, v0)
    b.t = 11
    b.step(9)
    for i, (u0, v0) in states.items():
        uo, vo = oracle.step(u0, v0, 9, t0=11, F=F[i], k=k[i], noise=0.1, seed=9 + i, **BASE)
        ub, vb = b.read(i)
        assert maxabs(ub, uo) <= 1e-10 and maxabs(vb, vo) <= 1e-10
    b.close()


def test_batch_full_config_sampled():
    # the batched workload: 256 instances, L_i on {32..128}, F_i, k_i drawn
    # from the seeded generator, noise 0.1, run 40 steps; sampled instances
    # are bitwise equal to single-grid runs and match the oracle
    need_cuda()
    Ls, F, k = inputs.batch_instances(256, seed=0)
    b = gs.GrayScottBatch(Ls, F, k, noise=0.1, seed=42, dtype="f32", **BASE)
    b.step(40)
    for i in (0, 1, 100, 255):
        s = gs.GrayScott(Ls[i], F=F[i], k=k[i], noise=0.1, seed=42 + i, dtype="f32", **BASE)
        s.step(40)
        us, vs = s.read()
        ub, vb = b.read(i)
        np.testing.assert_array_equal(ub, us)
        np.testing.assert_array_equal(vb, vs)
        s.close()
    i = min(range(256), key=lambda j: Ls[j])
    u0, v0 = oracle.init(Ls[i])
    uo, vo = oracle.step(u0, v0, 40, F=F[i], k=k[i], noise=0.1, seed=42 + i, **BASE)
    ub, vb = b.read(i)
    assert maxabs(ub, uo) <= 1e-4 and maxabs(vb, vo) <= 1e-4
    b.close()


def test_batch_tail_split_alternating_pieces_bitwise():
    """The last grid / 2 work items of a launch are cut along z into four
    pieces that march in alternating directions: 40 grids of 128^3 are 2560
    items (16 runs of 1024 cells x 4 z-chunks each), the last 152 of a
    304-CTA launch become 608 pieces.  Instances whose items are cut, and one
    that is not, evolve bit for bit like single grids."""
    need_cuda()
    n, L = 40, 128
    F = list(np.linspace(0.02, 0.05, n))
    k = list(np.linspace(0.05, 0.065, n))
    b = gs.GrayScottBatch([L] * n, F, k, noise=0.1, seed=9, dtype="f32", **BASE)
    b.step(3)
    info = b.info
    base = n * (L * L // 1024) * (L // 32)
    m = min(info["grid"] // 2, base)
    assert info["items"] == base - m + 4 * m  # the last items were cut
    for i in (0, n - 2, n - 1):
        s = gs.GrayScott(L, F=F[i], k=k[i], noise=0.1, seed=9 + i, dtype="f32", **BASE)
        s.step(3)
        us, vs = s.read()
        ub, vb = b.read(i)
        np.testing.assert_array_equal(ub, us)
        np.testing.assert_array_equal(vb, vs)
        s.close()
    b.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_batch_bounded_waits_report_timeout(mode):
    # mode 1: the producer issues no copies; mode 2: CTA 0 never arrives at the
    # grid barrier.  Both must end in GS_ETIMEOUT, not a hang, and the batch
    # must work again afterwards.
    b, Ls, F, k = small_batch("f32", noise=0.0)
    gs.gs_batch_set_fault(b.handle, mode, 2_000_000)
    b.step(3)
    with pytest.raises(gs.GsError) as e:
        b.sync()
    assert e.value.status == gs.GS_ETIMEOUT
    gs.gs_batch_set_fault(b.handle, 0, 2_000_000_000)
    b.init()
    b.step(4)
    u, v = b.read(2)
    u0, v0 = oracle.init(Ls[2])
    uo, vo = oracle.step(u0, v0, 4, F=F[2], k=k[2], noise=0.0, seed=5 + 2, **BASE)
    assert maxabs(u, uo) <= 1e-4 and maxabs(v, vo) <= 1e-4
    b.close()


def test_batch_argument_errors():
    need_cuda()
    with pytest.raises(gs.GsError) as e:
        gs.GrayScottBatch([8, 10], [0.02, 0.02], [0.05, 0.05], dtype="f32")
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError):
        gs.GrayScottBatch([512], [0.02], [0.05], dtype="f32")
    b = gs.GrayScottBatch([8], [0.02], [0.05], dtype="f32")
    with pytest.raises(gs.GsError) as e:
        gs.gs_batch_read(b.handle, 1, gs.GS_U, np.empty(8 ** 3, dtype=np.float32))
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError):
        gs.gs_batch_read(b.handle, 0, gs.GS_U, np.empty(5, dtype=np.float32))
    b.close()


@pytest.mark.parametrize("tz,stages", [(3, 3), (16, 4), (64, 6), (256, 8)])
def test_batch_plan_changes_no_bits(tz, stages):
    """Any z-chunk / ring depth evolves every instance bit for bit like the default plan."""
    ref, Ls, _, _ = small_batch("f32")
    ref.step(13)
    b, _, _, _ = small_batch("f32")
    gs.gs_batch_set_plan(b.handle, tz, stages)
    b.step(13)
    for i in range(len(Ls)):
        ur, vr = ref.read(i)
        ub, vb = b.read(i)
        np.testing.assert_array_equal(ub, ur)
        np.testing.assert_array_equal(vb, vr)
    for bad in [(0, 6), (257, 6), (32, 2), (32, 9)]:
        with pytest.raises(gs.GsError):
            gs.gs_batch_set_plan(b.handle, *bad)
    b.step(2)  # still usable after the rejected plans
    ref.close()
    b.close()


def test_batch_autotune_keeps_state_and_results():
    need_cuda()
    Ls = [8, 16, 32, 48, 64]
    F = list(np.linspace(0.02, 0.05, len(Ls)))
    k = list(np.linspace(0.06, 0.045, len(Ls)))
    a = gs.GrayScottBatch(Ls, F, k, noise=0.1, seed=11, **BASE)
    b = gs.GrayScottBatch(Ls, F, k, noise=0.1, seed=11, **BASE)
    a.step(3)
    b.step(3)
    before = [a.read(i) for i in range(len(Ls))]
    plan = a.autotune(steps_per_trial=4)
    assert plan["tile_z"] in (16, 32, 64, 128) and plan["stages"] in (4, 6, 8) and plan["us_per_step"] > 0
    assert a.t == 3
    for i in range(len(Ls)):
        np.testing.assert_array_equal(a.read(i)[0], before[i][0])
        np.testing.assert_array_equal(a.read(i)[1], before[i][1])
    a.step(7)
    b.step(7)
    for i in range(len(Ls)):
        np.testing.assert_array_equal(a.read(i)[0], b.read(i)[0])
        np.testing.assert_array_equal(a.read(i)[1], b.read(i)[1])
    a.close()
    b.close()
