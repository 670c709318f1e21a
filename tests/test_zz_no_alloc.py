"""The allocation-free batched step against the allocating batched path.

gs_batch_step_noalloc serves callers that cannot allocate device memory on
their hot path; it keeps its tables in a fixed device array instead of
allocating them.  Its results must equal gs_batch_step's on two calls in a
row (the second one resuming from the first's state), it must not change the
device's free memory, and it must refuse batches beyond its fixed limits.
This file is collected last so a stop at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_2309_10292_gb300 import gs
from tests.gpu_util import need_cuda

pytestmark = pytest.mark.gpu

BASE = dict(Du=0.2, Dv=0.1, dt=1.0)


def _fill_arena(torch, ref, Ls, offs, arena):
    for i, L in enumerate(Ls):
        u, v = ref.read(i)
        n = L ** 3
        arena[offs[i][0]:offs[i][0] + n] = torch.from_numpy(u.ravel()).to(arena.device)
        arena[offs[i][1]:offs[i][1] + n] = torch.from_numpy(v.ravel()).to(arena.device)


def _fill_set(torch, ref, Ls, offs, arena, cur):
    for i, L in enumerate(Ls):
        u, v = ref.read(i)
        n = L ** 3
        arena[offs[i][2 * cur]:offs[i][2 * cur] + n] = torch.from_numpy(u.ravel()).to(arena.device)
        arena[offs[i][2 * cur + 1]:offs[i][2 * cur + 1] + n] = torch.from_numpy(v.ravel()).to(arena.device)


def _arena_state(arena, offs, i, L, cur):
    n = L ** 3
    u = arena[offs[i][2 * cur]:offs[i][2 * cur] + n].cpu().numpy().reshape(L, L, L)
    v = arena[offs[i][2 * cur + 1]:offs[i][2 * cur + 1] + n].cpu().numpy().reshape(L, L, L)
    return u, v


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_equals_batch_step_two_calls(dtype):
    torch = need_cuda()
    v4 = dtype == "f32"
    Ls = [8, 16, 32, 48, 12 if v4 else 6, 64, 24, 4 if v4 else 2, 96, 128]
    F = list(np.linspace(0.01, 0.06, len(Ls)))
    k = list(np.linspace(0.07, 0.04, len(Ls)))
    ref = gs.GrayScottBatch(Ls, F, k, noise=0.1, seed=5, dtype=dtype, **BASE)
    offs, total = gs.noalloc_arena_offsets(Ls, dtype)
    tdt = torch.float32 if v4 else torch.float64
    arena = torch.zeros(total, dtype=tdt, device="cuda")
    _fill_arena(torch, ref, Ls, offs, arena)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    # call 1: 10 steps from step 0 in set 0 -> state in set 0
    gs.gs_batch_step_noalloc(Ls, F, k, BASE["Du"], BASE["Dv"], BASE["dt"], 0.1, 5, dtype, arena,
                             0, 0, 10, stream)
    ref.step(10)
    for i, L in enumerate(Ls):
        ua, va = _arena_state(arena, offs, i, L, 0)
        ur, vr = ref.read(i)
        np.testing.assert_array_equal(ua, ur)
        np.testing.assert_array_equal(va, vr)

    # call 2: 7 more steps resuming at step 10 -> state in set 1; no device memory taken
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    gs.gs_batch_step_noalloc(Ls, F, k, BASE["Du"], BASE["Dv"], BASE["dt"], 0.1, 5, dtype, arena,
                             10, 0, 7, stream)
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    ref.step(7)
    for i, L in enumerate(Ls):
        ua, va = _arena_state(arena, offs, i, L, 1)
        ur, vr = ref.read(i)
        np.testing.assert_array_equal(ua, ur)
        np.testing.assert_array_equal(va, vr)
    ref.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_from_second_buffer_set_odd_steps_largest_L(dtype):
    # entry with the state in buffer set 1 at a nonzero step, an odd step
    # count (the state ends in set 0), and the largest instance the call
    # takes (L = 256; for FP64 its y tile is two rows)
    torch = need_cuda()
    v4 = dtype == "f32"
    Ls = [256, 16, 40 if v4 else 10, 64]
    F = [0.02, 0.035, 0.05, 0.03]
    k = [0.048, 0.06, 0.065, 0.05]
    ref = gs.GrayScottBatch(Ls, F, k, noise=0.1, seed=11, dtype=dtype, **BASE)
    ref.step(3)  # state at step 3
    offs, total = gs.noalloc_arena_offsets(Ls, dtype)
    tdt = torch.float32 if v4 else torch.float64
    arena = torch.full((total,), float("nan"), dtype=tdt, device="cuda")
    _fill_set(torch, ref, Ls, offs, arena, 1)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for call, n in enumerate((5, 2)):
        cur = 1 if call == 0 else 0
        gs.gs_batch_step_noalloc(Ls, F, k, BASE["Du"], BASE["Dv"], BASE["dt"], 0.1, 11, dtype, arena,
                                 ref.t, cur, n, stream)
        ref.step(n)
        for i, L in enumerate(Ls):
            ua, va = _arena_state(arena, offs, i, L, 0)
            ur, vr = ref.read(i)
            np.testing.assert_array_equal(ua, ur)
            np.testing.assert_array_equal(va, vr)
    ref.close()


def test_noalloc_rejects_batches_beyond_its_limits():
    torch = need_cuda()
    arena = torch.zeros(1024, dtype=torch.float32, device="cuda")
    with pytest.raises(gs.GsError) as e:
        gs.gs_batch_step_noalloc([8] * 257, [0.02] * 257, [0.05] * 257, 0.2, 0.1, 1.0, 0.0, 0, "f32",
                                 arena, 0, 0, 1)
    assert e.value.status == gs.GS_EINVAL and "256" in str(e.value)
    with pytest.raises(gs.GsError) as e:
        gs.gs_batch_step_noalloc([256] * 200, [0.02] * 200, [0.05] * 200, 0.2, 0.1, 1.0, 0.0, 0, "f32",
                                 arena, 0, 0, 1)
    assert e.value.status == gs.GS_EINVAL and "8192" in str(e.value)
