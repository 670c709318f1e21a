"""Out-of-bounds writes, caught without a sanitizer: the four field buffers
of a grid live inside one device allocation, separated by guard bands
filled with a NaN bit pattern.  Every kernel runs a few steps (odd and even
counts, so both buffers of each pair are written); the guard bands must keep
their bits and the fields must equal an ordinary run's bit for bit.
"""
import numpy as np
import pytest

from paper_2309_10292_gb300 import gs
from tests.gpu_util import PAPER, need_cuda

pytestmark = pytest.mark.gpu

GUARD = 64 * 1024  # bytes before, between and after the four fields
POISON = {"f32": 0x7FC0BEEF, "f64": 0x7FF8DEADBEEFCAFE}


def _guarded(torch, L, dtype):
    esz = 4 if dtype == "f32" else 8
    itype = torch.int32 if dtype == "f32" else torch.int64
    ftype = torch.float32 if dtype == "f32" else torch.float64
    field = -(-L ** 3 * esz // 256) * 256  # bytes, rounded up to 256
    total = GUARD + 4 * (field + GUARD)
    raw = torch.empty(total // esz, dtype=itype, device="cuda")
    assert raw.data_ptr() % 256 == 0
    raw.fill_(POISON[dtype])
    fields, guards, pos = [], [(0, GUARD // esz)], GUARD // esz
    for _ in range(4):
        n = field // esz
        fields.append(raw[pos:pos + L ** 3].view(ftype).view(L, L, L))
        guards.append((pos + L ** 3, pos + n + GUARD // esz))
        pos += n + GUARD // esz
    return raw, fields, guards


def _check_guards(raw, guards, dtype):
    want = POISON[dtype]
    host = raw.cpu().numpy()
    for a, b in guards:
        bad = np.nonzero(host[a:b] != want)[0]
        assert bad.size == 0, f"guard band [{a}, {b}) overwritten at {a + bad[:5]}"


CASES = [
    # (L, dtype, kernel, tiles, depth, arith, boundary)
    (17, "f32", gs.GS_KERNEL_NAIVE, (0, 0, 0), 0, None, None),
    (17, "f64", gs.GS_KERNEL_NAIVE, (0, 0, 0), 0, None, None),
    (40, "f32", gs.GS_KERNEL_ZMARCH, (32, 16, 16), 0, None, None),
    (40, "f64", gs.GS_KERNEL_ZMARCH, (16, 6, 7), 0, None, None),
    (40, "f64", gs.GS_KERNEL_ZMARCH, (32, 16, 16), 0, gs.GS_ARITH_DS, None),
    (40, "f64", gs.GS_KERNEL_ZMARCH, (16, 6, 7), 0, gs.GS_ARITH_FX, None),
    (17, "f64", gs.GS_KERNEL_NAIVE, (0, 0, 0), 0, gs.GS_ARITH_FX, None),
    (48, "f32", gs.GS_KERNEL_TBLOCK, (16, 16, 16), 2, None, None),
    (48, "f32", gs.GS_KERNEL_TBLOCK, (16, 16, 24), 3, None, None),
    (48, "f32", gs.GS_KERNEL_TBLOCK, (16, 8, 48), 5, None, None),
    (40, "f32", gs.GS_KERNEL_ZMARCH, (32, 8, 40), 0, None, gs.GS_BOUNDARY_HELD),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"L{c[0]}-{c[1]}-k{c[2]}-d{c[4]}-a{c[5]}-b{c[6]}")
def test_kernels_stay_inside_their_fields(case):
    torch = need_cuda()
    L, dtype, kernel, tiles, depth, arith, boundary = case
    prm = dict(PAPER, noise=0.1, seed=9)
    raw, fields, guards = _guarded(torch, L, dtype)
    stream = torch.cuda.current_stream()
    h = gs.gs_create_on(L, prm["Du"], prm["Dv"], prm["F"], prm["k"], prm["dt"], prm["noise"], prm["seed"],
                        dtype, *fields, stream=stream)
    ref = gs.GrayScott(L, dtype=dtype, **prm)
    try:
        for sim in (h, ref.handle):
            if boundary is not None:
                gs.gs_set_boundary(sim, boundary)
            if arith is not None:
                gs.gs_set_arith(sim, arith)
        gs.gs_set_plan(h, kernel, *tiles, depth)
        for n in (3, 4):  # an odd and an even count: both buffers of each field written
            gs.gs_step(h, n)
            ref.step(n)
            gs.gs_sync(h)
            _check_guards(raw, guards, dtype)
        out = np.empty((L, L, L), dtype=np.float32 if dtype == "f32" else np.float64)
        for f in (gs.GS_U, gs.GS_V):
            gs.gs_read(h, f, out)
            want = ref.read()[f]
            np.testing.assert_array_equal(out, want)
        assert np.isfinite(out).all()
    finally:
        gs.gs_destroy(h)
        ref.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_noalloc_stays_inside_its_instances(dtype):
    # a caller-owned arena between guard bands; the alignment padding between
    # the instances' fields is poisoned too and must keep its bits
    torch = need_cuda()
    v4 = dtype == "f32"
    Ls = [8, 12 if v4 else 6, 32, 48, 4 if v4 else 2, 64]
    F = list(np.linspace(0.01, 0.06, len(Ls)))
    k = list(np.linspace(0.07, 0.04, len(Ls)))
    base = dict(Du=0.2, Dv=0.1, dt=1.0)
    ref = gs.GrayScottBatch(Ls, F, k, noise=0.1, seed=3, dtype=dtype, **base)
    offs, total = gs.noalloc_arena_offsets(Ls, dtype)
    esz = 4 if v4 else 8
    g = GUARD // esz
    itype = torch.int32 if v4 else torch.int64
    ftype = torch.float32 if v4 else torch.float64
    raw = torch.empty(g + total + g, dtype=itype, device="cuda")
    raw.fill_(POISON[dtype])
    arena = raw[g:g + total].view(ftype)
    assert arena.data_ptr() % 256 == 0
    live = np.zeros(total, dtype=bool)
    for i, L in enumerate(Ls):
        u, v = ref.read(i)
        for j, f in enumerate((u, v)):
            arena[offs[i][j]:offs[i][j] + L ** 3] = torch.from_numpy(f.ravel()).to("cuda")
        for j in range(4):
            live[offs[i][j]:offs[i][j] + L ** 3] = True
    torch.cuda.synchronize()
    gs.gs_batch_step_noalloc(Ls, F, k, base["Du"], base["Dv"], base["dt"], 0.1, 3, dtype, arena, 0, 0, 5,
                             torch.cuda.current_stream())
    ref.step(5)
    host = raw.cpu().numpy()
    want = POISON[dtype]
    assert (host[:g] == want).all() and (host[g + total:] == want).all()
    pad = host[g:g + total][~live]
    assert (pad == want).all(), f"{int((pad != want).sum())} padding elements overwritten"
    for i, L in enumerate(Ls):  # the state after an odd step count is in set 1
        got = arena[offs[i][2]:offs[i][2] + L ** 3].cpu().numpy().reshape(L, L, L)
        np.testing.assert_array_equal(got, ref.read(i)[0])
    ref.close()


# ---------------------------------------------------------------------------
# Buffers the library allocates itself (gs_set_alloc_guard): the batch's
# arena and tables, every surrogate buffer
# ---------------------------------------------------------------------------
class _LibraryGuards:
    def __enter__(self):
        gs.gs_set_alloc_guard(GUARD)
        return self

    def __exit__(self, *exc):
        gs.gs_set_alloc_guard(0)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_step_stays_inside_its_arena(dtype):
    torch = need_cuda()
    v4 = dtype == "f32"
    Ls = [8, 12 if v4 else 6, 32, 48, 4 if v4 else 2, 64, 128, 96]
    F = list(np.linspace(0.01, 0.06, len(Ls)))
    k = list(np.linspace(0.07, 0.04, len(Ls)))
    prm = dict(Du=0.2, Dv=0.1, dt=1.0, noise=0.1, seed=3, dtype=dtype)
    ref = gs.GrayScottBatch(Ls, F, k, **prm)
    with _LibraryGuards():
        b = gs.GrayScottBatch(Ls, F, k, **prm)
    try:
        assert gs.gs_batch_guard_check(b.handle) == 0
        for n in (3, 4):
            b.step(n)
            ref.step(n)
            assert gs.gs_batch_guard_check(b.handle) == 0
        for i in range(len(Ls)):
            for got, want in zip(b.read(i), ref.read(i)):
                np.testing.assert_array_equal(got, want)
    finally:
        b.close()
        ref.close()


@pytest.mark.parametrize("depth", [2, 4])
def test_blocked_batch_stays_inside_its_arena(depth):
    # the temporally blocked kernel: its cp.async staging and 16-byte stores
    # stay inside each instance's fields; its tables sit between guard bands
    need_cuda()
    Ls = [8, 12, 32, 48, 4, 64, 128, 96]
    F = list(np.linspace(0.01, 0.06, len(Ls)))
    k = list(np.linspace(0.07, 0.04, len(Ls)))
    prm = dict(Du=0.2, Dv=0.1, dt=1.0, noise=0.1, seed=3, dtype="f32")
    ref = gs.GrayScottBatch(Ls, F, k, **prm)
    with _LibraryGuards():
        b = gs.GrayScottBatch(Ls, F, k, **prm)
        b.set_depth(depth)
    try:
        assert gs.gs_batch_guard_check(b.handle) == 0
        for n in (2 * depth, depth + 1):
            b.step(n)
            ref.step(n)
            assert gs.gs_batch_guard_check(b.handle) == 0
        for i in range(len(Ls)):
            for got, want in zip(b.read(i), ref.read(i)):
                np.testing.assert_array_equal(got, want)
    finally:
        b.close()
        ref.close()


def _guarded_pair(torch, shape):
    # two FP32 output fields between guard bands (caller-owned outputs)
    n = int(np.prod(shape))
    g = GUARD // 4
    field = -(-n // 64) * 64
    raw = torch.empty(g + 2 * (field + g), dtype=torch.int32, device="cuda")
    raw.fill_(POISON["f32"])
    outs = [raw[g + i * (field + g):g + i * (field + g) + n].view(torch.float32).view(shape) for i in range(2)]
    guards = [(0, g)] + [(g + i * (field + g) + n, g + (i + 1) * (field + g)) for i in range(2)]
    return raw, outs, guards


@pytest.mark.parametrize("L,backend", [(32, gs.GS_SURR_MMA), (128, gs.GS_SURR_TCGEN05),
                                       (128, gs.GS_SURR_MMA), (256, gs.GS_SURR_TCGEN05)])
def test_surrogate_buffers_stay_inside(L, backend):
    torch = need_cuda()
    from paper_2309_10292_gb300 import inputs
    params = inputs.surrogate_init_params(seed=3, last_scale=0.3)
    g = torch.Generator(device="cuda").manual_seed(L)
    u = torch.rand((1, L, L, L), device="cuda", generator=g)
    v = torch.rand((1, L, L, L), device="cuda", generator=g) * 0.5
    with _LibraryGuards():
        s = gs.Surrogate(params)
    ref = gs.Surrogate(params)
    try:
        for net in (s, ref):
            gs.gs_surr_set_backend(net.handle, backend)
        raw, (uo, vo), guards = _guarded_pair(torch, (1, L, L, L))
        gs.gs_surr_forward(s.handle, 1, L, u, v, [0.03], [0.05], uo, vo)
        ru, rv = ref.forward(u, v, [0.03], [0.05])
        assert gs.gs_surr_guard_check(s.handle) == 0
        _check_guards(raw, guards, "f32")
        assert torch.equal(uo, ru) and torch.equal(vo, rv)
        if L <= 128:  # one training step: every gradient buffer
            with _LibraryGuards():  # the training workspace is allocated now
                ls = s.train_step(u, v, [0.03], [0.05], ru, rv, 1e-4)
            lr_ = ref.train_step(u, v, [0.03], [0.05], ru, rv, 1e-4)
            assert gs.gs_surr_guard_check(s.handle) == 0
            # the loss and (on the mma.sync path) the weight gradients are summed
            # with atomics, in no fixed order
            assert ls == pytest.approx(lr_, rel=1e-9)
            np.testing.assert_allclose(gs.gs_surr_get_params(s.handle), gs.gs_surr_get_params(ref.handle),
                                       rtol=1e-5, atol=1e-8)
    finally:
        s.close()
        ref.close()
