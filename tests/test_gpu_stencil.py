"""GPU parity of the Gray-Scott stencil kernels against the FP64 CPU oracle.

Every call goes through the C-ABI (ctypes binding).  Tolerances: the GPU FP64
path must match the oracle within max-abs 1e-10 and the FP32 path within
1e-4 (stated per field); kernels must agree with each other bit for bit; the
noise draws are integer work and must match exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2309_10292_gb300 import gs, inputs
from tests.gpu_util import PAPER, maxabs, need_cuda

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}
V = {"f32": 4, "f64": 2}


def make(L, dtype, kernel=None, tiles=(0, 0, 0), **kw):
    need_cuda()
    prm = dict(PAPER)
    prm.update(kw)
    sim = gs.GrayScott(L, dtype=dtype, **prm)
    if kernel is not None:
        sim.set_plan(kernel, *tiles)
    return sim


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("seed,t", [(42, 0), (42, 1), (42, 999), (2 ** 40 + 3, 5)])
def test_noise_field_bitwise(dtype, seed, t):
    torch = need_cuda()
    n = 64 ** 3 + 5
    out = torch.empty(n, dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
    gs.gs_noise_field(seed, t, n, dtype, out)
    torch.cuda.synchronize()
    ref = oracle.noise_field(seed, t, n)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
def test_config1_parity_100_steps(dtype, kernel):
    # L=64, 100 steps, noise 0, centred cube: FP64 <= 1e-10, FP32 <= 1e-4
    L, n = 64, 100
    u0, v0 = oracle.init(L)
    uo, vo = oracle.step(u0, v0, n, **PAPER, noise=0.0, seed=0)
    sim = make(L, dtype, kernel, noise=0.0, seed=0)
    sim.step(n)
    u, v = sim.read()
    eu, ev = maxabs(u, uo), maxabs(v, vo)
    print(f"config1 {dtype} kernel={kernel}: max-abs u {eu:.3e} v {ev:.3e}")
    assert eu <= TOL[dtype] and ev <= TOL[dtype]
    assert sim.t == n


def _cases():
    out = []
    for L in (1, 2, 3, 4, 5, 8, 17, 32, 48, 64):
        for dtype in ("f64", "f32"):
            out.append((L, dtype, gs.GS_KERNEL_NAIVE, (0, 0, 0)))
    for dtype in ("f64", "f32"):
        v = V[dtype]
        for L, tiles in [(8, (8, 8, 8)), (8, (v, 3, 3)), (16, (8, 5, 7)), (32, (32, 8, 32)),
                         (48, (32, 5, 7)), (48, (16, 16, 48)), (64, (64, 1, 5)), (64, (16, 64, 9)),
                         (64, (8 if v == 4 else 4, 7, 64))]:
            out.append((L, dtype, gs.GS_KERNEL_ZMARCH, tiles))
    return out


@pytest.mark.parametrize("L,dtype,kernel,tiles", _cases())
def test_random_state_parity(L, dtype, kernel, tiles):
    # random initial state, noise on, 20 steps from step index 7
    n = 20
    u0, v0 = inputs.random_fields(L, seed=1000 + L, lo=0.0, hi=1.0)
    prm = dict(Du=0.2, Dv=0.1, F=0.035, k=0.06, dt=0.5, noise=0.1, seed=1234)
    uo, vo = oracle.step(u0, v0, n, t0=7, **prm)
    sim = make(L, dtype, kernel, tiles, **prm)
    sim.write(u0, v0)
    sim.t = 7
    sim.step(n)
    u, v = sim.read()
    assert maxabs(u, uo) <= TOL[dtype] and maxabs(v, vo) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("L,tiles", [(64, [(0, 0, 0), (32, 8, 16), (64, 4, 64), (16, 3, 5)]),
                                     (48, [(0, 0, 0), (16, 16, 7), (48, 16, 48)])])
def test_kernels_bitwise_equal(dtype, L, tiles):
    prm = dict(PAPER, noise=0.1, seed=7)
    ref = make(L, dtype, gs.GS_KERNEL_NAIVE, **prm)
    ref.step(30)
    ur, vr = ref.read()
    for t in tiles:
        sim = make(L, dtype, gs.GS_KERNEL_ZMARCH, t, **prm)
        sim.step(30)
        u, v = sim.read()
        np.testing.assert_array_equal(u, ur)
        np.testing.assert_array_equal(v, vr)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("L", [3, 16, 64])
def test_fixed_point_bitwise(dtype, L):
    sim = make(L, dtype, noise=0.0)
    sim.write(np.ones((L, L, L)), np.zeros((L, L, L)))
    sim.step(40)
    u, v = sim.read()
    assert np.all(u == 1.0) and np.all(v == 0.0)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_x_reflection_bitwise(dtype):
    L = 32
    sim = make(L, dtype, noise=0.0)
    sim.step(40)
    u, v = sim.read()
    np.testing.assert_array_equal(u, u[:, :, ::-1])
    np.testing.assert_array_equal(v, v[:, :, ::-1])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_resume_from_state_bitwise(dtype):
    L = 32
    prm = dict(PAPER, noise=0.1, seed=99)
    a = make(L, dtype, **prm)
    a.step(30)
    ua, va = a.read()
    b = make(L, dtype, **prm)
    b.step(13)
    ub, vb = b.read()
    c = make(L, dtype, **prm)
    c.write(ub, vb)
    c.t = 13
    c.step(17)
    uc, vc = c.read()
    np.testing.assert_array_equal(uc, ua)
    np.testing.assert_array_equal(vc, va)


@pytest.mark.parametrize("L,dtype", [(512, "f32"), (512, "f64"), (1024, "f32")])
def test_full_size_sampled_cells(L, dtype):
    # the benchmark's workload (centred cube, noise 0.1, seed 42, default plan)
    # checked at sampled cells against the oracle's light-cone computation
    n = 16
    prm = dict(PAPER, noise=0.1, seed=42)
    sim = make(L, dtype, **prm)
    assert sim.plan["kernel"] == gs.GS_KERNEL_ZMARCH
    sim.step(n)
    u, v = sim.read()
    rng = np.random.default_rng(L)
    centers = [(L // 2, L // 2, L // 2), (L // 2 - 9, L // 2 + 4, L // 2 - 1), (0, 0, 0),
               (L - 1, 5, L // 2)] + [tuple(int(c) for c in rng.integers(0, L, 3)) for _ in range(3)]
    m = 2
    for c in centers:
        uo, vo = oracle.window(L, c, m, n, **prm)
        idx = [(np.arange(-m, m + 1) + cc) % L for cc in c]
        sel = np.ix_(idx[2], idx[1], idx[0])
        assert maxabs(u[sel], uo) <= TOL[dtype], c
        assert maxabs(v[sel], vo) <= TOL[dtype], c
    del u, v
    sim.close()


def test_largest_grid_sampled_cells():
    # the largest edge (1625^3 cells: the noise counter is 32-bit), FP32:
    # 69 GB of fields; L is not a multiple of 4, so the one-thread-per-cell
    # kernel runs.  Planes around sampled cells are read with gs_slice.
    L, n, m = gs.GS_MAX_L, 3, 2
    assert L ** 3 < 2 ** 32 <= (L + 1) ** 3
    prm = dict(PAPER, noise=0.1, seed=42)
    sim = make(L, "f32", **prm)
    assert sim.plan["kernel"] == gs.GS_KERNEL_NAIVE
    sim.step(n)
    for c in [(L // 2, L // 2, L // 2), (0, 0, 0), (L - 1, 3, L - 2), (812, 809, 815)]:
        uo, vo = oracle.window(L, c, m, n, **prm)
        zs = [(c[2] + d) % L for d in range(-m, m + 1)]
        idx = [(np.arange(-m, m + 1) + cc) % L for cc in c[:2]]
        for fld, ref in ((gs.GS_U, uo), (gs.GS_V, vo)):
            planes = np.stack([sim.slice(fld, 2, z) for z in zs])  # [z][y][x]
            got = planes[np.ix_(range(len(zs)), idx[1], idx[0])]
            assert maxabs(got, ref) <= TOL["f32"], (c, fld)
    sim.close()
    with pytest.raises(gs.GsError):
        gs.GrayScott(L + 1, dtype="f32", **prm)


def test_step_zero_and_argument_errors():
    sim = make(8, "f32")
    sim.step(0)
    assert sim.t == 0
    with pytest.raises(gs.GsError) as e:
        gs.gs_read(sim.handle, gs.GS_U, np.empty(7, dtype=np.float32))
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError):
        gs.gs_step(sim.handle, -1)
    odd = make(17, "f32")
    with pytest.raises(gs.GsError) as e:
        odd.set_plan(gs.GS_KERNEL_ZMARCH)
    assert e.value.status == gs.GS_EINVAL
    assert odd.plan["kernel"] == gs.GS_KERNEL_NAIVE
    with pytest.raises(gs.GsError):
        sim.set_plan(gs.GS_KERNEL_ZMARCH, 6, 4, 4)  # tile_x not a multiple of 4


def test_bounded_wait_timeout_reports_and_recovers():
    # failure injection: the producer issues no copies, the consumers' bounded
    # waits expire, the next sync reports GS_ETIMEOUT and the context stays usable
    L = 32
    sim = make(L, "f32", gs.GS_KERNEL_ZMARCH, noise=0.0)
    gs.gs_set_fault(sim.handle, 1, 1_000_000)
    sim.step(1)
    with pytest.raises(gs.GsError) as e:
        sim.sync()
    assert e.value.status == gs.GS_ETIMEOUT
    gs.gs_set_fault(sim.handle, 0, 2_000_000_000)
    sim.init()
    sim.step(5)
    u, v = sim.read()
    u0, v0 = oracle.init(L)
    uo, vo = oracle.step(u0, v0, 5, **PAPER, noise=0.0, seed=0)
    assert maxabs(u, uo) <= 1e-4 and maxabs(v, vo) <= 1e-4


def test_grids_on_two_streams_step_at_the_same_time():
    # each grid's z-march and blocked kernels draw work units from that grid's
    # own counter, so two grids stepping at once on two streams leave each
    # other's results bit for bit as when they step one after the other
    import torch
    L = 96
    prm = dict(PAPER, noise=0.1, seed=5)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    grids = []
    for st, plan in ((s1, (gs.GS_KERNEL_ZMARCH, 32, 4, 16)), (s2, (gs.GS_KERNEL_TBLOCK, 32, 8, 32, 2))):
        g = gs.GrayScott(L, dtype="f32", stream=st, **prm)
        g.set_plan(*plan)
        grids.append(g)
    for _ in range(8):
        for g in grids:
            g.step(4)
    outs = [g.read() for g in grids]
    refs = []
    for plan in ((gs.GS_KERNEL_ZMARCH, 32, 4, 16), (gs.GS_KERNEL_TBLOCK, 32, 8, 32, 2)):
        r = make(L, "f32", **prm)
        r.set_plan(*plan)
        r.step(32)
        refs.append(r.read())
        r.close()
    for (u, v), (ur, vr) in zip(outs, refs):
        np.testing.assert_array_equal(u, ur)
        np.testing.assert_array_equal(v, vr)
    for g in grids:
        g.close()


# ---------------------------------------------------------------------------
# Temporal blocking: `depth` fused steps per HBM pass (FP32)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,tiles,depth,n", [(32, (16, 8, 32), 2, 9), (32, (8, 4, 5), 3, 10),
                                             (48, (16, 8, 7), 4, 11), (64, (64, 16, 64), 2, 6),
                                             (64, (32, 8, 13), 4, 8), (16, (4, 2, 3), 2, 5),
                                             (32, (16, 8, 32), 5, 12), (32, (8, 4, 7), 6, 14),
                                             (48, (16, 8, 9), 7, 15), (32, (16, 8, 32), 8, 17),
                                             (24, (4, 2, 5), 8, 9)])
def test_tblock_bitwise_equal_to_plain(L, tiles, depth, n):
    prm = dict(PAPER, noise=0.1, seed=3)
    ref = make(L, "f32", gs.GS_KERNEL_NAIVE, **prm)
    ref.step(n)
    ur, vr = ref.read()
    sim = make(L, "f32", **prm)
    sim.set_plan(gs.GS_KERNEL_TBLOCK, *tiles, depth)
    assert sim.plan["kernel"] == gs.GS_KERNEL_TBLOCK and sim.plan["depth"] == depth
    sim.step(n)  # n // depth blocked passes, the rest single steps
    u, v = sim.read()
    np.testing.assert_array_equal(u, ur)
    np.testing.assert_array_equal(v, vr)
    assert sim.t == n


def test_tblock_config1_parity():
    L, n = 64, 100
    u0, v0 = oracle.init(L)
    uo, vo = oracle.step(u0, v0, n, **PAPER, noise=0.0, seed=0)
    sim = make(L, "f32", noise=0.0, seed=0)
    sim.set_plan(gs.GS_KERNEL_TBLOCK, 32, 8, 32, 4)
    sim.step(n)
    u, v = sim.read()
    assert maxabs(u, uo) <= 1e-4 and maxabs(v, vo) <= 1e-4


@pytest.mark.parametrize("depth,tile", [(2, (64, 16)), (4, (64, 8)), (8, (16, 8))])
def test_tblock_full_size_sampled_cells(depth, tile):
    # the L=1024 FP32 workload with temporal blocking, sampled against the oracle
    L, n = 1024, 16
    prm = dict(PAPER, noise=0.1, seed=42)
    sim = make(L, "f32", **prm)
    sim.set_plan(gs.GS_KERNEL_TBLOCK, *tile, 64, depth)
    sim.step(n)
    u, v = sim.read()
    m = 2
    for c in [(L // 2, L // 2, L // 2), (0, 0, 0), (L - 1, 63, 64), (64, 15, L - 1), (300, 700, 5)]:
        uo, vo = oracle.window(L, c, m, n, **prm)
        idx = [(np.arange(-m, m + 1) + cc) % L for cc in c]
        sel = np.ix_(idx[2], idx[1], idx[0])
        assert maxabs(u[sel], uo) <= 1e-4 and maxabs(v[sel], vo) <= 1e-4, c
    sim.close()


def test_tblock_rejects_unsupported_plans():
    sim = make(64, "f64")
    with pytest.raises(gs.GsError) as e:
        sim.set_plan(gs.GS_KERNEL_TBLOCK, 32, 8, 32, 2)
    assert e.value.status == gs.GS_EINVAL
    s32 = make(48, "f32")
    for bad in [(32, 8, 8, 2), (16, 7, 8, 2), (16, 8, 8, 9), (16, 8, 8, 1)]:
        with pytest.raises(gs.GsError):
            s32.set_plan(gs.GS_KERNEL_TBLOCK, *bad)
    assert s32.plan["kernel"] == gs.GS_KERNEL_ZMARCH
    s64 = make(64, "f32")
    with pytest.raises(gs.GsError, match="shared memory"):
        s64.set_plan(gs.GS_KERNEL_TBLOCK, 32, 16, 8, 8)  # depth 8 on a 32 x 16 tile: ~405 KB


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_autotune_restores_state_and_keeps_fastest_plan(dtype):
    L = 64
    prm = dict(PAPER, noise=0.1, seed=8)
    a = make(L, dtype, **prm)
    a.step(7)
    u0, v0 = a.read()
    best, trials = a.autotune(steps_per_trial=12)
    assert a.t == 7
    u1, v1 = a.read()
    np.testing.assert_array_equal(u0, u1)
    np.testing.assert_array_equal(v0, v1)
    assert len(trials) > 3
    fastest = min(trials, key=lambda r: r["us_per_step"])
    assert best["us_per_step"] == fastest["us_per_step"]
    assert a.plan == best  # every field, the tuner's time included
    kinds = {r["kernel"] for r in trials}
    assert gs.GS_KERNEL_NAIVE in kinds and gs.GS_KERNEL_ZMARCH in kinds
    if dtype == "f32":
        assert gs.GS_KERNEL_TBLOCK in kinds
    a.step(13)
    ref = make(L, dtype, gs.GS_KERNEL_NAIVE, **prm)
    ref.step(20)
    ua, va = a.read()
    ur, vr = ref.read()
    np.testing.assert_array_equal(ua, ur)
    np.testing.assert_array_equal(va, vr)
    a.set_plan(best["kernel"], best["tile_x"], best["tile_y"], best["tile_z"], best["depth"])
    assert a.plan["us_per_step"] == 0.0  # a plan set by hand carries no tuner time


# ---------------------------------------------------------------------------
# FP64 fields in double-single (GS_ARITH_DS), fixed-point (GS_ARITH_FX) and
# fixed-point-with-remainder (GS_ARITH_FXF) arithmetic
# ---------------------------------------------------------------------------
ARITHS = [gs.GS_ARITH_DS, gs.GS_ARITH_FX, gs.GS_ARITH_FXF]
ARITH_IDS = ["ds", "fx", "fxf"]


def make_ar(arith, L, kernel=None, tiles=(0, 0, 0), **kw):
    sim = make(L, "f64", kernel, tiles, **kw)
    sim.arith = arith
    return sim


# partial tiles in x and y (the z-march kernel converts each staged plane in
# place, its own cells and the halo entries each thread alone reads)
@pytest.mark.parametrize("arith", ARITHS, ids=ARITH_IDS)
@pytest.mark.parametrize("tiles", [(32, 16, 16), (16, 6, 7), (8, 4, 40), (40, 1, 3)])
def test_conv_arith_zmarch_partial_tiles_bitwise_equal_plain(arith, tiles):
    L, n = 40, 12
    prm = dict(PAPER, noise=0.1, seed=11)
    u0, v0 = inputs.random_fields(L, seed=5, lo=0.0, hi=1.0)
    a = make_ar(arith, L, gs.GS_KERNEL_NAIVE, **prm)
    b = make_ar(arith, L, gs.GS_KERNEL_ZMARCH, tiles, **prm)
    for s in (a, b):
        s.write(u0, v0)
        s.step(n)
    ua, va = a.read()
    ub, vb = b.read()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    uo, vo = oracle.step(u0, v0, n, **prm)
    assert max(maxabs(ub, uo), maxabs(vb, vo)) <= TOL["f64"]


@pytest.mark.parametrize("arith", ARITHS, ids=ARITH_IDS)
@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
def test_conv_arith_config1_parity(arith, kernel):
    L, n = 64, 100
    u0, v0 = oracle.init(L)
    uo, vo = oracle.step(u0, v0, n, **PAPER, noise=0.0, seed=0)
    sim = make_ar(arith, L, kernel, noise=0.0, seed=0)
    assert sim.arith == arith
    sim.step(n)
    u, v = sim.read()
    err = max(maxabs(u, uo), maxabs(v, vo))
    print(f"arith {arith} config 1: max-abs error vs oracle {err:.3e}")
    assert err <= TOL["f64"]


@pytest.mark.parametrize("arith", ARITHS, ids=ARITH_IDS)
@pytest.mark.parametrize("L", [48, 17, 5, 2])
def test_conv_arith_random_state_parity_with_noise(arith, L):
    # dt = 0.5: the products du dt are taken (dt = 1 skips them)
    prm = dict(Du=0.2, Dv=0.1, F=0.035, k=0.06, dt=0.5, noise=0.1, seed=77)
    u0, v0 = inputs.random_fields(L, seed=600 + L, lo=0.0, hi=1.0)
    sim = gs.GrayScott(L, dtype="f64", **prm)
    sim.arith = arith
    sim.write(u0, v0)
    sim.t = 7
    sim.step(40)
    u, v = sim.read()
    uo, vo = oracle.step(u0, v0, 40, t0=7, **prm)
    err = max(maxabs(u, uo), maxabs(v, vo))
    print(f"arith {arith} L={L}: max-abs error vs oracle {err:.3e}")
    assert err <= TOL["f64"]


@pytest.mark.parametrize("arith", ARITHS, ids=ARITH_IDS)
def test_conv_arith_kernels_bitwise_equal_and_close_to_ieee(arith):
    L, n = 64, 60
    prm = dict(PAPER, noise=0.1, seed=3)
    a = make_ar(arith, L, gs.GS_KERNEL_NAIVE, **prm)
    b = make_ar(arith, L, gs.GS_KERNEL_ZMARCH, **prm)
    c = make(L, "f64", gs.GS_KERNEL_ZMARCH, **prm)
    for s in (a, b, c):
        s.step(n)
    ua, va = a.read()
    ub, vb = b.read()
    uc, vc = c.read()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    d = max(maxabs(ua, uc), maxabs(va, vc))
    print(f"arith {arith} vs IEEE FP64 after {n} steps: {d:.3e}")
    assert 0 < d <= 1e-11


@pytest.mark.parametrize("arith", ARITHS, ids=ARITH_IDS)
def test_conv_arith_full_size_sampled_cells(arith):
    L, n, m = 512, 16, 2
    prm = dict(PAPER, noise=0.1, seed=42)
    sim = make_ar(arith, L, **prm)
    sim.step(n)
    for c in [(L // 2, L // 2, L // 2), (0, 0, 0), (L - 1, 5, L // 2)]:
        uo, vo = oracle.window(L, c, m, n, **prm)
        zs = [(c[2] + d) % L for d in range(-m, m + 1)]
        idx = [(np.arange(-m, m + 1) + cc) % L for cc in c[:2]]
        for fld, ref in ((gs.GS_U, uo), (gs.GS_V, vo)):
            planes = np.stack([sim.slice(fld, 2, z) for z in zs])
            assert maxabs(planes[np.ix_(range(len(zs)), idx[1], idx[0])], ref) <= TOL["f64"], (c, fld)
    sim.close()


@pytest.mark.parametrize("arith", ARITHS, ids=ARITH_IDS)
@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
def test_conv_arith_packed_between_the_steps_of_a_call(kernel, arith):
    # the FP64 arithmetics other than IEEE keep the fields in their own packed
    # form between the steps of one gs_step call and round them to FP64 only
    # at its end: n steps in one call and in n calls differ by those
    # roundings, and both match the oracle
    L, n = 32, 30
    prm = dict(PAPER, noise=0.1, seed=21)
    u0, v0 = inputs.random_fields(L, seed=8, lo=0.0, hi=1.0)
    one = make_ar(arith, L, kernel, **prm)
    many = make_ar(arith, L, kernel, **prm)
    for s in (one, many):
        s.write(u0, v0)
    one.step(n)
    for _ in range(n):
        many.step(1)
    assert one.t == many.t == n
    u1, v1 = one.read()
    un, vn = many.read()
    uo, vo = oracle.step(u0, v0, n, **prm)
    e1 = max(maxabs(u1, uo), maxabs(v1, vo))
    en = max(maxabs(un, uo), maxabs(vn, vo))
    d = max(maxabs(u1, un), maxabs(v1, vn))
    print(f"arith {arith}, {n} steps: one call {e1:.3e}, {n} calls {en:.3e} from the oracle; apart {d:.3e}")
    assert e1 <= TOL["f64"] and en <= TOL["f64"] and d <= 1e-11
    # a second call continues from FP64 fields exactly as a fresh object would
    fresh = make_ar(arith, L, kernel, **prm)
    fresh.write(u1, v1)
    fresh.t = n
    one.step(5)
    fresh.step(5)
    np.testing.assert_array_equal(one.read()[0], fresh.read()[0])
    np.testing.assert_array_equal(one.read()[1], fresh.read()[1])


def test_conv_arith_only_for_fp64_fields():
    s32 = make(16, "f32")
    for ar in ARITHS:
        with pytest.raises(gs.GsError) as e:
            s32.arith = ar
        assert e.value.status == gs.GS_EINVAL and s32.arith == gs.GS_ARITH_IEEE
    s64 = make(16, "f64")
    with pytest.raises(gs.GsError):
        s64.arith = 5


@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
@pytest.mark.parametrize("arith,bad", [(gs.GS_ARITH_FX, 2048.0), (gs.GS_ARITH_FXF, 4.5), (gs.GS_ARITH_FXF, -4.0)],
                         ids=["fx", "fxf", "fxf-neg"])
def test_fixed_point_reports_values_outside_its_range(kernel, arith, bad):
    # |u| >= 1024 (FX) or >= 4 (FXF) cannot be held in the fixed-point
    # format: the next check reports it once, and the object stays usable
    L = 16
    sim = make_ar(arith, L, kernel, noise=0.0, seed=0)
    u0, v0 = inputs.random_fields(L, seed=3, lo=0.0, hi=1.0)
    u0[3, 4, 5] = bad
    sim.write(u0, v0)
    sim.step(1)
    with pytest.raises(gs.GsError) as e:
        sim.sync()
    assert e.value.status == gs.GS_EINVAL and "fixed-point range" in str(e.value)
    sim.init()
    sim.step(2)
    sim.sync()
    sim.close()


@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
def test_fxf_reports_results_outside_its_range(kernel):
    # inputs inside the range (a plane of u = 3.9) that one step pushes
    # past 4 (the oracle's step from the same fields reaches |u| 4.09 and
    # |v| 4.75): the check of the step's results reports it
    L = 16
    sim = make_ar(gs.GS_ARITH_FXF, L, kernel, noise=0.5, seed=4)
    u0, v0 = inputs.random_fields(L, seed=8, lo=0.0, hi=1.0)
    u0[3, :, :] = 3.9
    sim.write(u0, v0)
    sim.step(1)
    with pytest.raises(gs.GsError) as e:
        sim.sync()
    assert e.value.status == gs.GS_EINVAL and "fixed-point range" in str(e.value)
    sim.init()
    sim.step(2)
    sim.sync()
    sim.close()


# ---------------------------------------------------------------------------
# Plan cache (gs_autotune_cached)
# ---------------------------------------------------------------------------
def test_plan_cache_tunes_once_per_configuration(tmp_path):
    need_cuda()
    path = str(tmp_path / "plans.txt")
    with open(path, "w") as f:
        f.write("not a plan line\ngs-plan-v1 too few fields\n")
    a = make(24, "f32", noise=0.1, seed=1)
    best, hit = a.autotune_cached(path, steps_per_trial=1)
    assert not hit and best["us_per_step"] > 0
    lines = [l for l in open(path) if l.startswith("gs-plan-v1 ") and len(l.split()) == 9]
    assert len(lines) == 1 and "/L24/f32/ieee/periodic/noise" in lines[0]
    # same configuration: the cached plan, no timing, same fields afterwards
    b = make(24, "f32", noise=0.1, seed=1)
    best2, hit2 = b.autotune_cached(path, steps_per_trial=1)
    assert hit2 and best2 == best
    assert b.plan["kernel"] == best["kernel"] and b.plan["tile_x"] == best["tile_x"]
    for s in (a, b):
        s.step(5)
    ua, va = a.read()
    ub, vb = b.read()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    # another configuration (no noise) is a miss and appends a second line
    c = make(24, "f32", noise=0.0, seed=1)
    _, hit3 = c.autotune_cached(path, steps_per_trial=1)
    assert not hit3
    assert sum(1 for l in open(path) if l.startswith("gs-plan-v1 ") and len(l.split()) == 9) == 2
    # a directory is not a writable cache file
    d = make(16, "f32")
    with pytest.raises(gs.GsError) as e:
        d.autotune_cached(str(tmp_path), steps_per_trial=1)
    assert e.value.status == gs.GS_EIO


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_async_copies_match_blocking_ones_on_two_streams(dtype):
    # two grids on two streams: async write -> steps -> async read per grid,
    # both enqueued before either stream is waited on; the fields must equal
    # those of the blocking calls and the oracle
    import torch
    need_cuda()
    L, n = 40, 7
    u0, v0 = oracle.init(L)
    dt = np.float32 if dtype == "f32" else np.float64
    uo, vo = oracle.step(u0, v0, n, **PAPER, noise=0.1, seed=9)
    ref = make(L, dtype, noise=0.1, seed=9)
    ref.write(u0, v0)
    ref.step(n)
    ur, vr = ref.read()
    sims, bufs = [], []
    for i in range(2):
        sim = make(L, dtype, noise=0.1, seed=9, stream=torch.cuda.Stream())
        hin = [torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory() for a in (u0, v0)]
        hout = [torch.full((L, L, L), float("nan"), dtype=hin[0].dtype).pin_memory() for _ in range(2)]
        sims.append(sim)
        bufs.append((hin, hout))
    torch.cuda.synchronize()
    for sim, (hin, hout) in zip(sims, bufs):
        gs.gs_write_async(sim.handle, gs.GS_U, hin[0])
        gs.gs_write_async(sim.handle, gs.GS_V, hin[1])
        sim.step(n)
        gs.gs_read_async(sim.handle, gs.GS_U, hout[0])
        gs.gs_read_async(sim.handle, gs.GS_V, hout[1])
    for sim, (_, hout) in zip(sims, bufs):
        sim.sync()
        np.testing.assert_array_equal(hout[0].numpy(), ur)
        np.testing.assert_array_equal(hout[1].numpy(), vr)
        assert maxabs(hout[0].numpy(), uo) <= TOL[dtype] and maxabs(hout[1].numpy(), vo) <= TOL[dtype]
    with pytest.raises(gs.GsError) as e:
        gs.gs_read_async(sims[0].handle, gs.GS_U, torch.empty(7, dtype=hout[0].dtype))
    assert e.value.status == gs.GS_EINVAL


def test_fp64_fma_rate_is_measured():
    # the FP64 pipe's rate the bench divides by: positive, and within a wide
    # band around GB300's nominal 1.25 TFLOP/s (0.625 T FMA/s)
    need_cuda()
    r = gs.gs_measure_fp64_fma()
    print(f"FP64 FMA/s: {r:.4e}")
    assert 0.1 * 0.625e12 < r < 4 * 0.625e12
