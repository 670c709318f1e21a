"""GPU tests of the paper's kernel variants: the held outer layer (the paper's
kernel skips cells on the first and last layer of every axis) and the single
field without reaction or noise ("1-variable no random"), against the
oracle's pinned restatements."""
import numpy as np
import pytest

import oracle
from paper_2309_10292_gb300 import gs, inputs
from tests.gpu_util import PAPER, maxabs, need_cuda

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}


def faces(L):
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return (x == 0) | (y == 0) | (z == 0) | (x == L - 1) | (y == L - 1) | (z == L - 1)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
@pytest.mark.parametrize("L", [64, 20, 5])
def test_held_boundary_matches_oracle(dtype, kernel, L):
    need_cuda()
    if kernel == gs.GS_KERNEL_ZMARCH and L % (4 if dtype == "f32" else 2):
        pytest.skip("z-march needs L divisible by the vector width")
    prm = dict(PAPER, noise=0.1, seed=9)
    u0, v0 = inputs.random_fields(L, seed=L, lo=0.0, hi=1.0)
    sim = gs.GrayScott(L, dtype=dtype, **prm)
    sim.set_plan(kernel)
    sim.boundary = gs.GS_BOUNDARY_HELD
    sim.write(u0, v0)
    sim.t = 3
    sim.step(40)
    u, v = sim.read()
    uo, vo = oracle.step_held(u0, v0, 40, t0=3, **prm)
    assert maxabs(u, uo) <= TOL[dtype] and maxabs(v, vo) <= TOL[dtype]
    f = faces(L)
    np.testing.assert_array_equal(u[f], u0.astype(u.dtype)[f])
    np.testing.assert_array_equal(v[f], v0.astype(v.dtype)[f])
    sim.close()


@pytest.mark.parametrize("arith", [gs.GS_ARITH_DS, gs.GS_ARITH_FX, gs.GS_ARITH_FXF], ids=["ds", "fx", "fxf"])
@pytest.mark.parametrize("kernel", [gs.GS_KERNEL_NAIVE, gs.GS_KERNEL_ZMARCH])
def test_held_boundary_in_the_other_fp64_arithmetics(arith, kernel):
    # a held grid rounds to FP64 after every step (the faces are copied from
    # the FP64 input), whatever the arithmetic: equal across kernels and to
    # the oracle, and the faces untouched
    need_cuda()
    L = 24
    prm = dict(PAPER, noise=0.1, seed=13)
    u0, v0 = inputs.random_fields(L, seed=4, lo=0.0, hi=1.0)
    sims = []
    for kern in (gs.GS_KERNEL_NAIVE, kernel):
        sim = gs.GrayScott(L, dtype="f64", **prm)
        sim.arith = arith
        sim.set_plan(kern)
        sim.boundary = gs.GS_BOUNDARY_HELD
        sim.write(u0, v0)
        sim.step(30)
        sims.append(sim)
    (ua, va), (ub, vb) = sims[0].read(), sims[1].read()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    uo, vo = oracle.step_held(u0, v0, 30, **prm)
    assert maxabs(ua, uo) <= 1e-10 and maxabs(va, vo) <= 1e-10
    f = faces(L)
    np.testing.assert_array_equal(ua[f], u0[f])
    for sim in sims:
        sim.close()


def test_held_boundary_kernels_bitwise_equal_and_config1():
    need_cuda()
    L = 64
    prm = dict(PAPER, noise=0.0, seed=0)
    a = gs.GrayScott(L, dtype="f64", **prm)
    a.set_plan(gs.GS_KERNEL_NAIVE)
    a.boundary = gs.GS_BOUNDARY_HELD
    b = gs.GrayScott(L, dtype="f64", **prm)
    b.boundary = gs.GS_BOUNDARY_HELD
    a.step(100)
    b.step(100)
    ua, va = a.read()
    ub, vb = b.read()
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    u0, v0 = oracle.init(L)
    uo, vo = oracle.step_held(u0, v0, 100, **prm)
    assert maxabs(ua, uo) <= 1e-10 and maxabs(va, vo) <= 1e-10


def test_held_boundary_refuses_temporal_blocking():
    need_cuda()
    sim = gs.GrayScott(32, dtype="f32", **PAPER)
    sim.set_plan(gs.GS_KERNEL_TBLOCK, 16, 8, 32, 2)
    with pytest.raises(gs.GsError):
        sim.boundary = gs.GS_BOUNDARY_HELD
    assert sim.boundary == gs.GS_BOUNDARY_PERIODIC
    sim.set_plan(gs.GS_KERNEL_ZMARCH)
    sim.boundary = gs.GS_BOUNDARY_HELD
    with pytest.raises(gs.GsError):
        sim.set_plan(gs.GS_KERNEL_TBLOCK, 16, 8, 32, 2)
    best, trials = sim.autotune(steps_per_trial=12)
    assert all(t["kernel"] != gs.GS_KERNEL_TBLOCK for t in trials)
    with pytest.raises(gs.GsError):
        sim.boundary = 7
    sim.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("held", [False, True])
@pytest.mark.parametrize("L", [64, 48, 7, 2])
def test_single_field_matches_oracle(dtype, held, L):
    need_cuda()
    f0, _ = inputs.random_fields(L, seed=50 + L, lo=0.0, hi=1.0)
    s = gs.SingleField(L, D=0.2, dt=1.0, dtype=dtype,
                       boundary=gs.GS_BOUNDARY_HELD if held else gs.GS_BOUNDARY_PERIODIC)
    s.write(f0)
    s.step(60)
    f = s.read()
    fo = oracle.diffuse(f0, 60, D=0.2, dt=1.0, held=held)
    assert maxabs(f, fo) <= TOL[dtype]
    assert s.info["zmarch"] == (L % (4 if dtype == "f32" else 2) == 0)
    assert s.info["steps"] == 60
    s.close()


def test_single_field_full_size_sampled():
    # a large FP64 grid (the bench runs L=1024): a Dirichlet mode's closed form
    need_cuda()
    L, n, D, dt = 512, 10, 0.2, 1.0
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij", sparse=True)
    m = (1, 2, 3)
    mode = (np.sin(np.pi * m[0] * x / (L - 1)) * np.sin(np.pi * m[1] * y / (L - 1))
            * np.sin(np.pi * m[2] * z / (L - 1)))
    f0 = 0.5 + 0.25 * mode
    s = gs.SingleField(L, D=D, dt=dt, dtype="f64", boundary=gs.GS_BOUNDARY_HELD)
    s.write(f0)
    del f0
    s.step(n)
    f = s.read()
    lam = -sum(1 - np.cos(np.pi * md / (L - 1)) for md in m) / 3.0
    expect = 0.5 + 0.25 * (1 + dt * D * lam) ** n * mode
    assert maxabs(f, expect) <= 1e-12
    s.close()
