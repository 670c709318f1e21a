"""Pins for the CPU oracle: each check ties it to something other than itself.

Simulation pins follow Eq. (1)-(3) of the paper (forward Euler, normalised
7-point Laplacian) with periodic wrap; each is a property fixed by the
mathematics (fixed point, symmetry, closed form, conservation, light cone,
translation equivariance) or an independent brute force, chosen so that a
dropped term, a wrong sign, a wrong neighbour index or a swapped operand
fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2309_10292_gb300 import inputs

P = inputs.PAPER_PARAMS
M32 = 0xFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Independent numpy restatement of the counter hash (written separately from
# gs_oracle.c from the same published definition).
# ---------------------------------------------------------------------------
def np_fmix32(h):
    h = np.asarray(h, dtype=np.uint64) & M32
    h = h ^ (h >> np.uint64(16))
    h = (h * np.uint64(0x85EBCA6B)) & np.uint64(M32)
    h = h ^ (h >> np.uint64(13))
    h = (h * np.uint64(0xC2B2AE35)) & np.uint64(M32)
    h = h ^ (h >> np.uint64(16))
    return h


def np_noise(seed, t, cells):
    lo, hi = seed & M32, (seed >> 32) & M32
    a = int(np_fmix32(lo ^ int(np_fmix32((t & M32) ^ 0x9E3779B9))))
    b = int(np_fmix32(hi ^ int(np_fmix32(a ^ 0x7F4A7C15))))
    c = np.asarray(cells, dtype=np.uint64)
    h = np_fmix32(np_fmix32(c ^ np.uint64(a)) ^ np.uint64(b))
    m = (h >> np.uint64(8)).astype(np.int64)
    return (2 * m + 1 - 2 ** 24).astype(np.float64) / 2.0 ** 24


def test_fmix32_published_vectors(orc):
    path = os.path.join(GOLDEN, "murmur3_fmix32.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for seed, expected in rows:
        assert orc.fmix32(int(seed, 16)) == int(expected, 16)


def test_fmix32_matches_numpy_restatement(orc):
    rng = np.random.default_rng(1)
    for h in rng.integers(0, 2 ** 32, size=200):
        assert orc.fmix32(int(h)) == int(np_fmix32(int(h)))


@pytest.mark.parametrize("seed,t", [(42, 0), (42, 1), (42, 999), (0, 7), (2 ** 40 + 3, 5)])
def test_noise_field_matches_numpy_restatement(orc, seed, t):
    n = 16 ** 3
    r = orc.noise_field(seed, t, n)
    np.testing.assert_array_equal(r, np_noise(seed, t, np.arange(n)))
    assert orc.noise_r(seed, t, 123) == r[123]


def test_noise_distribution_exact(orc):
    r = orc.noise_field(42, 3, 64 ** 3)
    assert np.all(r > -1.0) and np.all(r < 1.0)
    scaled = r * 2 ** 24
    assert np.all(scaled == np.round(scaled))
    assert np.all(np.mod(scaled, 2) == 1)  # odd numerators only
    assert abs(r.mean()) < 5e-3
    assert abs(r.var() - 1.0 / 3.0) < 5e-3
    # different steps give different fields, no shift structure between them
    r2 = orc.noise_field(42, 4, 64 ** 3)
    assert not np.array_equal(r, r2)
    assert abs(np.corrcoef(r, r2)[0, 1]) < 1e-2
    assert abs(np.corrcoef(r[1:], r2[:-1])[0, 1]) < 1e-2


def test_noise_code_map_is_centred():
    # the map m -> (2m + 1 - 2^24) / 2^24 over all 2^24 codes: mean exactly 0,
    # extremes +-(1 - 2^-24)
    m = np.arange(2 ** 24, dtype=np.int64)
    r = (2 * m + 1 - 2 ** 24) / 2.0 ** 24
    assert r.sum() == 0.0
    assert r.min() == -(1 - 2.0 ** -24) and r.max() == 1 - 2.0 ** -24


# ---------------------------------------------------------------------------
# Simulation pins
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L", [1, 2, 3, 8])
def test_fixed_point_is_exact(orc, L):
    u = np.ones((L, L, L))
    v = np.zeros((L, L, L))
    u2, v2 = orc.step(u, v, 25, **P, noise=0.0, seed=1)
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(v2, v)


def test_init_centred_cube(orc):
    u, v = orc.init(64)
    cube = np.zeros((64, 64, 64), dtype=bool)
    cube[29:35, 29:35, 29:35] = True
    assert np.all(u[cube] == 0.25) and np.all(v[cube] == 0.33)
    assert np.all(u[~cube] == 1.0) and np.all(v[~cube] == 0.0)


def test_octahedral_symmetry(orc):
    L = 16
    u0, v0 = orc.init(L)
    u, v = orc.step(u0, v0, 30, **P, noise=0.0, seed=0)
    assert not np.allclose(u, u0)
    # x reflection: x- and x+ are summed first, so the result is bitwise symmetric
    np.testing.assert_array_equal(u, u[:, :, ::-1])
    np.testing.assert_array_equal(v, v[:, :, ::-1])
    # the other 47 maps hold up to summation order
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product([False, True], repeat=3):
            for f in (u, v):
                g = np.transpose(f, perm)
                for ax, fl in enumerate(flips):
                    if fl:
                        g = np.flip(g, axis=ax)
                np.testing.assert_allclose(g, f, rtol=0, atol=1e-13)


def _mode(L, m):
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return np.sin(2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / L)


def _lam(L, m):
    return -sum(1 - np.cos(2 * np.pi * md / L) for md in m) / 3.0


@pytest.mark.parametrize("L,m", [(16, (1, 2, 3)), (12, (0, 1, 0)), (9, (4, 0, 2))])
def test_sine_mode_diffusion_closed_form(orc, L, m):
    c, A, n, Du, dt = 0.5, 0.1, 40, 0.2, 1.0
    s = _mode(L, m)
    u0 = c + A * s
    v0 = np.zeros_like(u0)
    u, v = orc.step(u0, v0, n, Du=Du, Dv=0.1, F=0.0, k=0.0, dt=dt, noise=0.0, seed=0)
    g = 1 + dt * Du * _lam(L, m)
    np.testing.assert_allclose(u, c + A * g ** n * s, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(v, 0.0)


def test_sine_mode_with_feed(orc):
    L, m, c, A, n = 12, (1, 1, 0), 0.6, 0.05, 30
    Du, F, dt = 0.2, 0.03, 0.5
    s = _mode(L, m)
    u, v = orc.step(c + A * s, np.zeros((L, L, L)), n, Du=Du, Dv=0.1, F=F, k=0.05, dt=dt,
                    noise=0.0, seed=0)
    expect = 1 + (c - 1) * (1 - dt * F) ** n + A * (1 + dt * (Du * _lam(L, m) - F)) ** n * s
    np.testing.assert_allclose(u, expect, rtol=0, atol=1e-12)


def test_v_mode_with_kill(orc):
    L, m, c, A, n = 10, (2, 0, 1), 0.3, 0.1, 30
    Dv, k, dt = 0.1, 0.05, 1.0
    s = _mode(L, m)
    u, v = orc.step(np.zeros((L, L, L)), c + A * s, n, Du=0.2, Dv=Dv, F=0.0, k=k, dt=dt,
                    noise=0.0, seed=0)
    expect = c * (1 - dt * k) ** n + A * (1 + dt * (Dv * _lam(L, m) - k)) ** n * s
    np.testing.assert_allclose(v, expect, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(u, 0.0)


def brute_force(u, v, nsteps, Du, Dv, F, k, dt, noise, seed, t0=0):
    """Explicit neighbour-matrix restatement of Eq. (1)-(3) with periodic wrap."""
    L = u.shape[0]
    n = L ** 3
    A = np.zeros((n, n))
    for z, y, x in itertools.product(range(L), repeat=3):
        i = x + L * (y + L * z)
        for dx, dy, dz in [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
            A[i, (x + dx) % L + L * ((y + dy) % L + L * ((z + dz) % L))] += 1.0
    uf, vf = u.reshape(-1).copy(), v.reshape(-1).copy()
    for s in range(nsteps):
        r = np_noise(seed, t0 + s, np.arange(n))
        lu = (A @ uf - 6 * uf) / 6
        lv = (A @ vf - 6 * vf) / 6
        du = Du * lu - uf * vf * vf + F * (1 - uf) + noise * r
        dv = Dv * lv + uf * vf * vf - (F + k) * vf
        uf, vf = uf + dt * du, vf + dt * dv
    return uf.reshape(u.shape), vf.reshape(v.shape)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("noise", [0.0, 0.1])
def test_brute_force_tiny_grids(orc, L, noise):
    u0, v0 = inputs.random_fields(L, seed=100 + L, lo=0.0, hi=1.0)
    args = dict(Du=0.2, Dv=0.1, F=0.035, k=0.06, dt=0.5, noise=noise, seed=77)
    ub, vb = brute_force(u0, v0, 12, t0=3, **args)
    uo, vo = orc.step(u0, v0, 12, t0=3, **args)
    np.testing.assert_allclose(uo, ub, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vo, vb, rtol=0, atol=1e-14)


def _l1_dist_to_cube(L):
    lo, hi = L // 2 - 3, L // 2 + 2
    d = np.zeros(L, dtype=np.int64)
    for i in range(L):
        if lo <= i <= hi:
            continue
        d[i] = min((lo - i) % L, (i - hi) % L)
    z, y, x = np.meshgrid(d, d, d, indexing="ij")
    return x + y + z


def test_light_cone(orc):
    L, t = 32, 7
    u0, v0 = orc.init(L)
    dist = _l1_dist_to_cube(L)
    u, v = orc.step(u0, v0, t, **P, noise=0.0, seed=0)
    out = dist > t
    assert np.all(u[out] == 1.0) and np.all(v[out] == 0.0)
    assert np.all(u[dist == t] != 1.0)  # the front has moved exactly t cells
    u, v = orc.step(u0, v0, t, **P, noise=0.1, seed=5)
    assert np.all(v[out] == 0.0)
    assert np.all(v[dist == t] != 0.0)


def test_translation_equivariance(orc):
    L = 16
    u0, v0 = orc.init(L)
    shift = (3, 5, 7)
    ua, va = orc.step(u0, v0, 15, **P, noise=0.0, seed=0)
    ub, vb = orc.step(np.roll(u0, shift, axis=(0, 1, 2)), np.roll(v0, shift, axis=(0, 1, 2)),
                      15, **P, noise=0.0, seed=0)
    np.testing.assert_array_equal(ub, np.roll(ua, shift, axis=(0, 1, 2)))
    np.testing.assert_array_equal(vb, np.roll(va, shift, axis=(0, 1, 2)))


def test_conservation_pure_diffusion(orc):
    L = 16
    u0, _ = inputs.random_fields(L, seed=3)
    u, v = orc.step(u0, np.zeros_like(u0), 50, Du=0.2, Dv=0.1, F=0.0, k=0.0, dt=1.0,
                    noise=0.0, seed=0)
    assert abs(u.sum() - u0.sum()) <= 1e-12 * abs(u0.sum())
    assert np.all(np.isfinite(u))


def test_step_composition_and_step_index(orc):
    # n steps at once == a steps, then n-a steps starting at step index a
    L = 6
    u0, v0 = inputs.random_fields(L, seed=9)
    args = dict(**P, noise=0.1, seed=11)
    ua, va = orc.step(u0, v0, 9, **args)
    u1, v1 = orc.step(u0, v0, 4, **args)
    ub, vb = orc.step(u1, v1, 5, t0=4, **args)
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(va, vb)
    uc, _ = orc.step(u1, v1, 5, t0=0, **args)
    assert not np.array_equal(uc, ub)


@pytest.mark.parametrize("L,center,m,n", [(16, (3, 0, 15), 1, 5), (12, (6, 6, 6), 2, 4),
                                          (5, (0, 0, 0), 1, 7)])
def test_window_equals_full_grid(orc, L, center, m, n):
    # light-cone window (with its own wrap when the window exceeds L) gives the
    # same bits as the full periodic grid at the sampled cells
    args = dict(**P, noise=0.1, seed=3)
    u0, v0 = orc.init(L)
    uf, vf = orc.step(u0, v0, n, t0=2, **args)
    uw, vw = orc.window(L, center, m, n, t0=2, **args)
    idx = [(np.arange(-m, m + 1) + c) % L for c in center]
    sel = np.ix_(idx[2], idx[1], idx[0])
    np.testing.assert_array_equal(uw, uf[sel])
    np.testing.assert_array_equal(vw, vf[sel])
    ur, vr = inputs.random_fields(L, seed=4)
    uf, vf = orc.step(ur, vr, n, **args)
    uw, vw = orc.window(L, center, m, n, u0=ur, v0=vr, **args)
    np.testing.assert_array_equal(uw, uf[sel])
    np.testing.assert_array_equal(vw, vf[sel])


def test_plausible_ranges_noise(orc):
    # loose plausibility only (the paper's Listing 1 ranges come from a different
    # boundary, RNG and size): the state stays bounded and v >= 0
    L = 32
    u0, v0 = orc.init(L)
    u, v = orc.step(u0, v0, 200, **P, noise=0.1, seed=42)
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(v))
    assert -0.5 < u.min() and u.max() < 2.0
    assert v.min() >= -1e-12 and v.max() < 1.0


# ---------------------------------------------------------------------------
# Surrogate primitives
# ---------------------------------------------------------------------------
def fft_conv(x, w, b):
    """Circular correlation via numpy's FFT: y[p] = sum_d w[d] x[p + d]."""
    N, L, _, _, Cin = x.shape
    Cout = w.shape[2]
    y = np.zeros((N, L, L, L, Cout))
    for ci in range(Cin):
        X = np.fft.fftn(x[..., ci], axes=(1, 2, 3))
        for co in range(Cout):
            K = np.zeros((L, L, L))
            for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
                tap = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)
                K[(-dz) % L, (-dy) % L, (-dx) % L] += w[tap, ci, co]
            y[..., co] += np.real(np.fft.ifftn(X * np.fft.fftn(K)[None], axes=(1, 2, 3)))
    return y + (0 if b is None else b)


# ---------------------------------------------------------------------------
# The paper's kernel variants: outer layer held, one field without noise
# ---------------------------------------------------------------------------
def _faces(L):
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return (x == 0) | (y == 0) | (z == 0) | (x == L - 1) | (y == L - 1) | (z == L - 1)


def _dmode(L, m):
    """Dirichlet mode: zero on the first and last layer of every axis (m_d >= 1)."""
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return (np.sin(np.pi * m[0] * x / (L - 1)) * np.sin(np.pi * m[1] * y / (L - 1))
            * np.sin(np.pi * m[2] * z / (L - 1)))


def _dlam(L, m):
    return -sum(1 - np.cos(np.pi * md / (L - 1)) for md in m) / 3.0


def test_held_faces_unchanged_and_interior_as_periodic(orc):
    L = 10
    u0, v0 = inputs.random_fields(L, seed=5, lo=0.0, hi=1.0)
    args = dict(Du=0.2, Dv=0.1, F=0.035, k=0.06, dt=0.5, noise=0.1, seed=77)
    uh, vh = orc.step_held(u0, v0, 9, t0=2, **args)
    f = _faces(L)
    np.testing.assert_array_equal(uh[f], u0[f])
    np.testing.assert_array_equal(vh[f], v0[f])
    assert np.all(uh[~f] != u0[~f])
    # one step: interior cells see no wrap, so they equal the periodic step bit for bit
    u1, v1 = orc.step_held(u0, v0, 1, t0=2, **args)
    up, vp = orc.step(u0, v0, 1, t0=2, **args)
    np.testing.assert_array_equal(u1[~f], up[~f])
    np.testing.assert_array_equal(v1[~f], vp[~f])


def test_held_fixed_point(orc):
    L = 7
    u = np.ones((L, L, L))
    v = np.zeros((L, L, L))
    uh, vh = orc.step_held(u, v, 5, Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0, noise=0.0, seed=0)
    np.testing.assert_array_equal(uh, 1.0)
    np.testing.assert_array_equal(vh, 0.0)


@pytest.mark.parametrize("L,m", [(12, (1, 2, 1)), (9, (3, 1, 2))])
def test_held_dirichlet_mode_closed_form(orc, L, m):
    c, A, n, Du, dt = 0.4, 0.1, 30, 0.2, 1.0
    s = _dmode(L, m)
    u, v = orc.step_held(c + A * s, np.zeros((L, L, L)), n, Du=Du, Dv=0.1, F=0.0, k=0.0, dt=dt,
                         noise=0.0, seed=0)
    g = 1 + dt * Du * _dlam(L, m)
    np.testing.assert_allclose(u, c + A * g ** n * s, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(v, 0.0)


def _held_matrix(L):
    """Neighbour-count matrix of the interior cells; rows of face cells are empty."""
    n = L ** 3
    A = np.zeros((n, n))
    f = _faces(L).reshape(-1)
    for z, y, x in itertools.product(range(L), repeat=3):
        i = x + L * (y + L * z)
        if f[i]:
            continue
        for dx, dy, dz in [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
            A[i, (x + dx) + L * ((y + dy) + L * (z + dz))] += 1.0
    return A, f


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 6])
def test_held_brute_force_tiny_grids(orc, L):
    u0, v0 = inputs.random_fields(L, seed=300 + L, lo=0.0, hi=1.0)
    args = dict(Du=0.2, Dv=0.1, F=0.035, k=0.06, dt=0.5, noise=0.1, seed=7)
    A, f = _held_matrix(L)
    n = L ** 3
    uf, vf = u0.reshape(-1).copy(), v0.reshape(-1).copy()
    for s in range(6):
        r = np_noise(7, 4 + s, np.arange(n))
        lu = (A @ uf - 6 * uf) / 6
        lv = (A @ vf - 6 * vf) / 6
        du = args["Du"] * lu - uf * vf * vf + args["F"] * (1 - uf) + args["noise"] * r
        dv = args["Dv"] * lv + uf * vf * vf - (args["F"] + args["k"]) * vf
        uf = np.where(f, uf, uf + args["dt"] * du)
        vf = np.where(f, vf, vf + args["dt"] * dv)
    uo, vo = orc.step_held(u0, v0, 6, t0=4, **args)
    np.testing.assert_allclose(uo.reshape(-1), uf, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vo.reshape(-1), vf, rtol=0, atol=1e-14)


@pytest.mark.parametrize("L,m", [(16, (1, 2, 3)), (9, (4, 0, 2))])
def test_diffuse_periodic_mode_closed_form(orc, L, m):
    c, A, n, D, dt = 0.5, 0.2, 40, 0.3, 0.8
    s = _mode(L, m)
    f = orc.diffuse(c + A * s, n, D=D, dt=dt)
    np.testing.assert_allclose(f, c + A * (1 + dt * D * _lam(L, m)) ** n * s, rtol=0, atol=1e-12)


@pytest.mark.parametrize("L,m", [(12, (1, 1, 1)), (9, (2, 3, 1))])
def test_diffuse_held_dirichlet_closed_form(orc, L, m):
    c, A, n, D, dt = -0.2, 0.3, 25, 0.2, 1.0
    s = _dmode(L, m)
    f = orc.diffuse(c + A * s, n, D=D, dt=dt, held=True)
    np.testing.assert_allclose(f, c + A * (1 + dt * D * _dlam(L, m)) ** n * s, rtol=0, atol=1e-12)


def test_diffuse_conserves_and_matches_the_two_field_step(orc):
    L = 11
    f0, _ = inputs.random_fields(L, seed=9, lo=0.0, hi=1.0)
    f = orc.diffuse(f0, 20, D=0.2, dt=1.0)
    assert abs(f.sum() - f0.sum()) <= 1e-12 * f0.sum()
    # same arithmetic as Eq. 1-2 with v = 0, F = k = 0 and no noise
    u, _ = orc.step(f0, np.zeros_like(f0), 20, Du=0.2, Dv=0.1, F=0.0, k=0.0, dt=1.0, noise=0.0, seed=0)
    np.testing.assert_array_equal(f, u)


@pytest.mark.parametrize("L", [1, 2, 3, 5])
@pytest.mark.parametrize("held", [False, True])
def test_diffuse_brute_force_tiny_grids(orc, L, held):
    f0, _ = inputs.random_fields(L, seed=400 + L, lo=0.0, hi=1.0)
    n = L ** 3
    if held:
        A, fm = _held_matrix(L)
    else:
        A = np.zeros((n, n))
        fm = np.zeros(n, dtype=bool)
        for z, y, x in itertools.product(range(L), repeat=3):
            i = x + L * (y + L * z)
            for dx, dy, dz in [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
                A[i, (x + dx) % L + L * ((y + dy) % L + L * ((z + dz) % L))] += 1.0
    g = f0.reshape(-1).copy()
    for _ in range(7):
        g = np.where(fm, g, g + 0.5 * (0.25 * ((A @ g - 6 * g) / 6)))
    fo = orc.diffuse(f0, 7, D=0.25, dt=0.5, held=held)
    np.testing.assert_allclose(fo.reshape(-1), g, rtol=0, atol=1e-14)


@pytest.mark.parametrize("L", [3, 4, 6])
def test_conv_fwd_matches_fft(orc, L):
    x = inputs.random_tensor((2, L, L, L, 3), seed=1)
    w = inputs.random_tensor((27, 3, 2), seed=2)
    b = inputs.random_tensor((2,), seed=3)
    np.testing.assert_allclose(orc.conv3d_fwd(x, w, b), fft_conv(x, w, b), rtol=0, atol=1e-12)


def test_conv_single_tap_is_a_shift(orc):
    L = 5
    x = inputs.random_tensor((1, L, L, L, 1), seed=4)
    for dz, dy, dx in [(1, 0, 0), (0, -1, 0), (0, 0, 1), (-1, 1, -1)]:
        w = np.zeros((27, 1, 1))
        w[9 * (dz + 1) + 3 * (dy + 1) + (dx + 1), 0, 0] = 1.0
        y = orc.conv3d_fwd(x, w, None)
        np.testing.assert_array_equal(y, np.roll(x, (-dz, -dy, -dx), axis=(1, 2, 3)))


def test_conv_adjoints(orc):
    L = 4
    x = inputs.random_tensor((2, L, L, L, 3), seed=5)
    g = inputs.random_tensor((2, L, L, L, 5), seed=6)
    w = inputs.random_tensor((27, 3, 5), seed=7)
    y = orc.conv3d_fwd(x, w, None)
    dx = orc.conv3d_bwd_data(g, w)
    dw, db = orc.conv3d_bwd_weight(x, g)
    lhs = np.sum(y * g)
    assert abs(lhs - np.sum(x * dx)) < 1e-10 * max(1.0, abs(lhs))
    assert abs(lhs - np.sum(w * dw)) < 1e-10 * max(1.0, abs(lhs))
    np.testing.assert_allclose(db, g.sum(axis=(0, 1, 2, 3)), rtol=1e-13)


def test_surrogate_gradients_finite_differences(orc):
    L, N = 4, 2
    params = inputs.surrogate_init_params(seed=3, last_scale=1.0)
    u, v = inputs.random_fields(L, seed=8, lo=0.0, hi=1.0)
    u = np.stack([u, 1 - u]); v = np.stack([v, 0.5 * v])
    F, k = np.array([0.02, 0.05]), np.array([0.048, 0.06])
    tgt = inputs.random_tensor((N, L, L, L, 2), seed=9, lo=0.0, hi=1.0)

    def loss_of(pp):
        out, _ = orc.surrogate_forward(pp, u, v, F, k)
        return orc.mse_loss(out, tgt)[0]

    out, cache = orc.surrogate_forward(params, u, v, F, k)
    _, dout = orc.mse_loss(out, tgt)
    grads = orc.surrogate_backward(cache, dout)
    rng = np.random.default_rng(0)
    h = 1e-6
    for l in range(6):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in params[l][0].shape)
            pp = [(w.copy(), b.copy()) for w, b in params]
            pp[l][0][idx] += h
            lp = loss_of(pp)
            pp[l][0][idx] -= 2 * h
            lm = loss_of(pp)
            fd = (lp - lm) / (2 * h)
            an = grads[l][0][idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (l, idx, fd, an)
        j = rng.integers(0, params[l][1].shape[0])
        pp = [(w.copy(), b.copy()) for w, b in params]
        pp[l][1][j] += h
        lp = loss_of(pp)
        pp[l][1][j] -= 2 * h
        lm = loss_of(pp)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[l][1][j]) <= 1e-6 * max(1e-3, abs(fd))


def _rest_of_network(orc, params, h, l, u, v):
    # the network's layers l .. 5 applied to a given h_l (composed here from the
    # convolution primitive, independently of surrogate_forward/backward)
    for j in range(l, 5):
        h = h + np.maximum(orc.conv3d_fwd(h, params[j][0], params[j][1]), 0.0)
    return np.stack([u, v], axis=-1) + orc.conv3d_fwd(h, params[5][0], params[5][1])


def test_surrogate_activation_gradients_finite_differences(orc):
    # dL/dh_l returned by surrogate_backward against central differences of
    # the loss in single entries of h_l
    L, N = 4, 1
    params = inputs.surrogate_init_params(seed=6, last_scale=1.0)
    u, v = inputs.random_fields(L, seed=10, lo=0.0, hi=1.0)
    u, v = u[None], v[None]
    F, k = np.array([0.03]), np.array([0.055])
    tgt = inputs.random_tensor((N, L, L, L, 2), seed=11, lo=0.0, hi=1.0)
    out, cache = orc.surrogate_forward(params, u, v, F, k)
    _, dout = orc.mse_loss(out, tgt)
    _, dhs = orc.surrogate_backward(cache, dout, return_dh=True)
    rng = np.random.default_rng(1)
    h = 1e-6
    for l in range(1, 6):
        for _ in range(3):
            idx = (0,) + tuple(int(i) for i in rng.integers(0, L, 3)) + (int(rng.integers(0, 32)),)
            hp = cache["hs"][l].copy()
            hp[idx] += h
            lp = orc.mse_loss(_rest_of_network(orc, params, hp, l, u, v), tgt)[0]
            hp[idx] -= 2 * h
            lm = orc.mse_loss(_rest_of_network(orc, params, hp, l, u, v), tgt)[0]
            fd = (lp - lm) / (2 * h)
            an = dhs[l - 1][idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (l, idx, fd, an)


def test_surrogate_backward_bf16_emulation(orc):
    # rounding dL/dout and every dz_l to bfloat16 keeps the gradients within a
    # few bfloat16 rounding errors of the exact ones, and the last layer's
    # bias gradient is then exactly the sum of the rounded dL/dout
    L, N = 4, 2
    params = inputs.surrogate_init_params(seed=4, last_scale=1.0)
    u, v = inputs.random_fields(L, seed=12, lo=0.0, hi=1.0)
    u = np.stack([u, 1 - u]); v = np.stack([v, 0.5 * v])
    F, k = np.array([0.02, 0.05]), np.array([0.048, 0.06])
    tgt = inputs.random_tensor((N, L, L, L, 2), seed=13, lo=0.0, hi=1.0)
    out, cache = orc.surrogate_forward(params, u, v, F, k)
    _, dout = orc.mse_loss(out, tgt)
    g0, d0 = orc.surrogate_backward(cache, dout, return_dh=True)
    g1, d1 = orc.surrogate_backward(cache, dout, emulate_bf16=True, return_dh=True)
    for l in range(6):
        for j in range(2):
            rel = np.linalg.norm(g1[l][j] - g0[l][j]) / np.linalg.norm(g0[l][j])
            assert 0 < rel < 2 ** -6, (l, j, rel)
    for a, b in zip(d0, d1):
        assert 0 < np.linalg.norm(a - b) / np.linalg.norm(a) < 2 ** -6
    np.testing.assert_allclose(g1[5][1], orc.bf16_round(dout).sum(axis=(0, 1, 2, 3)), rtol=1e-13, atol=0)
    assert np.abs(g1[5][1] - dout.sum(axis=(0, 1, 2, 3))).max() > 0


def test_surrogate_zero_last_layer_is_identity(orc):
    L = 4
    params = inputs.surrogate_init_params(seed=1)
    params[5] = (np.zeros_like(params[5][0]), np.zeros(2))
    u, v = inputs.random_fields(L, seed=2)
    out, _ = orc.surrogate_forward(params, u[None], v[None], np.array([0.03]), np.array([0.05]))
    np.testing.assert_array_equal(out[0, ..., 0], u)
    np.testing.assert_array_equal(out[0, ..., 1], v)


def test_bf16_round_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-5, 5, size=5000),
                        [0.0, -0.0, 1.0, 65504.0, 3.3895313892515355e38]])
    a32 = a.astype(np.float32)
    # exact ties at every 16-bit boundary: low half 0x8000
    bits = (rng.integers(0, 2 ** 31, size=1000).astype(np.uint32) & np.uint32(0x7F7F0000)) | np.uint32(0x8000)
    ties = bits.view(np.float32)
    x = np.concatenate([a32, ties]).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(orc.bf16_round(x), ref)


def test_adam_constant_gradient_closed_form(orc):
    # with a constant gradient the bias-corrected moments are exactly g and g^2,
    # so each step moves p by lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.01, 2.0])
    m = np.zeros(3); v = np.zeros(3)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        p, m, v = orc.adam_update(p, g, m, v, t, lr=lr, eps=eps)
    np.testing.assert_allclose(p, np.array([1.0, -2.0, 0.5]) - 5 * lr * g / (np.abs(g) + eps),
                               rtol=0, atol=1e-12)


def test_mse_loss_gradient(orc):
    out = np.array([[1.0, 2.0], [3.0, 5.0]])
    tgt = np.array([[1.0, 1.0], [1.0, 1.0]])
    l, g = orc.mse_loss(out, tgt)
    assert l == (0 + 1 + 4 + 16) / 4
    np.testing.assert_array_equal(g, 2 * (out - tgt) / 4)
