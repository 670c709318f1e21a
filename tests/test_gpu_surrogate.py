"""GPU tests of the learned surrogate's tensor-core kernels against the FP64 oracle.

The oracle composes the network from its circular convolutions with bfloat16
rounding emulated where the GPU stores bfloat16 (input, weights, hidden
activations); what remains is FP32 accumulation order and the bfloat16
rounding of back-propagated gradients, covered by the stated tolerances.
"""
import numpy as np
import pytest

import oracle
from paper_2309_10292_gb300 import gs, inputs, surrogate
from tests.gpu_util import PAPER, need_cuda

pytestmark = pytest.mark.gpu


def _fields(N, L, seed):
    u = np.stack([inputs.random_fields(L, seed=seed + n, lo=0.0, hi=1.0)[0] for n in range(N)])
    v = np.stack([inputs.random_fields(L, seed=seed + n, lo=0.0, hi=0.5)[1] for n in range(N)])
    return u.astype(np.float32), v.astype(np.float32)


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("L,N", [(16, 2), (32, 1)])
def test_forward_matches_oracle(L, N):
    torch = need_cuda()
    params = inputs.surrogate_init_params(seed=L, last_scale=1.0)
    u, v = _fields(N, L, 10 * L)
    F, k = [0.02, 0.05][:N], [0.048, 0.061][:N]
    s = gs.Surrogate(params)
    pu, pv = s.forward(_dev(torch, u), _dev(torch, v), F, k)
    out, _ = oracle.surrogate_forward(params, u.astype(np.float64), v.astype(np.float64), F, k, emulate_bf16=True)
    d_orc = out - np.stack([u, v], axis=-1)
    d_gpu = np.stack([pu.cpu().numpy(), pv.cpu().numpy()], axis=-1) - np.stack([u, v], axis=-1)
    scale = np.abs(d_orc).max()
    err = np.abs(d_gpu - d_orc)
    print(f"L={L} N={N}: max |d| {scale:.3e}, max err {err.max():.3e}, mean err {err.mean():.3e}")
    assert err.max() <= 2e-2 * scale
    assert err.mean() <= 2e-3 * scale
    s.close()


def test_forward_full_size_sampled_cells():
    # the run size (L=256): sampled cells against the oracle network evaluated on
    # a 13^3 window (the network's receptive field has radius 6)
    torch = need_cuda()
    L = 256
    params = inputs.surrogate_init_params(seed=5, last_scale=1.0)
    rng = np.random.default_rng(0)
    u = rng.uniform(0, 1, (1, L, L, L)).astype(np.float32)
    v = rng.uniform(0, 0.5, (1, L, L, L)).astype(np.float32)
    s = gs.Surrogate(params)
    pu, pv = s.forward(_dev(torch, u), _dev(torch, v), [0.03], [0.055])
    pu, pv = pu.cpu().numpy(), pv.cpu().numpy()
    for c in [(0, 0, 0), (255, 128, 7), (100, 200, 255), (128, 128, 128)]:
        idx = [(np.arange(-6, 7) + cc) % L for cc in c]
        sel = np.ix_(idx[2], idx[1], idx[0])
        wu, wv = u[0][sel][None].astype(np.float64), v[0][sel][None].astype(np.float64)
        out, _ = oracle.surrogate_forward(params, wu, wv, [0.03], [0.055], emulate_bf16=True)
        du_o = out[0, 6, 6, 6, 0] - wu[0, 6, 6, 6]
        dv_o = out[0, 6, 6, 6, 1] - wv[0, 6, 6, 6]
        x, y, z = c
        du_g = pu[0, z, y, x] - u[0, z, y, x]
        dv_g = pv[0, z, y, x] - v[0, z, y, x]
        tol = 2e-2 * max(abs(du_o), abs(dv_o), 1e-3)
        assert abs(du_g - du_o) <= tol and abs(dv_g - dv_o) <= tol, (c, du_g, du_o, dv_g, dv_o)
    s.close()


# Gradient parity runs on networks whose every forward sum is exact in FP32
# as in FP64: sparse weights of +-1/4, +-1/2, biases on a 1/64 grid, fields
# and targets on a 1/16 grid, 20F = 0.5 and 20k = 1 (inputs.dyadic_fields,
# inputs.surrogate_dyadic_params).  Layer l's pre-activation z_l is then a
# multiple of q_l = 2^-(6 + 2l), and the oracle checks that the sum of its
# terms' magnitudes stays below 2^22 q_l, so neither side rounds a forward
# sum: both see the same activations, the same ReLU masks (a random network
# flips masks wherever |z| is within the FP32-vs-FP64 difference, and the
# gradient there is ambiguous) and the same dL/dout.  The data gradients
# are sums of few dyadic terms too and come out exact (equal to the oracle's
# bit for bit, as measured); the weight and bias gradients sum over every
# cell and differ by FP32 accumulation order, about 1e-6 of the largest
# entry.  Element by element, per tensor:
#   |gpu - oracle| <= GRAD_ATOL * max|oracle| + GRAD_RTOL * |oracle|
GRAD_RTOL = 1e-4
GRAD_ATOL = 1e-5
F_DY, K_DY = 0.025, 0.05  # 20 F and 20 k exactly representable


def _assert_close(g, o, what):
    g, o = np.asarray(g, dtype=np.float64), np.asarray(o, dtype=np.float64)
    scale = np.abs(o).max()
    err = np.abs(g - o)
    bound = GRAD_ATOL * scale + GRAD_RTOL * np.abs(o)
    worst = float((err / np.maximum(bound, 1e-300)).max())
    print(f"{what}: max |o| {scale:.3e} max err {err.max():.3e} worst err/bound {worst:.3f}")
    assert scale > 0, what
    assert np.all(err <= bound), (what, worst)


def _assert_exact_forward_sums(params, cache):
    # oracle side only: every layer's sum of term magnitudes below 2^22 q_l
    for l in range(6):
        q = 2.0 ** -(6 + 2 * l)
        absum = oracle.conv3d_fwd(np.abs(cache["hs"][l]), np.abs(params[l][0]), np.abs(params[l][1]))
        assert absum.max() < 2.0 ** 22 * q, (l, absum.max() / (2.0 ** 22 * q))


def _dyadic_case(N, L, seed):
    params = inputs.surrogate_dyadic_params(seed=seed)
    u = inputs.dyadic_fields((N, L, L, L), seed=seed + 100).astype(np.float32)
    v = inputs.dyadic_fields((N, L, L, L), seed=seed + 200, hi=0.5).astype(np.float32)
    tu = inputs.dyadic_fields((N, L, L, L), seed=seed + 300).astype(np.float32)
    tv = inputs.dyadic_fields((N, L, L, L), seed=seed + 400, hi=0.5).astype(np.float32)
    return params, u, v, tu, tv, [F_DY] * N, [K_DY] * N


def _trace_buffer(torch, N, L):
    return torch.zeros(5 * N * L ** 3 * 32, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("L,N,seed", [(16, 1, 0), (16, 2, 1), (32, 1, 2)])
def test_gradients_match_oracle(L, N, seed):
    # every layer's dW, db and data gradient dL/dh_l, element by element
    # (mma.sync path: L is not a multiple of 128)
    torch = need_cuda()
    params, u, v, tu, tv, F, k = _dyadic_case(N, L, seed)
    out, cache = oracle.surrogate_forward(params, u.astype(np.float64), v.astype(np.float64), F, k,
                                          emulate_bf16=True)
    _assert_exact_forward_sums(params, cache)
    s = gs.Surrogate(params)
    dh = _trace_buffer(torch, N, L)
    gs.gs_surr_trace_grads(s.handle, dh, dh.numel())
    loss_gpu = s.grad(_dev(torch, u), _dev(torch, v), F, k, _dev(torch, tu), _dev(torch, tv))
    grads = s.grads()
    ou, ov = _dev(torch, u), _dev(torch, v)
    gs.gs_surr_get_train_output(s.handle, ou, ov, N * L ** 3)
    gs.gs_surr_trace_grads(s.handle, None)
    # exact forward sums: the training forward pass equals the oracle's bit for bit
    np.testing.assert_array_equal(np.stack([ou.cpu().numpy(), ov.cpu().numpy()], axis=-1), out)
    loss_o, dout = oracle.mse_loss(out, np.stack([tu, tv], axis=-1).astype(np.float64))
    go, dho = oracle.surrogate_backward(cache, dout, emulate_bf16=True, return_dh=True)
    # the loss adds FP32 per-thread partial sums (in FP64 across threads)
    assert abs(loss_gpu - loss_o) <= 1e-6 * loss_o
    for l in range(6):
        _assert_close(grads[l][0], go[l][0], f"layer {l} dW")
        _assert_close(grads[l][1], go[l][1], f"layer {l} db")
    dhg = dh.cpu().numpy().reshape(5, N, L, L, L, 32)
    for l in range(1, 6):
        _assert_close(dhg[l - 1], dho[l - 1], f"dL/dh_{l}")
    s.close()


def _window_index(lo, r, n, L):
    # per axis (x, y, z): the n cells starting r cells before lo, periodic
    return [(np.arange(n) - r + c) % L for c in lo]


@pytest.mark.parametrize("backend", [gs.GS_SURR_TCGEN05])
def test_training_gradients_at_L128_match_oracle(backend):
    # L = 128, the tensor-core training path.  The loss target equals the
    # network's own prediction except in a 4^3 box (across the periodic x and
    # z wrap), so dL/dout is known in closed form, zero outside the box, and
    # every gradient is supported within 6 cells of the box: the oracle
    # evaluates the network on that 16^3 window and its gradients are the
    # full grid's.
    torch = need_cuda()
    L, r, seed = 128, 6, 3
    params = inputs.surrogate_dyadic_params(seed=seed)
    u = inputs.dyadic_fields((1, L, L, L), seed=seed + 100).astype(np.float32)
    v = inputs.dyadic_fields((1, L, L, L), seed=seed + 200, hi=0.5).astype(np.float32)
    F, k = [F_DY], [K_DY]
    lo = np.array([126, 62, 127])  # box corner (x, y, z); cells lo .. lo + 3, periodic
    box = [(np.arange(4) + c) % L for c in lo]
    # target - prediction in the box, [field][z][y][x], on the 1/16 grid
    delta = inputs.dyadic_fields((2, 4, 4, 4), seed=seed + 500, lo=-0.5, hi=0.5)

    # the window: the box and r = 6 cells on each side, 16^3 cells; the box
    # is at window cells r .. r+3 along each axis
    wx, wy, wz = _window_index(lo, r, 16, L)
    sel = np.ix_(wz, wy, wx)
    wu = u[0][sel][None].astype(np.float64)
    wv = v[0][sel][None].astype(np.float64)
    out, cache = oracle.surrogate_forward(params, wu, wv, F, k, emulate_bf16=True)
    _assert_exact_forward_sums(params, cache)
    dout = np.zeros((1, 16, 16, 16, 2))
    for f in range(2):
        dout[0, r:r + 4, r:r + 4, r:r + 4, f] = -delta[f] / L ** 3  # 2 (pred - target) / (2 L^3)
    go, dho = oracle.surrogate_backward(cache, dout, emulate_bf16=True, return_dh=True)

    s = gs.Surrogate(params)
    gs.gs_surr_set_backend(s.handle, backend)
    ud, vd = _dev(torch, u), _dev(torch, v)
    s.grad(ud, vd, F, k, ud, vd)
    ou, ov = torch.empty_like(ud), torch.empty_like(vd)
    gs.gs_surr_get_train_output(s.handle, ou, ov, L ** 3)
    # in the box (whose receptive field is the window) the prediction equals the oracle's
    win_pred = np.stack([ou[0].cpu().numpy()[sel], ov[0].cpu().numpy()[sel]], axis=-1)
    np.testing.assert_array_equal(win_pred[r:r + 4, r:r + 4, r:r + 4], out[0, r:r + 4, r:r + 4, r:r + 4])
    tu, tv = ou.clone(), ov.clone()
    zi, yi, xi = np.ix_(box[2], box[1], box[0])
    tzyx = tuple(torch.from_numpy(np.broadcast_to(a, (4, 4, 4)).copy()).cuda() for a in (zi, yi, xi))
    tu[0][tzyx] += torch.from_numpy(delta[0]).float().cuda()
    tv[0][tzyx] += torch.from_numpy(delta[1]).float().cuda()
    dh = _trace_buffer(torch, 1, L)
    gs.gs_surr_trace_grads(s.handle, dh, dh.numel())
    s.grad(ud, vd, F, k, tu, tv)
    grads = s.grads()
    gs.gs_surr_trace_grads(s.handle, None)

    for l in range(6):
        _assert_close(grads[l][0], go[l][0], f"L=128 layer {l} dW")
        _assert_close(grads[l][1], go[l][1], f"L=128 layer {l} db")
    dhg = dh.view(5, L, L, L, 32)
    tz, ty, tx = (torch.from_numpy(a).cuda() for a in (wz, wy, wx))
    for l in range(1, 6):
        full = dhg[l - 1]
        win = full[tz][:, ty][:, :, tx]
        _assert_close(win.cpu().numpy(), dho[l - 1][0], f"L=128 dL/dh_{l}")
        # nothing outside the window
        assert float(full.abs().sum()) == pytest.approx(float(win.abs().sum()), rel=1e-5, abs=0)
    s.close()


def test_adam_step_matches_oracle():
    torch = need_cuda()
    L = 16
    params = inputs.surrogate_init_params(seed=2, last_scale=1.0)
    u, v = _fields(1, L, 1)
    tu, tv = _fields(1, L, 2)
    s = gs.Surrogate(params)
    s.grad(_dev(torch, u), _dev(torch, v), [0.03], [0.05], _dev(torch, tu), _dev(torch, tv))
    g = s.grads()
    p0 = s.params()
    gs.gs_surr_adam(s.handle, 1e-3)
    p1 = s.params()
    for l in range(6):
        for j in range(2):
            exp, _, _ = oracle.adam_update(p0[l][j], g[l][j], 0.0 * g[l][j], 0.0 * g[l][j], 1, lr=1e-3)
            np.testing.assert_allclose(p1[l][j], exp, rtol=0, atol=2e-6)
    s.close()


def test_training_reduces_loss_and_beats_persistence():
    # train on the stencil's own trajectories and show what the network gains
    # over predicting "no change" on held-out pairs
    need_cuda()
    pool = surrogate.TrajectoryPool(L=32, n=8, seed=3, warm=(60, 400))
    s = gs.Surrogate(inputs.surrogate_init_params(seed=0))
    before = surrogate.evaluate(s, pool, pairs=4)
    # the untrained network is exactly "no change" (zero final layer)
    assert before["rms_network"] == before["rms_persistence"]
    losses, _ = surrogate.train(s, pool, iters=1500, lr=1e-3, batch=2, warmup=100)
    after = surrogate.evaluate(s, pool, pairs=8)
    print("before", before, "after", after, "loss", losses[0], losses[-1])
    assert np.mean(losses[-50:]) < 0.3 * np.mean(losses[:10])
    # measured about 0.46 of the no-change error (RMS over both fields)
    assert after["rms_network"] < 0.7 * after["rms_persistence"]
    assert after["max_network"] < after["max_persistence"]
    pool.close()
    s.close()


def test_run_with_checks_and_fallback():
    need_cuda()
    L = 32
    sim = gs.GrayScott(L, noise=0.0, seed=0, dtype="f32", **PAPER)
    sim.step(100)
    s = gs.Surrogate(inputs.surrogate_init_params(seed=1))
    # impossible tolerance: every check falls back, segments alternate
    rep = s.run(sim, PAPER["F"], PAPER["k"], 256, check_every=64, tol=1e-12)
    assert sim.t == 100 + 256
    assert rep["surrogate_steps"] + rep["stencil_steps"] == 256
    assert rep["checks"] >= 1 and rep["fallbacks"] == rep["checks"]
    assert rep["stencil_steps"] > 0
    # loose tolerance: no fallback, 3 of every 4 applications kept
    rep2 = s.run(sim, PAPER["F"], PAPER["k"], 128, check_every=64, tol=1e9)
    assert rep2["fallbacks"] == 0 and rep2["surrogate_steps"] == 96 and rep2["stencil_steps"] == 32
    u, v = sim.read()
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(v))
    s.close()
    sim.close()


# ---------------------------------------------------------------------------
# The checked run (gs_surr_run) against the oracle: network applications from
# oracle.surrogate_forward, stencil segments from oracle.step, chained in the
# order the run takes them.  The network part carries the forward pass's
# tolerance (bfloat16 activations: 2e-2 of the update's scale); the stencil
# steps after it add only FP32 rounding.
# ---------------------------------------------------------------------------
RUN_PARAMS = dict(Du=0.2, Dv=0.1, F=0.035, k=0.06, dt=1.0)


def _oracle_net(params, u, v):
    out, _ = oracle.surrogate_forward(params, u[None], v[None], [RUN_PARAMS["F"]], [RUN_PARAMS["k"]],
                                      emulate_bf16=True)
    return out[0, ..., 0], out[0, ..., 1]


def _oracle_steps(u, v, n, t0):
    return oracle.step(u, v, n, noise=0.0, seed=0, t0=t0, **RUN_PARAMS)


def _run_case(L, seed):
    # a developed pattern: 300 stencil steps from the centred cube with small
    # random perturbations (the oracle starts from the same state)
    u0, v0 = oracle.init(L)
    du, dv = inputs.random_fields(L, seed=seed, lo=-0.05, hi=0.05)
    u0, v0 = u0 + du, np.clip(v0 + dv, 0.0, None)
    u0, v0 = _oracle_steps(u0, v0, 300, 0)
    params = inputs.surrogate_init_params(seed=seed, last_scale=0.05)
    return u0, v0, params


def _sim_from(torch, L, u, v, t):
    sim = gs.GrayScott(L, noise=0.0, seed=0, dtype="f32", **RUN_PARAMS)
    sim.write(u.astype(np.float32), v.astype(np.float32))
    sim.t = t
    return sim


def test_checked_run_kept_segment_matches_oracle():
    # L = 32 (mma.sync path), one segment of 32 steps, no fallback: the run
    # keeps one network application, then checks a second one against 16
    # stencil steps from the same state and keeps the stencil's state
    torch = need_cuda()
    L = 32
    u0, v0, params = _run_case(L, 1)
    u0, v0 = u0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64)
    sim = _sim_from(torch, L, u0, v0, 300)
    s = gs.Surrogate(params)
    rep = s.run(sim, RUN_PARAMS["F"], RUN_PARAMS["k"], 32, check_every=32, tol=1e9)
    assert rep["surrogate_applications"] == 1 and rep["surrogate_steps"] == 16
    assert rep["stencil_steps"] == 16 and rep["checks"] == 1 and rep["fallbacks"] == 0
    assert sim.t == 332
    ug, vg = sim.read()
    u1, v1 = _oracle_net(params, u0, v0)               # kept application
    scale = max(np.abs(u1 - u0).max(), np.abs(v1 - v0).max())  # the network's change
    nu, nv = _oracle_net(params, u1, v1)               # checked application
    u2, v2 = _oracle_steps(u1, v1, 16, 316)            # the stencil's state is kept
    check_err = max(np.abs(nu - u2).max(), np.abs(nv - v2).max())
    err = max(np.abs(ug - u2).max(), np.abs(vg - v2).max())
    print(f"kept segment: scale {scale:.3e} max err {err:.3e}; check error {check_err:.4e} vs "
          f"{rep['max_check_error']:.4e}")
    assert err <= 2e-2 * scale
    assert rep["max_check_error"] == pytest.approx(check_err, rel=2e-2)
    assert rep["last_check_error"] == rep["max_check_error"]
    s.close()
    sim.close()


def test_checked_run_fallback_segment_matches_oracle():
    # the same start with an impossible tolerance: the first segment's check
    # fails, so the second segment is 32 plain stencil steps
    torch = need_cuda()
    L = 32
    u0, v0, params = _run_case(L, 2)
    u0, v0 = u0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64)
    sim = _sim_from(torch, L, u0, v0, 300)
    s = gs.Surrogate(params)
    rep = s.run(sim, RUN_PARAMS["F"], RUN_PARAMS["k"], 64, check_every=32, tol=1e-12)
    assert rep["surrogate_steps"] == 16 and rep["stencil_steps"] == 48
    assert rep["checks"] == 1 and rep["fallbacks"] == 1
    ug, vg = sim.read()
    u, v = _oracle_net(params, u0, v0)
    scale = max(np.abs(u - u0).max(), np.abs(v - v0).max())  # the network's change
    u, v = _oracle_steps(u, v, 16, 316)
    u, v = _oracle_steps(u, v, 32, 332)
    err = max(np.abs(ug - u).max(), np.abs(vg - v).max())
    print(f"fallback: scale {scale:.3e} max err {err:.3e}")
    assert err <= 2e-2 * scale
    s.close()
    sim.close()


def test_checked_run_at_L128_sampled_cells_match_oracle():
    # L = 128 (tensor-core path): one segment of 32 steps = one kept
    # application, then the checked one and 16 stencil steps.  Sampled cells
    # from their light cone: the network on a 45^3 window (radius 16 + 6)
    # is exact on its inner 33^3 cells, and 16 stencil steps on those are
    # exact at the centre
    torch = need_cuda()
    L = 128
    rng = np.random.default_rng(5)
    u0, v0 = oracle.init(L)
    du, dv = inputs.random_fields(L, seed=3, lo=-0.05, hi=0.05)
    u0 = (u0 + du).astype(np.float32).astype(np.float64)
    v0 = np.clip(v0 + dv, 0.0, None).astype(np.float32).astype(np.float64)
    params = inputs.surrogate_init_params(seed=6, last_scale=0.05)
    sim = _sim_from(torch, L, u0, v0, 0)
    s = gs.Surrogate(params)
    rep = s.run(sim, RUN_PARAMS["F"], RUN_PARAMS["k"], 32, check_every=32, tol=1e9)
    assert rep["surrogate_steps"] == 16 and rep["stencil_steps"] == 16 and rep["checks"] == 1
    ug, vg = sim.read()
    cells = [(0, 0, 0), (127, 64, 3), (61, 62, 63)] + [tuple(int(x) for x in rng.integers(0, L, 3))]
    for (x, y, z) in cells:
        R = 22
        idx = [(np.arange(-R, R + 1) + c) % L for c in (x, y, z)]
        sel = np.ix_(idx[2], idx[1], idx[0])
        nu, nv = _oracle_net(params, u0[sel], v0[sel])
        iu, iv = nu[6:-6, 6:-6, 6:-6], nv[6:-6, 6:-6, 6:-6]      # exact 33^3
        fu, fv = _oracle_steps(iu, iv, 16, 16)
        c = 16
        s0 = (slice(6, -6),) * 3
        scale = max(np.abs(iu - u0[sel][s0]).max(), np.abs(iv - v0[sel][s0]).max())  # the network's change
        tol = 2e-2 * scale
        print((x, y, z), ug[z, y, x], fu[c, c, c], vg[z, y, x], fv[c, c, c], tol)
        assert abs(ug[z, y, x] - fu[c, c, c]) <= tol and abs(vg[z, y, x] - fv[c, c, c]) <= tol
    s.close()
    sim.close()


def test_weights_file_round_trip_and_refusals(tmp_path):
    need_cuda()
    params = inputs.surrogate_init_params(seed=12, last_scale=1.0)
    a = gs.Surrogate(params)
    path = str(tmp_path / "w.gssurr")
    a.save(path)
    b = gs.Surrogate()
    b.load(path)
    np.testing.assert_array_equal(gs.gs_surr_get_params(b.handle), gs.gs_surr_get_params(a.handle))
    raw = open(path, "rb").read()
    assert raw[:8] == b"GSSURR01" and len(raw) == 12 + 4 * gs.gs_surr_param_count()
    for name, data, status in [("magic", b"XXXXXXXX" + raw[8:], gs.GS_EINVAL),
                               ("short", raw[:100], gs.GS_EIO),
                               ("long", raw + b"\0", gs.GS_EINVAL)]:
        bad = str(tmp_path / name)
        open(bad, "wb").write(data)
        with pytest.raises(gs.GsError) as e:
            b.load(bad)
        assert e.value.status == status, name
    with pytest.raises(gs.GsError) as e:
        b.load(str(tmp_path / "missing"))
    assert e.value.status == gs.GS_EIO
    a.close()
    b.close()


def test_surrogate_argument_errors():
    torch = need_cuda()
    s = gs.Surrogate()
    x = torch.zeros((1, 20, 20, 20), device="cuda")
    with pytest.raises(gs.GsError) as e:
        s.forward(x, x, [0.02], [0.05])
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError):
        gs.gs_surr_set_params(s.handle, np.zeros(10, dtype=np.float32))
    sim = gs.GrayScott(32, noise=0.0, dtype="f64", **PAPER)
    with pytest.raises(gs.GsError):
        s.run(sim, 0.02, 0.048, 64)
    s.close()


# ---------------------------------------------------------------------------
# 5th-generation tensor-core (tcgen05) forward path, L % 128 == 0
# ---------------------------------------------------------------------------
# L = 128: three boxes per slab row; 256: a 136-cell box plus the wrapped
# halo (both end segments); 384: also one 144-cell box (the middle segment)
@pytest.mark.parametrize("L,N", [(128, 1), (128, 2), (256, 1), (384, 1)])
def test_tcgen05_forward_matches_mma_path_and_oracle(L, N):
    torch = need_cuda()
    params = inputs.surrogate_init_params(seed=21, last_scale=1.0)
    rng = np.random.default_rng(N)
    u = rng.uniform(0, 1, (N, L, L, L)).astype(np.float32)
    v = rng.uniform(0, 0.5, (N, L, L, L)).astype(np.float32)
    F, k = [0.03, 0.045][:N], [0.055, 0.062][:N]
    s = gs.Surrogate(params)
    gs.gs_surr_set_backend(s.handle, gs.GS_SURR_TCGEN05)
    tu, tv = s.forward(_dev(torch, u), _dev(torch, v), F, k)
    gs.gs_surr_sync(s.handle)
    gs.gs_surr_set_backend(s.handle, gs.GS_SURR_MMA)
    mu, mv = s.forward(_dev(torch, u), _dev(torch, v), F, k)
    tu, tv, mu, mv = (t.cpu().numpy() for t in (tu, tv, mu, mv))
    d_t = np.stack([tu - u, tv - v])
    d_m = np.stack([mu - u, mv - v])
    scale = np.abs(d_m).max()
    err = np.abs(d_t - d_m)
    print(f"tcgen05 vs mma.sync: max |d| {scale:.3e} max err {err.max():.3e} mean {err.mean():.3e}")
    assert err.max() <= 2e-2 * scale and err.mean() <= 1e-3 * scale
    for n in range(N):
        # (x, y, z): segment edges in x (127 | 128, L - 1), wrap rows in y and z
        for c in [(0, 0, 0), (127, 5, 64), (64, 127, 127), (L - 1, L - 4, L // 2), (L // 2, 0, L - 1)]:
            idx = [(np.arange(-6, 7) + cc) % L for cc in c]
            sel = np.ix_(idx[2], idx[1], idx[0])
            wu, wv = u[n][sel][None].astype(np.float64), v[n][sel][None].astype(np.float64)
            out, _ = oracle.surrogate_forward(params, wu, wv, [F[n]], [k[n]], emulate_bf16=True)
            x, y, z = c
            for ch, (tt, base) in enumerate(((tu, u), (tv, v))):
                d_o = out[0, 6, 6, 6, ch] - base[n, z, y, x]
                d_g = tt[n, z, y, x] - base[n, z, y, x]
                assert abs(d_g - d_o) <= 2e-2 * max(abs(d_o), 1e-3), (n, c, ch, d_g, d_o)
    s.close()


def test_tcgen05_training_gradients_match_mma_path():
    # the two convolution paths on the same L = 128 training step, element by
    # element (the forward pass of both is exact on these inputs)
    torch = need_cuda()
    L = 128
    params, u, v, tu, tv, F, k = _dyadic_case(1, L, 4)
    u, v, tu, tv = (_dev(torch, a) for a in (u, v, tu, tv))
    s = gs.Surrogate(params)
    res = []
    for backend in (gs.GS_SURR_TCGEN05, gs.GS_SURR_MMA):
        gs.gs_surr_set_backend(s.handle, backend)
        dh = _trace_buffer(torch, 1, L)
        gs.gs_surr_trace_grads(s.handle, dh, dh.numel())
        loss = s.grad(u, v, F, k, tu, tv)
        res.append((loss, s.grads(), dh))
        gs.gs_surr_trace_grads(s.handle, None)
    (lt, gt, dt), (lm, gm, dm) = res
    assert lt == lm
    for l in range(6):
        for j, name in ((0, "dW"), (1, "db")):
            _assert_close(gt[l][j], gm[l][j], f"tcgen05 vs mma.sync layer {l} {name}")
    assert torch.equal(dt, dm)
    s.close()
