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


@pytest.mark.parametrize("L,N", [(16, 1), (16, 2)])
def test_gradients_match_oracle(L, N):
    torch = need_cuda()
    params = inputs.surrogate_init_params(seed=7 + L, last_scale=1.0)
    u, v = _fields(N, L, 3 * L)
    tu, tv = _fields(N, L, 5 * L)
    F, k = [0.025, 0.04][:N], [0.05, 0.065][:N]
    s = gs.Surrogate(params)
    loss_gpu = s.grad(_dev(torch, u), _dev(torch, v), F, k, _dev(torch, tu), _dev(torch, tv))
    grads = s.grads()
    out, cache = oracle.surrogate_forward(params, u.astype(np.float64), v.astype(np.float64), F, k,
                                          emulate_bf16=True)
    loss_o, dout = oracle.mse_loss(out, np.stack([tu, tv], axis=-1).astype(np.float64))
    go = oracle.surrogate_backward(cache, dout)
    assert abs(loss_gpu - loss_o) <= 1e-2 * loss_o
    for l in range(6):
        for gg, oo, name in ((grads[l][0], go[l][0], "w"), (grads[l][1], go[l][1], "b")):
            rel = np.linalg.norm(gg - oo) / max(np.linalg.norm(oo), 1e-30)
            cos = float(np.sum(gg * oo) / (np.linalg.norm(gg) * np.linalg.norm(oo) + 1e-30))
            print(f"layer {l} {name}: rel {rel:.2e} cos {cos:.6f}")
            assert rel <= 3e-2 and cos >= 0.999, (l, name, rel, cos)
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
    torch = need_cuda()
    L = 128
    params = inputs.surrogate_init_params(seed=4, last_scale=1.0)
    rng = np.random.default_rng(7)
    u = _dev(torch, rng.uniform(0, 1, (1, L, L, L)))
    v = _dev(torch, rng.uniform(0, 0.5, (1, L, L, L)))
    ut = _dev(torch, rng.uniform(0, 1, (1, L, L, L)))
    vt = _dev(torch, rng.uniform(0, 0.5, (1, L, L, L)))
    s = gs.Surrogate(params)
    gs.gs_surr_set_backend(s.handle, gs.GS_SURR_TCGEN05)
    lt = s.grad(u, v, [0.03], [0.05], ut, vt)
    gt = s.grads()
    gs.gs_surr_set_backend(s.handle, gs.GS_SURR_MMA)
    lm = s.grad(u, v, [0.03], [0.05], ut, vt)
    gm = s.grads()
    assert abs(lt - lm) <= 1e-3 * lm
    for l in range(6):
        for j in range(2):
            rel = np.linalg.norm(gt[l][j] - gm[l][j]) / np.linalg.norm(gm[l][j])
            assert rel <= 1e-2, (l, j, rel)
    s.close()
