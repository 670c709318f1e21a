"""Training and evaluation loop of the 16-step surrogate (orchestration only).

Training data are trajectories of the stencil itself: independent FP32 grids
(noise 0, the network cannot predict noise) with (F, k) drawn like the
batched workload, started from the centred cube and advanced by libgs; each
training pair is (state at t, state at t + 16).  Every forward, backward and
optimizer step runs in libgs's CUDA kernels; this module only moves device
pointers around.
"""
from __future__ import annotations

import time

import numpy as np

from . import gs, inputs

K = 16


class TrajectoryPool:
    """Independent stencil runs that advance K steps each time a pair is drawn.

    Runs start from the centred cube after a random warm-up in `warm` and
    restart once they pass warm[1] steps, so the pairs stay drawn from the
    same range of times.
    """

    def __init__(self, L=128, n=8, seed=0, warm=(100, 1200), Du=0.2, Dv=0.1, dt=1.0):
        import torch
        _, Fs, ks = inputs.batch_instances(n, seed=seed)
        self.rng = np.random.default_rng(seed + 1)
        self.L = L
        self.warm = warm
        self.F, self.k = Fs, ks
        self.sims = []
        for i in range(n):
            s = gs.GrayScott(L, Du=Du, Dv=Dv, F=Fs[i], k=ks[i], dt=dt, noise=0.0, seed=seed + i, dtype="f32")
            s.step(int(self.rng.integers(warm[0], warm[1])))
            self.sims.append(s)
        self.next = 0
        torch.cuda.synchronize()

    def _restart_if_old(self, s):
        if s.t > self.warm[1]:
            s.init()
            s.step(int(self.rng.integers(self.warm[0], self.warm[1])))

    def draw(self, N):
        """N pairs as stacked tensors (x_u, x_v, y_u, y_v) [N, L, L, L] and their F, k."""
        import torch
        xu, xv, yu, yv, F, k = [], [], [], [], [], []
        for _ in range(N):
            i = self.next
            self.next = (self.next + 1) % len(self.sims)
            s = self.sims[i]
            self._restart_if_old(s)
            u, v = s.tensors()
            xu.append(u.clone())
            xv.append(v.clone())
            s.step(K)
            u, v = s.tensors()
            yu.append(u.clone())
            yv.append(v.clone())
            F.append(self.F[i])
            k.append(self.k[i])
        return (torch.stack(xu), torch.stack(xv), torch.stack(yu), torch.stack(yv), F, k)

    def close(self):
        for s in self.sims:
            s.close()


def lr_at(it: int, iters: int, lr: float, warmup: int, decay_to: float) -> float:
    """Linear warm-up over `warmup` iterations, then exponential decay to lr * decay_to."""
    if it < warmup:
        return lr * (it + 1) / warmup
    frac = (it - warmup) / max(1, iters - warmup - 1)
    return lr * (decay_to ** frac)


def train(surr: "gs.Surrogate", pool: TrajectoryPool, iters: int, lr: float = 3e-4, batch: int = 2,
          lr_decay_to: float = 0.05, warmup: int = 50, log_every: int = 0):
    """Adam on pairs drawn from the pool; returns the loss history and wall time."""
    import torch
    losses = []
    t0 = time.perf_counter()
    for it in range(iters):
        lr_it = lr_at(it, iters, lr, warmup, lr_decay_to)
        xu, xv, yu, yv, F, k = pool.draw(batch)
        losses.append(surr.train_step(xu, xv, F, k, yu, yv, lr_it))
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {losses[-1]:.3e} lr {lr_it:.2e}", flush=True)
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def evaluate(surr: "gs.Surrogate", pool: TrajectoryPool, pairs: int = 4):
    """RMS and max error of the network and of persistence (u(t+16) ~ u(t)) on fresh pairs."""
    import torch
    err_net, err_id, mx_net, mx_id = [], [], [], []
    for _ in range(pairs):
        xu, xv, yu, yv, F, k = pool.draw(1)
        pu, pv = surr.forward(xu, xv, F, k)
        tgt = torch.stack([yu, yv])
        net = torch.stack([pu, pv]) - tgt
        ide = torch.stack([xu, xv]) - tgt
        err_net.append(float(net.pow(2).mean().sqrt()))
        err_id.append(float(ide.pow(2).mean().sqrt()))
        mx_net.append(float(net.abs().max()))
        mx_id.append(float(ide.abs().max()))
    return {"rms_network": float(np.mean(err_net)), "rms_persistence": float(np.mean(err_id)),
            "max_network": float(np.max(mx_net)), "max_persistence": float(np.max(mx_id))}


def time_forward(L: int = 256, reps: int = 5, backend: str = "tcgen05", seed: int = 0) -> dict:
    """Time one network application on a random L^3 state (seeded weights with
    a non-zero last layer); returns ms per application and TFLOP/s."""
    import torch
    be = {"auto": gs.GS_SURR_AUTO, "mma": gs.GS_SURR_MMA, "tcgen05": gs.GS_SURR_TCGEN05}[backend]
    s = gs.Surrogate(inputs.surrogate_init_params(seed=seed, last_scale=1.0))
    gs.gs_surr_set_backend(s.handle, be)
    g = torch.Generator(device="cuda").manual_seed(seed)
    u = torch.rand((1, L, L, L), device="cuda", generator=g)
    v = torch.rand((1, L, L, L), device="cuda", generator=g) * 0.3
    s.forward(u, v, [0.02], [0.05])
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        s.forward(u, v, [0.02], [0.05])
    b.record(st)
    gs.gs_surr_sync(s.handle)
    ms = a.elapsed_time(b) / reps
    flop = 2.0 * 27 * (4 * 32 + 4 * 32 * 32 + 32 * 2) * L ** 3
    s.close()
    return {"L": L, "backend": backend, "ms": ms, "tflops": flop / ms / 1e9}


# useful FLOP per cell of one training step: the forward pass, the data
# gradients of layers 5..1 and the weight gradients of all six layers
TRAIN_FLOP_PER_CELL = (2 * 27 * (4 * 32 + 4 * 32 * 32 + 32 * 2) + 2 * 27 * (2 * 32 + 4 * 32 * 32)
                       + 2 * 27 * (4 * 32 + 4 * 32 * 32 + 32 * 2))


def time_train_step(L: int = 128, N: int = 1, reps: int = 10, backend: str = "tcgen05", seed: int = 0) -> dict:
    """Time one training step (forward, every gradient, Adam) on N random
    L^3 pairs after three untimed steps; returns ms per step and useful TFLOP/s."""
    import torch
    be = {"auto": gs.GS_SURR_AUTO, "mma": gs.GS_SURR_MMA, "tcgen05": gs.GS_SURR_TCGEN05}[backend]
    s = gs.Surrogate(inputs.surrogate_init_params(seed=seed, last_scale=0.1))
    gs.gs_surr_set_backend(s.handle, be)
    g = torch.Generator(device="cuda").manual_seed(seed)
    u, v, tu, tv = (torch.rand((N, L, L, L), device="cuda", generator=g) * (1.0 if i % 2 == 0 else 0.5)
                    for i in range(4))
    F, k = [0.03] * N, [0.05] * N
    for _ in range(3):
        s.train_step(u, v, F, k, tu, tv, 1e-5)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        s.train_step(u, v, F, k, tu, tv, 1e-5)
    b.record(st)
    gs.gs_surr_sync(s.handle)
    ms = a.elapsed_time(b) / reps
    s.close()
    return {"L": L, "N": N, "backend": backend, "ms_per_step": ms,
            "tflops": TRAIN_FLOP_PER_CELL * N * L ** 3 / ms / 1e9}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="time the surrogate's forward pass or one training step")
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--N", type=int, default=1, help="grids per training step (--train)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--train", action="store_true", help="time a training step instead of the forward pass")
    ap.add_argument("--backend", default="tcgen05", choices=["auto", "mma", "tcgen05"])
    args = ap.parse_args()
    if args.train:
        print(json.dumps(time_train_step(args.L, args.N, args.reps, args.backend)))
    else:
        print(json.dumps(time_forward(args.L, args.reps, args.backend)))
