"""Time one stencil configuration from the command line (cell updates per
second, CUDA events on the grid's stream), e.g.

    python -m paper_2309_10292_gb300.timing --L 256 --dtype f64 --arith ds \
        --plan zmarch,128,8,32 --steps 6

prints one JSON line with the plan and the rate; with --batch it times the
batched workload instead (256 instances, L_i on {32, 48, 64, 96, 128}), e.g.

    python -m paper_2309_10292_gb300.timing --batch --depth 2 --tile-z 64 --steps 6

All compute runs in libgs.
"""
from __future__ import annotations

import argparse
import json

KERNELS = {"naive": 1, "zmarch": 2, "tblock": 3}


def main(argv=None):
    import torch

    from paper_2309_10292_gb300 import gs
    ap = argparse.ArgumentParser(description="time the Gray-Scott stencil on one grid")
    ap.add_argument("--L", type=int, default=512)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--arith", default="ieee", choices=["ieee", "ds", "fx", "fxf"])
    ap.add_argument("--noise", type=float, default=0.1)
    ap.add_argument("--plan", default="", help="kernel,tile_x,tile_y,tile_z[,depth[,stages]]; empty: autotune")
    ap.add_argument("--steps", type=int, default=100, help="timed steps")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", action="store_true", help="time the 256-instance batched launch")
    ap.add_argument("--depth", type=int, default=1, help="--batch: temporal-blocking depth")
    ap.add_argument("--tile-z", type=int, default=32, help="--batch: z-chunk per work item")
    ap.add_argument("--stages", type=int, default=8, help="--batch: TMA ring depth (depth 1)")
    a = ap.parse_args(argv)
    if a.batch:
        return time_batch(a)
    sim = gs.GrayScott(a.L, Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0, noise=a.noise, seed=42, dtype=a.dtype)
    if a.arith != "ieee":
        sim.arith = {"ds": gs.GS_ARITH_DS, "fx": gs.GS_ARITH_FX, "fxf": gs.GS_ARITH_FXF}[a.arith]
    if a.plan:
        f = a.plan.split(",")
        nums = [int(x) for x in f[1:]] + [0] * (5 - len(f[1:]))
        plan = {"kernel": KERNELS[f[0]], "tile_x": nums[0], "tile_y": nums[1], "tile_z": nums[2],
                "depth": nums[3] or 1, "stages": nums[4], "us_per_step": 0.0}
        gs.gs_set_plan_full(sim.handle, plan)
    else:
        sim.autotune()
    sim.step(a.warmup)
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    sim.step(a.steps)
    t1.record(stream)
    sim.sync()
    ms = t0.elapsed_time(t1)
    out = {"L": a.L, "dtype": a.dtype, "arith": a.arith, "noise": a.noise, "plan": sim.plan,
           "steps": a.steps, "ms": ms, "gcups": a.L ** 3 * a.steps / (ms / 1e3) / 1e9}
    sim.close()
    print(json.dumps(out))


def time_batch(a):
    import torch

    from paper_2309_10292_gb300 import gs, inputs
    Ls, F, k = inputs.batch_instances(256, seed=0)
    b = gs.GrayScottBatch(Ls, F, k, Du=0.2, Dv=0.1, dt=1.0, noise=a.noise, seed=42, dtype="f32")
    gs.gs_batch_set_plan(b.handle, a.tile_z, a.stages)
    b.set_depth(a.depth)
    b.step(a.steps)  # capture + warm-up with the timed step count
    b.sync()
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    b.step(a.steps)
    t1.record(stream)
    b.sync()
    ms = t0.elapsed_time(t1)
    cells = sum(L ** 3 for L in Ls)
    out = {"batch": len(Ls), "cells": cells, "noise": a.noise, "depth": a.depth, "tile_z": a.tile_z,
           "steps": a.steps, "ms": ms, "gcups": cells * a.steps / (ms / 1e3) / 1e9, "info": b.info}
    b.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
