"""Benchmark of the Gray-Scott stencil hot path on GB300.

Default workload (one bench step): the plain FP32 stencil on a periodic
512^3 grid (134M cells, four 0.54 GB field buffers, larger than L2), noise
0.1 from the counter hash with seed 42, Du=0.2 Dv=0.1 F=0.02 k=0.048 dt=1:
re-initialise to the centred cube, then 1000 time steps.  Metric: giga
cell-updates per second (GCUPS) and the fraction of the measured HBM
roofline (16 B per cell-step in FP32, 32 B in FP64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas: the plain grid does not shard), and rank 0 prints one JSON line
with value = total cell updates of all ranks / max time over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gray-Scott GCUPS & % HBM peak; surrogate/batched vs plain time at fixed error"
PARAMS = dict(Du=0.2, Dv=0.1, F=0.02, k=0.048, dt=1.0)
L_MAIN, NSTEPS, NOISE, SEED = 512, 1000, 0.1, 42
KERNEL_SRC = [os.path.join(ROOT, "paper_2309_10292_gb300", "csrc", f) for f in ("gs_stencil.cu", "gs_common.cuh")]
PROFILE = os.path.join(ROOT, "profiles", "gs_zmarch_f32_L512.md")


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """Largest value of x over all ranks (x itself when running alone)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: float, seconds_max: float) -> float:
    """Aggregate throughput: units processed by all ranks over the slowest rank's time."""
    return ws * units_per_rank / seconds_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_digest() -> str:
    """sha256 (16 hex digits) of every library source and header: names the
    exact code a bench line measured."""
    import glob
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2309_10292_gb300", "csrc", "*")) +
                    glob.glob(os.path.join(ROOT, "include", "*.h"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def kernel_digest() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


TBLOCK_PROFILE = os.path.join(ROOT, "profiles", "gs_tblock_issue_L512.md")
TBLOCK_SRC = [os.path.join(ROOT, "paper_2309_10292_gb300", "csrc", f) for f in ("gs_tblock.cu", "gs_tblock.cuh", "gs_common.cuh")]


def profiled_issue():
    """Warp instructions per cell update of the temporally blocked and z-march
    plans from the committed ncu summary, if it was taken on the current
    temporal-blocking source (else None): {plan string: count}."""
    if not os.path.exists(TBLOCK_PROFILE):
        return None
    text = open(TBLOCK_PROFILE).read()
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    w = re.search(r"warp_inst_per_update:\s*(.*)", text)
    h = hashlib.sha256()
    for f in TBLOCK_SRC:
        h.update(open(f, "rb").read())
    if not m or not w or m.group(1) != h.hexdigest()[:16]:
        return None
    return {k: float(v) for k, v in (item.split("=") for item in w.group(1).split())}


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not b or m.group(1) != kernel_digest():
        return None
    return float(b.group(1))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int, log_dir: str | None = None):
        self.proc = None
        self.path = os.path.join(log_dir or tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"), f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(target_s: float = 12.0, L: int = L_MAIN):
    """Time the FP64 CPU oracle on a bounded sample of the workload."""
    import numpy as np

    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    u, v = oracle.init(L)
    # step 0 warms the threads and pages; then chunks of 1, 2, 4, ... steps
    # continue the trajectory until the timed sample reaches target_s
    u, v = oracle.step(u, v, 1, **PARAMS, noise=NOISE, seed=SEED, t0=0)
    n, dt, chunk = 0, 0.0, 1
    while dt < target_s and n < 2000:
        t0 = time.perf_counter()
        u, v = oracle.step(u, v, chunk, **PARAMS, noise=NOISE, seed=SEED, t0=1 + n)
        dt += time.perf_counter() - t0
        n += chunk
        chunk = min(2 * chunk, 2000 - n) if dt < target_s / 2 else max(1, min(chunk, 2000 - n))
    assert np.isfinite(u).all()
    return {"value": L ** 3 * n / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle, L={L}, steps 1..{n} of the noise-0.1 centred-cube run "
                      f"({n} time steps, {dt:.1f} s, {threads} OpenMP threads)"}


def main_workload(L: int, time_steps: int) -> str:
    """The headline workload, named the same in both arms' config."""
    return (f"plain stencil FP32, L={L} ({L ** 3} cells), periodic, noise {NOISE} "
            f"(counter hash, seed {SEED}), Du=0.2 Dv=0.1 F=0.02 k=0.048 dt=1, "
            f"centred-cube start, {time_steps} time steps per bench step")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build_oracle()
    threads = oracle.set_threads(os.cpu_count() or 1)
    L = L_MAIN
    u, v = oracle.init(L)
    # 16 time steps per bench step (about 1 s on 16 cores): long enough that the
    # per-call copies of the FP64 fields in and out of the oracle do not dominate
    per_step_time_steps = 16
    times = []
    t = 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        u, v = oracle.step(u, v, per_step_time_steps, **PARAMS, noise=NOISE, seed=SEED, t0=t)
        dt = time.perf_counter() - t0
        t += per_step_time_steps
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = L ** 3 * per_step_time_steps * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": main_workload(L, args.time_steps), "L": L, "time_steps": args.time_steps,
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                         "sample": f"the FP64 oracle on a bounded sample of that workload: {per_step_time_steps} "
                                   f"of its time steps per bench step at L={L}, timed on {threads} threads"},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_batched(args, stream, hbm_peak):
    """Batched workload: 256 instances, L_i on {32,48,64,96,128}, F_i ~ U[0.01,0.06],
    k_i ~ U[0.04,0.07] (seeded), noise 0.1, 2000 steps in one persistent graph launch,
    against per-instance launches of the single-grid kernel."""
    import numpy as np
    import torch

    from paper_2309_10292_gb300 import gs, inputs
    Ls, F, k = inputs.batch_instances(256, seed=0)
    base = dict(Du=PARAMS["Du"], Dv=PARAMS["Dv"], dt=PARAMS["dt"])
    cells = sum(L ** 3 for L in Ls)
    nsteps, nseq = args.batch_steps, max(1, args.batch_steps // 10)
    b = gs.GrayScottBatch(Ls, F, k, noise=NOISE, seed=SEED, dtype="f32", **base)
    plan = b.autotune(steps_per_trial=20)  # z-chunk and ring depth of the persistent launch
    b.step(nsteps)  # capture + warm-up
    b.sync()
    b.init()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    b.step(nsteps)
    ev[1].record(stream)
    b.sync()
    t_pers = ev[0].elapsed_time(ev[1]) / 1e3
    info = b.info
    # per-instance launches (the same kernel a single grid uses), fewer steps
    b.init()
    b.step_sequential(2)
    b.sync()
    b.init()
    ev[2].record(stream)
    b.step_sequential(nseq)
    ev[3].record(stream)
    b.sync()
    t_seq = ev[2].elapsed_time(ev[3]) / 1e3
    # bitwise check persistent vs sequential after nseq steps on sampled instances
    c = gs.GrayScottBatch(Ls, F, k, noise=NOISE, seed=SEED, dtype="f32", **base)
    c.step(nseq)
    equal = all(np.array_equal(b.read(i)[0], c.read(i)[0]) and np.array_equal(b.read(i)[1], c.read(i)[1])
                for i in (0, 7, 128, 255))
    c.close()
    b.close()
    noise0 = bench_batched_noise0(Ls, F, k, base, cells, max(12, nsteps // 2), stream)
    g_pers = cells * nsteps / t_pers / 1e9
    g_seq = cells * nseq / t_seq / 1e9
    return {"workload": f"256 instances, L_i uniform on {{32,48,64,96,128}} ({cells} cells), "
                        f"F_i~U[0.01,0.06], k_i~U[0.04,0.07], noise {NOISE}, FP32, {nsteps} steps",
            "value": g_pers, "unit": "GCUPS", "time_s": t_pers,
            "hbm_frac": g_pers * 16.0 / hbm_peak,
            "sequential_value": g_seq, "sequential_steps": nseq,
            "sequential_launches_per_step": len(Ls),
            "speedup_vs_sequential": g_pers / g_seq,
            "bitwise_equal_to_sequential": bool(equal),
            "persistent_grid": info["grid"], "work_items_per_step": info["items"], "plan": plan,
            "cooperative_attribute": info["cooperative"], "graph_launches": 1, "noise0": noise0}


def bench_batched_noise0(Ls, F, k, base, cells, nsteps, stream):
    """The same 256 instances without noise (no counter hash per cell
    update), where the temporally blocked form can pay: the autotuner's plan
    (depth included) against the best one-step-per-pass plan of a short
    sweep (z-chunk 16 or 32, ring depth 6 or 8), both timed over the same
    steps."""
    import torch

    from paper_2309_10292_gb300 import gs
    b = gs.GrayScottBatch(Ls, F, k, noise=0.0, seed=SEED, dtype="f32", **base)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed():
        b.init()
        b.step(nsteps)  # capture + warm-up
        b.sync()
        b.init()
        ev[0].record(stream)
        b.step(nsteps)
        ev[1].record(stream)
        b.sync()
        return cells * nsteps / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e9

    plan = b.autotune(steps_per_trial=24)
    tuned = timed()
    one = {}
    b.set_depth(1)
    for tz in (16, 32):
        for stages in (6, 8):
            gs.gs_batch_set_plan(b.handle, tz, stages)
            one[f"z{tz}_s{stages}"] = timed()
    b.close()
    return {"plan": plan, "value": tuned, "unit": "GCUPS", "steps": nsteps,
            "depth1_value": max(one.values()), "depth1_by_plan": one,
            "note": "noise 0: the same instances without the counter hash; value = the tuned plan"}


def bench_snapshot(args, stream):
    """Output stage: L=256 FP32 (noise 0.1), 4000 steps with a snapshot of U
    and V every 500 (9 records, 134 MB each, to a temporary file, written by
    the library's writer thread while the stencil runs) against the same
    steps without.  The interval gives each record more stencil time than
    its write takes, as the paper's infrequent output does."""
    import shutil
    import tempfile
    import time

    import torch

    from paper_2309_10292_gb300 import gs, snapshot
    L, n, every = 256, 4000, 500
    sim = gs.GrayScott(L, dtype="f32", noise=NOISE, seed=SEED, **PARAMS)
    sim.set_plan(gs.GS_KERNEL_ZMARCH, 256, 4, 64)
    sim.step(20)
    torch.cuda.synchronize()
    sim.init()
    t0 = time.perf_counter()
    sim.step(n)
    sim.sync()
    plain = time.perf_counter() - t0
    d = tempfile.mkdtemp(prefix="gs_snap_")
    try:
        path = os.path.join(d, "run.gs")
        sim.init()
        t0 = time.perf_counter()
        with sim.snapshots(path) as w:
            w.write()
            for _ in range(n // every):
                sim.step(every)
                w.write()
            sim.sync()
            t_steps = time.perf_counter() - t0  # the stencil's own time with the writer running
            w.flush()
            info = w.info()
        t_all = time.perf_counter() - t0
        hdr, recs = snapshot.read(path, load_fields=False)
        size = os.path.getsize(path)
    finally:
        shutil.rmtree(d, ignore_errors=True)
    sim.close()
    return {"workload": f"L={L} FP32, {n} steps, snapshot of U and V every {every} steps ({len(recs)} records)",
            "records": len(recs), "file_bytes": size, "stencil_s_plain": plain, "stencil_s_with_snapshots": t_steps,
            "overhead_frac": t_steps / plain - 1.0, "total_s_with_flush": t_all,
            "write_gb_s": info["bytes"] / t_all / 1e9,
            "note": "host wall-clock times; device-to-host copies and file writes overlap the stencil"}


def bench_paper_variants(args, stream, hbm_peak):
    """The paper's own kernel forms on this GPU, with its effective-bandwidth
    accounting (Eq. 4a, 4b: fetch = L^3 - 8 - 12 (L - 2), write = (L - 2)^3
    elements per variable): the 2-variable application kernel (outer layer
    held, noise 0.1) and the 1-variable no-random update, FP64 like the
    paper's runs and FP32, at L = 1024.  The paper's MI250x figures (Table 2,
    one GCD): Julia 2-variable 312 GB/s (111.07 ms), Julia 1-variable no
    random 312 GB/s (54.03 ms), HIP 1-variable 599 GB/s (28.74 ms), peak
    1600 GB/s."""
    import torch

    from paper_2309_10292_gb300 import gs
    L, n = 1024, 6
    out = {"L": L, "steps": n, "accounting": "paper Eq. 4a-4b effective bytes / kernel time",
           "paper_mi250x_gb_s": {"julia_2var": 312, "julia_1var_no_random": 312, "hip_1var": 599, "peak": 1600},
           "paper_mi250x_ms": {"julia_2var": 111.07, "julia_1var_no_random": 54.03, "hip_1var": 28.74}}

    def eff_bytes(esz, nvar):
        return nvar * ((L ** 3 - 8 - 12 * (L - 2)) + (L - 2) ** 3) * esz

    def timed(step, sync):
        step(2)
        sync()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(n)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    for dtype, esz in (("f64", 8), ("f32", 4)):
        sim = gs.GrayScott(L, dtype=dtype, noise=NOISE, seed=SEED, **PARAMS)
        sim.boundary = gs.GS_BOUNDARY_HELD
        if dtype == "f32":
            sim.autotune(steps_per_trial=12)  # (temporal blocking is skipped: periodic only)
        ms = timed(sim.step, sim.sync)
        plan = sim.plan
        sim.close()
        torch.cuda.empty_cache()
        out[f"two_var_{dtype}"] = {"ms_per_step": ms, "effective_gb_s": eff_bytes(esz, 2) / ms / 1e6,
                                   "plan": {k: plan[k] for k in ("kernel", "tile_x", "tile_y", "tile_z", "stages")},
                                   "gcups": L ** 3 / ms / 1e6,
                                   "hbm_frac": eff_bytes(esz, 2) / ms / 1e6 / hbm_peak}
        one = gs.SingleField(L, D=PARAMS["Du"], dt=PARAMS["dt"], dtype=dtype, boundary=gs.GS_BOUNDARY_HELD)
        ms = timed(one.step, one.sync)
        info = one.info
        one.close()
        torch.cuda.empty_cache()
        out[f"one_var_{dtype}"] = {"ms_per_step": ms, "effective_gb_s": eff_bytes(esz, 1) / ms / 1e6,
                                   "gcups": L ** 3 / ms / 1e6,
                                   "hbm_frac": eff_bytes(esz, 1) / ms / 1e6 / hbm_peak,
                                   "kernel": "z-march single field" if info["zmarch"] else "one thread per cell"}
    return out


def _large_run(L, n, noise, stream, hbm_peak):
    """Autotune (plain, z-march, temporal blocking at depths 2-8) and time n
    steps of an L^3 FP32 grid from the centred-cube start."""
    import torch

    from paper_2309_10292_gb300 import gs
    sim = gs.GrayScott(L, dtype="f32", noise=noise, seed=SEED, **PARAMS)
    best, trials = sim.autotune(steps_per_trial=12)
    by_depth = {}
    for r in trials:
        d = r["depth"] if r["kernel"] == gs.GS_KERNEL_TBLOCK else 1
        if d not in by_depth or r["us_per_step"] < by_depth[d]["us_per_step"]:
            by_depth[d] = r
    sim.step(4)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(n)
    b.record(stream)
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1e3
    g = L ** 3 * n / s / 1e9
    depth = best["depth"] if best["kernel"] == gs.GS_KERNEL_TBLOCK else 1
    sim.close()
    return {"value": g, "unit": "GCUPS", "time_s": s, "plan": best,
            "hbm_frac_per_pass": g * 16.0 / depth / hbm_peak,
            "single_pass_roofline_frac": g * 16.0 / hbm_peak,
            "best_gcups_by_depth": {str(d): L ** 3 / r["us_per_step"] / 1e3 for d, r in sorted(by_depth.items())},
            "tuned_candidates": len(trials)}


def bench_large(args, stream, hbm_peak):
    """L=1024 FP32 (four 4.3 GB fields), noise 0.1, plan autotuned over the plain,
    z-march and temporally blocked (depth 2-8) kernels, 500 steps; and the same
    grid without noise, where the lighter per-cell arithmetic lets temporal
    blocking pass the single-step HBM roofline."""
    L, n = 1024, args.large_steps
    out = {"workload": f"plain stencil FP32, L={L}, noise {NOISE}, {n} steps, autotuned plan"}
    out.update(_large_run(L, n, NOISE, stream, hbm_peak))
    out["noise0"] = {"workload": f"the same grid and plan search without noise (noise 0), {n} steps"}
    out["noise0"].update(_large_run(L, n, 0.0, stream, hbm_peak))
    # issue roofline of the temporally blocked plans (noise on): warp
    # instructions per update from the committed ncu counts, against the
    # issue ceiling of 4 warp instructions per clock per SM at the SM clock
    # sampled during the bench
    inst = profiled_issue()
    if inst is not None:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        clk = (getattr(args, "sm_mhz_seen", None) or 2070.0) * 1e6
        peak = 4 * sms * clk / 1e9  # G warp instructions / s
        hbm_bound = hbm_peak / 16.0
        rows = {}
        for plan, i in inst.items():
            rows[plan] = {"warp_inst_per_update": i, "issue_bound_gcups": peak / i}
        d3 = inst.get("tblock,32,32,64,3")
        out["issue_roofline"] = {
            "bound": "issue", "unit": "G warp instructions/s", "peak": peak,
            "peak_kind": "4 warp instructions per clock per SM x SMs x the sampled SM clock",
            "plans": rows, "single_step_hbm_bound_gcups": hbm_bound,
            "depth3_achieved_issue_fraction": 0.734,
            "depth3_warp_inst_needed_to_pass_single_step": (peak * 0.734 / hbm_bound) if d3 else None,
            "source": os.path.relpath(TBLOCK_PROFILE, ROOT)}
    return out


def bench_surrogate(args, stream):
    """Surrogate: train on L=128 stencil trajectories, then advance an L=256 FP32
    grid (noise 0) by N steps with the checked surrogate run and compare its
    time-to-state and error with the plain FP32 stencil and the FP64 stencil."""
    import numpy as np
    import torch

    from paper_2309_10292_gb300 import gs, inputs, surrogate
    p = dict(PARAMS)
    F, k = p.pop("F"), p.pop("k")
    # training
    pool = surrogate.TrajectoryPool(L=128, n=16, seed=11, warm=(200, 1500))
    net = gs.Surrogate(inputs.surrogate_init_params(seed=0))
    # one training step (forward, every data and weight gradient, Adam) on a
    # fixed batch of 2 pairs, timed alone with CUDA events
    xu, xv, yu, yv, Fb, kb = pool.draw(args.surr_batch)
    timer = gs.Surrogate(inputs.surrogate_init_params(seed=1, last_scale=0.1))
    for _ in range(3):
        timer.train_step(xu, xv, Fb, kb, yu, yv, 1e-5)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(10):
        timer.train_step(xu, xv, Fb, kb, yu, yv, 1e-5)
    b.record(stream)
    torch.cuda.synchronize()
    step_s = a.elapsed_time(b) / 1e4
    timer.close()
    del xu, xv, yu, yv
    train_flop = surrogate.TRAIN_FLOP_PER_CELL * args.surr_batch * 128 ** 3
    losses, t_train = surrogate.train(net, pool, iters=args.surr_iters, lr=1e-3, batch=args.surr_batch,
                                      warmup=100)
    ev = surrogate.evaluate(net, pool, pairs=8)
    pool.close()
    seg = max(1, len(losses) // 20)
    curve = [float(np.mean(losses[i:i + seg])) for i in range(0, len(losses), seg)]
    L, n, warm = 256, args.surr_steps, 300
    # forward throughput at L=256
    x = torch.rand((1, L, L, L), device="cuda")
    y = torch.rand((1, L, L, L), device="cuda") * 0.3
    net.forward(x, y, [F], [k])
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(3):
        net.forward(x, y, [F], [k])
    b.record(stream)
    torch.cuda.synchronize()
    fwd_s = a.elapsed_time(b) / 3e3
    flop = 2 * 27 * (4 * 32 + 4 * 32 * 32 + 32 * 2) * L ** 3
    del x, y
    # time-to-state: plain FP32 stencil (autotuned plan), surrogate run, FP64 stencil
    def fresh(dtype):
        sim = gs.GrayScott(L, F=F, k=k, noise=0.0, seed=0, dtype=dtype, **p)
        sim.step(warm)
        return sim
    plain = fresh("f32")
    plain.autotune(steps_per_trial=12)
    tuned = plain.plan
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain.step(n)
    plain.sync()
    t_plain = time.perf_counter() - t0
    up, vp = plain.read()
    plain.close()
    def checked_run(tol):
        s32 = fresh("f32")
        # the surrogate's stencil checks and fallbacks use the same tuned plan
        s32.set_plan(tuned["kernel"], tuned["tile_x"], tuned["tile_y"], tuned["tile_z"], tuned["depth"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = net.run(s32, F, k, n, check_every=64, tol=tol)
        t = time.perf_counter() - t0
        us, vs = s32.read()
        s32.close()
        return rep, t, us, vs
    rep, t_surr, us, vs = checked_run(args.surr_tol)
    tighter = args.surr_tol / 2
    rep_t, t_t, ut, vt = checked_run(tighter)
    s64 = fresh("f64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s64.step(n)
    s64.sync()
    t_fp64 = time.perf_counter() - t0
    u64, v64 = s64.read()
    s64.close()
    sds = fresh("f64")
    sds.arith = gs.GS_ARITH_DS
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sds.step(n)
    sds.sync()
    t_ds = time.perf_counter() - t0
    sds.close()
    net.close()
    err = lambda a, b: float(max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()))
    rms = lambda a, b: float(np.sqrt(np.mean((a[0] - b[0]) ** 2) + np.mean((a[1] - b[1]) ** 2)))
    return {"workload": f"surrogate trained for {args.surr_iters} steps of {args.surr_batch} pairs of L=128 "
                        f"stencil trajectories (16 runs, F, k as the batched workload, noise 0); run on L={L} "
                        f"FP32 from step {warm}, {n} steps, check every 64 steps against 16 stencil steps, "
                        f"tol {args.surr_tol}",
            "train_step_ms_L128": step_s * 1e3, "train_step_batch": args.surr_batch,
            "train_step_tflops": train_flop / step_s / 1e12,
            "train_time_s": t_train, "train_loss_first": float(np.mean(losses[:10])),
            "train_loss_last": float(np.mean(losses[-10:])), "train_loss_curve": curve,
            "heldout_max_network": ev["max_network"], "heldout_max_no_change": ev["max_persistence"],
            "tighter_tol": {"tol": tighter, "report": rep_t, "time_s": t_t,
                            "max_abs_error_vs_fp32_stencil": err((ut, vt), (up, vp)),
                            "rms_error_vs_fp32_stencil": rms((ut, vt), (up, vp))},
            "rms_error_vs_fp32_stencil": rms((us, vs), (up, vp)),
            "heldout_rms_network": ev["rms_network"], "heldout_rms_no_change": ev["rms_persistence"],
            "forward_ms_L256": fwd_s * 1e3,
            "forward_tflops": flop / fwd_s / 1e12,
            "time_to_state_s": {"surrogate_run": t_surr, "plain_fp32": t_plain, "plain_fp64_ieee": t_fp64,
                                "plain_fp64_double_single": t_ds},
            "plain_plan": tuned,
            "speedup_vs_plain": t_plain / t_surr,
            "report": rep,
            "max_abs_error_vs_fp32_stencil": err((us, vs), (up, vp)),
            "max_abs_error_vs_fp64_stencil": err((us, vs), (u64, v64)),
            "fp32_stencil_vs_fp64_stencil": err((up, vp), (u64, v64))}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2309_10292_gb300 import gs

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    L = args.L
    cells = L ** 3

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sim = gs.GrayScott(L, dtype="f32", noise=NOISE, seed=SEED, **PARAMS)
    if args.plan:
        # explicit plan (profiling runs): kernel name, tile_x, tile_y, tile_z, depth/stages
        kind, *nums = args.plan.split(",")
        kern = {"naive": gs.GS_KERNEL_NAIVE, "zmarch": gs.GS_KERNEL_ZMARCH, "tblock": gs.GS_KERNEL_TBLOCK}[kind]
        tx, ty, tz, last = (int(x) for x in nums)
        gs.gs_set_plan_full(sim.handle, dict(kernel=kern, tile_x=tx, tile_y=ty, tile_z=tz,
                                             depth=last if kern == gs.GS_KERNEL_TBLOCK else 1,
                                             stages=last if kern == gs.GS_KERNEL_ZMARCH else 0))
        tune_best, tune_trials = {"us_per_step": None}, []
    else:
        tune_best, tune_trials = sim.autotune(steps_per_trial=24)
    plan = sim.plan
    # warm-up (untimed)
    for _ in range(args.warmup):
        sim.init()
        sim.step(args.time_steps)
    barrier()
    launches0 = gs.gs_launch_count(sim.handle)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local, args.clocks_log) if rank == 0 else None
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        a, b, c = ev[i]
        a.record(stream)
        sim.init()
        b.record(stream)
        sim.step(args.time_steps)
        c.record(stream)
    t_end.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    args.sm_mhz_seen = clk["sm_mhz"] if clk else None
    launches = gs.gs_launch_count(sim.handle) - launches0
    stencil_launches = launches - args.steps  # one init launch per bench step
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), ws, dev)
    step_ms = sum(b.elapsed_time(c) for (_, b, c) in ev)
    value = whole_job_rate(ws, cells * args.time_steps * args.steps, total_ms / 1e3) / 1e9
    per_launch_s = step_ms / 1e3 / stencil_launches
    hbm_peak, peak_kind = load_peaks()
    alg_bytes = 16.0 * cells  # one read and one write of u and v per pass
    achieved = alg_bytes / per_launch_s / 1e9
    kname = {gs.GS_KERNEL_NAIVE: "gs_naive_kernel<float, noise>", gs.GS_KERNEL_ZMARCH: "gs_zmarch_kernel<float, noise>",
             gs.GS_KERNEL_TBLOCK: f"gs_tblock_kernel<noise, {plan['depth']}>"}[plan["kernel"]]
    traffic = profiled_traffic() if plan["kernel"] == gs.GS_KERNEL_ZMARCH else None

    # end to end through the C-ABI with host buffers: every bench step copies
    # the initial state in from pinned host memory, runs the 1000 steps and
    # copies the final state out.  Two grids on two streams take the bench
    # steps in turn, so one grid's host copies overlap the other's compute;
    # a grid's stepping waits (device event) for the other grid's stepping,
    # so the two never compete for HBM, and a grid's output buffers are
    # reused only after the host has waited for its previous result.
    u0 = torch.empty((L, L, L), dtype=torch.float32).pin_memory()
    v0 = torch.empty_like(u0).pin_memory()
    sim.init()
    gs.gs_read(sim.handle, gs.GS_U, u0)
    gs.gs_read(sim.handle, gs.GS_V, v0)
    sim2 = gs.GrayScott(L, dtype="f32", noise=NOISE, seed=SEED, stream=torch.cuda.Stream(dev), **PARAMS)
    gs.gs_set_plan_full(sim2.handle, plan)
    sim2.step(args.warmup)  # the second grid's first launches, outside the timed region like the first's
    sims = [sim, sim2]
    outs = [[torch.empty_like(u0).pin_memory() for _ in range(2)] for _ in sims]
    e2e_steps = max(1, min(args.steps, 6))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    stepped = None  # event after the previous bench step's stencil launches
    for i in range(e2e_steps):
        j = i % 2
        s, (uo, vo) = sims[j], outs[j]
        if i >= 2:
            s.sync()  # the previous result in uo/vo has reached the host
        gs.gs_write_async(s.handle, gs.GS_U, u0)
        gs.gs_write_async(s.handle, gs.GS_V, v0)
        gs.gs_set_step(s.handle, 0)
        if stepped is not None:
            s.stream.wait_event(stepped)
        s.step(args.time_steps)
        stepped = torch.cuda.Event()
        stepped.record(s.stream)
        gs.gs_read_async(s.handle, gs.GS_U, uo)
        gs.gs_read_async(s.handle, gs.GS_V, vo)
    for s in sims:
        s.sync()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    uo, vo = outs[(e2e_steps - 1) % 2]
    if e2e_steps >= 2:  # both grids ran the same problem from the same inputs
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    sim2.close()
    e2e_value = whole_job_rate(ws, cells * args.time_steps * e2e_steps, e2e_s) / 1e9
    assert np.isfinite(uo.numpy()).all()

    extra = {}
    if rank == 0 and not args.no_fp64:
        # FP64 runs of the same workload (oracle-matching precision), shorter:
        # IEEE FP64 arithmetic, and double-single arithmetic on the FP32 pipe
        ref64 = {}

        def fp64_rate(arith):
            # GCUPS, and the max-abs difference of the final fields (5 + n64
            # steps from the centred cube) from the IEEE FP64 run's
            s64 = gs.GrayScott(L, dtype="f64", noise=NOISE, seed=SEED, **PARAMS)
            s64.arith = arith
            if arith != gs.GS_ARITH_IEEE:
                s64.autotune(steps_per_trial=4)  # the converting kernels favour other tiles
            s64.step(5)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64.step(n64)
            b.record(stream)
            torch.cuda.synchronize()
            u, v = s64.tensors()
            if arith == gs.GS_ARITH_IEEE:
                ref64["u"], ref64["v"] = u.clone(), v.clone()
                diff = 0.0
            else:
                diff = max(float((u - ref64["u"]).abs().max()), float((v - ref64["v"]).abs().max()))
            s64.close()
            return cells * n64 / (a.elapsed_time(b) / 1e3) / 1e9, diff

        n64 = 1000  # the L = 512 workload's step count (one gs_step call)
        # the FP64 pipe's measured rate (FMAs per second), clocks sampled meanwhile
        csamp = Clocks(torch.cuda.current_device())
        fp64_ops = max(gs.gs_measure_fp64_fma(stream) for _ in range(6))
        fp64_clocks = csamp.stop()
        g64, _ = fp64_rate(gs.GS_ARITH_IEEE)
        g64ds, d64ds = fp64_rate(gs.GS_ARITH_DS)
        g64fx, d64fx = fp64_rate(gs.GS_ARITH_FX)
        g64fxf, d64fxf = fp64_rate(gs.GS_ARITH_FXF)
        ref64.clear()
        # precision: the FP32 result of the whole workload (the e2e run's
        # output) against the same run in IEEE FP64 on the GPU
        s64 = gs.GrayScott(L, dtype="f64", noise=NOISE, seed=SEED, **PARAMS)
        s64.step(args.time_steps)
        u64, v64 = s64.read()
        s64.close()
        du = float(np.abs(uo.numpy().astype(np.float64) - u64).max())
        dv = float(np.abs(vo.numpy().astype(np.float64) - v64).max())
        del u64, v64
        extra["accuracy"] = {"fp32_vs_fp64_max_abs": {"u": du, "v": dv}, "time_steps": args.time_steps,
                             "note": "the FP32 workload's final fields against the same run in IEEE FP64 "
                                     "on the GPU (the FP64 kernels match the FP64 oracle within 1e-10, tested)"}
        extra["fp64"] = {"value": g64, "unit": "GCUPS", "time_steps": n64,
                         "hbm_frac": g64 * 32.0 / hbm_peak, "note": "same workload in FP64 (IEEE arithmetic)",
                         # the FP64 pipe bounds it: 22 FP64 operations per cell (11 adds,
                         # 9 FMAs, 2 multiplies; one pipe issue each) against the
                         # measured FMA issue rate of the pipe
                         "alu_roofline": {"bound": "alu", "achieved": g64 * 22.0, "peak": fp64_ops / 1e9,
                                          "unit": "G FP64 operations/s", "frac": g64 * 22.0 / (fp64_ops / 1e9),
                                          "peak_kind": "measured (gs_measure_fp64_fma: independent FMA chains)",
                                          "peak_clocks": fp64_clocks,
                                          "nominal_peak": 625.0},
                         "double_single": {"value": g64ds, "unit": "GCUPS", "hbm_frac": g64ds * 32.0 / hbm_peak,
                                           "max_abs_vs_ieee_fp64": d64ds,
                                           "note": "FP64 fields, double-single arithmetic on the FP32 pipe "
                                                   "(within 1e-13 of the FP64 oracle after 100 steps, tested)"},
                         "fixed_point": {"value": g64fx, "unit": "GCUPS", "hbm_frac": g64fx * 32.0 / hbm_peak,
                                         "max_abs_vs_ieee_fp64": d64fx,
                                         "note": "FP64 fields, 64-bit fixed point on the integer pipes: exact "
                                                 "neighbour sums (within 1e-14 of the FP64 oracle after 100 steps, "
                                                 "tested)"},
                         "fixed_point_remainder": {"value": g64fxf, "unit": "GCUPS",
                                                   "hbm_frac": g64fxf * 32.0 / hbm_peak,
                                                   "max_abs_vs_ieee_fp64": d64fxf,
                                                   "note": "FP64 fields, 32-bit fixed point with an FP32 "
                                                           "remainder: exact integer neighbour sums, float-pair "
                                                           "products (within 3e-13 of the FP64 oracle after 100 steps, "
                                                           "tested)"},
                         "compared_after_steps": 5 + n64}

    if rank == 0 and not args.no_batch:
        extra["batched"] = bench_batched(args, stream, hbm_peak)
    if rank == 0 and not args.no_large:
        extra["l1024"] = bench_large(args, stream, hbm_peak)
    if rank == 0 and not args.no_surrogate:
        extra["surrogate"] = bench_surrogate(args, stream)
    if rank == 0 and not args.no_snapshot:
        extra["snapshot"] = bench_snapshot(args, stream)
    if rank == 0 and not args.no_variants:
        extra["paper_variants"] = bench_paper_variants(args, stream, hbm_peak)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": main_workload(L, args.time_steps),
                       "L": L, "time_steps": args.time_steps,
                       "plan": plan,
                       "autotune": {"candidates": len(tune_trials), "best_us_per_step": tune_best["us_per_step"]},
                       "l2": "inputs larger than L2 (4 field buffers of %.2f GB)" % (cells * 4 / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "source_sha256_16": source_digest()},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic,
                         "kernel": kname, "launches": stencil_launches,
                         "steps_per_launch": plan["depth"] if plan["kernel"] == gs.GS_KERNEL_TBLOCK else 1,
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": per_launch_s * 1e3},
            "e2e": {"value": e2e_value, "unit": "GCUPS", "h2d_bytes_per_step": 2 * cells * 4,
                    "d2h_bytes_per_step": 2 * cells * 4, "steps": e2e_steps,
                    "overlap": "two grids on two streams take the steps in turn (async copies; a grid steps after the other grid's steps)"},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    sim.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=L_MAIN)
    ap.add_argument("--time-steps", type=int, default=NSTEPS)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 side measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances measurement")
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--no-large", action="store_true", help="skip the L=1024 measurement")
    ap.add_argument("--large-steps", type=int, default=500)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate measurement")
    ap.add_argument("--no-snapshot", action="store_true", help="skip the snapshot-writer measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the paper-variant kernels (L=1024 FP64/FP32)")
    ap.add_argument("--clocks-log", default=None, help="directory for the raw nvidia-smi clock samples")
    ap.add_argument("--plan", default="", help="fixed plan instead of autotuning, e.g. zmarch,128,8,64,6")
    ap.add_argument("--surr-iters", type=int, default=6000)
    ap.add_argument("--surr-batch", type=int, default=2)
    ap.add_argument("--surr-steps", type=int, default=1024)
    ap.add_argument("--surr-tol", type=float, default=0.2)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
