#!/usr/bin/env python
"""Benchmark of the TaylorGrid query forward + coefficient backward on GB300.

Workload (one step): a 256^3 order-2 FP32 TaylorGrid (1 channel, 10
coefficients per vertex, 671 MB), 2^24 uniform points, upstream dL/df ~ N(0,1).
A step bins the points by brick (tg_batch_bin), evaluates f at every point
(tg_query_binned, Eq. 2 - Eq. 4) and scatters dL/df back onto the
coefficients (tg_query_backward_binned). Inputs are larger than L2 (points
201 MB, grid 671 MB, gradient 671 MB).

At N = 1 the line also carries, under "configs", the other workloads of the
method measured the same way (an SDF fit step with Adam, the query forward
alone at orders 0-2 and FP32/BF16, a ray-marching training step, and a
serving trace of fit jobs and queries against the same jobs run one at a
time); --no-extras / --no-serving skip them.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica (weak scaling, no collective on
the data path); the timed region is bracketed by barriers and the max over
ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RES, ORDER, C, K = 256, 2, 1, 10
N_POINTS = 1 << 24
METRIC = "TaylorGrid fwd+bwd Mpts/s & %HBM peak; fit-job p50/p99 latency vs plain FP32"
WORKLOAD = "query fwd+bwd, 256^3 order-2 FP32 TaylorGrid, 2^24 uniform points"
CPU_SAMPLE = 1 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(n_points: int, n_vertices: int):
    """Compulsory-traffic model: each point's inputs/outputs once, each touched vertex once.

    forward:  12 B (xyz) + 4 B (f) per point + K*4 B per touched vertex
    backward: 12 B (xyz) + 4 B (dL/df) per point + 2*K*4 B per touched vertex (gradient read-modify-write)
    """
    touched = n_vertices * (1.0 - np.exp(-8.0 * n_points / n_vertices))
    fwd = 16.0 * n_points + K * 4.0 * touched
    bwd = 16.0 * n_points + 2.0 * K * 4.0 * touched
    return fwd, bwd


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1])); mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda() else "gloo")
    return world, rank, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seeds(rank: int):
    """Seeds of one replica's inputs: (points, upstream). Every rank draws its own points."""
    return 1 + rank, 4 + rank


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(n_points: int, coefs64):
    """One fwd+bwd of the oracle on n_points of the workload's points (seed 1) and upstream (seed 4)."""
    import oracle
    import workloads as W
    pts = W.uniform_points(1, n_points)
    up = W.normal(4, W.STREAM_UPSTREAM, np.arange(n_points, dtype=np.uint64)).reshape(-1, 1)
    t0 = time.perf_counter()
    oracle.query(3, RES, ORDER, C, coefs64, pts, want_grad=False)
    oracle.query_backward(3, RES, ORDER, C, pts, up)
    return time.perf_counter() - t0


def host_grid_fp64():
    """A 256^3 order-2 grid of N(0,1) coefficients for the reference arm, which runs without a GPU. The oracle's
    arithmetic does not depend on the values, so numpy's generator stands in for the device's (its values
    differ from the GPU grid's; the main line's baseline runs on the GPU grid's own coefficients)."""
    return np.random.default_rng(0).standard_normal(RES ** 3 * C * K)


def threads_used() -> int:
    """OpenMP threads of the oracle: OMP_NUM_THREADS if set, else every core this process may run on (nproc)."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    env = os.environ.get("OMP_NUM_THREADS")
    return min(int(env), n) if env else n


def oracle_rate(coefs64, steps: int, warmup: int, sample: int = CPU_SAMPLE):
    """Steady-state oracle throughput: `warmup` untimed samples of sample / 16 points, then `steps` timed samples."""
    for _ in range(warmup):
        oracle_sample(sample // 16, coefs64)
    total = sum(oracle_sample(sample, coefs64) for _ in range(steps))
    return sample * steps / total / 1e6, total


def cpu_baseline_of(coefs32, steps: int = 5, warmup: int = 3):
    """The oracle timed on the given grid in a fresh process (no CUDA context, no torch thread pool beside the
    oracle's OpenMP threads), on `steps` samples of CPU_SAMPLE points after `warmup` smaller untimed ones."""
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    try:
        np.save(path, coefs32)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-from", path,
                            "--steps", str(steps), "--warmup", str(warmup)], capture_output=True, text=True,
                           check=True)
    finally:
        os.unlink(path)
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_cpu_baseline(path: str, steps: int, warmup: int):
    coefs64 = np.load(path).astype(np.float64)
    value, _ = oracle_rate(coefs64, steps, warmup)
    print(json.dumps({"value": value, "unit": "Mpts/s", "cores": threads_used(), "kind": "oracle",
                      "sample": f"{steps} x {CPU_SAMPLE} of the 2^24 points (the first {CPU_SAMPLE} of the "
                                f"workload's points and upstream) after {warmup} untimed warm-up samples, on the "
                                "coefficients of the GPU's grid, in a process of its own"}), flush=True)


def run_oracle_timings():
    """The FP64 oracle on the fits of the other configurations, timed on the host cores: the whole config-1 fit
    (32^3 order 2, sphere, 2^16 points per step, L1, Adam lr 1e-2, 100 steps), and samples of the 256^3 fit
    step (2^20 points, L1 + 0.1 eikonal, Adam) and of the ray-march training step (160^3 density order 2 +
    colour order 1, 8192 rays x 256 samples, both Adam steps), extrapolated to 2000 and 3000 steps. Inputs are
    generated before each timed region."""
    import oracle
    import workloads as W
    out = {"cores": threads_used()}
    # config 1, the whole fit
    shape = W.sphere_shape()
    res, order, n, steps = 32, 2, 1 << 16, 100
    batches = [W.sdf_points(shape, seed=1, step=k, n=n) for k in range(steps)]
    p = W.init_coefs(3, res, order, 1, seed=0, std=1e-3).astype(np.float64)
    m, v = np.zeros_like(p), np.zeros_like(p)
    t0 = time.perf_counter()
    for k in range(steps):
        g, _ = oracle.sdf_step(res, order, p, batches[k], shape.spheres, shape.boxes, 0.0)
        oracle.adam(p, g, m, v, 1e-2, step=k + 1)
    t1 = time.perf_counter()
    ev = W.sdf_points(shape, seed=2, step=0, n=1 << 14)
    f, _, _, _ = oracle.query(3, res, order, 1, p, ev, want_grad=False)
    err = float(np.abs(f[:, 0] - oracle.sdf_union(shape.spheres, shape.boxes, ev.astype(np.float64))).mean())
    out["config1_fit"] = {"s": t1 - t0, "steps": steps, "mean_abs_sdf_error": err, "kind": "measured"}
    # config 2, a sample of the 256^3 fit step
    shape = W.union_shape(0)
    res, n, k_s = 256, 1 << 20, 2
    batches = [W.sdf_points(shape, seed=1, step=k, n=n) for k in range(k_s)]
    p = W.init_coefs(3, res, 2, 1, seed=0, std=1e-3).astype(np.float64)
    m, v = np.zeros_like(p), np.zeros_like(p)
    t0 = time.perf_counter()
    for k in range(k_s):
        g, _ = oracle.sdf_step(res, 2, p, batches[k], shape.spheres, shape.boxes, 0.1)
        oracle.adam(p, g, m, v, 5e-3, step=k + 1)
    per = (time.perf_counter() - t0) / k_s
    out["config2_fit"] = {"s_per_step": per, "sampled_steps": k_s, "s_2000_steps_extrapolated": 2000 * per,
                          "kind": "extrapolated from the sampled steps"}
    del p, m, v, g
    # config 4, a sample of the ray-march training step
    res, R, S = 160, 8192, 256
    dco = W.init_coefs(3, res, 2, 1, seed=0, std=0.5).astype(np.float64)
    cco = W.init_coefs(3, res, 1, 3, seed=1, std=0.5).astype(np.float64)
    r_s = 1024                                   # rays rendered per sample; the step's 8192 scale linearly
    o, d = W.random_rays(7, R, radius=1.5, spread=0.35)
    tgt = np.random.default_rng(0).random((R, 3)).astype(np.float32)
    md, vd, mc, vc = (np.zeros_like(a) for a in (dco, dco, cco, cco))
    t0 = time.perf_counter()
    _, _, dg, cg = oracle.render(res, 2, dco, 1, cco, o[:r_s], d[:r_s], S, seed=0, target=tgt[:r_s])
    t1 = time.perf_counter()
    oracle.adam(dco, dg, md, vd, 0.1, step=1)
    oracle.adam(cco, cg, mc, vc, 0.03, step=1)
    t2 = time.perf_counter()
    per = (t1 - t0) * R / r_s + (t2 - t1)
    out["config4_render_fit"] = {"s_per_step": per, "sampled": f"{r_s} of the step's {R} rays (scaled by {R // r_s}) "
                                 "and both Adam steps in full", "s_3000_steps_extrapolated": 3000 * per,
                                 "kind": "extrapolated from the sampled step"}
    print(json.dumps(out), flush=True)


def oracle_timings_of():
    """run_oracle_timings in a process of its own (no CUDA context beside the oracle's threads)."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-timings"], capture_output=True,
                       text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args, world, rank):
    if rank != 0:
        return
    value, total = oracle_rate(host_grid_fp64(), args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_points_per_step": CPU_SAMPLE},
        "cpu_baseline": {"value": value, "unit": "Mpts/s", "cores": threads_used(), "kind": "oracle",
                         "sample": f"{CPU_SAMPLE} of the 2^24 points per step (the first {CPU_SAMPLE} of the "
                                   "workload's points and upstream), on a 256^3 order-2 grid of N(0,1) coefficients "
                                   "(numpy's generator: values differ from the GPU grid's, the arithmetic does not)"},
        "e2e": {"value": value, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tg.load()
    launches_per_step = 7      # 5 binning kernels, forward, backward

    g = tg.tg_create(3, RES, ORDER, C, "f32", seed=0, init_std=1.0)
    N = N_POINTS
    seed_pts, seed_up = replica_seeds(rank)
    pts_np = W.uniform_points(seed_pts, N)
    up_np = W.normal(seed_up, W.STREAM_UPSTREAM, np.arange(N, dtype=np.uint64)).astype(np.float32).reshape(-1, 1)
    P = torch.from_numpy(pts_np).to(dev)
    U = torch.from_numpy(up_np).to(dev)
    out = torch.empty((N, 1), device=dev)
    grad = torch.zeros(g.n_coefs, device=dev)
    batch = tg.tg_batch_create(3, RES, N)
    stream = torch.cuda.current_stream()

    # one step = bin, forward, backward. The headline runs in binned order: f
    # is written, and dL/df read, in the batch's brick order (tg_batch_order
    # maps a slot to its input index), as the training paths use it; the
    # input-order variant (f scattered to, dL/df gathered from, input
    # positions) is timed beside it.
    def calls_of(binned):
        return [("bin", lambda pts, up: tg.tg_batch_bin(batch, pts)),
                ("forward", lambda pts, up: tg.tg_query_binned(g, batch, out=out, binned_order=binned)),
                ("backward", lambda pts, up: tg.tg_query_backward_binned(g, batch, up, grad, binned_order=binned))]

    def timed(binned, steps, warmup, clk=None):
        calls = calls_of(binned)
        for _ in range(warmup):
            for _, call in calls:
                call(P, U)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        kev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for s in range(steps):
            for k, (_, call) in enumerate(calls):
                kev[s][k].record(stream)
                call(P, U)
            kev[s][-1].record(stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = max_over_ranks(world, ev[0].elapsed_time(ev[1])) / steps
        kernels = {name: statistics.mean(e[k].elapsed_time(e[k + 1]) for e in kev) for k, (name, _) in enumerate(calls)}
        return ms, kernels

    # device-timed region
    with Clocks(local) as clk:
        ms, kernels = timed(True, args.steps, args.warmup)
    clocks = clk.summary()
    value = world * N / (ms * 1e-3) / 1e6
    ms_in, kernels_in = timed(False, args.steps, 3)

    # End to end through the public API: every step copies its inputs from pinned
    # host memory and reads f back to pinned host memory. Two buffer sets and two
    # copy streams let step k+1's host-to-device copy and step k-1's read-back run
    # while step k computes, as a caller streaming batches would.
    pts_h = torch.from_numpy(pts_np).pin_memory()
    up_h = torch.from_numpy(up_np).pin_memory()
    outs_h = [torch.empty((N, 1), dtype=torch.float32).pin_memory() for _ in range(2)]
    bufs = [(torch.empty_like(P), torch.empty_like(U), torch.empty_like(out)) for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    in_ready, computed, read_back = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    used = [False, False]

    def e2e_step(k):
        b = k % 2
        Pb, Ub, Ob = bufs[b]
        if used[b]:
            h2d.wait_event(computed[b])            # step k-2 no longer reads these inputs
        with torch.cuda.stream(h2d):
            Pb.copy_(pts_h, non_blocking=True)
            Ub.copy_(up_h, non_blocking=True)
            in_ready[b].record(h2d)
        stream.wait_event(in_ready[b])
        if used[b]:
            stream.wait_event(read_back[b])        # step k-2's f has left this buffer
        tg.tg_batch_bin(batch, Pb)
        tg.tg_query_binned(g, batch, out=Ob, binned_order=True)
        tg.tg_query_backward_binned(g, batch, Ub, grad, binned_order=True)
        computed[b].record(stream)
        d2h.wait_event(computed[b])
        with torch.cuda.stream(d2h):
            outs_h[b].copy_(Ob, non_blocking=True)
            read_back[b].record(d2h)
        used[b] = True

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(h2d)                                 # before the first timed copy
    for k in range(args.steps):
        e2e_step(2 + k)
    e1.record(d2h)                                 # after the last read-back
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(world, e0.elapsed_time(e1)) / args.steps
    barrier(world)
    # the order of points inside a brick differs between binnings (shared-memory ranks), so the last
    # end-to-end f is taken back to input order with that step's own permutation before the comparison
    perm = tg.tg_batch_order(batch).long().cpu()
    f_e2e = torch.empty_like(outs_h[0])
    f_e2e[perm] = outs_h[(1 + args.steps) % 2]
    tg.tg_batch_bin(batch, P)
    tg.tg_query_binned(g, batch, out=out)
    assert torch.equal(f_e2e, out.cpu()), "end-to-end f differs from the device-timed f"

    hbm, peak_kind = peaks()
    fwd_bytes, bwd_bytes = algorithmic_bytes(N, RES ** 3)
    dom = max(kernels, key=kernels.get)
    dom_bytes = {"forward": fwd_bytes, "backward": bwd_bytes}.get(dom)
    achieved = (dom_bytes / (kernels[dom] * 1e-3) / 1e9) if dom_bytes else None
    line = {
        "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_gpu": N, "res": RES, "order": ORDER, "channels": C,
                   "l2": "inputs larger than L2 (points 201 MB, grid 671 MB, gradient 671 MB)",
                   "parallelism": f"replicas x{world}"},
        "order": "binned: f written and dL/df read in the batch's brick order",
        "kernel_ms": {k: round(v, 4) for k, v in kernels.items()},
        "input_order": {"value": world * N / (ms_in * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms_in,
                        "kernel_ms": {k: round(v, 4) for k, v in kernels_in.items()},
                        "note": "f scattered to and dL/df gathered from the points' input positions"},
        "roofline": {"bound": "hbm", "kernel": KERNEL_NAMES[dom], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "peak_kind": peak_kind,
                     "traffic": TRAFFIC.get(dom),
                     "model": "compulsory bytes: 16 B/point + K*4 B (fwd) or 2*K*4 B (bwd) per touched vertex"},
        "step_roofline": {"bytes": fwd_bytes + bwd_bytes, "achieved_gbs": (fwd_bytes + bwd_bytes) / (ms * 1e-3) / 1e9,
                          "frac": (fwd_bytes + bwd_bytes) / (ms * 1e-3) / 1e9 / hbm},
        "alu_roofline": alu_roofline(tg, N, kernels["forward"]),
        "clocks": clocks,
        "e2e": {"value": world * N / (ms_e2e * 1e-3) / 1e6, "unit": "Mpts/s",
                "h2d_bytes_per_step": int(pts_np.nbytes + up_np.nbytes), "d2h_bytes_per_step": int(N * 4),
                "pipelined": "step k+1 copy-in and step k-1 read-back overlap step k's kernels"},
        "gpu_launches": launches_per_step * args.steps,
    }
    if rank == 0 and world == 1 and not args.no_extras:     # single-GPU runs only: the same on every N
        line["configs"] = {"fit_step_256_o2": bench_fit_step(), "query_only_256": bench_query_only(),
                           "query_pair_c_abi_256": bench_query_pair(), "query_pair_2d_1024": bench_query_2d(),
                           "render_160": bench_render(), "render_fit_160_400x400": bench_render_fit(),
                           "recon_256_union": bench_recon(), "fit_256_o2_from_scratch": bench_fit_from_scratch()}
        if not args.no_serving:
            line["configs"]["serving"] = bench_serving()
            line["configs"]["serving_burst"] = bench_burst()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_of(tg.tg_get_coefs(g).cpu().numpy())      # the very grid the GPU ran on
        if not args.no_extras:
            line["oracle_timings"] = oracle_timings_of()
    if rank == 0:
        print(json.dumps(line), flush=True)


def alu_roofline(tg, n_points: int, fwd_ms: float):
    """The forward against the measured FP32 FMA peak (tg_measure_fp32_peak), on an operation-count model of
    Eq. 2 - Eq. 4 at order 2, one channel: per corner the 10-term series as 10 multiply-adds (20 FLOP) on the
    offset products (3 offsets and 6 products, 9 FLOP) and the blend (2 FLOP); per point the 8 corner weights
    (12 multiplies) and the index rule (6). 8 x 31 + 18 = 266 FLOP per point."""
    flop_per_point = 8 * 31 + 18
    peak = tg.tg_measure_fp32_peak()
    achieved = n_points * flop_per_point / (fwd_ms * 1e-3) / 1e12
    return {"kernel": "brick_fwd_kernel (tg_query_binned)", "flop_per_point": flop_per_point,
            "model": "operation count of Eq. 2 - Eq. 4 at order 2",
            "achieved_tflops": achieved, "peak_tflops": peak, "peak_kind": "measured (tg_measure_fp32_peak)",
            "frac": achieved / peak}


def _time_ms(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def bench_fit_step(steps=10, warmup=3):
    """SDF fitting step at 256^3 order 2, 2^20 points, L1 + 0.1 eikonal, Adam (FP32 / BF16 / FP16 storage)."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    shape = W.union_shape(0)
    dsh = tg.DeviceShape(shape.spheres, shape.boxes, shape.area_cdf())
    n = 1 << 20
    out = {}
    for dt in ["f32", "bf16", "f16"]:
        g = tg.tg_create(3, RES, ORDER, 1, dt, seed=0, init_std=1e-3)
        batch = tg.tg_batch_create(3, RES, n)
        grad = torch.zeros(g.n_coefs, device="cuda")
        loss = torch.zeros(2, device="cuda")
        k = [0]

        def step():
            tg.tg_sdf_step(g, batch, dsh, grad, loss, n=n, seed=1, step=k[0], lambda_eik=0.1)
            tg.tg_adam_step(g, grad, lr=5e-3, step=k[0] + 1)
            k[0] += 1
        ms = _time_ms(step, steps, warmup)
        out[dt] = {"ms_per_step": ms, "Mpts_per_s": n / (ms * 1e-3) / 1e6}
        if dt == "f32":       # the paper's full objective: Eq. 7 weight (k = 100), lambda_1 1e-4, TV lambda_2 2e-5
            def step_full():
                tg.tg_sdf_step(g, batch, dsh, grad, loss, n=n, seed=1, step=k[0], lambda_eik=1e-4, k_weight=100.0)
                tg.tg_tv_step(g, 2e-5, grad)
                tg.tg_adam_step(g, grad, lr=3e-3, step=k[0] + 1)
                k[0] += 1
            ms = _time_ms(step_full, steps, warmup)
            out["f32_paper_objective"] = {"ms_per_step": ms, "Mpts_per_s": n / (ms * 1e-3) / 1e6}
            def step_lazy():   # the same step with lazy Adam (untouched coefficients keep parameter and moments)
                tg.tg_sdf_step(g, batch, dsh, grad, loss, n=n, seed=1, step=k[0], lambda_eik=0.1)
                tg.tg_adam_step_lazy(g, grad, lr=5e-3, step=k[0] + 1)
                k[0] += 1
            ms = _time_ms(step_lazy, steps, warmup)
            out["f32_lazy_adam"] = {"ms_per_step": ms, "Mpts_per_s": n / (ms * 1e-3) / 1e6}
            ms_adam = _time_ms(lambda: tg.tg_adam_step(g, grad, lr=5e-3, step=1), steps, warmup)
            adam_bytes = 32.0 * g.n_coefs          # read p, g, m, v; write p, m, v and the zeroed g
            out["adam_kernel"] = {"ms": ms_adam, "algorithmic_GB": adam_bytes / 1e9,
                                  "achieved_GBps": adam_bytes / (ms_adam * 1e-3) / 1e9,
                                  "frac_of_measured_hbm_peak": adam_bytes / (ms_adam * 1e-3) / 1e9 / peaks()[0]}
            ms_tv = _time_ms(lambda: tg.tg_tv_step(g, 2e-5, grad), steps, warmup)
            tv_bytes = 12.0 * g.n_coefs            # read theta, read + write the gradient
            out["tv_kernel"] = {"ms": ms_tv, "algorithmic_GB": tv_bytes / 1e9,
                                "achieved_GBps": tv_bytes / (ms_tv * 1e-3) / 1e9,
                                "frac_of_measured_hbm_peak": tv_bytes / (ms_tv * 1e-3) / 1e9 / peaks()[0]}
        del g, batch, grad
    return {"workload": "SDF fit step, 256^3 order 2, 2^20 points (half uniform, half near-surface), "
                        "L1 + 0.1 eikonal, Adam; sample+bin+forward+loss+backward+Adam", **out}


def bench_query_only(steps=5, warmup=2):
    """Forward-only query throughput, 2^24 uniform points, 256^3, orders 0/1/2, FP32 vs BF16 storage."""
    import torch

    import paper_2402_14415_gb300 as tg
    n = N_POINTS
    P = torch.rand((n, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    outp = torch.empty((n, 1), device="cuda")
    batch = tg.tg_batch_create(3, RES, n)
    res = {}
    for order in (0, 1, 2):
        for dt in ("f32", "bf16"):
            g = tg.tg_create(3, RES, order, 1, dt, seed=0, init_std=1.0)

            def step():
                tg.tg_batch_bin(batch, P)
                tg.tg_query_binned(g, batch, out=outp)
            ms = _time_ms(step, steps, warmup)
            res[f"order{order}_{dt}"] = round(n / (ms * 1e-3) / 1e6, 1)
            if order == 2:    # the same points presorted by brick (the sort untimed), then bin + forward timed
                tg.tg_batch_bin(batch, P)
                Ps = tg.tg_batch_points(batch)
                tg.tg_batch_bin(batch, Ps)
                outs = torch.empty_like(outp)

                def step_sorted():
                    tg.tg_batch_bin(batch, Ps)
                    tg.tg_query_binned(g, batch, out=outs)
                ms = _time_ms(step_sorted, steps, warmup)
                res[f"order2_{dt}_presorted"] = round(n / (ms * 1e-3) / 1e6, 1)
                t0 = time.perf_counter()              # the presort itself, timed: one bin and one gather
                tg.tg_batch_bin(batch, P)
                Ps = tg.tg_batch_points(batch)
                torch.cuda.synchronize()
                res[f"order2_{dt}_presort_ms"] = round(1e3 * (time.perf_counter() - t0), 3)
                del Ps, outs
            del g
    return {"workload": "query forward (bin + binned forward, input order), 256^3, 2^24 uniform points; "
                        "_presorted: the points presorted by brick (sort untimed), _presort_ms: that sort",
            "unit": "Mpts/s", **res}


def bench_query_2d(steps=5, warmup=2, res2=1024):
    """The 2-D path: tg_query + tg_query_backward (point-parallel kernels) on 2^24 uniform points, 1024^2
    order 2 FP32 (6 coefficients per vertex, a 25 MB grid that stays in L2)."""
    import torch

    import paper_2402_14415_gb300 as tg
    n = N_POINTS
    gen = torch.Generator(device="cuda").manual_seed(5)
    P = torch.rand((n, 2), device="cuda", generator=gen)
    U = torch.randn((n, 1), device="cuda", generator=gen)
    out = torch.empty((n, 1), device="cuda")
    g = tg.tg_create(2, res2, 2, 1, "f32", seed=0, init_std=1.0)
    grad = torch.zeros(g.n_coefs, device="cuda")
    ms_f = _time_ms(lambda: tg.tg_query(g, P, out=out), steps, warmup)

    def pair():
        tg.tg_query(g, P, out=out)
        tg.tg_query_backward(g, P, U, grad)
    ms = _time_ms(pair, steps, warmup)
    return {"workload": f"2-D query pair (tg_query + tg_query_backward), {res2}^2 order 2 FP32, 2^24 uniform points",
            "unit": "Mpts/s", "forward": round(n / (ms_f * 1e-3) / 1e6, 1), "pair": round(n / (ms * 1e-3) / 1e6, 1)}


def bench_query_pair(steps=5, warmup=2):
    """The C-ABI pair tg_query + tg_query_backward on 2^24 uniform points at 256^3 order 2 FP32: each call
    bins into the grid's own batch (large 3-D batches) - against the point-parallel kernels on the same points."""
    import torch

    import paper_2402_14415_gb300 as tg
    n = N_POINTS
    gen = torch.Generator(device="cuda").manual_seed(3)
    P = torch.rand((n, 3), device="cuda", generator=gen)
    U = torch.randn((n, 1), device="cuda", generator=gen)
    out = torch.empty((n, 1), device="cuda")
    g = tg.tg_create(3, RES, ORDER, 1, "f32", seed=0, init_std=1.0)
    grad = torch.zeros(g.n_coefs, device="cuda")

    def pair():
        tg.tg_query(g, P, out=out)
        tg.tg_query_backward(g, P, U, grad)
    ms = _time_ms(pair, steps, warmup)
    chunk = (1 << 18) - 1                 # below the binning threshold: the point-parallel kernels

    def pair_pp():
        for i in range(0, n, chunk):
            tg.tg_query(g, P[i:i + chunk], out=out[i:i + chunk])
            tg.tg_query_backward(g, P[i:i + chunk], U[i:i + chunk], grad)
    ms_pp = _time_ms(pair_pp, 2, 1)
    return {"workload": "tg_query + tg_query_backward, 256^3 order 2 FP32, 2^24 uniform points", "unit": "Mpts/s",
            "binned_by_the_calls": round(n / (ms * 1e-3) / 1e6, 1), "ms": round(ms, 3),
            "point_parallel": round(n / (ms_pp * 1e-3) / 1e6, 1), "ms_point_parallel": round(ms_pp, 3)}


def blob_gt(scene, rays_o, rays_d, n_samples=1024, bg=1.0, chunk=1024, dtype=None):
    """Ground-truth colours of the synthetic blob scene (the Synthetic-NeRF stand-in): density
    sum_k a_k exp(-1/2 (x - mu_k)^T P_k (x - mu_k)), colour the density-weighted mean of the blobs' rgb,
    composited along each ray by midpoint quadrature over its [near, far] in the unit cube (bg on a miss).
    Plain torch on the GPU, FP64 (or `dtype`), in chunks of rays; the exponent of every (sample, blob) pair
    is one row of a matrix product of the sample's monomials (xx, yy, zz, xy, xz, yz, x, y, z, 1) with
    per-blob coefficients. It only makes the training targets. In FP32 the monomial form loses about 1e-7 of
    |x^T P x| <= 3 / 0.02^2 to cancellation, a relative error below 1e-3 in a blob's density."""
    import torch
    dtype = dtype or torch.float64
    tiny = torch.finfo(dtype).tiny
    mu, P, amp, rgb = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in scene)
    Pm = torch.einsum("bac,bc->ba", P, mu)                                       # P mu
    coef = torch.stack([P[:, 0, 0], P[:, 1, 1], P[:, 2, 2], 2 * P[:, 0, 1], 2 * P[:, 0, 2], 2 * P[:, 1, 2],
                        -2 * Pm[:, 0], -2 * Pm[:, 1], -2 * Pm[:, 2], (mu * Pm).sum(1)], 0)   # (10, B)
    coef, amp, rgb = coef.to(dtype), amp.to(dtype), rgb.to(dtype)
    out = []
    for i in range(0, rays_o.shape[0], chunk):
        o, d = rays_o[i:i + chunk].to(dtype), rays_d[i:i + chunk].to(dtype)
        inv = 1.0 / torch.where(d == 0, torch.full_like(d, 1e-30), d)
        t0, t1 = (0.0 - o) * inv, (1.0 - o) * inv
        near = torch.clamp(torch.minimum(t0, t1).amax(1), min=0.0)
        far = torch.maximum(t0, t1).amin(1)
        hit = far > near
        dt = torch.where(hit, (far - near) / n_samples, torch.zeros_like(far))
        ts = near[:, None] + (torch.arange(n_samples, device="cuda", dtype=dtype)[None] + 0.5) * dt[:, None]
        x = o[:, None, :] + ts[..., None] * d[:, None, :]                        # (r, n, 3)
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        mono = torch.stack([X * X, Y * Y, Z * Z, X * Y, X * Z, Y * Z, X, Y, Z, torch.ones_like(X)], -1)
        q = mono @ coef                                                          # (r, n, B)
        s = amp * torch.exp(-0.5 * torch.clamp(q, min=0.0))
        sig = s.sum(-1)
        col = (s @ rgb) / torch.clamp(sig, min=tiny)[..., None]
        tau = sig * dt[:, None]
        T = torch.exp(-(torch.cumsum(tau, 1) - tau))
        w = T * (1 - torch.exp(-tau))
        C = (w[..., None] * col).sum(1) + torch.exp(-tau.sum(1))[:, None] * bg
        out.append(torch.where(hit[:, None], C, torch.full_like(C, bg)).float())
    return torch.cat(out)


def bench_render(steps=5, warmup=2):
    """Ray-march training step: 8192 rays x 256 samples, 160^3 density (order 2) + colour (order 1, 3 ch), BF16."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    res, R, S = 160, 8192, 256
    dg = tg.tg_create(3, res, 2, 1, "bf16", seed=0, init_std=0.5)
    cg = tg.tg_create(3, res, 1, 3, "bf16", seed=1, init_std=0.5)
    o, d = W.random_rays(7, R, radius=1.5, spread=0.35)
    ro, rd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    target = torch.rand((R, 3), device="cuda")
    batch = tg.tg_batch_create(3, res, R * S)
    dgr = torch.zeros(dg.n_coefs, device="cuda")
    cgr = torch.zeros(cg.n_coefs, device="cuda")
    loss = torch.zeros(1, device="cuda")
    k = [0]

    def step():
        tg.tg_render_rays(dg, cg, ro, rd, S=S, seed=k[0], target=target, batch=batch, density_grad=dgr,
                          color_grad=cgr, loss_sum=loss)
        tg.tg_adam_step(dg, dgr, lr=1e-2, step=k[0] + 1)
        tg.tg_adam_step(cg, cgr, lr=1e-2, step=k[0] + 1)
        k[0] += 1
    ms = _time_ms(step, steps, warmup)
    fwd = _time_ms(lambda: tg.tg_render_rays(dg, cg, ro, rd, S=S, seed=1), steps, warmup)
    return {"workload": "ray-march training step, 8192 rays x 256 samples, 160^3 BF16 density o2 + colour o1 (3 ch)",
            "train_ms_per_step": ms, "train_Msamples_per_s": R * S / (ms * 1e-3) / 1e6,
            "forward_ms": fwd, "forward_Msamples_per_s": R * S / (fwd * 1e-3) / 1e6}


def bench_fit_from_scratch(steps=2000, n_pts=1 << 20):
    """The 256^3 order-2 fit from scratch as configured: 2000 Adam steps at lr 5e-3, L1 + 0.1 eikonal, 2^20
    points per step, on the union shape (24 spheres, 8 boxes), with FP32, BF16 and FP16 storage; mean |SDF
    error| on 2^16 and volumetric IoU on 2^20 uniform points after the last step."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    from paper_2402_14415_gb300.fit import fit_sdf
    shape = W.union_shape(0)
    dsh = tg.DeviceShape(shape.spheres, shape.boxes, shape.area_cdf())
    ev = torch.rand((1 << 20, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
    out = {}
    for dt in ("f32", "bf16", "f16"):
        g = tg.tg_create(3, RES, ORDER, 1, dt, seed=0, init_std=1e-3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fit_sdf(g, dsh, steps, n_pts, lr=5e-3, lambda_eik=0.1, eval_pts=ev[:1 << 16], eval_every=steps)
        torch.cuda.synchronize()
        out[dt] = {"fit_s": time.perf_counter() - t0, "mean_abs_sdf_error": r.final_error,
                   "iou": tg.tg_sdf_iou(g, dsh, ev)}
        del g
    for dt in ("bf16", "f16"):
        out[dt]["error_vs_f32"] = out[dt]["mean_abs_sdf_error"] / out["f32"]["mean_abs_sdf_error"]
    return {"workload": f"union shape, 256^3 order 2 from scratch, {steps} steps, Adam lr 5e-3, L1 + 0.1 eikonal, "
                        "2^20 points per step", **out}


def bench_recon(coarse_steps=1500, fine_steps=500, n_pts=1 << 20, M=256, n_samples=1 << 16, fine_lr=1e-4):
    """Reconstruction metrics of the union shape (24 spheres, 8 boxes) fitted coarse to fine as Sec. 4.1 trains:
    128^3 order 2 for 1500 steps (Adam lr 5e-3), re-expanded onto 256^3 (tg_resample), 500 more steps (lr 1e-4;
    a fresh Adam at the coarse rate adds more noise than it removes), L1 + 0.1 eikonal, 2^20 points per step. Then the paper's metrics on stand-in data: volumetric IoU on 2^20 uniform
    points, mean |SDF error| on 2^16, and the Chamfer distance between 2^16 area-weighted points of the
    extracted mesh (M^3 lattice, marching tetrahedra) and 2^16 points on the target surface."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    from paper_2402_14415_gb300.fit import fit_sdf
    shape = W.union_shape(0)
    dsh = tg.DeviceShape(shape.spheres, shape.boxes, shape.area_cdf())
    gen = torch.Generator(device="cuda").manual_seed(2)
    ev = torch.rand((1 << 20, 3), device="cuda", generator=gen)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    coarse = tg.tg_create(3, 128, ORDER, 1, "f32", seed=0, init_std=1e-3)
    fit_sdf(coarse, dsh, coarse_steps, n_pts, lr=5e-3, lambda_eik=0.1)
    g = tg.tg_create(3, RES, ORDER, 1, "f32", seed=0, init_std=0.0)
    tg.tg_resample(coarse, g)
    r = fit_sdf(g, dsh, fine_steps, n_pts, lr=fine_lr, lambda_eik=0.1, seed=3, eval_pts=ev[:1 << 16],
                eval_every=fine_steps)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    iou = tg.tg_sdf_iou(g, dsh, ev)
    _, count = tg.tg_extract_mesh(g, M, 0.0, max_tris=0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tris, _ = tg.tg_extract_mesh(g, M, 0.0, max_tris=count)
    b.record()
    torch.cuda.synchronize()
    ms_mesh = a.elapsed_time(b)
    gt = tg.tg_sample_sdf_points(dsh, seed=9, step=0, n=2 * n_samples, jitter=0.0)[n_samples:]
    gt = gt[tg.tg_sdf_eval_target(dsh, gt).abs() < 1e-5].contiguous()   # drops the sampler's uniform fallbacks
    a.record()
    mp = tg.tg_sample_mesh(tris, n_samples, seed=10)
    sa, sb = tg.tg_chamfer(mp, gt)
    b.record()
    torch.cuda.synchronize()
    cd = sa / mp.shape[0] + sb / gt.shape[0]
    return {"workload": f"union shape fitted coarse to fine: 128^3 order 2 for {coarse_steps} steps (Adam lr 5e-3), "
                        f"resampled to 256^3, {fine_steps} steps (lr {fine_lr:g}); 2^20 points per step, L1 + 0.1 "
                        f"eikonal; mesh at {M}^3 by marching tetrahedra",
            "fit_s": fit_s, "mean_abs_sdf_error": r.final_error, "iou": iou, "triangles": count,
            "chamfer_l2": cd, "chamfer_points": [int(mp.shape[0]), int(gt.shape[0])],
            "mesh_extract_ms": ms_mesh, "sample_and_chamfer_ms": a.elapsed_time(b)}


def bench_render_fit(steps=3000, res=160, R=8192, S=256, side=400, lr=(0.1, 0.03)):
    """The ray-marching fit of the synthetic blob scene: 100 cameras at side x side pixels on a sphere of radius
    1.5 (every 10th held out), targets rendered by blob_gt with 1024 midpoint samples (FP32 at 400 x 400: the
    14.4 M training pixels would take minutes in FP64), density (order 2) + colour (order 1, 3 ch) BF16 grids,
    MSE photometric loss, Adam; PSNR on the held-out views."""
    import math

    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    scene = W.blob_scene(4)
    cams_tr = [k for k in range(100) if k % 10 != 0]
    cams_te = [k for k in range(100) if k % 10 == 0]
    o_tr, d_tr = (torch.from_numpy(a).cuda() for a in W.camera_rays(100, side, side, cams=cams_tr))
    o_te, d_te = (torch.from_numpy(a).cuda() for a in W.camera_rays(100, side, side, cams=cams_te))
    gdt = torch.float32 if side > 100 else torch.float64
    gt_tr, gt_te = (blob_gt(scene, o, d, dtype=gdt, chunk=4096 if side > 100 else 1024)
                    for o, d in ((o_tr, d_tr), (o_te, d_te)))
    dg = tg.tg_create(3, res, 2, 1, "bf16", seed=0, init_std=1e-3)
    cg = tg.tg_create(3, res, 1, 3, "bf16", seed=1, init_std=1e-3)
    batch = tg.tg_batch_create(3, res, R * S)
    dgr = torch.zeros(dg.n_coefs, device="cuda")
    cgr = torch.zeros(cg.n_coefs, device="cuda")
    loss = torch.zeros(1, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        idx = torch.randint(0, o_tr.shape[0], (R,), device="cuda", generator=gen)
        tg.tg_render_rays(dg, cg, o_tr[idx].contiguous(), d_tr[idx].contiguous(), S=S, seed=k,
                          target=gt_tr[idx].contiguous(), batch=batch, density_grad=dgr, color_grad=cgr, loss_sum=loss)
        tg.tg_adam_step(dg, dgr, lr=lr[0], step=k + 1)
        tg.tg_adam_step(cg, cgr, lr=lr[1], step=k + 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sq = 0.0
    for i in range(0, o_te.shape[0], 1 << 16):
        rgb = tg.tg_render_rays(dg, cg, o_te[i:i + (1 << 16)].contiguous(), d_te[i:i + (1 << 16)].contiguous(), S=S,
                                seed=1 << 40)
        sq += float(((rgb - gt_te[i:i + (1 << 16)]) ** 2).sum())
    psnr = -10 * math.log10(sq / (o_te.shape[0] * 3))
    return {"workload": f"ray-march fit of 64 Gaussian blobs: {res}^3 BF16 density o2 + colour o1, {R} rays x {S} "
                        f"samples, {steps} steps, Adam lr {lr}; 90 training / 10 held-out cameras at {side}x{side} "
                        f"(targets by 1024-sample midpoint quadrature in {str(gdt).split('.')[-1]})",
            "ms_per_step": ms, "held_out_psnr_db": psnr}


def bench_serving(n_jobs=40, rate=20.0, budget=64 << 30, seed=5, slots=32, deadline_s=120.0):
    """Poisson arrivals of fit jobs (70 %) and queries (30 %) through the server, against the same trace run
    one job at a time with FP32 storage."""
    import math

    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    rng = np.random.default_rng(seed)
    t, trace = 0.0, []
    for k in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        if rng.random() < 0.7 or not any(e["kind"] == "fit" for e in trace):
            trace.append({"kind": "fit", "t": t, "res": int(rng.choice([32, 64, 128, 256])),
                          "order": int(rng.choice([1, 2])), "dtype": str(rng.choice(["bf16", "f32"])),
                          "shape": W.union_shape(100 + k), "seed": 100 + k})
        else:
            n = int(math.exp(rng.uniform(math.log(1e4), math.log(1e6))))
            fits = [i for i, e in enumerate(trace) if e["kind"] == "fit"]
            trace.append({"kind": "query", "t": t, "n": n, "of": int(rng.choice(fits)),
                          "pts": torch.rand((n, 3), device="cuda")})

    def run(force_fp32, max_running, smallest_first=False, lazy=False):
        srv = tg.Server(budget_bytes=budget, max_running=max_running, smallest_first=smallest_first)
        ids, outs = {}, []
        t0 = srv.time()
        i = 0
        while True:
            now = srv.time() - t0
            while i < len(trace) and trace[i]["t"] <= now:
                e = trace[i]
                if e["kind"] == "fit":
                    sh = e["shape"]
                    ids[i] = srv.fit_job(sh.spheres, sh.boxes, sh.area_cdf(), res=e["res"], order=e["order"],
                                         dtype="f32" if force_fp32 else e["dtype"], seed=e["seed"],
                                         points_per_step=1 << 16, eval_points=1 << 14, eval_every=10,
                                         max_steps=1000, tol=2e-3, lr=5e-3, lambda_eik=0.0, lazy_adam=lazy)
                else:
                    out = torch.empty(e["n"], device="cuda")
                    outs.append(out)
                    ids[i] = srv.query_job(ids[e["of"]], e["pts"], out)
                i += 1
            pending = srv.step()
            if i == len(trace) and pending == 0:
                break
            if srv.time() - t0 > deadline_s:
                srv.close()
                raise RuntimeError(f"serving trace did not drain within {deadline_s} s")
        makespan = srv.time() - t0
        lat = {"fit": [], "query": []}
        pts, errs, steps = 0, [], []
        for k, jid in ids.items():
            r = srv.poll(jid)
            lat[trace[k]["kind"]].append(r["t_done"] - (t0 + trace[k]["t"]))
            pts += r["points"]
            if trace[k]["kind"] == "fit":
                errs.append(r["error"])
                steps.append(r["steps"])
        srv.close()
        pct = lambda a, q: float(np.percentile(a, q)) if a else None
        return {"fit_p50_s": pct(lat["fit"], 50), "fit_p99_s": pct(lat["fit"], 99),
                "query_p50_s": pct(lat["query"], 50), "query_p99_s": pct(lat["query"], 99),
                "makespan_s": makespan, "Mpts_per_s": pts / makespan / 1e6,
                "fit_steps_total": int(sum(steps)), "fit_reached_tol": int(sum(e < 2e-3 for e in errs)),
                "fit_final_error_median": pct(errs, 50)}
    served = run(False, slots, smallest_first=True)
    served_lazy = run(False, slots, smallest_first=True, lazy=True)
    alone = run(True, 1)
    return {"workload": f"{n_jobs} Poisson arrivals at {rate}/s: 70% SDF fit jobs (res 32/64/128/256, order 1/2, "
                        "BF16/FP32, 2^16 points/step, L1, until mean |SDF error| < 2e-3 or 1000 steps), 30% queries "
                        "of 1e4-1e6 points; 64 GB admission budget",
            "served": {"slots": slots, "admission": "smallest job first", **served},
            "served_lazy_adam": {"slots": slots, "admission": "smallest job first", **served_lazy},
            "one_at_a_time_fp32": alone}


def bench_burst(n_jobs=24, steps=200, budget=64 << 30, deadline_s=120.0):
    """Saturation throughput: n_jobs SDF fit jobs submitted at once (res 64 / 96, order 1 / 2, BF16 / FP32,
    2^16 points per step, a fixed number of steps), run three ways: advanced in groups (one launch per stage per
    group of equal order and dtype), each job alone on its own stream (TG_FIT_DETERMINISTIC), and one job at a
    time."""
    import paper_2402_14415_gb300 as tg
    import workloads as W
    mix = [(64 + 32 * (k % 2), 1 + (k // 2) % 2, ("bf16", "f32")[(k // 4) % 2]) for k in range(n_jobs)]

    def run(max_running, deterministic):
        srv = tg.Server(budget_bytes=budget, max_running=max_running)
        t0 = srv.time()
        ids = []
        for k, (res, order, dtype) in enumerate(mix):
            sh = W.union_shape(300 + k)
            ids.append(srv.fit_job(sh.spheres, sh.boxes, sh.area_cdf(), res=res, order=order, dtype=dtype,
                                   seed=300 + k, points_per_step=1 << 16, eval_points=1 << 14, eval_every=10,
                                   max_steps=steps, tol=0.0, lr=5e-3, deterministic=deterministic))
        srv.run_until_idle(timeout_s=deadline_s)
        makespan = srv.time() - t0
        rs = [srv.poll(j) for j in ids]
        srv.close()
        assert all(r["state"] == "done" and r["steps"] == steps for r in rs), rs
        pts = sum(r["points"] for r in rs)
        return {"makespan_s": makespan, "Mpts_per_s": pts / makespan / 1e6}
    grouped = run(n_jobs, False)
    own = run(n_jobs, True)
    serial = run(1, False)
    return {"workload": f"{n_jobs} SDF fit jobs submitted at once (res 64/96, order 1/2, BF16/FP32, 2^16 points/step, "
                        f"L1, {steps} steps each)",
            "grouped": grouped, "own_stream_each": own, "one_at_a_time": serial}


def profile_once():
    """One untimed pass of every kernel of the step (value and spatial-gradient variants)."""
    import torch

    import paper_2402_14415_gb300 as tg
    tg.load()
    n = int(sys.argv[sys.argv.index("--profile-points") + 1]) if "--profile-points" in sys.argv else N_POINTS
    g = tg.tg_create(3, RES, ORDER, C, "f32", seed=0, init_std=1.0)
    gen = torch.Generator(device="cuda").manual_seed(0)
    P = torch.rand((n, 3), device="cuda", generator=gen)
    U = torch.randn((n, 1), device="cuda", generator=gen)
    UG = torch.randn((n, 1, 3), device="cuda", generator=gen)
    out = torch.empty((n, 1), device="cuda")
    gx = torch.empty((n, 1, 3), device="cuda")
    grad = torch.zeros(g.n_coefs, device="cuda")
    batch = tg.tg_batch_create(3, RES, n)
    # the bench step's launches, in its order: bin, forward, backward (binned order), then the input-order pair
    tg.tg_batch_bin(batch, P)
    tg.tg_query_binned(g, batch, out=out, binned_order=True)
    tg.tg_query_backward_binned(g, batch, U, grad, binned_order=True)
    tg.tg_query_binned(g, batch, out=out)
    tg.tg_query_backward_binned(g, batch, U, grad)
    # spatial-gradient variants of the two brick kernels
    tg.tg_query_binned(g, batch, out=out, grad_x=gx)
    tg.tg_query_backward_binned(g, batch, U, grad, dL_dgradx=UG)
    # the point-parallel pair on the same unsorted points (no binning; warp-aggregated FP32 reductions):
    # calls captured into a CUDA graph never bin, so the pair is captured and replayed once
    pair = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pair):
        tg.tg_query(g, P, out=out)
        tg.tg_query_backward(g, P, U, grad)
    pair.replay()
    tg.tg_adam_step(g, grad, lr=1e-3, step=1)
    tg.tg_tv_step(g, 2e-5, grad)              # the total variation term of the paper's fit objective
    torch.cuda.synchronize()
    print("profile pass done, timeouts:", tg.tg_batch_timeouts(batch))


def profile_fit(dtype="f32"):
    """Three SDF fit steps (256^3 order 2, 2^20 points, L1 + 0.1 eikonal, Adam) for ncu: two warm-up steps, then
    the profiled one (capture with -s <launches of two steps>)."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    shape = W.union_shape(0)
    dsh = tg.DeviceShape(shape.spheres, shape.boxes, shape.area_cdf())
    n = 1 << 20
    g = tg.tg_create(3, RES, ORDER, 1, dtype, seed=0, init_std=1e-3)
    batch = tg.tg_batch_create(3, RES, n)
    grad = torch.zeros(g.n_coefs, device="cuda")
    loss = torch.zeros(2, device="cuda")
    for k in range(3):
        tg.tg_sdf_step(g, batch, dsh, grad, loss, n=n, seed=1, step=k, lambda_eik=0.1)
        tg.tg_adam_step(g, grad, lr=5e-3, step=k + 1)
    torch.cuda.synchronize()
    print("profile fit pass done, timeouts:", tg.tg_batch_timeouts(batch))


def profile_render():
    """Three ray-march training steps (8192 rays x 256 samples, 160^3 BF16 density o2 + colour o1 x 3, both Adam
    steps) for ncu: two warm-up steps, then the profiled one."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    res, R, S = 160, 8192, 256
    dg = tg.tg_create(3, res, 2, 1, "bf16", seed=0, init_std=0.5)
    cg = tg.tg_create(3, res, 1, 3, "bf16", seed=1, init_std=0.5)
    o, d = W.random_rays(7, R, radius=1.5, spread=0.35)
    ro, rd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    target = torch.rand((R, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    batch = tg.tg_batch_create(3, res, R * S)
    dgr = torch.zeros(dg.n_coefs, device="cuda")
    cgr = torch.zeros(cg.n_coefs, device="cuda")
    loss = torch.zeros(1, device="cuda")
    for k in range(3):
        tg.tg_render_rays(dg, cg, ro, rd, S=S, seed=k, target=target, batch=batch, density_grad=dgr,
                          color_grad=cgr, loss_sum=loss)
        tg.tg_adam_step(dg, dgr, lr=0.1, step=k + 1)
        tg.tg_adam_step(cg, cgr, lr=0.03, step=k + 1)
    torch.cuda.synchronize()
    print("profile render pass done")


def profile_serve(steps=3):
    """Six SDF fit jobs of one group (order 2, FP32, res 64 / 96, 2^16 points per step) through the server for a
    few steps, for ncu captures of the batched step's kernels."""
    import torch

    import paper_2402_14415_gb300 as tg
    import workloads as W
    srv = tg.Server(budget_bytes=16 << 30, max_running=16)
    ids = []
    for k in range(6):
        sh = W.union_shape(300 + k)
        ids.append(srv.fit_job(sh.spheres, sh.boxes, sh.area_cdf(), res=64 + 32 * (k % 2), order=2, dtype="f32",
                               seed=300 + k, points_per_step=1 << 16, eval_points=1 << 14, eval_every=10,
                               max_steps=steps, tol=0.0, lr=5e-3))
    srv.run_until_idle(timeout_s=60)
    torch.cuda.synchronize()
    print("profile serve pass done:", [srv.poll(j)["steps"] for j in ids])
    srv.close()


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# full-size launches (binned order) captured by `ncu ... python bench.py --profile`
# (profiles/query_step_256_o2_2e24_full.md); None once the kernel has changed since.
TRAFFIC = {"forward": 0.939709696e9 + 0.064290304e9, "backward": 1.006815e9 + 0.612811264e9, "bin": None}
KERNEL_NAMES = {"bin": "bin_* (5 kernels, tg_batch_bin)", "forward": "brick_fwd_kernel (tg_query_binned)",
                "backward": "brick_bwd_fast_kernel (tg_query_backward_binned)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the fit / query-only / render lines")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving trace (about 25 s)")
    ap.add_argument("--profile", action="store_true",
                    help="run each kernel of the step once, untimed (for ncu captures)")
    ap.add_argument("--profile-points", type=int, default=N_POINTS)
    ap.add_argument("--profile-fit", choices=["f32", "bf16", "f16"], default=None,
                    help="run three SDF fit steps at 256^3 order 2 in this storage dtype (for ncu captures)")
    ap.add_argument("--profile-render", action="store_true",
                    help="run three ray-march training steps at 160^3 (for ncu captures)")
    ap.add_argument("--profile-serve", action="store_true",
                    help="run six fit jobs of one group through the server for three steps (for ncu captures)")
    ap.add_argument("--cpu-baseline-from", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-timings", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_baseline_from:
        return run_cpu_baseline(args.cpu_baseline_from, args.steps, args.warmup)
    if args.oracle_timings:
        return run_oracle_timings()
    args.warmup = max(args.warmup, 3)
    if args.profile:
        return profile_once()
    if args.profile_fit:
        return profile_fit(args.profile_fit)
    if args.profile_render:
        return profile_render()
    if args.profile_serve:
        return profile_serve()
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
