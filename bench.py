"""Benchmark: voxel-transducer pairs/s of the closed-form operator A and its
adjoint A^T on the c2 system (128^3 voxels at 0.1 mm, 128-element cylindrically
focused array rotated over 180 angles = 23,040 positions, 1024 samples at
40 MHz, U = 11, dl = U, blob phantom).

One step is one pass of the whole path, s = A x then z = A^T s, over one batch
of the positions (``--batch-angles`` rotation angles x 128 elements); steps
walk through the angles.  value = pairs processed / device time, where one A
or one A^T of a batch processes N x K_batch pairs.  Inputs are resident in HBM
for ``value``; ``e2e`` repeats the step through the C ABI with x in pinned
host memory and z copied back.  The L2 is flushed (a 256 MB write) between
timed steps.

Under torchrun each rank takes its own batches (weak scaling, no data-path
collective); rank 0 prints one JSON line.  ``--impl reference`` times the FP64
CPU oracle on the host cores instead, on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_29253_gb300 import workloads as W  # noqa: E402

METRIC = "voxel-transducer pairs/s for A and A^T (closed form)"
N_ANGLES = 180
# FP32 floating-point operations of one quadrant-edge area evaluation of the
# cylinder path: 2 per FFMA, 1 per FADD / FMUL, 4 per FFMA2, 2 per FADD2 /
# FMUL2 (MUFU operations not counted), from the instruction counters of one
# adj_geom_kernel launch on the c2 geometry (64^3 grid, 128 positions,
# 1.450e9 evaluations): 165.5 (166.4 for the forward kernel).
FLOPS_PER_QUAD_EVAL = 166
# DRAM read + write bytes of one adj_geom_kernel launch of the default
# workload (128^3 x 512 positions), one-pass ncu capture of this kernel
# version (29.38 MB read + 16.85 MB written).
ADJ_TRAFFIC_BYTES = 41.94e6  # adj_geom_kernel DRAM read + write per launch (ncu, full c2 batch)
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch-angles", type=int, default=4)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-voxels", type=int, default=1024)
    p.add_argument("--grid", type=int, default=128,
                   help="voxels per axis over the same 12.8 mm cube (128 = the c2 grid; smaller for profiling)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the convolution, batched-FISTA and c3 comparisons after the main timing")
    p.add_argument("--extras", default="conv,fista,c3,c5,exp1",
                   help="comma-separated extra lines to run: conv, fista, c3, c5, exp1")
    p.add_argument("--fista-problems", type=int, default=8)
    p.add_argument("--fista-iters", type=int, default=10)
    p.add_argument("--c3-positions", type=int, default=128)
    p.add_argument("--c5-positions", type=int, default=16)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def batches(args, rank, world, total_steps):
    """Angle batches for this rank: rank r takes batches r, r + world, ..."""
    from paper_2609_29253_gb300 import shard

    return shard.angle_batches(N_ANGLES, args.batch_angles, rank, world, total_steps)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def physical_gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local < len(ids) and ids[local].isdigit():
            return int(ids[local])
    return local


def oracle_sample(w, taps, n_vox, seed=0):
    """Time the FP64 oracle on A and A^T restricted to a seeded voxel subset."""
    import oracle

    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.N, size=min(n_vox, w.N), replace=False)).astype(np.int64)
    xs = w.x[idx].astype(np.float64)
    t0 = time.perf_counter()
    s, _ = oracle.forward(w, taps, xs, vox_idx=idx)
    oracle.adjoint(w, taps, s, vox_idx=idx)
    dt = time.perf_counter() - t0
    pairs = 2 * idx.size * w.K
    return pairs / dt, dt, idx.size, oracle.num_threads()


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    ang = batches(args, 0, 1, 1)[0]
    w = c2w(args, ang)
    taps = oracle.taps_for(w)
    for _ in range(args.warmup):
        oracle_sample(w, taps, 64)
    vals, times = [], []
    for i in range(args.steps):
        v, dt, nv, cores = oracle_sample(w, taps, args.cpu_sample_voxels, seed=i)
        vals.append(v)
        times.append(dt)
    value = statistics.mean(vals)
    sample = (f"{args.cpu_sample_voxels} seeded voxels x {w.K} positions ({args.batch_angles} angles), "
              f"A then A^T, FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, w),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def c2w(args, angles, with_x=True):
    """The c2 workload on a --grid^3 grid over the same 12.8 mm cube."""
    w = W.c2(angles=angles, with_x=False)
    if args.grid != 128:
        n = (args.grid,) * 3
        pitch = 12.8e-3 / args.grid
        w = w.with_(n=n, pitch=pitch, origin=W.centred_origin(n, pitch))
    if with_x:
        w = w.with_(x=W.blob_phantom(w.n, w.origin, w.pitch, 200, 0))
    return w


def cuda_ms(fn, reps=3, warm=1):
    """Mean device time (ms) of fn() on the current stream, CUDA events."""
    import torch

    for _ in range(warm):
        fn()
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def rel_l2(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / b.norm())


def conv_compare(api, plan, w, taps, x, dev):
    """The temporal convolution of A and of A^T on one batch: FP64-accumulated
    CUDA-core kernels of the plain plan against the tcgen05 BF16 split
    Toeplitz kernels of a PAT_FLAG_CONV_TC plan (same f and s)."""
    tc = api.Plan(w, taps=taps, conv_tc=True, device=dev)
    f = plan.forward_geometric(x)
    s_plain = plan.conv_forward(f)
    s_tc = tc.conv_forward(f)
    v_plain = plan.conv_adjoint(s_plain)
    v_tc = tc.conv_adjoint(s_plain)
    out = {"workload": f"the main batch: K {w.K} rows, U L {w.UL} fine bins -> L {w.L}, {w.T + w.U - 1} taps",
           "forward_ms": {"fp64_cuda_cores": cuda_ms(lambda: plan.conv_forward(f)),
                          "tcgen05_bf16x3": cuda_ms(lambda: tc.conv_forward(f))},
           "adjoint_ms": {"fp64_cuda_cores": cuda_ms(lambda: plan.conv_adjoint(s_plain)),
                          "tcgen05_bf16x3": cuda_ms(lambda: tc.conv_adjoint(s_plain))},
           "rel_l2_tc_vs_fp64": {"forward": rel_l2(s_tc, s_plain), "adjoint": rel_l2(v_tc, v_plain)},
           "step_ms_with_tc": cuda_ms(lambda: (tc.forward(x), tc.adjoint(s_plain)), reps=1)}
    out["tc_error"] = api._lib.pat_plan_get_info(tc.handle)["tc_error"]
    out["all_c2_rows"] = conv_all_rows(api, taps, dev)
    return out


def conv_all_rows(api, taps, dev):
    """The same convolutions over all 23,040 c2 positions in one launch (a
    plan of the c2 time axis and array on an 8^3 grid; the convolution does
    not depend on the grid), seeded random f, as the tensor cores see a whole
    c2 application: 360 x 8 output tiles instead of the batch's 8 x 8.
    FLOP/s counts the tensor-core work as issued (three BF16 products per
    Toeplitz tile, ~4x the banded multiply-adds)."""
    import torch

    n = (8, 8, 8)
    w = W.c2(with_x=False).with_(n=n, origin=W.centred_origin(n, 0.1e-3))
    plan = api.Plan(w, taps=taps, device=dev)
    tc = api.Plan(w, taps=taps, conv_tc=True, device=dev)
    g = torch.Generator(device=dev).manual_seed(7)
    f = torch.randn((w.K, w.UL), device=dev, generator=g)
    s_plain = plan.conv_forward(f)
    s_tc = tc.conv_forward(f)
    v_plain = plan.conv_adjoint(s_plain)
    v_tc = tc.conv_adjoint(s_plain)
    t_tc = cuda_ms(lambda: tc.conv_forward(f), reps=3)
    nw = w.T + w.U - 1
    kw = -(-(127 * w.U + nw) // 64) * 64  # Toeplitz contraction length per 128-sample tile
    flops = 3 * 2 * 128 * 64 * kw * (-(-w.L // 128)) * (-(-w.K // 64))
    out = {"workload": f"all c2 positions: K {w.K} rows, U L {w.UL} -> L {w.L}, {nw} taps, random f",
           "forward_ms": {"fp64_cuda_cores": cuda_ms(lambda: plan.conv_forward(f), reps=3), "tcgen05_bf16x3": t_tc},
           "adjoint_ms": {"fp64_cuda_cores": cuda_ms(lambda: plan.conv_adjoint(s_plain), reps=3),
                          "tcgen05_bf16x3": cuda_ms(lambda: tc.conv_adjoint(s_plain), reps=3)},
           "rel_l2_tc_vs_fp64": {"forward": rel_l2(s_tc, s_plain), "adjoint": rel_l2(v_tc, v_plain)},
           "tcgen05_forward_tflops": flops / (t_tc * 1e-3) / 1e12,
           "tc_error": api._lib.pat_plan_get_info(tc.handle)["tc_error"]}
    return out


def fista_compare(api, dev, n_prob, iters):
    """Batched reconstruction (c4-shaped, reduced sizes): n_prob problems of
    uneven grids, position counts and lengths, s = A x + 1 % noise.  Time per
    iteration of all problems: one pat_recon per problem enqueued on the
    legacy stream (plain FP32 operator, no graph), against pat_recon_batch
    (one CUDA graph per iteration, a branch per problem) with the plain and
    with the tensor-core-convolution plans."""
    import torch

    ws = [W.c4_problem(p, n_range=(24, 40), k_range=(128, 384)) for p in range(n_prob)]
    plans = [api.Plan(w, device=dev) for w in ws]
    plans_tc = [api.Plan(w, taps=p.taps, conv_tc=True, device=dev) for w, p in zip(ws, plans)]
    g = torch.Generator(device=dev).manual_seed(1234)
    s_list, lam, steps = [], [], []
    for w, p in zip(ws, plans):
        s0 = p.forward(torch.from_numpy(w.x).to(dev))
        s = s0 + 0.01 * s0.abs().max() * torch.randn(s0.shape, device=dev, generator=g)
        s_list.append(s.contiguous())
        z = p.adjoint(s.contiguous())
        lam.append(float(1e-3 * z.abs().max()))
        v = torch.ones(w.N, device=dev)
        for _ in range(20):
            v = p.adjoint(p.forward((v.double() / v.double().norm()).float()))
        steps.append(float(1.0 / (1.05 * (float(v.double().norm()) + lam[-1]))))
        if not (math.isfinite(lam[-1]) and math.isfinite(steps[-1])):
            raise RuntimeError(f"{w.name}: lambda {lam[-1]}, step {steps[-1]}, |s0| {float(s0.abs().max())}, "
                               f"finite s0 {bool(torch.isfinite(s0).all())}, finite z {bool(torch.isfinite(z).all())}, "
                               f"finite v {bool(torch.isfinite(v).all())}, |x| {float(np.abs(w.x).max())}")
    x0 = [torch.zeros(p.N, device=dev) for p in plans]

    def seq():
        return [p.recon(s, x, iters=iters, lambda_R=l, step=t) for p, s, x, l, t in zip(plans, s_list, x0, lam, steps)]

    side = torch.cuda.Stream(device=dev)

    def batched(ps):
        with torch.cuda.stream(side):
            r = api.recon_batch(ps, s_list, x0, iters=iters, lambdas=lam, steps=steps)
        side.synchronize()
        return r

    def wall(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / iters, r

    t_seq, r_seq = wall(seq)
    t_b, r_b = wall(lambda: batched(plans))
    t_tc, r_tc = wall(lambda: batched(plans_tc))
    d_b = max(rel_l2(a, b) for a, b in zip(r_b, r_seq))
    d_tc = max(rel_l2(a, b) for a, b in zip(r_tc, r_seq))
    pairs = sum(w.N * w.K for w in ws)
    return {"workload": "; ".join(w.name for w in ws), "problems": n_prob, "iterations": iters,
            "pairs_per_iteration": 2 * pairs,
            "ms_per_iteration": {"plain_fp32_sequential": t_seq, "graph_batched": t_b,
                                 "graph_batched_tcgen05_conv": t_tc},
            "speedup_vs_plain": {"graph_batched": t_seq / t_b, "graph_batched_tcgen05_conv": t_seq / t_tc},
            "max_rel_l2_vs_plain": {"graph_batched": d_b, "graph_batched_tcgen05_conv": d_tc},
            "timing": "wall clock per iteration over all problems, host to device completion, step sizes fixed"}


def c3_line(api, dev, n_pos):
    """The precision-split system (c3): 256^3 voxels at 0.08 mm, planar 3x3 mm
    elements on a 40 mm hemisphere, L 2048, tcgen05 BF16 split convolution;
    one batch of the first n_pos positions."""
    import torch

    w = W.c3(with_x=False, rotations=1)
    w = w.with_tx(w.tx[:n_pos])
    w = w.with_(x=W.blob_phantom(w.n, w.origin, w.pitch, 200, 0))
    plan = api.Plan(w, conv_tc=True, device=dev)
    x = torch.from_numpy(w.x).to(dev)
    s = plan.forward(x)
    t_f = cuda_ms(lambda: plan.forward(x, out=s), reps=2)
    z = torch.empty(w.N, device=dev)
    t_a = cuda_ms(lambda: plan.adjoint(s, out=z), reps=2)
    pairs = w.N * w.K
    return {"workload": f"c3: 256^3 @ 0.08 mm, first {w.K} of 5,120 planar 3x3 mm positions, L 2048 @ 40 MHz, "
                        f"U 11, dl 11, tcgen05 BF16 split convolution",
            "forward_pairs_per_s": pairs / (t_f * 1e-3), "adjoint_pairs_per_s": pairs / (t_a * 1e-3),
            "ms": {"forward": t_f, "adjoint": t_a}, "mean_bins_per_pair": plan.info["pair_bins"] / pairs,
            "tc_error": api._lib.pat_plan_get_info(plan.handle)["tc_error"]}


def c5_line(api, dev, n_pos):
    """The full-scale system (c5): 512^3 voxels at 0.05 mm (134M), the c2
    array rotated over 128 angles, L 4096 at 50 MHz; the first n_pos
    positions of one angle, closed form (surface method) against the point
    method with 16 x 16 points per element (Alg. 2) on a quarter of them."""
    import torch

    w = W.c5(with_x=False, n_angles=128)
    w = w.with_tx(w.tx[:n_pos])
    w = w.with_(x=W.blob_phantom(w.n, w.origin, w.pitch, 200, 0))
    x = torch.from_numpy(w.x).to(dev)
    plan = api.Plan(w, device=dev)
    s = plan.forward(x)
    t_f = cuda_ms(lambda: plan.forward(x, out=s), reps=1)
    z = torch.empty(w.N, device=dev)
    t_a = cuda_ms(lambda: plan.adjoint(s, out=z), reps=1)
    n_pt = max(1, n_pos // 4)
    wp = w.with_tx(w.tx[:n_pt]).with_(method=W.METHOD_POINT, q1=16, q2=16)
    pplan = api.Plan(wp, taps=plan.taps, device=dev)
    sp = pplan.forward(x)
    t_pf = cuda_ms(lambda: pplan.forward(x, out=sp), reps=1)
    pairs = w.N * w.K
    return {"workload": f"c5: 512^3 @ 0.05 mm, first {w.K} of 16,384 cylindrical positions, L 4096 @ 50 MHz, U 11, "
                        f"dl 11; point method 16 x 16 on the first {n_pt}",
            "closed_form": {"forward_pairs_per_s": pairs / (t_f * 1e-3), "adjoint_pairs_per_s": pairs / (t_a * 1e-3),
                            "ms": {"forward": t_f, "adjoint": t_a}},
            "point_16x16": {"forward_pairs_per_s": w.N * n_pt / (t_pf * 1e-3), "ms": {"forward": t_pf},
                            "point_evaluations_per_s": w.N * n_pt * 256 / (t_pf * 1e-3)},
            "mean_bins_per_pair": plan.info["pair_bins"] / pairs}


def exp1_line(api, dev):
    """The paper's Experiment 1 system (fine grid: 98,415 voxels x 215
    cylindrical elements, 2688 samples at 62.5 MHz): one A plus one A^T with
    the exact areas, the paper's lookup tables (1000 x 1000), the trapezoidal
    approximation, Piecewise-Planes with 30 planes and the point method with
    25 x 25 points (Q = 625), each with its
    distance to the exact A x.  The paper's own per-iteration times (A100,
    FP64, one A and one A^T assumed per iteration) are context, not targets."""
    import torch

    w = W.exp1("fine")
    x = torch.from_numpy(w.x).to(dev)
    taps = api.system_taps(w, dev)
    ops = {"exact": api.Plan(w, taps=taps, device=dev),
           "lut_1000x1000": api.Plan(w.with_(method=W.METHOD_LUT, q1=1000, q2=1000), taps=taps, device=dev),
           "trapezoidal": api.Plan(w.with_(method=W.METHOD_TRAPEZOID), taps=taps, device=dev),
           "piecewise_planes_30": api.Plan(w, taps=taps, piecewise_planes=30, device=dev),
           "point_625": api.Plan(w.with_(method=W.METHOD_POINT, q1=25, q2=25), taps=taps, device=dev)}
    s_ex = ops["exact"].forward(x)
    out = {"workload": w.name, "pairs_per_application": w.N * w.K}
    for name, p in ops.items():
        s = p.forward(x)
        z = torch.empty(w.N, device=dev)
        t = cuda_ms(lambda: (p.forward(x, out=s), p.adjoint(s, out=z)), reps=3)
        out[name] = {"ms_A_plus_AT": t, "rel_l2_vs_exact": rel_l2(s, s_ex),
                     "quad_evals_per_application": p.info["quad_evals"]}
    out["paper_a100_fp64_ms_per_iteration"] = {"exact": 2021, "lut": 192, "trapezoidal": 145, "point_625": 533,
                                               "piecewise_planes_30": 1256}
    return out


def config(args, w):
    grid = "" if args.grid == 128 else f" [reduced grid {args.grid}^3 for profiling]"
    return {"workload": "c2: 128^3 voxels @ 0.1 mm, 128-element cylindrical array (R 20 mm, 10 mm elevation, "
                        "0.3 mm pitch) x 180 angles = 23,040 positions, L 1024 @ 40 MHz, U 11, dl 11, closed form" + grid,
            "batch": f"{args.batch_angles} angles x 128 elements = {128 * args.batch_angles} positions per step",
            "N": w.N, "K_batch": w.K, "L": w.L, "U": w.U, "dl": w.dl,
            "l2": "flushed between timed steps (256 MB write)", "parallelism": f"transducer batches over {args.gpus} GPU(s)"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2609_29253_gb300 import _lib, api

    total = args.warmup + args.steps
    angle_sets = batches(args, rank, world, total)
    w0 = c2w(args, angle_sets[0])
    x = torch.from_numpy(w0.x).to(dev)
    taps = api.system_taps(w0, dev)
    plans = []
    for ang in angle_sets:
        plans.append(api.Plan(c2w(args, ang, with_x=False).with_(x=w0.x), taps=taps, device=dev))
    K = plans[0].K
    s = torch.empty((K, w0.L), dtype=torch.float32, device=dev)
    z = torch.empty(w0.N, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(p):
        p.forward(x, out=s)
        p.adjoint(s, out=z)

    for i in range(args.warmup):
        step(plans[i])
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(physical_gpu_index(local))
    if rank == 0:
        clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        p = plans[args.warmup + i]
        e0, e1, e2 = ev[i]
        e0.record(stream)
        p.forward(x, out=s)
        e1.record(stream)
        p.adjoint(s, out=z)
        e2.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop() if rank == 0 else None
    t_fwd = [a.elapsed_time(b) for a, b, _ in ev]
    t_adj = [b.elapsed_time(c) for _, b, c in ev]
    t_step = sum(t_fwd) + sum(t_adj)  # ms, device time of the K steps
    if world > 1:
        tt = torch.tensor([t_step], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step = float(tt)
    pairs_step = 2 * w0.N * K
    value = pairs_step * args.steps * world / (t_step * 1e-3)

    # per-launch work of the dominant kernels (scan counts of the plans)
    qe = statistics.mean(p.info["quad_evals"] for p in plans[args.warmup:])
    ae = statistics.mean(p.info["area_evals"] for p in plans[args.warmup:])
    mean_fwd = statistics.mean(t_fwd) * 1e-3
    mean_adj = statistics.mean(t_adj) * 1e-3
    flops = qe * FLOPS_PER_QUAD_EVAL
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the clock seen
    ach = flops / mean_adj / 1e12
    # the same denominators measured by the library's own dependent-chain kernels (after the timed region)
    mp = _lib.pat_measure_peaks()
    measured = {"fp32_ffma_tflops": mp["fp32_ffma_flops"] / 1e12, "fp32_ffma2_tflops": mp["fp32_ffma2_flops"] / 1e12,
                "fp64_dfma_tflops": mp["fp64_dfma_flops"] / 1e12, "sfu_rsqrt_tops": mp["sfu_rsqrt_ops"] / 1e12,
                "frac_of_measured_ffma": ach / (mp["fp32_ffma_flops"] / 1e12)}

    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(w0.x).pin_memory()
        zh = torch.empty(w0.N, dtype=torch.float32).pin_memory()
        xd = torch.empty_like(x)
        p = plans[args.warmup]
        for _ in range(1):
            xd.copy_(xh, non_blocking=True)
            p.forward(xd, out=s)
            p.adjoint(s, out=z)
            zh.copy_(z, non_blocking=True)
        torch.cuda.synchronize(dev)
        ts = []
        for i in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            xd.copy_(xh, non_blocking=True)
            plans[args.warmup + i].forward(xd, out=s)
            plans[args.warmup + i].adjoint(s, out=z)
            zh.copy_(z, non_blocking=True)
            torch.cuda.synchronize(dev)
            ts.append(time.perf_counter() - t0)
        e2e = {"value": pairs_step * args.steps / sum(ts), "unit": "pairs/s", "h2d_bytes_per_step": 4 * w0.N,
               "d2h_bytes_per_step": 4 * w0.N}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        wcpu = c2w(args, angle_sets[args.warmup], with_x=False).with_(x=w0.x)
        v, dt, nv, cores = oracle_sample(wcpu, taps, args.cpu_sample_voxels)
        cpu = {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{nv} seeded voxels x {wcpu.K} positions, A then A^T, FP64 ({dt:.1f} s)"}

    extras = {}
    want = set(e.strip() for e in args.extras.split(",") if e.strip())
    if rank == 0 and not args.no_extras:
        if "conv" in want:
            extras["conv_tcgen05"] = conv_compare(api, plans[args.warmup],
                                                  c2w(args, angle_sets[args.warmup], with_x=False).with_(x=w0.x), taps,
                                                  x, dev)
        if "fista" in want:
            extras["fista_batched"] = fista_compare(api, dev, args.fista_problems, args.fista_iters)
        if "c3" in want:
            extras["c3_precision_split"] = c3_line(api, dev, args.c3_positions)
        if "c5" in want and args.c5_positions > 0:
            extras["c5_full_scale_subset"] = c5_line(api, dev, args.c5_positions)
        if "exp1" in want:
            extras["exp1_operators"] = exp1_line(api, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config(args, w0),
                "forward_pairs_per_s": w0.N * K / mean_fwd, "adjoint_pairs_per_s": w0.N * K / mean_adj,
                "area_evals_per_s": ae / mean_adj, "mean_bins_per_pair": plans[args.warmup].info["pair_bins"] / (w0.N * K),
                "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                             "traffic": ADJ_TRAFFIC_BYTES if (args.grid == 128 and args.batch_angles == 4) else None,
                             "kernel": "adj_geom_kernel", "flops_per_unit": FLOPS_PER_QUAD_EVAL,
                             "units_per_launch": qe, "unit_name": "quadrant-edge area evaluation",
                             "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x median SM clock under load",
                             "measured_peaks": measured},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 4 * args.steps,
                "clocks": clk, "wall_s_timed": t_wall}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
