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
# adj_geom_kernel launch of this kernel version on the c2 geometry at the
# bench's grid (128^3 voxels, one angle of 128 positions, 1.1629e10
# evaluations): 139.5 (143.0 on a 64^3 grid).
FLOPS_PER_QUAD_EVAL = 139.5
# Warp instructions issued per evaluation by the same launch (smsp__inst_executed:
# 7.639e10 for 1.1629e10 evaluations): the kernel is bound by instruction issue,
# so the line also reports the fraction of the SMs' issue slots it fills
# (152 SMs x 4 schedulers x 1 warp instruction per cycle).
WARP_INSTS_PER_QUAD_EVAL = 6.569
ISSUE_PER_SM_PER_CYCLE = 4
# DRAM read + write bytes of one adj_geom_kernel launch of the default
# workload (128^3 x 512 positions), one-pass ncu capture of this kernel
# version (32.61 MB read + 44.06 MB written).
ADJ_TRAFFIC_BYTES = 76.67e6  # adj_geom_kernel DRAM read + write per launch (ncu, full c2 batch)
# FP32 flops executed per planar quadrant-edge evaluation by adj_geom_kernel on
# the c3 line's 128 positions (same counters): 87.1 (86.0 for the forward).
FLOPS_PER_PLANE_EVAL = 87.1
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
    p.add_argument("--extras", default="conv,fista,c3,c5,exp1,c1,full",
                   help="comma-separated extra lines to run: conv, fista, c3, c5, exp1, c1, full")
    p.add_argument("--fista-first", type=int, default=4, help="first problem of the c4 set")
    p.add_argument("--fista-problems", type=int, default=4)
    p.add_argument("--fista-iters", type=int, default=2)
    p.add_argument("--fista-power", type=int, default=5, help="power iterations for the step size")
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


def oracle_sample(w, taps, n_vox, seed=0, outputs=False):
    """Time the FP64 oracle on A and A^T restricted to a seeded voxel subset
    (taps: the oracle's own system kernel)."""
    import oracle

    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.N, size=min(n_vox, w.N), replace=False)).astype(np.int64)
    xs = w.x[idx].astype(np.float64)
    t0 = time.perf_counter()
    s, _ = oracle.forward(w, taps, xs, vox_idx=idx)
    z, _ = oracle.adjoint(w, taps, s, vox_idx=idx)
    dt = time.perf_counter() - t0
    pairs = 2 * idx.size * w.K
    if outputs:
        return pairs / dt, dt, idx.size, oracle.num_threads(), (idx, s, z)
    return pairs / dt, dt, idx.size, oracle.num_threads()


def oracle_parity(api, dev, plan, w, sample, want):
    """Distances of the CUDA path to the FP64 oracle (rel L2), measured in the
    CPU-baseline leg, the one part of this script that runs the oracle, on
    samples the oracle computes in seconds:
      * the headline batch: A x over the oracle sample's voxels (x zero
        elsewhere, all rows) and A^T of the oracle's s at those voxels;
      * c3 (tcgen05 split and plain FP32 plans, first 128 positions): two
        whole rows of A x and A^T at 256 seeded voxels, per output;
      * c1: the closed form (dl 1) and the 64 x 64 point method, whole s.
    Both sides compute their own system kernel."""
    import torch

    import oracle

    out = {}
    idx, s_ref, z_ref = sample
    xs = torch.zeros(w.N, device=dev)
    xs[torch.from_numpy(idx).to(dev)] = torch.from_numpy(w.x[idx]).to(dev)
    s_gpu = plan.forward(xs)
    z_gpu = plan.adjoint(torch.from_numpy(s_ref.astype(np.float32)).to(dev))
    zg = z_gpu.cpu().numpy()[idx]
    out["c2_batch"] = {"sample": f"{idx.size} seeded voxels x {w.K} positions",
                       "A_rel_l2": float(np.linalg.norm(s_gpu.cpu().numpy() - s_ref) / np.linalg.norm(s_ref)),
                       "AT_rel_l2": float(np.linalg.norm(zg - z_ref) / np.linalg.norm(z_ref))}
    if "c3" in want:
        w3 = c3_batch(128)
        taps3 = oracle.taps_for(w3)
        ks = np.array([5, 77])
        x64 = w3.x.astype(np.float64)
        rows = np.stack([oracle.forward(w3.with_tx(w3.tx[k:k + 1]), taps3, x64)[0][0] for k in ks])
        rng = np.random.default_rng(5)
        y = rng.standard_normal((w3.K, w3.L)).astype(np.float32)
        vidx = np.sort(rng.choice(w3.N, size=256, replace=False)).astype(np.int64)
        zr, _ = oracle.adjoint(w3, taps3, y.astype(np.float64), vox_idx=vidx)
        x3 = torch.from_numpy(w3.x).to(dev)
        res = {"sample": "rows 5 and 77 of A x (all 16.7M voxels); A^T of a seeded y at 256 seeded voxels"}
        for name, tc in (("tcgen05_split", True), ("plain_fp32", False)):
            p3 = api.Plan(w3, conv_tc=tc, device=dev)
            s3 = p3.forward(x3).cpu().numpy()[ks]
            z3 = p3.adjoint(torch.from_numpy(y).to(dev)).cpu().numpy()[vidx]
            res[name] = {"A_rows_rel_l2": [float(np.linalg.norm(s3[i] - rows[i]) / np.linalg.norm(rows[i]))
                                           for i in range(len(ks))],
                         "AT_rel_l2": float(np.linalg.norm(z3 - zr) / np.linalg.norm(zr))}
            del p3
        out["c3"] = res
    if "c1" in want:
        res = {}
        for name, wc in (("closed_form_dl_1", W.c1(dl=1)), ("point_64x64", W.c1(method=W.METHOD_POINT, q=(64, 64),
                                                                                      dl=1))):
            ref, _ = oracle.forward(wc, oracle.taps_for(wc), wc.x.astype(np.float64))
            pc = api.Plan(wc, device=dev)
            got = pc.forward(torch.from_numpy(wc.x).to(dev)).cpu().numpy()
            res[name] = {"A_rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
        out["c1"] = res
    return out


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
    # the adjoint's input: the same signals scaled to a maximum of 1 (the
    # system kernel is of order 1e-20, so h-bar^- applied to s of this random
    # f, itself about 1e-19, would fall below FP32's normal range on any path)
    y = s_plain / s_plain.abs().max()
    v_plain = plan.conv_adjoint(y)
    v_tc = tc.conv_adjoint(y)
    t_tc = cuda_ms(lambda: tc.conv_forward(f), reps=3)
    # the split-plane kernel pat_forward uses: f as BF16 hi and lo planes (the
    # epilogue's output format), brought into the tensor cores by tensor-map copies
    planes = tc.conv_split(f)
    s_sp = tc.conv_forward_split(planes)
    t_sp = cuda_ms(lambda: tc.conv_forward_split(planes), reps=5)
    sp_bytes = 2 * 2 * w.K * w.UL + 4 * w.K * w.L  # planes read once, s written
    hbm = measured_hbm_gbs()
    nw = w.T + w.U - 1
    kw = -(-(127 * w.U + nw) // 64) * 64  # Toeplitz contraction length per 128-sample tile
    flops = 3 * 2 * 128 * 64 * kw * (-(-w.L // 128)) * (-(-w.K // 64))
    out = {"workload": f"all c2 positions: K {w.K} rows, U L {w.UL} -> L {w.L}, {nw} taps, random f; "
                       "adjoint of its s scaled to unit maximum",
           "forward_ms": {"fp64_cuda_cores": cuda_ms(lambda: plan.conv_forward(f), reps=3), "tcgen05_bf16x3": t_tc},
           "adjoint_ms": {"fp64_cuda_cores": cuda_ms(lambda: plan.conv_adjoint(y), reps=3),
                          "tcgen05_bf16x3": cuda_ms(lambda: tc.conv_adjoint(y), reps=3)},
           "rel_l2_tc_vs_fp64": {"forward": rel_l2(s_tc, s_plain), "adjoint": rel_l2(v_tc, v_plain)},
           "tcgen05_forward_tflops": flops / (t_tc * 1e-3) / 1e12,
           "split_plane_forward": {"ms": t_sp, "rel_l2_vs_fp64": rel_l2(s_sp, s_plain),
                                   "bytes": sp_bytes, "gb_per_s": sp_bytes / (t_sp * 1e-3) / 1e9,
                                   "hbm_peak_gb_per_s": hbm,
                                   "frac_of_hbm": (sp_bytes / (t_sp * 1e-3) / 1e9) / hbm if hbm else None,
                                   "method_tflops": 2.0 * w.K * w.L * nw / (t_sp * 1e-3) / 1e12,
                                   "tiles": (-(-w.L // 128)) * (-(-w.K // 256))},
           "tc_error": api._lib.pat_plan_get_info(tc.handle)["tc_error"]}
    return out


def issue_line(quad_evals, seconds, sm_mhz):
    """Issue-slot view of the dominant kernel beside its FP32 roofline: warp
    instructions issued per launch (the per-evaluation count from the
    instruction counters times the plan's evaluations) over the launch's
    CUDA-event time, against 152 SMs x 4 schedulers x one instruction per cycle
    at the clock seen."""
    got = quad_evals * WARP_INSTS_PER_QUAD_EVAL / seconds / 1e9
    peak = SM_COUNT * ISSUE_PER_SM_PER_CYCLE * sm_mhz * 1e6 / 1e9
    return {"achieved": got, "peak": peak, "unit": "G warp instructions/s", "frac": got / peak,
            "warp_insts_per_unit": WARP_INSTS_PER_QUAD_EVAL}


def measured_hbm_gbs():
    """The HBM copy bandwidth of this GPU pool (MEASURED_PEAKS.json), else the
    6.8 TB/s fallback of one earlier GB300 measurement."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def fista_compare(api, dev, first, n_prob, iters, power):
    """Batched reconstruction on problems of the c4 set (grids 48^3-160^3,
    1,024-8,192 planar or cylindrical positions, L 1024 or 2048, tube
    phantoms), problems first .. first + n_prob - 1, s = A x + 1 % noise,
    lambda_R = 1e-3 |A^T s|_inf, step from `power` power iterations.  Time per
    iteration of all problems: one pat_recon per problem enqueued on the legacy
    stream (plain FP32 operator, no graph), against pat_recon_batch (one CUDA
    graph per iteration, a branch per problem) with the plain and with the
    tensor-core-convolution plans.  busy_fraction: the problems' A and A^T
    device times (CUDA events, one launch sequence each) over the sequential
    iteration's wall time; 1 - busy is the idle share that persistent
    kernels or batching could recover."""
    import torch

    ws = [W.c4_problem(p) for p in range(first, first + n_prob)]
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
        for _ in range(power):
            v = p.adjoint(p.forward((v.double() / v.double().norm()).float()))
        steps.append(float(1.0 / (1.05 * (float(v.double().norm()) + lam[-1]))))
        if not (math.isfinite(lam[-1]) and math.isfinite(steps[-1])):
            raise RuntimeError(f"{w.name}: lambda {lam[-1]}, step {steps[-1]}")
    x0 = [torch.zeros(p.N, device=dev) for p in plans]
    # device time of one A and one A^T per problem
    ops_ms = []
    for p, s in zip(plans, s_list):
        x = torch.zeros(p.N, device=dev)
        ops_ms.append(cuda_ms(lambda: (p.forward(x), p.adjoint(s)), reps=1, warm=1))

    def seq():
        return [p.recon(s, x, iters=iters, lambda_R=l, step=t) for p, s, x, l, t in zip(plans, s_list, x0, lam, steps)]

    side = torch.cuda.Stream(device=dev)

    def batched(ps):
        with torch.cuda.stream(side):
            r = api.recon_batch(ps, s_list, x0, iters=iters, lambdas=lam, steps=steps)
        side.synchronize()
        return r

    def wall(fn):
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
    return {"workload": "; ".join(w.name for w in ws),
            "selection": f"c4 problems {first}..{first + n_prob - 1} (seeds 1000 + p) of the 32 drawn from the "
                         f"stated ranges; {iters} iterations each, step from {power} power iterations",
            "problems": n_prob, "iterations": iters, "pairs_per_iteration": 2 * pairs,
            "ms_per_iteration": {"plain_fp32_sequential": t_seq, "graph_batched": t_b,
                                 "graph_batched_tcgen05_conv": t_tc},
            "speedup_vs_plain": {"graph_batched": t_seq / t_b, "graph_batched_tcgen05_conv": t_seq / t_tc},
            "max_rel_l2_vs_plain": {"graph_batched": d_b, "graph_batched_tcgen05_conv": d_tc},
            "ms_A_plus_AT_per_problem": ops_ms, "busy_fraction_sequential": sum(ops_ms) / t_seq,
            "pairs_per_s_sequential": 2 * pairs / (t_seq * 1e-3),
            "timing": "wall clock per iteration over all problems, host to device completion, step sizes fixed"}


def plane_roofline(quad_evals, ms):
    """FP32 roofline of a planar A^T (its geometry kernel is 99 % of it): the
    executed flops per evaluation measured with ncu's counters, over the FP32
    peak at the maximum SM clock."""
    ach = quad_evals * FLOPS_PER_PLANE_EVAL / (ms * 1e-3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "flops_per_unit": FLOPS_PER_PLANE_EVAL, "units": quad_evals,
            "unit_name": "planar quadrant-edge area evaluation", "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}


def c3_line(api, dev, n_pos):
    """The precision-split system (c3): 256^3 voxels at 0.08 mm, planar 3x3 mm
    elements on a 40 mm hemisphere, L 2048, tcgen05 BF16 split convolution;
    one batch of the first n_pos positions, against the plain FP32 plan
    (FP64-accumulated convolution on the CUDA cores) on the same positions."""
    import torch

    w = c3_batch(n_pos)
    plan = api.Plan(w, conv_tc=True, device=dev)
    plain = api.Plan(w, taps=plan.taps, device=dev)
    x = torch.from_numpy(w.x).to(dev)
    s = plan.forward(x)
    t_f = cuda_ms(lambda: plan.forward(x, out=s), reps=2)
    z = torch.empty(w.N, device=dev)
    t_a = cuda_ms(lambda: plan.adjoint(s, out=z), reps=2)
    s_p = plain.forward(x)
    t_pf = cuda_ms(lambda: plain.forward(x, out=s_p), reps=2)
    z_p = torch.empty(w.N, device=dev)
    t_pa = cuda_ms(lambda: plain.adjoint(s, out=z_p), reps=2)
    pairs = w.N * w.K
    return {"workload": f"c3: 256^3 @ 0.08 mm, first {w.K} of 5,120 planar 3x3 mm positions, L 2048 @ 40 MHz, "
                        f"U 11, dl 11, tcgen05 BF16 split convolution",
            "forward_pairs_per_s": pairs / (t_f * 1e-3), "adjoint_pairs_per_s": pairs / (t_a * 1e-3),
            "ms": {"forward": t_f, "adjoint": t_a}, "mean_bins_per_pair": plan.info["pair_bins"] / pairs,
            "plain_fp32": {"ms": {"forward": t_pf, "adjoint": t_pa},
                           "forward_pairs_per_s": pairs / (t_pf * 1e-3), "adjoint_pairs_per_s": pairs / (t_pa * 1e-3)},
            "rel_l2_split_vs_plain_fp32": {"forward": rel_l2(s, s_p), "adjoint": rel_l2(z, z_p)},
            "roofline_adjoint_geometry": plane_roofline(plan.info["quad_evals"], t_a),
            "tc_error": api._lib.pat_plan_get_info(plan.handle)["tc_error"]}


def c3_batch(n_pos):
    w = W.c3(with_x=False, rotations=1)
    w = w.with_tx(w.tx[:n_pos])
    return w.with_(x=W.blob_phantom(w.n, w.origin, w.pitch, 200, 0))


def c5_line(api, dev, n_pos):
    """The full-scale system (c5): 512^3 voxels at 0.05 mm (134M), the c2
    array rotated over 128 angles, L 4096 at 50 MHz; the first n_pos
    positions of one angle, closed form (surface method) against the point
    method with 16 x 16 points per element (Alg. 2) on a quarter of them.
    The point method bins each point per fine bin, so its distance to the
    closed form is reported both against the closed form at the same
    binning (dl = 1: the quadrature error, Prop. 2) and at the operating
    point dl = U (which adds Remark 1's grouping)."""
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
    plan1 = api.Plan(w.with_tx(w.tx[:n_pt]).with_(dl=1), taps=plan.taps, device=dev)
    s1 = plan1.forward(x)
    pairs = w.N * w.K
    return {"workload": f"c5: 512^3 @ 0.05 mm, first {w.K} of 16,384 cylindrical positions, L 4096 @ 50 MHz, U 11, "
                        f"dl 11; point method 16 x 16 on the first {n_pt}",
            "closed_form": {"forward_pairs_per_s": pairs / (t_f * 1e-3), "adjoint_pairs_per_s": pairs / (t_a * 1e-3),
                            "ms": {"forward": t_f, "adjoint": t_a}},
            "point_16x16": {"forward_pairs_per_s": w.N * n_pt / (t_pf * 1e-3), "ms": {"forward": t_pf},
                            "point_evaluations_per_s": w.N * n_pt * 256 / (t_pf * 1e-3)},
            "point_16x16_vs_closed_form_rel_l2": {"same_binning_dl_1": rel_l2(sp, s1),
                                                  "operating_point_dl_11": rel_l2(sp, s[:n_pt])},
            "mean_bins_per_pair": plan.info["pair_bins"] / pairs}


def c1_line(api, dev):
    """The c1 system (16^3 voxels at 0.1 mm, 32 planar 1 x 1 mm elements on a
    10 mm Fibonacci sphere, L 256 at 40 MHz): the closed form against the
    64 x 64 point quadrature of the surface (Alg. 2), at the same binning
    (dl = 1) and with the closed form at its operating point dl = U."""
    import torch

    w1 = W.c1(dl=1)
    x = torch.from_numpy(w1.x).to(dev)
    taps = api.system_taps(w1, dev)
    closed1 = api.Plan(w1, taps=taps, device=dev)
    closed11 = api.Plan(W.c1(), taps=taps, device=dev)
    point = api.Plan(W.c1(method=W.METHOD_POINT, q=(64, 64), dl=1), taps=taps, device=dev)
    out = {"workload": w1.name + "; closed form (dl 1 and 11) and 64 x 64 points per element"}
    res = {}
    for name, p in (("closed_form_dl_1", closed1), ("closed_form_dl_11", closed11), ("point_64x64", point)):
        s = p.forward(x)
        z = torch.empty(w1.N, device=dev)
        res[name] = s
        out[name] = {"ms_A_plus_AT": cuda_ms(lambda: (p.forward(x, out=s), p.adjoint(s, out=z)), reps=3)}
    out["point_64x64_vs_closed_form_rel_l2"] = {"same_binning_dl_1": rel_l2(res["point_64x64"], res["closed_form_dl_1"]),
                                                "operating_point_dl_11": rel_l2(res["point_64x64"],
                                                                                res["closed_form_dl_11"])}
    return out


def full_line(api, dev, x2):
    """Whole applications of the headline systems: one A and one A^T over all
    23,040 c2 positions (128^3 voxels), and over all 5,120 c3 positions
    (256^3 voxels, tcgen05 BF16 split convolution), CUDA events, clocks
    sampled during the run."""
    import torch

    out = {}
    w2 = W.c2(with_x=False)
    w3 = W.c3(with_x=False)
    w3 = w3.with_(x=W.blob_phantom(w3.n, w3.origin, w3.pitch, 200, 0))
    for name, w, x, tc in (("c2_all_23040_positions", w2, x2, False),
                           ("c3_all_5120_positions", w3, None, True)):
        t0 = time.perf_counter()
        plan = api.Plan(w, conv_tc=tc, device=dev)
        t_plan = time.perf_counter() - t0
        if x is None:
            x = torch.from_numpy(w.x).to(dev)
        s = torch.empty((w.K, w.L), device=dev)
        z = torch.empty(w.N, device=dev)
        clk = ClockSampler(physical_gpu_index(torch.cuda.current_device()))
        clk.start()
        t_f = cuda_ms(lambda: plan.forward(x, out=s), reps=1, warm=0)
        t_a = cuda_ms(lambda: plan.adjoint(s, out=z), reps=1, warm=0)
        c = clk.stop()
        pairs = w.N * w.K
        out[name] = {"ms": {"A": t_f, "AT": t_a, "A_plus_AT": t_f + t_a}, "pairs": pairs,
                     "pairs_per_s": 2 * pairs / ((t_f + t_a) * 1e-3), "forward_pairs_per_s": pairs / (t_f * 1e-3),
                     "adjoint_pairs_per_s": pairs / (t_a * 1e-3), "plan_creation_s": t_plan, "clocks": c,
                     "tc_error": api._lib.pat_plan_get_info(plan.handle)["tc_error"] if tc else None}
        del plan, s, z
        torch.cuda.empty_cache()
    return out


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
        v, dt, nv, cores, smp = oracle_sample(wcpu, oracle.taps_for(wcpu), args.cpu_sample_voxels, outputs=True)
        cpu = {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{nv} seeded voxels x {wcpu.K} positions, A then A^T, FP64 ({dt:.1f} s)"}
        want_p = set(e.strip() for e in args.extras.split(",")) if not args.no_extras else set()
        cpu["parity"] = oracle_parity(api, dev, plans[args.warmup], wcpu, smp, want_p)

    extras = {}
    want = set(e.strip() for e in args.extras.split(",") if e.strip())
    if rank == 0 and not args.no_extras:
        if "conv" in want:
            extras["conv_tcgen05"] = conv_compare(api, plans[args.warmup],
                                                  c2w(args, angle_sets[args.warmup], with_x=False).with_(x=w0.x), taps,
                                                  x, dev)
        if "fista" in want:
            extras["fista_batched"] = fista_compare(api, dev, args.fista_first, args.fista_problems, args.fista_iters,
                                                    args.fista_power)
        if "c3" in want:
            extras["c3_precision_split"] = c3_line(api, dev, args.c3_positions)
            if cpu and "c3" in cpu.get("parity", {}):
                extras["c3_precision_split"]["rel_l2_vs_fp64_oracle"] = cpu["parity"]["c3"]
        if "c5" in want and args.c5_positions > 0:
            extras["c5_full_scale_subset"] = c5_line(api, dev, args.c5_positions)
        if "exp1" in want:
            extras["exp1_operators"] = exp1_line(api, dev)
        if "c1" in want:
            extras["c1_closed_vs_quadrature"] = c1_line(api, dev)
            if cpu and "c1" in cpu.get("parity", {}):
                extras["c1_closed_vs_quadrature"]["rel_l2_vs_fp64_oracle"] = cpu["parity"]["c1"]
        if "full" in want and args.grid == 128:
            extras["full_applications"] = full_line(api, dev, x)

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
                             "measured_peaks": measured,
                             "issue": issue_line(qe, mean_adj, sm_mhz)},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 4 * args.steps,
                "clocks": clk, "wall_s_timed": t_wall}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
