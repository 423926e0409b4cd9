"""Benchmark of the Batch-BFS / BCTS search on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload atari|precision] [--precision fp32|bf16|fp8|fp32_simt]

One step = one full search (Alg. 1 expansion, root / depth-1 / leaf Q-network,
backup with the Eq. 7 correction) over one batch of roots.  Default workload:
32 roots from seeded synthetic sprite-environment states, |A| = 18, d = 3
(5,832 leaves per root), gamma = 0.99, correction c = 1, FP32-class arithmetic,
He-initialised Nature-DQN weights from seed 1234 (synthetic stand-ins for
Atari states and pre-trained Rainbow weights).

Prints ONE JSON line on rank 0.  `value` = leaf nodes per second over all ranks
(device time, inputs resident in HBM); `e2e` = the same through bcts_search
with host buffers (host->device roots and device->host actions + values in the
timed region).  Under torchrun every rank searches its own 32 roots (weak
scaling, no collective on the data path; a barrier and a max over ranks of the
elapsed time only).

--impl reference times the oracle (plain FP64 C, OpenMP) on this host's cores
on a bounded sample of the same workload.
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

from paper_2107_01715_b300 import inputs  # noqa: E402

METRIC = "leaf nodes/sec & decisions/sec (A=18, d=3/4) vs plain FP32; p50/p99 latency, 1 B300"
WORKLOADS = {
    "atari": dict(n=32, A=18, d=3, gamma=0.99, c=1.0, precision="fp32",
                  name="plain Batch-BFS at Atari scale: 32 roots, |A|=18, d=3, FP32, correction on"),
    "precision": dict(n=8, A=18, d=4, gamma=0.99, c=1.0, precision="bf16",
                      name="precision form: 8 roots, |A|=18, d=4, leaf Q-net in reduced precision"),
    "batched": dict(n=256, A=18, d=4, gamma=0.99, c=1.0, precision="bf16",
                    name="batched form: 256 roots, d uniform in {1,2,3,4}, |A| in {4,9,18}, BF16, graph-replayed"),
    "sweep": dict(n=1, A=18, d=0, gamma=0.99, c=1.0, precision="fp32",
                  name="time per tree-search operation vs depth (one root per search), as in Sec. 4's runtime "
                       "experiment: sprite world A=18 d=1..5, DNN forward model A=2 d=2..16 and A=10 d=1..6"),
    "pruned": dict(n=32, A=18, d=4, keep=32, gamma=0.99, c=1.0, precision="fp32",
                   name="pruned search: 32 roots, |A|=18, d=4, 32 nodes kept per root action and level, FP32"),
    "dnn": dict(n=16, A=10, d=5, gamma=0.99, c=1.0, precision="fp32",
                name="DNN forward model (Sec. 4): 16 roots, |A|=10, d=5, 100-wide state, 3 hidden layers of 100, FP32"),
    "stream": dict(n=1 << 20, A=18, frames=100_000, backup_roots=1024, backup_d=4, gamma=0.99, c=1.0,
                   precision="fp32",
                   name="streaming kernels alone: Alg. 1's expansion of 1,048,576 parents x |A|=18 "
                        "(bcts_expand), the renderer on 100,000 states (bcts_render) and the backup with the "
                        "BCTS correction over 1,024 roots x 18^4 leaves (bcts_backup)"),
    "serving": dict(n=1024, A=18, d=4, gamma=0.99, c=1.0, precision="bf16", rate=500.0, seconds=4.0,
                    budget=120 << 30,
                    name="serving form: Poisson requests from 1024 episodes, d in {2,3,4}, |A|=18, BF16, "
                         "120 GB frame budget"),
}
L2_BYTES = 126 * 2 ** 20
DTYPES = {"fp32": "f32 (bf16x3 split products, f32 accumulate)", "bf16": "bf16", "fp8": "e4m3", "fp32_simt": "f32"}
# Multiply-accumulates per node of each kernel class in the method's own network
# (Nature-DQN; conv1 over a whole 4-frame stack for the roots and depth-1 nodes).  The
# parents' partial maps and the leaves' conv1 run no contraction: streaming passes over
# the sprite tables, bound by their DRAM bytes alone.
ALG_MACS = {"conv1": 400 * 32 * 256, "conv1_partial": 0, "conv1_leaf": 0,
            "conv2": 81 * 64 * 512, "conv3": 49 * 64 * 576, "fc1": 512 * 3136}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per node of the leaf-level
# kernel classes from one ncu capture of the current kernel version at 4 roots, A = 18,
# d = 3 (launches over 23,328 leaves; traffic grows in proportion to the nodes a launch
# processes).  A class whose kernel changed after its capture has no entry here.
TRAFFIC_PER_NODE = {"fp32/conv1_leaf": 53939.0, "bf16/conv1_leaf": 27170.0, "fp8/conv1_leaf": 13745.0,
                    "fp32/conv2": 70771.0, "bf16/conv2": 34762.0, "fp8/conv2": 16775.0,
                    "fp32/conv3": 31903.0, "fp32/fc1": 13443.0}
# Output rows each precision's default kernel computes per output row it keeps: the
# window and tap-pair kernels run on a grid padded to the input's width and height
# (conv2: 100 rows per 81, conv3: 81 per 49), and the tap-pair tiles keep 127 of 128.
EXEC_PAD = {"fp32/conv2": 100 / 81 * 128 / 127, "bf16/conv2": 100 / 81, "bf16/conv3": 81 / 49,
            "fp8/conv2": 100 / 81}


def layer_model(cls, precision, A):
    """Roofline terms of one node of a kernel class: (algorithmic MACs, tensor MMAs
    executed per MAC, algorithmic DRAM bytes read, written).  Activation maps are bf16
    (2 bytes), bf16 hi + lo in the FP32-class split mode (4 bytes), E4M3 in FP8 (1 byte);
    the partial conv1 map of a parent is FP32 and each of its A children reads it, so a
    leaf's share is 1/A of it; the fc1 output is FP32 (in the split mode, whose fc1
    epilogue folds fc2 in, two halves' partial Q-values: 2 x 18 FP32).  Weights stay resident in shared
    memory (read once per CTA).  The split mode executes 2 bf16 MMAs per conv1 MAC
    (pixels are exact in bf16) and 3 per MAC elsewhere, times the padding of the
    default kernel's output grid (EXEC_PAD)."""
    e = {"fp32": 4, "bf16": 2, "fp8": 1}.get(precision, 4)
    c1, c2, c3, f1 = 400 * 32, 81 * 64, 49 * 64, 512
    fc1_out = 2 * 18 * 4 if precision == "fp32" else f1 * 4
    rw = {"conv1": (80, c1 * e), "conv1_partial": (80, c1 * 4), "conv1_leaf": (80 + c1 * 4 / A, c1 * e),
          "conv2": (c1 * e, c2 * e), "conv3": (c2 * e, c3 * e), "fc1": (c3 * e, fc1_out),
          "fc2": (fc1_out, 4)}.get(cls, (0, 0))
    macs = ALG_MACS.get(cls, A * 512 if cls == "fc2" else 0)
    mma = (2 if cls.startswith("conv1") else 3) if precision == "fp32" else 1
    mma *= EXEC_PAD.get(f"{precision}/{cls}", 1.0)
    return macs, mma, rw[0], rw[1]


def class_nodes(cls, n, A, d, prof_cnt):
    """Nodes one search step sends through a kernel class: every root, depth-1 node and leaf
    runs the Q-network once; with partial maps the leaves' conv1 is split into the parents'
    partial maps (depth d-1) and the leaves' last slot."""
    leaves = n * A ** d if d >= 2 else 0
    total = n + n * A + leaves
    partial = prof_cnt.get("conv1_leaf", 0) > 0
    if cls == "conv1":
        return total - leaves if partial else total
    if cls == "conv1_partial":
        return n * A ** (d - 1) if partial else 0
    if cls == "conv1_leaf":
        return leaves if partial else 0
    return total


def roofline_for(dom, precision, A, nodes, ms, launches, pk, pk_kind):
    """Roofline of the dominant kernel class.  `achieved` counts the method's own work:
    algorithmic FLOPs (2 x the layer's MACs per node) for a contraction, algorithmic DRAM
    bytes otherwise, over the class's CUDA-event time.  The binding resource is the one
    whose minimum time is longer: the FLOPs the kernel executes (split mode: 2-3 bf16 MMAs
    per MAC) at the tensor peak of the operand type, or the algorithmic bytes at the
    measured copy bandwidth.  `executed_frac` is the executed MMA rate against the same
    peak."""
    macs, mma, rd, wr = layer_model(dom, precision, A)
    secs = ms / 1e3
    bytes_ = (rd + wr) * nodes
    hbm = pk["hbm_gbs"]
    alg_flops = 2.0 * macs * nodes
    if precision == "fp32_simt":
        peak_t = pk.get("sm_max_mhz", 2032.0) * 1e6 * 148 * 128 * 2 / 1e12
        t_note, t_bound = "FP32 FMA: 148 SMs x 128 lanes x 2 FLOP x max SM clock", "alu"
        exec_flops = alg_flops
    else:
        ratio = 2.0 if precision == "fp8" else 1.0  # nominal dense fp8 / bf16 = 4.5 / 2.25
        peak_t = pk["bf16_tflops_sustained"] * ratio
        exec_flops = alg_flops * mma
        t_bound = "tensor"
        t_note = "bf16 dense sustained" + (" x 2 (nominal fp8/bf16 ratio)" if ratio > 1 else "")
    t_tensor = exec_flops / (peak_t * 1e12)
    t_hbm = bytes_ / (hbm * 1e9)
    per_launch = nodes / max(launches, 1)
    tpn = TRAFFIC_PER_NODE.get(f"{precision}/{dom}")
    common = {"kernel": dom, "traffic": tpn * per_launch if tpn else None,
              "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per node from one capture of "
                                 "this kernel version (4 roots, A=18, d=3), x nodes per launch; not measured in "
                                 "this run") if tpn else "no ncu capture of the current version of this kernel",
              "algorithmic_bytes_per_launch": (rd + wr) * per_launch,
              "algorithmic_flops_per_launch": alg_flops / max(launches, 1),
              "executed_flops_per_launch": exec_flops / max(launches, 1),
              "avg_launch_ms": ms / max(launches, 1), "launches": launches,
              "min_time_ms": {"tensor_or_alu_executed": 1e3 * t_tensor, "hbm": 1e3 * t_hbm},
              "hbm_achieved_gbs": bytes_ / secs / 1e9}
    if t_hbm >= t_tensor:
        ach = bytes_ / secs / 1e9
        return dict(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                    peak_note=f"STREAM-style copy bandwidth (of {pk_kind})", **common)
    ach = alg_flops / secs / 1e12
    return dict(bound=t_bound, achieved=ach, peak=peak_t, unit="TFLOP/s", frac=ach / peak_t,
                executed_frac=exec_flops / secs / 1e12 / peak_t,
                peak_note=f"{t_note} (of {pk_kind}); achieved counts the method's FLOPs (2 x MACs)", **common)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="atari", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the other forms' measurements on the line")
    ap.add_argument("--frames", action="store_true",
                    help="the frame path: every node's frame rendered to device memory, conv1 on the tensor cores")
    ap.add_argument("--roots", type=int, default=None, help="override the root count (smaller profiling cases)")
    ap.add_argument("--rate", type=float, default=None, help="serving: mean request rate (req/s)")
    ap.add_argument("--seconds", type=float, default=None, help="serving: length of the arrival stream (s)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self, max_mhz):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": max_mhz, "reasons": ["nvidia-smi unavailable"]}
        sm, reasons, power = [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    max_mhz = float(parts[2])
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max_mhz,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def dist_setup(gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BCTS_BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float, device):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(W, wl, target_s=15.0):
    """The oracle as it stands on this host's cores, on a bounded sample: one root
    (A^d leaves + the root and depth-1 evaluations) of the same workload."""
    import oracle
    oracle.build()
    roots = inputs.root_states([0])
    t0 = time.perf_counter()
    oracle.search(roots, W, wl["A"], wl["d"], float(np.float32(wl["gamma"])), wl["c"])
    dt = time.perf_counter() - t0
    leaves = wl["A"] ** wl["d"]
    return {"value": leaves / dt, "unit": "leaf nodes/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"1 root (seed 0) of the workload: {leaves} leaves + {1 + wl['A']} root/depth-1 "
                      f"Q evaluations, FP64, {dt:.1f} s"}


def run_dnn(args, wl):
    """Batch-BFS over the DNN forward model: device-resident roots, per-kernel
    events, ALU roofline of the forward-model layers (FP32 CUDA cores)."""
    import torch
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2107_01715_b300 import bcts
    n, A, d = wl["n"], wl["A"], wl["d"]
    W = inputs.dnn_weights(A)
    ctx = bcts.bcts_dnn_create(W, A, d, wl["gamma"], wl["c"])
    roots = inputs.dnn_root_states(range(rank * n, rank * n + n))
    d_roots = torch.from_numpy(roots).to(dev)
    d_act = torch.empty(n, dtype=torch.int32, device=dev)
    d_val = torch.empty(n * A, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    leaves = n * A ** d
    expanded = sum(n * A ** i for i in range(1, d + 1))  # children produced by the forward model

    def step():
        bcts.bcts_dnn_search_device(ctx, d_roots, n, d_act, d_val, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        bcts.bcts_dnn_profile(ctx, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
    prof_ms, prof_cnt, launches = bcts.bcts_dnn_profile(ctx, False)
    total_s = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in ev) / 1e3, dev)
    value = world * leaves * args.steps / total_s
    e2e_times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        bcts.bcts_dnn_search(ctx, roots)
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * leaves * args.steps / max_over_ranks(world, sum(e2e_times), dev)
    if rank != 0:
        ctx.close()
        return
    pk, pk_kind = peaks()
    # forward-model MACs per child: W1's state part once per parent (shared by A
    # children), layers 2 and 3, and the 101-row output layer
    macs_child = 100 * 100 / A + 2 * 100 * 100 + 101 * 100
    flops = 2.0 * macs_child * expanded * args.steps
    mlp_s = prof_ms["dnn_mlp"] / 1e3
    peak = pk.get("sm_max_mhz", 2032.0) * 1e6 * 148 * 128 * 2 / 1e12
    achieved = flops / mlp_s / 1e12 if mlp_s > 0 else None
    roofline = {"kernel": "dnn_mlp", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "traffic_note": "no ncu capture of this kernel class",
                "peak_note": "FP32 FMA: 148 SMs x 128 lanes x 2 FLOP x max SM clock (of " + pk_kind + " clock)",
                "algorithmic_flops_per_launch": flops / max(prof_cnt["dnn_mlp"], 1),
                "avg_launch_ms": prof_ms["dnn_mlp"] / max(prof_cnt["dnn_mlp"], 1), "launches": prof_cnt["dnn_mlp"]}
    cb = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        # a bounded sample: the workload's roots one by one until about 10 s of CPU work
        t0 = time.perf_counter()
        k = 0
        while k < n and time.perf_counter() - t0 < 10.0:
            oracle.dnn_search(roots[k:k + 1], W, A, d, float(np.float32(wl["gamma"])), wl["c"])
            k += 1
        dt = time.perf_counter() - t0
        cb = {"value": k * A ** d / dt, "unit": "leaf nodes/s", "cores": oracle.threads(), "kind": "oracle",
              "sample": f"{k} roots of the workload: {k * A ** d} leaves, "
                        f"{k * sum(A ** i for i in range(1, d + 1))} forward-model steps, FP64, {dt:.1f} s"}
    line = {"metric": METRIC, "value": value, "unit": "leaf nodes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["name"], "roots_per_step": n, "A": A, "d": d, "leaves_per_step": leaves,
                       "forward_model_steps_per_step": expanded,
                       "l2": "flushed between steps (256 MB write)"},
            "decisions_per_s": world * n * args.steps / total_s,
            "e2e": {"value": e2e_value, "unit": "leaf nodes/s", "h2d_bytes_per_step": n * 400,
                    "d2h_bytes_per_step": n * 4 + n * A * 4},
            "gpu_launches": launches,
            "kernel_ms": prof_ms, "kernel_launches": prof_cnt, "roofline": roofline, "cpu_baseline": cb,
            "clocks": _clock_line(clk, pk)}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_pruned(args, wl):
    """Pruned search at a depth the full tree would not reach in the same time:
    device-resident roots, per-kernel events; the unit is scored leaves."""
    import torch
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2107_01715_b300 import bcts
    n, A, d, keep = wl["n"], wl["A"], wl["d"], wl["keep"]
    precision = args.precision or wl["precision"]
    W = inputs.qnet_weights(A, seed=1234)
    ctx = bcts.bcts_create(W, A, d, wl["gamma"], wl["c"], precision=precision)
    roots = inputs.root_states(range(rank * n, rank * n + n))
    d_roots = torch.from_numpy(roots.view(np.uint8).copy()).to(dev)
    d_act = torch.empty(n, dtype=torch.int32, device=dev)
    d_val = torch.empty(n * A, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    # candidates per group and level: A at level 2, min(keep, C) * A afterwards
    cands, S = [], 1
    for i in range(2, d + 1):
        C = S * A
        cands.append(C)
        S = min(keep, C)
    leaves = n * A * cands[-1]
    scored = n + n * A + n * A * sum(cands)  # Q-network evaluations per search

    def step():
        bcts.bcts_search_pruned_device(ctx, d_roots, n, keep, d_act, d_val, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        bcts.bcts_profile(ctx, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
    prof_ms, prof_cnt, launches = bcts.bcts_profile(ctx, False)
    total_s = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in ev) / 1e3, dev)
    value = world * leaves * args.steps / total_s
    e2e = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        bcts.bcts_search_pruned(ctx, roots, keep)
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    e2e_value = world * leaves * args.steps / max_over_ranks(world, sum(e2e), dev)
    if rank != 0:
        ctx.close()
        return
    pk, pk_kind = peaks()
    dom = max(prof_ms, key=lambda k: prof_ms[k])
    roofline = None
    if prof_ms[dom] > 0:
        roofline = roofline_for(dom, precision, A, scored * args.steps, prof_ms[dom], prof_cnt[dom], pk, pk_kind)
    line = {"metric": METRIC, "value": value, "unit": "leaf nodes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES.get(precision, precision), "data": "synthetic",
            "config": {"workload": wl["name"], "roots_per_step": n, "A": A, "d": d, "keep": keep,
                       "leaves_per_step": leaves, "q_evaluations_per_step": scored, "full_tree_leaves": n * A ** d,
                       "precision": precision, "l2": "flushed between steps (256 MB write)"},
            "decisions_per_s": world * n * args.steps / total_s,
            "e2e": {"value": e2e_value, "unit": "leaf nodes/s", "h2d_bytes_per_step": n * 80,
                    "d2h_bytes_per_step": n * 4 + n * A * 4},
            "gpu_launches": launches, "kernel_ms": prof_ms, "kernel_launches": prof_cnt, "roofline": roofline,
            "cpu_baseline": None, "clocks": _clock_line(clk, pk)}
    print(json.dumps(line), flush=True)
    ctx.close()


def stream_measure(bcts, torch, wl, warmup, steps, roots_override=None, rank=0, local=0, world=1):
    """The HBM-bound kernels on their own, at sizes where bandwidth rather than launch
    latency decides: the expansion (one thread per child: read the parent's 80-byte
    state and R, write the child's state and R) through bcts_expand, the renderer
    (read a state, write its 28,224-byte frame stack) through bcts_render, and the
    backup with the BCTS correction through bcts_backup (8 bytes per leaf).  Inside a
    search they run on the levels' node counts; here each is timed alone with CUDA
    events, inputs and outputs larger than L2."""
    dev = torch.device("cuda", local)
    P, A = wl["n"], wl["A"]
    F = min(wl["frames"], P // 10)  # rendered from the first children (a reduced --roots case shrinks both)
    base = inputs.root_states(range(rank * 4096, rank * 4096 + 4096))
    parents = np.resize(base, P)  # 4,096 seeded states repeated: the kernels' work does not depend on repeats
    d_par = torch.from_numpy(parents.view(np.uint8).copy()).to(dev)
    d_parR = torch.zeros(P, dtype=torch.float32, device=dev)
    d_child = torch.empty(P * A * 80, dtype=torch.uint8, device=dev)
    d_childR = torch.empty(P * A, dtype=torch.float32, device=dev)
    d_frames = torch.empty(F * inputs.FRAME_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    reps = max(1, min(steps, 20))
    ops = {"expand": (lambda: bcts.bcts_expand(d_par, d_parR, P, A, 0.99, d_child, d_childR, None, stream),
                      P * (80 + 4) + P * A * (80 + 4), P * A, "children"),
           "render": (lambda: bcts.bcts_render(d_child, F, d_frames, stream),
                      F * (80 + inputs.FRAME_BYTES), F, "frame stacks")}
    # backup: seeded leaf rewards and max-Q values of nb roots x A^db leaves (Alg. 1 order)
    nb, db = wl["backup_roots"], wl["backup_d"]
    if roots_override:
        nb = max(1, nb * roots_override // WORKLOADS["stream"]["n"])
    LB = nb * A ** db
    gen = torch.Generator(device=dev).manual_seed(5)
    b_R = torch.randint(-1, 2, (LB,), device=dev, generator=gen).float() * 0.99
    b_q = torch.rand(LB, device=dev, generator=gen)
    b_q0, b_r1, b_m1 = (torch.rand(nb * A, device=dev, generator=gen) for _ in range(3))
    b_act = torch.empty(nb, dtype=torch.int32, device=dev)
    b_val = torch.empty(nb * A, dtype=torch.float32, device=dev)
    ops["backup"] = (lambda: bcts.bcts_backup(b_R, b_q, b_q0, b_r1, b_m1, nb, A, db, 0.99, 1.0, b_act, b_val,
                                              stream=stream),
                     LB * 8 + nb * A * (3 * 4 + 4) + nb * 4, nb, "decisions")
    pk, pk_kind = peaks()
    out = {}
    with torch.cuda.stream(stream):
        with ClockSampler(local) as clk:
            for name, (fn, nbytes, units, unit_name) in ops.items():
                for _ in range(warmup):
                    fn()
                stream.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
                barrier(world)
                for i in range(reps):
                    ev[i][0].record(stream)
                    fn()
                    ev[i][1].record(stream)
                stream.synchronize()
                ms = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in ev) / reps, dev)
                ach = nbytes / (ms / 1e3) / 1e9
                out[name] = {"avg_launch_ms": ms, "algorithmic_bytes_per_launch": nbytes, "units_per_launch": units,
                             "unit": unit_name, "rate_per_s": world * units / (ms / 1e3),
                             "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                          "frac": ach / pk["hbm_gbs"],
                                          "peak_note": f"STREAM-style copy bandwidth (of {pk_kind})"}}
    del d_child, d_frames, b_R, b_q
    return {"kernels": out, "parents": P, "A": A, "render_states": F, "backup_leaves": LB, "reps": reps,
            "clocks": clk.summary(pk.get("sm_max_mhz", 2032.0))}


def run_stream(args, wl):
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(torch.device("cuda", local))
    from paper_2107_01715_b300 import bcts
    m = stream_measure(bcts, torch, wl, args.warmup, args.steps, args.roots, rank, local, world)
    if rank != 0:
        return
    e = m["kernels"]["expand"]
    line = {"metric": "expansion children/s, render frame stacks/s and backup decisions/s (the search's HBM-bound "
                      "kernels alone)",
            "value": e["rate_per_s"], "unit": "children/s", "n_gpus": world, "steps": m["reps"],
            "warmup": args.warmup, "ms_per_step": e["avg_launch_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int16 states, uint8 frames, f32 values", "data": "synthetic",
            "config": {"workload": wl["name"], "parents": m["parents"], "A": m["A"], "render_states": m["render_states"],
                       "backup_leaves": m["backup_leaves"],
                       "l2": "no flush: every launch reads and writes more than the 126 MB L2"},
            "roofline": dict(e["roofline"], kernel="expand_kernel"), "kernels": m["kernels"],
            "gpu_launches": 4 * (m["reps"] + args.warmup), "clocks": m["clocks"], "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_sweep(args, wl):
    """Device time of one decision (one root, whole Batch-BFS search) per depth, for the
    sprite world (FP32-class) and the DNN forward model (FP32), with the FP64 oracle's
    depth-first search on the host cores where it finishes in seconds."""
    import torch
    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2107_01715_b300 import bcts
    import oracle
    oracle.build()
    stream = torch.cuda.Stream(device=dev)
    reps = max(args.steps, 3)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(2):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / reps

    rows = []
    A = 18
    W = inputs.qnet_weights(A, seed=1234)
    roots = inputs.root_states([0])
    d_roots = torch.from_numpy(roots.view(np.uint8).copy()).to(dev)
    d_act = torch.empty(1, dtype=torch.int32, device=dev)
    d_val = torch.empty(64, dtype=torch.float32, device=dev)
    def host_ms(fn):
        for _ in range(3):  # eager, captured, replayed
            fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return 1e3 * (time.perf_counter() - t0) / reps

    for d in range(1, 6):
        ctx = bcts.bcts_create(W, A, d, 0.99, 1.0, precision="fp32")
        ms = timed(lambda: bcts.bcts_search_device(ctx, d_roots, 1, d_act, d_val, stream))
        hms = host_ms(lambda: bcts.bcts_search(ctx, roots))
        ctx.close()
        cpu = None
        if d <= 3:
            t0 = time.perf_counter()
            oracle.search(roots, W, A, d, float(np.float32(0.99)), 1.0)
            cpu = 1e3 * (time.perf_counter() - t0)
        rows.append({"env": "sprite", "A": A, "d": d, "leaves": A ** d, "gpu_ms": ms, "host_api_ms": hms,
                     "oracle_dfs_ms": cpu})
    for A, depths in ((2, range(2, 17, 2)), (10, range(1, 7))):
        Wd = inputs.dnn_weights(A)
        r = inputs.dnn_root_states([0])
        d_r = torch.from_numpy(r).to(dev)
        for d in depths:
            ctx = bcts.bcts_dnn_create(Wd, A, d, 0.99, 1.0)
            ms = timed(lambda: bcts.bcts_dnn_search_device(ctx, d_r, 1, d_act, d_val, stream))
            ctx.close()
            cpu = None
            if A ** d <= 20000:
                t0 = time.perf_counter()
                oracle.dnn_search(r, Wd, A, d, float(np.float32(0.99)), 1.0)
                cpu = 1e3 * (time.perf_counter() - t0)
            rows.append({"env": "dnn", "A": A, "d": d, "leaves": A ** d, "gpu_ms": ms, "oracle_dfs_ms": cpu})
    if rank != 0:
        return
    big = rows[4]  # sprite world, d = 5: the largest single-root search of the sweep
    line = {"metric": METRIC, "value": big["leaves"] / (big["gpu_ms"] / 1e3), "unit": "leaf nodes/s",
            "n_gpus": world, "steps": reps, "warmup": 2, "ms_per_step": big["gpu_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES["fp32"], "data": "synthetic",
            "config": {"workload": wl["name"], "value_is": "sprite world, A=18, d=5, one root"},
            "sweep": rows, "cpu_baseline": {"kind": "oracle", "cores": oracle.threads(),
                                            "sample": "the oracle's DFS per depth where it finishes in seconds"}}
    print(json.dumps(line), flush=True)


def run_reference(args, wl):
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    W = inputs.qnet_weights(wl["A"], seed=1234)
    times = []
    cb = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(W, wl)
        if i >= args.warmup:
            times.append(wl["A"] ** wl["d"] / r["value"])
            cb = r
    total = sum(times)
    leaves = wl["A"] ** wl["d"] * len(times)
    value = leaves / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "leaf nodes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"] + " (oracle sample: 1 root per step)", "roots_per_step": 1,
                       "A": wl["A"], "d": wl["d"]},
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": "leaf nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Root-value tolerances per precision, |v - v_oracle| <= tol * max(|v_oracle|, 1): the
# FP32-class bound of the FP32 path; BF16 / FP8 leaf Q-networks carry their operand
# rounding (8 / 4 significant bits) through four layers.  The same figures as the tests'.
PRECISION_TOL = {"fp32": 1e-4, "bf16": 2e-2, "fp8": 8e-2}


def working_set_gb(n, A, d, precision):
    """DRAM bytes one search streams through besides the weights: the two deepest node
    levels (80-byte states + R), the parents' FP32 partial conv1 maps and one
    Q-network pass's activation maps (the library's pass: the whole level when its
    maps fit in 1/16 of the device memory, else equal passes of that size)."""
    e = {"fp32": 4, "bf16": 2, "fp8": 1}.get(precision, 4)
    leaves = n * A ** d
    parents = n * A ** max(d - 1, 0)
    per_leaf = (400 * 32 + 81 * 64 + 49 * 64) * e + 512 * 4
    try:
        import torch
        mem = torch.cuda.get_device_properties(0).total_memory if torch.cuda.is_available() else 0
    except Exception:
        mem = 0
    cap = max(32768, int((mem or 288e9) / 16) // per_leaf)
    passes = -(-leaves // cap)
    chunk = -(-leaves // passes)
    return (84 * (leaves + parents) + parents * 400 * 32 * 4 +
            chunk * per_leaf) / 1e9


def report_vs_oracle(bcts, W, wl):
    """Root values and actions of the FP32-class, BF16 and FP8 leaf Q-networks against
    the stored FP64 oracle values (written by tests/golden/make_oracle_values.py, which
    calls only the oracle): the precision workload's 8 roots at d = 4, and a separate
    line for 256 more roots at d = 2.  Errors are relative, |v - v_oracle| /
    max(|v_oracle|, 1), with the correction on (c = 1, Eq. 3) and off (c = 0, Eq. 2).
    A root's action counts towards the agreement wherever the oracle's top-2 value
    margin exceeds the precision's tolerance (PRECISION_TOL)."""
    gamma = float(np.float32(wl["gamma"]))
    out = {"tolerance": PRECISION_TOL, "vs": "stored FP64 oracle values"}
    for fname, label in (("oracle_precision8_a18_d4.json", "8 roots, A=18, d=4 (the precision form)"),
                         ("oracle_precision256_a18_d2.json", "256 roots, A=18, d=2 (additional roots)")):
        path = os.path.join(ROOT, "tests", "golden", fname)
        if not os.path.exists(path):
            out[label] = "stored oracle values missing"
            continue
        with open(path) as f:
            g = json.load(f)
        A, d, c = g["A"], g["d"], g["correction"]
        Wg = inputs.qnet_weights(A, seed=g["weights_seed"])
        roots = inputs.root_states(g["seeds"])
        ref_v = np.array([r["values"] for r in g["roots"]])
        ref_u = np.array([r["v_uncorrected"] for r in g["roots"]])
        ref_a = np.array([r["action"] for r in g["roots"]])
        srt = np.sort(ref_v, axis=1)
        margin = (srt[:, -1] - srt[:, -2]) / np.maximum(np.abs(srt[:, -1]), 1.0)
        res = {"roots": len(roots), "oracle_margin_quantiles": np.quantile(margin, [0.1, 0.5, 0.9]).tolist()}
        for prec, tol in PRECISION_TOL.items():
            vals = {}
            for cc in (c, 0.0):
                cx = bcts.bcts_create(Wg, A, d, gamma, cc, precision=prec)
                vals[cc] = bcts.bcts_search(cx, roots)
                cx.close()
            act, v1 = vals[c]
            _, v0 = vals[0.0]
            e1 = np.abs(v1 - ref_v) / np.maximum(np.abs(ref_v), 1.0)
            e0 = np.abs(v0 - ref_u) / np.maximum(np.abs(ref_u), 1.0)
            counted = margin > tol
            res[prec] = {"max_rel_err_c1": float(e1.max()), "p99_rel_err_c1": float(np.quantile(e1, 0.99)),
                         "mean_rel_err_c1": float(e1.mean()), "max_rel_err_c0": float(e0.max()),
                         "within_tolerance": bool((e1 <= tol).all() and (e0 <= tol).all()),
                         "roots_with_margin_above_tol": int(counted.sum()),
                         "action_agreement_where_margin_above_tol":
                             float((act[counted] == ref_a[counted]).mean()) if counted.any() else None,
                         "action_agreement_all_roots": float((act == ref_a).mean())}
        out[label] = res
    return out


def run_ours(args, wl):
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2107_01715_b300 import bcts
    precision = args.precision or wl["precision"]
    n, A, d = wl["n"], wl["A"], wl["d"]
    W = inputs.qnet_weights(A, seed=1234)
    ctx = bcts.bcts_create(W, A, d, wl["gamma"], wl["c"], precision=precision,
                           flags=bcts.BCTS_FLAG_FRAMES if args.frames else 0)
    roots = inputs.root_states(range(rank * n, rank * n + n))  # each rank its own roots
    d_roots = torch.from_numpy(roots.view(np.uint8).copy()).to(dev)
    d_act = torch.empty(n, dtype=torch.int32, device=dev)
    d_val = torch.empty(n * A, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    leaves = n * A ** d

    def step():
        bcts.bcts_search_device(ctx, d_roots, n, d_act, d_val, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):  # eager, then captured into a CUDA graph by the library
            step()
        stream.synchronize()
        bcts.bcts_profile(ctx, False)  # reset the launch count; recording off (the user's path)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            t_wall0 = time.perf_counter()
            for i in range(args.steps):
                flush.zero_()  # L2 flush between steps, outside the timed events
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            stream.synchronize()
            t_wall = time.perf_counter() - t_wall0
        torch.cuda.synchronize()
        barrier(world)
        _, _, launches = bcts.bcts_profile(ctx, True)  # timed-region launches; record from here
        # a second pass of the same steps with per-kernel events (eager) for the roofline
        for i in range(args.steps):
            flush.zero_()
            step()
        stream.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    prof_ms, prof_cnt, _ = bcts.bcts_profile(ctx, False)
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(world, total_s, dev)
    value = world * leaves * args.steps / total_s
    decisions = world * n * args.steps / total_s

    # end to end: host roots in, host actions + values out, every step
    e2e_times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        act, val = bcts.bcts_search(ctx, roots)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_times.append(dt)
    e2e_total = max_over_ranks(world, sum(e2e_times), dev)
    e2e_value = world * leaves * args.steps / e2e_total

    if rank != 0:
        ctx.close()
        return

    pk, pk_kind = peaks()
    # dominant kernel class by device time inside the timed region
    dom = max(prof_ms, key=lambda k: prof_ms[k])
    roofline = None
    if prof_ms[dom] > 0:
        nodes = args.steps * class_nodes(dom, n, A, d, prof_cnt)
        roofline = roofline_for(dom, precision, A, nodes, prof_ms[dom], prof_cnt[dom], pk, pk_kind)
    plain = None
    if not args.no_plain and precision != "fp32_simt":
        # the plain FP32 method: CUDA-core Q-network, one root per launch
        pctx = bcts.bcts_create(W, A, d, wl["gamma"], wl["c"], precision="fp32_simt")
        one = [d_roots[i * 80:(i + 1) * 80] for i in range(n)]
        with torch.cuda.stream(stream):
            bcts.bcts_search_device(pctx, one[0], 1, d_act, d_val, stream)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(n):
                bcts.bcts_search_device(pctx, one[i], 1, d_act[i:i + 1], d_val[i * A:(i + 1) * A], stream)
            e1.record(stream)
            stream.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": leaves / (pms / 1e3), "unit": "leaf nodes/s", "ms_per_step": pms,
                 "how": "FP32 CUDA-core Q-network, one root per bcts_search_device call, same roots"}
        pctx.close()

    cb = None
    if not args.no_cpu_baseline:
        cb = cpu_baseline(W, wl)

    precision_report = None
    if args.workload == "precision":
        precision_report = report_vs_oracle(bcts, W, wl)
    forms = None
    if args.workload == "atari" and not args.no_extras and not args.frames and args.roots is None:
        forms = forms_measure(bcts, torch, wl)

    lat = sorted(step_ms)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]
    clocks = clk.summary(pk.get("sm_max_mhz"))
    line = {
        "metric": METRIC, "value": value, "unit": "leaf nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES.get(precision, precision),
        "data": "synthetic",
        "config": {"workload": wl["name"], "roots_per_step": n, "A": A, "d": d, "gamma": wl["gamma"],
                   "correction": wl["c"], "leaves_per_step": leaves, "precision": precision,
                   "l2": "flushed between steps (256 MB write); per-step DRAM working set "
                         f"{working_set_gb(n, A, d, precision):.2f} GB (node levels, partial conv1 maps, "
                         "one leaf chunk's activation maps) > 126 MB L2"},
        "decisions_per_s": decisions,
        "latency_ms": {"p50": p50, "p99": p99, "what": f"one search of the {n}-root batch, device time"},
        "e2e": {"value": e2e_value, "unit": "leaf nodes/s", "h2d_bytes_per_step": int(n * 80),
                "d2h_bytes_per_step": int(n * 4 + n * A * 4),
                "ms_per_step": 1e3 * e2e_total / args.steps},
        "gpu_launches": launches,
        "kernel_ms": prof_ms, "kernel_launches": prof_cnt,
        "roofline": roofline,
        "plain_fp32": plain,
        "speedup_vs_plain_fp32": (value / plain["value"]) if plain else None,
        "cpu_baseline": cb,
        "precision_report": precision_report,
        "forms": forms,
        "clocks": clocks,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def _clock_line(clk, pk):
    return clk.summary(pk.get("sm_max_mhz"))


def batched_measure(bcts, wl, precision, steps, warmup, rank=0, local=0, world=1):
    """Batched form: one bcts_search_mixed call per step over 256 mixed roots (d uniform
    in {1,2,3,4}, |A| in {4,9,18}); host wall clock per call, inputs and outputs
    through host memory."""
    W = inputs.qnet_weights(18, seed=1234)
    ctx = bcts.bcts_create(W, 18, 4, wl["gamma"], wl["c"], precision=precision)
    roots, ds, As = inputs.mixed_roots(wl["n"], seed=7 + rank)
    leaves = int(sum(int(a) ** int(d) for a, d in zip(As, ds)))
    for _ in range(warmup):
        bcts.bcts_search_mixed(ctx, roots, ds, As)  # eager, tuned, captured, then replayed
    bcts.bcts_profile(ctx, False)
    pk, _ = peaks()
    barrier(world)
    with ClockSampler(local) as clk:
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            bcts.bcts_search_mixed(ctx, roots, ds, As)
            times.append(time.perf_counter() - t0)
    _, _, launches = bcts.bcts_profile(ctx, False)
    ctx.close()
    lat = sorted(times)
    return {"leaves_per_step": leaves, "roots_per_step": wl["n"], "precision": precision, "steps": steps,
            "total_s": sum(times), "leaf_nodes_per_s": leaves * steps / sum(times),
            "decisions_per_s": wl["n"] * steps / sum(times),
            "depth_hist": {str(k): int((ds == k).sum()) for k in (1, 2, 3, 4)},
            "A_hist": {str(k): int((As == k).sum()) for k in (4, 9, 18)},
            "latency_ms": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[-1],
                           "what": "one bcts_search_mixed call of the 256-root batch, host wall clock"},
            "gpu_launches": launches, "clocks": _clock_line(clk, pk)}


def run_batched(args, wl):
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_2107_01715_b300 import bcts
    precision = args.precision or wl["precision"]
    m = batched_measure(bcts, wl, precision, args.steps, args.warmup, rank, local, world)
    total = max_over_ranks(world, m["total_s"], torch.device("cuda", local))
    if rank == 0:
        leaves = m["leaves_per_step"]
        line = {"metric": METRIC, "value": world * leaves * args.steps / total, "unit": "leaf nodes/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": precision, "data": "synthetic",
                "config": {"workload": wl["name"], "roots_per_step": wl["n"], "leaves_per_step": leaves,
                           "depth_hist": m["depth_hist"], "A_hist": m["A_hist"],
                           "l2": f"{leaves} leaves per step, working set far above the 126 MB L2"},
                "decisions_per_s": world * wl["n"] * args.steps / total, "latency_ms": m["latency_ms"],
                "e2e": {"value": world * leaves * args.steps / total, "unit": "leaf nodes/s",
                        "h2d_bytes_per_step": wl["n"] * 80, "d2h_bytes_per_step": wl["n"] * (4 + 18 * 4)},
                "gpu_launches": m["gpu_launches"], "clocks": m["clocks"]}
        print(json.dumps(line), flush=True)


def search_measure(bcts, torch, W, A, d, n, gamma, c, precision, steps, warmup, flags=0, seed0=0):
    """Device-time throughput of bcts_search_device over n seeded roots (inputs in
    device memory, L2 flushed between steps), with per-kernel-class time from a
    second, profiled pass."""
    ctx = bcts.bcts_create(W, A, d, gamma, c, precision=precision, flags=flags)
    roots = inputs.root_states(range(seed0, seed0 + n))
    d_roots = torch.from_numpy(roots.view(np.uint8).copy()).cuda()
    d_act = torch.empty(n, dtype=torch.int32, device="cuda")
    d_val = torch.empty(n * A, dtype=torch.float32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for _ in range(warmup):
            bcts.bcts_search_device(ctx, d_roots, n, d_act, d_val, st)
        st.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(st)
            bcts.bcts_search_device(ctx, d_roots, n, d_act, d_val, st)
            ev[i][1].record(st)
        st.synchronize()
        bcts.bcts_profile(ctx, True)
        for i in range(steps):
            flush.zero_()
            bcts.bcts_search_device(ctx, d_roots, n, d_act, d_val, st)
        st.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    kms, kcnt, _ = bcts.bcts_profile(ctx, False)
    ctx.close()
    leaves = n * A ** d
    return {"leaf_nodes_per_s": leaves * steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
            "decisions_per_s": n * steps / (sum(ms) / 1e3), "leaves_per_step": leaves, "steps": steps,
            "kernel_ms_per_step": {k: v / steps for k, v in kms.items() if v > 0},
            "kernel_launches_per_step": {k: v / steps for k, v in kcnt.items() if v > 0}}


def forms_measure(bcts, torch, wl_default):
    """The other configurations the metric names, measured in the default run so that
    they appear on its line: the frame path of the headline workload, the precision
    form (8 roots, A = 18, d = 4) in BF16 / FP8 / FP32-class with its report against
    the stored oracle values, the batched form, the serving form at a rate below
    saturation, and the streaming kernels (expansion, renderer, backup) alone."""
    out = {}
    pk, pk_kind = peaks()
    g, cc = wl_default["gamma"], wl_default["c"]
    W18 = inputs.qnet_weights(18, seed=1234)
    # frame path: every node's frame rendered to device memory, conv1 on the tensor cores
    fp = search_measure(bcts, torch, W18, 18, 3, 32, g, cc, "fp32", 20, 3, flags=bcts.BCTS_FLAG_FRAMES)
    # frames it renders per step: the roots' stacks, then every inner node's and leaf's newest frame
    fr_bytes = 32 * 28224 + sum(32 * 18 ** i for i in range(1, 4)) * 7056
    rms = fp["kernel_ms_per_step"].get("render", 0.0)
    fp["render_in_search"] = {"bytes_written_per_step": fr_bytes, "ms_per_step": rms,
                              "gbs": fr_bytes / (rms / 1e3) / 1e9 if rms else None,
                              "frac_of_copy_bandwidth": fr_bytes / (rms / 1e3) / 1e9 / pk["hbm_gbs"] if rms else None}
    fp["what"] = ("the headline workload (32 roots, A=18, d=3, FP32-class) with BCTS_FLAG_FRAMES: node frames "
                  "rendered per level, conv1 as tcgen05 GEMMs over them (roots / depth-1 whole stacks, parents' "
                  "partial maps, leaves' newest slot)")
    out["frame_path"] = fp
    # precision form: 8 roots, A = 18, d = 4
    wp = WORKLOADS["precision"]
    prec = {}
    for p in ("bf16", "fp8", "fp32"):
        prec[p] = search_measure(bcts, torch, W18, 18, wp["d"], wp["n"], g, cc, p, 10, 3)
    prec["vs_oracle"] = report_vs_oracle(bcts, W18, wp)
    out["precision_form"] = prec
    # batched form
    out["batched_form"] = batched_measure(bcts, WORKLOADS["batched"], "bf16", 5, 3)
    # serving form, below saturation
    ws = WORKLOADS["serving"]
    out["serving_form"] = serving_measure(bcts, ws, "bf16", 300.0, 2.0)
    # the streaming kernels alone (a quarter of the stream workload's sizes)
    out["streaming_kernels"] = stream_measure(bcts, torch, dict(WORKLOADS["stream"], n=1 << 18, frames=25_000,
                                                                backup_roots=256), 2, 10)
    return out


def serving_measure(bcts, wl, precision, rate, seconds, rank=0, local=0, world=1):
    """Serving form: Poisson arrivals from simulated episodes through bcts_submit /
    bcts_poll; episodes advance by the returned action (bcts_env_step).  Returns the
    measurement (decisions/s, leaf nodes/s, p50/p99 latency, the plain FP32
    one-request-at-a-time baseline on a bounded sample, launches, clocks)."""
    A = 18
    W = inputs.qnet_weights(A, seed=1234)
    ctx = bcts.bcts_create(W, A, 4, wl["gamma"], wl["c"], precision=precision,
                           frame_budget_bytes=wl["budget"], max_roots=64)
    episodes = inputs.root_states(range(10000 + rank * wl["n"], 10000 + rank * wl["n"] + wl["n"]))
    g = inputs.splitmix64(4242 + rank)

    def uniform():
        return (next(g) >> 11) / float(1 << 53)

    # warm-up: every depth alone, then two full-size mixed bursts, so that both
    # workers have sized their buffers before the clock
    for d in (2, 3, 4):
        t = bcts.bcts_submit(ctx, episodes[:1], d, A)
        bcts.bcts_poll(ctx, t, A, timeout_us=-1)
    for _ in range(2):
        tks = [bcts.bcts_submit(ctx, episodes[i:i + 1], (2, 3, 4)[i % 3], A) for i in range(256)]
        for t in tks:
            bcts.bcts_poll(ctx, t, A, timeout_us=-1)
    bcts.bcts_profile(ctx, False)  # reset the launch counters (owner and serving workers)
    busy = set()
    pending = {}  # ticket -> (episode, submit time)
    lat, done_leaves, completed = [], 0, 0
    t0 = time.perf_counter()
    next_arrival = t0
    pk, _ = peaks()
    barrier(world)
    with ClockSampler(local) as clk:
        while True:
            now = time.perf_counter()
            # an arrival needs an idle episode; while every episode waits for its
            # decision, arrivals are deferred (their latency still counts from the
            # scheduled arrival time)
            while next_arrival <= now and next_arrival - t0 < seconds and len(busy) < wl["n"]:
                e = int(next(g) % wl["n"])
                while e in busy:
                    e = (e + 1) % wl["n"]
                d = (2, 3, 4)[next(g) % 3]
                tk = bcts.bcts_submit(ctx, episodes[e:e + 1], d, A)
                pending[tk] = (e, next_arrival, d)
                busy.add(e)
                next_arrival += -np.log(1.0 - uniform()) / rate
            # passes complete roughly in arrival order: poll the oldest tickets and
            # stop after a run of still-pending ones
            misses = 0
            for tk in list(pending):
                rc, a, _ = bcts.bcts_poll(ctx, tk, A, timeout_us=0)
                if rc == bcts.BCTS_OK:
                    e, ts, d = pending.pop(tk)
                    lat.append(time.perf_counter() - ts)
                    done_leaves += A ** d
                    completed += 1
                    episodes[e], _ = bcts.bcts_env_step(episodes[e], a)
                    busy.discard(e)
                else:
                    misses += 1
                    if misses >= 192:
                        break
            if next_arrival - t0 >= seconds and not pending:
                break
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
    _, _, served_launches = bcts.bcts_profile(ctx, False)
    ctx.close()
    # plain FP32 sequential baseline on a bounded sample of the same kind of requests
    pctx = bcts.bcts_create(W, A, 4, wl["gamma"], wl["c"], precision="fp32_simt")
    seq_roots = inputs.root_states(range(20000, 20012))
    tseq0 = time.perf_counter()
    seq_leaves = 0
    for i in range(len(seq_roots)):
        d = (2, 3, 4)[i % 3]
        bcts.bcts_search_mixed(pctx, seq_roots[i:i + 1], np.array([d], np.int32), np.array([A], np.int32))
        seq_leaves += A ** d
    tseq = time.perf_counter() - tseq0
    pctx.close()
    lat.sort()
    return {"offered_rate_req_s": rate, "arrival_seconds": seconds, "episodes": wl["n"], "precision": precision,
            "decisions": completed, "wall_s": wall, "decisions_per_s": completed / wall,
            "leaf_nodes_per_s": done_leaves / wall,
            "latency_ms": {"p50": 1e3 * lat[len(lat) // 2] if lat else None,
                           "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
                           "what": "submit to completion seen by the poller, host wall clock"},
            "plain_fp32_sequential": {"decisions_per_s": len(seq_roots) / tseq,
                                      "leaf_nodes_per_s": seq_leaves / tseq,
                                      "how": "one request at a time, FP32 CUDA-core Q-network, d cycling 2,3,4"},
            "gpu_launches": served_launches, "clocks": _clock_line(clk, pk)}


def run_serving(args, wl):
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_2107_01715_b300 import bcts
    precision = args.precision or wl["precision"]
    m = serving_measure(bcts, wl, precision, args.rate or wl["rate"], args.seconds or wl["seconds"], rank, local,
                        world)
    if rank == 0:
        line = {"metric": METRIC, "value": m["decisions_per_s"], "unit": "decisions/s", "n_gpus": world,
                "steps": m["decisions"], "warmup": 3, "ms_per_step": 1e3 * m["wall_s"] / max(m["decisions"], 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": precision,
                "data": "synthetic",
                "config": {"workload": wl["name"], "offered_rate_req_s": m["offered_rate_req_s"],
                           "arrival_seconds": m["arrival_seconds"], "episodes": wl["n"]},
                "leaf_nodes_per_s": m["leaf_nodes_per_s"], "latency_ms": m["latency_ms"],
                "plain_fp32_sequential": m["plain_fp32_sequential"],
                "e2e": {"value": m["decisions_per_s"], "unit": "decisions/s", "h2d_bytes_per_step": 80,
                        "d2h_bytes_per_step": 4 + 18 * 4},
                "gpu_launches": m["gpu_launches"], "clocks": m["clocks"]}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    wl = dict(WORKLOADS[args.workload])
    if args.roots:
        wl["n"] = args.roots
        wl["name"] += f" [reduced to {args.roots} roots]"
    if args.impl == "reference":
        run_reference(args, wl)
    elif args.workload == "batched":
        run_batched(args, wl)
    elif args.workload == "serving":
        run_serving(args, wl)
    elif args.workload == "dnn":
        run_dnn(args, wl)
    elif args.workload == "pruned":
        run_pruned(args, wl)
    elif args.workload == "sweep":
        run_sweep(args, wl)
    elif args.workload == "stream":
        run_stream(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
