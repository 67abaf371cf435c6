"""Benchmark of the cone-beam operators (forward projection, matched adjoint, voxel-driven BP).

Workload: 256^3 FP32 random-ellipsoid phantom (20 ellipsoids, 0.5 mm voxels), circular cone beam,
360 views over 2 pi, SID 750 mm, SDD 1200 mm, 512 x 512 detector with 0.6 mm pixels.

One step = A x (forward projection), A^T r (matched adjoint of a random cotangent) and the
voxel-driven back-projection of the sinogram, all FP32, inputs resident in HBM. The sinogram
(377 MB) exceeds L2; the volume (64 MiB) does not, so L2 is flushed (256 MiB write) before every
timed step. Every kernel is timed with CUDA events on the launching stream.

  value            forward projection throughput, G ray-samples/s (samples inside the support box)
  bp_gupdates      voxel-driven BP throughput, G voxel-view updates/s
  fwd_adj_ms       forward + adjoint time per iteration, ms
  e2e              forward projection through the C ABI with host buffers (copies timed)

`--impl reference` times the FP64 CPU oracle on bounded samples of the same workload.
With torchrun (N > 1) every rank projects its own volume (independent problems, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="cone-beam 256^3 circular, 360 views, 512x512 detector", volume=[256, 256, 256],
                voxel_mm=0.5, views=360, angular_range="2pi", sid_mm=750.0, sdd_mm=1200.0, detector=[512, 512],
                pixel_mm=0.6, phantom="20 random ellipsoids, seed 3", dt_mm=0.25)
METRIC = "cone-beam FP G ray-samples/s and BP G voxel-view updates/s; fwd+adjoint ms/iter"
# Algorithmic work per unit (FP32 operations counted as FLOP, an FMA as 2):
FP_FLOP_PER_SAMPLE = 34     # 3 position FMA (6), 3 floor + 3 frac (6), 7 lerps (21), accumulate (1)
FP_SMEM_BYTES_PER_SAMPLE = 32   # eight FP32 interpolation operands
ADJ_FLOP_PER_SAMPLE = 33    # 3 position FMA (6), 3 frac (3), 1 - a (2), z split (2), 12 weight products, 8 adds
ADJ_RED_PER_SAMPLE = 8      # one scatter-add per trilinear corner
BP_FLOP_PER_UPDATE = 18     # projection 3 FMA (6), reciprocal and 2 products (3), 3 bilinear lerps (6), weight, add
# On-chip rates per clock per SM measured on GB300 (2070 MHz) with
# python -m paper_2511_08427_gb300.peaks (every lane of 4 CTAs x 256 threads per SM, distinct banks or
# one cache line per warp request):
SMEM_RED_PER_CLK_SM = 28.32        # int32 red.shared.add
SMEM_LD_BYTES_PER_CLK_SM = 4 * 27.66   # 32-bit ld.shared
L1_LDG_PER_CLK_SM = 17.2           # 32-bit global loads hitting L1 (read-only path), one line per warp request
BP_LOADS_PER_UPDATE = 4            # bilinear detector operands


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, world: int, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(units_per_rank: float, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput in G units/s: every rank processed units_per_rank per step."""
    return world * units_per_rank * steps / seconds / 1e9


def build_inputs(seed_vol=3):
    from paper_2511_08427_gb300 import inputs
    vol = inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 64.0, seed_vol), (256, 256, 256),
                                      (0.5, 0.5, 0.5))
    return vol


def make_geometry():
    from paper_2511_08427_gb300.operators import Geometry
    return Geometry.cone_circular((256, 256, 256), (0.5, 0.5, 0.5), (512, 512), (0.6, 0.6), 360, 2 * math.pi,
                                  750.0, 1200.0)


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ------------------------------------------------------------------------------------------------

def oracle_sample_rate(vol, n_views: int, target_s: float = 10.0):
    """Time the FP64 oracle forward projection on the first views of the workload.
    Returns (G samples/s, samples, seconds, threads, views used)."""
    import oracle
    og_full = oracle.cone_circular((256, 256, 256), (0.5, 0.5, 0.5), (512, 512), (0.6, 0.6), 360, 2 * math.pi,
                                   750.0, 1200.0)
    threads = oracle.max_threads()
    v = np.ascontiguousarray(vol, dtype=np.float64)

    def sub(nv, start=0):
        idx = [(start + 7 * i) % 360 for i in range(nv)]
        return oracle.Geometry(og_full.vol_shape, og_full.vol_spacing, og_full.vol_offset, og_full.det_shape,
                               og_full.det_spacing, og_full.det_offset, 1, og_full.views[idx], og_full.dt)

    # detector rows subset to keep a call bounded: 1 view at a time, scaled by measured time
    g1 = sub(1)
    t0 = time.perf_counter()
    oracle.fp(g1, v)
    t1 = time.perf_counter() - t0
    nv = max(1, min(n_views, int(target_s / max(t1, 1e-3))))
    g = sub(nv, start=1)
    t0 = time.perf_counter()
    oracle.fp(g, v)
    dt = time.perf_counter() - t0
    samples = int(oracle.count_samples(g).sum())
    return samples / dt / 1e9, samples, dt, threads, nv


def oracle_single_core_rate(vol):
    """The FP64 oracle on one thread: forward projection of one view of the workload (a few seconds).
    Returns (G samples/s, samples, seconds)."""
    import oracle
    og = oracle.cone_circular((256, 256, 256), (0.5, 0.5, 0.5), (512, 512), (0.6, 0.6), 360, 2 * math.pi,
                              750.0, 1200.0)
    g = oracle.Geometry(og.vol_shape, og.vol_spacing, og.vol_offset, og.det_shape, og.det_spacing, og.det_offset,
                        1, og.views[[3]], og.dt)
    v = np.ascontiguousarray(vol, dtype=np.float64)
    n_all = oracle.max_threads()
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.fp(g, v)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(n_all)
    samples = int(oracle.count_samples(g).sum())
    return samples / dt / 1e9, samples, dt


def single_core_entry(vol):
    rate, s, dt = oracle_single_core_rate(vol)
    return {"value": rate, "unit": "G ray-samples/s", "cores": 1,
            "sample": f"FP64 oracle forward projection of 1 of 360 views on one thread ({s} samples, {dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vol = build_inputs()
    times, samples = [], []
    per_step = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    # every step times the oracle on a bounded sample (a few views) of the same workload
    for i in range(args.warmup + args.steps):
        rate, s, dt, threads, nv = oracle_sample_rate(vol, 64, target_s=per_step)
        if i >= args.warmup:
            times.append(dt)
            samples.append(s)
    value = sum(samples) / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "G ray-samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, kernel="FP64 CPU oracle, forward projection"),
            "cpu_baseline": {"value": value, "unit": "G ray-samples/s", "cores": threads, "kind": "oracle",
                             "sample": f"forward projection of {nv} views per step (of 360), full detector",
                             "single_core": single_core_entry(vol)},
            "e2e": {"value": value, "unit": "G ray-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def kernel_traffic(kernel: str, source: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, source), "rb") as f:
            digest = hashlib.sha1(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    return rec.get("dram_bytes_per_launch") if rec.get("source_sha1") == digest else None


def run_batched(dev, K: int = 3):
    """16 volumes of uneven sizes (96^3 ... 256^3, circular / helical orbits, 180-540 views, 256^2-512^2
    detectors) in one persistent launch per operator, FP32 and BF16 storage, plain and CUDA-graph replay."""
    import torch
    from paper_2511_08427_gb300 import inputs, operators as ops
    specs = inputs.batched_cone_workload()
    geoms, vols = [], []
    for w in specs:
        n = w["side"]
        geoms.append(ops.Geometry.cone_circular((n, n, n), (w["voxel_mm"],) * 3, (w["det"], w["det"]),
                                                (w["du"], w["du"]), w["views"], w["angular_range"], w["sid"],
                                                w["sdd"], helical_pitch=w["pitch"]))
        vols.append(inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 0.5 * n * w["voxel_mm"], w["seed"]),
                                                (n, n, n), (w["voxel_mm"],) * 3))
    samples = sum(g.count_samples() for g in geoms)
    out = {"workload": "16 cone-beam volumes 96^3..256^3, circular/helical, 180-540 views, 256^2-512^2 detectors",
           "samples_per_fp": samples}
    stream = torch.cuda.current_stream(dev)
    for dtype, tag in ((torch.float32, "f32"), (torch.bfloat16, "bf16")):
        plan = ops.Plan(geoms, dtype=dtype)
        xs = [torch.from_numpy(v).to(dev).to(dtype) for v in vols]
        sinos = [torch.empty(g.sinogram_shape, device=dev, dtype=dtype) for g in geoms]
        adj = [torch.empty(g.volume_shape, device=dev, dtype=dtype) for g in geoms]
        plan.forward_project(xs, sinos)
        plan.adjoint(sinos, adj)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        for _ in range(K):
            plan.forward_project(xs, sinos)
        ev[1].record(stream)
        for _ in range(K):
            plan.adjoint(sinos, adj)
        ev[2].record(stream)
        torch.cuda.synchronize()
        fp_ms = ev[0].elapsed_time(ev[1]) / K
        adj_ms = ev[1].elapsed_time(ev[2]) / K
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                plan.forward_project(xs, sinos)
                plan.adjoint(sinos, adj)
        stream.wait_stream(side)
        graph.replay()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(K):
            graph.replay()
        ev[1].record(stream)
        torch.cuda.synchronize()
        out[tag] = {"fp_ms": fp_ms, "adjoint_ms": adj_ms, "fp_gsamples_per_s": samples / (fp_ms * 1e-3) / 1e9,
                    "graph_fwd_adj_ms": ev[0].elapsed_time(ev[1]) / K, "grids": plan.info()["grids"]}
        del plan, xs, sinos, adj, graph
    return out

def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2511_08427_gb300 import _lib, operators as ops

    vol_np = build_inputs(seed_vol=3 + rank)
    g = make_geometry()
    # slab depth / buffer count chosen by the project's autotuner (cached per device and geometry)
    from paper_2511_08427_gb300 import autotune
    tuned = autotune.tune_forward(g)
    n_samples = g.count_samples()
    n_updates = 256 ** 3 * 360
    vol = torch.from_numpy(vol_np).to(dev)
    sino = torch.empty((360, 512, 512), device=dev)
    cot = torch.randn((360, 512, 512), device=dev, generator=torch.Generator(device=dev).manual_seed(22))
    adj = torch.empty_like(vol)
    bpv = torch.empty_like(vol)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        flush.fill_(1.0)
        if ev:
            ev[0].record(stream)
        ops.forward_project(vol, g, out=sino)
        if ev:
            ev[1].record(stream)
        ops.adjoint(cot, g, out=adj)
        if ev:
            ev[2].record(stream)
        ops.back_project(sino, g, out=bpv)
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            step(evs[i])
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    fp_ms = np.array([e[0].elapsed_time(e[1]) for e in evs])
    adj_ms = np.array([e[1].elapsed_time(e[2]) for e in evs])
    bp_ms = np.array([e[2].elapsed_time(e[3]) for e in evs])
    total_ms, fp_sum, adj_sum, bp_sum = max_over_ranks([total_ms, fp_ms.sum(), adj_ms.sum(), bp_ms.sum()], world, dev)
    K = args.steps
    fp_rate = job_rate(n_samples, world, K, fp_sum * 1e-3)
    bp_rate = job_rate(n_updates, world, K, bp_sum * 1e-3)

    # one gradient-descent iteration x <- x - alpha A^T (A x - p) on this workload, from x = 0.9 x_true:
    # unfused (projection, residual, adjoint, axpy) and fused (projection + pyronn_adjoint_update)
    p_meas = sino.clone()
    x_it = torch.zeros_like(vol)
    alpha_gd = 1e-4

    def gd_unfused():
        ops.forward_project(x_it, g, out=sino)
        ops.adjoint(sino - p_meas, g, out=adj)
        x_it.add_(adj, alpha=-alpha_gd)

    def gd_fused():
        ops.forward_project(x_it, g, out=sino)
        ops.adjoint_update(x_it, sino, g, -alpha_gd, sino_b=p_meas)

    gd_ms = {}
    for name, fn in (("unfused", gd_unfused), ("fused", gd_fused)):
        x_it.copy_(vol).mul_(0.9)   # both variants iterate from the same iterate
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(max(2, K // 2)):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        gd_ms[name] = e0.elapsed_time(e1) / max(2, K // 2)
    del p_meas, x_it

    def time_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # BF16 storage (FP32 arithmetic) forward projection of the same workload, and the FBP filter
    vol_bf, sino_bf = vol.bfloat16(), torch.empty(sino.shape, device=dev, dtype=torch.bfloat16)
    fp_bf16_ms = time_ms(lambda: ops.forward_project(vol_bf, g, out=sino_bf), max(3, K // 2))
    del vol_bf, sino_bf
    fbp_out = torch.empty_like(sino)
    fbp_ms = time_ms(lambda: ops.fbp_filter(sino, g, out=fbp_out), max(3, K // 2))
    del fbp_out

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    import ctypes
    h_vol = torch.from_numpy(vol_np).pin_memory()
    h_sino = torch.empty((360, 512, 512), dtype=torch.float32).pin_memory()
    L = _lib.lib()

    def e2e_call():
        _lib.check(L.pyronn_fp_host(g.handle, ctypes.c_void_p(h_vol.data_ptr()), ctypes.c_void_p(h_sino.data_ptr()),
                                    0, 1, ctypes.c_void_p(stream.cuda_stream)))

    for _ in range(2):
        e2e_call()
    n_e2e = max(3, K // 2)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_call()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_s = max_over_ranks([e2e_s], world, dev)[0]
    e2e_rate = job_rate(n_samples, world, 1, e2e_s)

    peaks, peak_src = measured_peaks()
    clk = clocks.summary()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 ALU peak from unit counts: SMs x 128 FP32 lanes x 2 FLOP per FMA x max SM clock
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    alu_peak_tflops = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    alu_src = f"{n_sm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (unit counts, max clock)"
    smem_peak_gbs = n_sm * SMEM_LD_BYTES_PER_CLK_SM * sm_max * 1e6 / 1e9
    red_peak = n_sm * SMEM_RED_PER_CLK_SM * sm_max * 1e6 / 1e9
    fp_s, adj_s, bp_s = fp_sum / K * 1e-3, adj_sum / K * 1e-3, bp_sum / K * 1e-3

    def alu_roofline(kernel, source, flop, seconds):
        achieved = flop / seconds / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / alu_peak_tflops, "traffic": kernel_traffic(kernel, source), "kernel": kernel,
                "launch_ms": seconds * 1e3, "peak_source": alu_src}

    rl_fp = alu_roofline("fp_tma_kernel", "paper_2511_08427_gb300/csrc/k_fp_tma.cu", n_samples * FP_FLOP_PER_SAMPLE, fp_s)
    rl_fp["flop_per_sample"] = FP_FLOP_PER_SAMPLE
    smem_gbs = n_samples * FP_SMEM_BYTES_PER_SAMPLE / fp_s / 1e9
    rl_fp["smem"] = {"achieved_gbs": smem_gbs, "peak_gbs": smem_peak_gbs, "frac": smem_gbs / smem_peak_gbs,
                     "bytes_per_sample": FP_SMEM_BYTES_PER_SAMPLE,
                     "peak_source": f"{n_sm} SMs x {SMEM_LD_BYTES_PER_CLK_SM:.1f} B/clk (measured 32-bit "
                                    f"ld.shared) x {sm_max:.0f} MHz"}
    rl_adj = alu_roofline("adjoint_slab_kernel", "paper_2511_08427_gb300/csrc/k_adjoint_slab.cu",
                          n_samples * ADJ_FLOP_PER_SAMPLE, adj_s)
    rl_adj["flop_per_sample"] = ADJ_FLOP_PER_SAMPLE
    red_rate = n_samples * ADJ_RED_PER_SAMPLE / adj_s / 1e9
    rl_adj["smem_reductions"] = {"achieved_gops": red_rate, "peak_gops": red_peak, "frac": red_rate / red_peak,
                                 "per_sample": ADJ_RED_PER_SAMPLE,
                                 "peak_source": f"{n_sm} SMs x {SMEM_RED_PER_CLK_SM} int32 red.shared/clk "
                                                f"(measured) x {sm_max:.0f} MHz"}
    rl_bp = alu_roofline("bp_brick_kernel", "paper_2511_08427_gb300/csrc/k_bp_brick.cu",
                         n_updates * BP_FLOP_PER_UPDATE, bp_s)
    rl_bp["flop_per_update"] = BP_FLOP_PER_UPDATE
    ldg_rate = n_updates * BP_LOADS_PER_UPDATE / bp_s / 1e9
    ldg_peak = n_sm * L1_LDG_PER_CLK_SM * sm_max * 1e6 / 1e9
    rl_bp["l1_loads"] = {"achieved_gops": ldg_rate, "peak_gops": ldg_peak, "frac": ldg_rate / ldg_peak,
                         "per_update": BP_LOADS_PER_UPDATE,
                         "peak_source": f"{n_sm} SMs x {L1_LDG_PER_CLK_SM} L1-hit 32-bit ld.global/clk (measured) "
                                        f"x {sm_max:.0f} MHz"}
    # kernels of one step: FP (plus the y-fastest copy it stages x-march slabs from), adjoint, BP
    fpc = g.fp_config()
    launches_per_step = 3 + (1 if fpc["kernel"] == 3 and fpc["y_fastest_x_march"] else 0)
    # the dominant kernel of the step (longest average launch)
    dominant = max((rl_fp, rl_adj, rl_bp), key=lambda r: r["launch_ms"])

    result = {
        "metric": METRIC, "value": fp_rate, "unit": "G ray-samples/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, l2="flushed before every timed step (256 MiB write)",
                       step="forward projection + matched adjoint + voxel-driven BP",
                       parallelism=f"{world} independent volume(s), one per GPU"),
        "bp_gupdates_per_s": bp_rate, "fwd_adj_ms_per_iter": (fp_sum + adj_sum) / K,
        "kernel_ms": {"fp": fp_sum / K, "adjoint": adj_sum / K, "bp": bp_sum / K},
        "gd_iteration_ms": gd_ms,
        "fp_bf16": {"ms": fp_bf16_ms, "gsamples_per_s": n_samples / (fp_bf16_ms * 1e-3) / 1e9},
        "fbp_filter_ms": fbp_ms,
        "samples_per_fp": n_samples, "updates_per_bp": n_updates,
        "e2e": {"value": e2e_rate, "unit": "G ray-samples/s", "h2d_bytes_per_step": int(vol_np.nbytes),
                "d2h_bytes_per_step": int(h_sino.numel() * 4), "call": "pyronn_fp_host"},
        "gpu_launches": launches_per_step * K,
        "clocks": clk,
        "roofline": dominant,
        "rooflines": {"fp": rl_fp, "adjoint": rl_adj, "bp": rl_bp},
    }
    result["autotune"] = {k: tuned[k] for k in ("depth", "buffers", "ms", "cached")}
    if not args.no_batched:
        result["batched"] = run_batched(dev, K=max(3, args.steps // 2))
    if rank == 0 and not args.no_cpu_baseline:
        rate, s, dt, threads, nv = oracle_sample_rate(vol_np, 64, target_s=args.ref_seconds)
        result["cpu_baseline"] = {"value": rate, "unit": "G ray-samples/s", "cores": threads, "kind": "oracle",
                                  "sample": f"FP64 oracle forward projection of {nv} of 360 views, full detector "
                                            f"({s} samples, {dt:.1f} s)",
                                  "single_core": single_core_entry(vol_np)}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
