"""Benchmark of the CT operators: ray-driven forward projection, matched adjoint, voxel-driven BP.

Headline workload (the largest configuration, arbitrary trajectory, Sec. 2.1 last sentence and
Sec. 2.4 "Flexible Trajectory Modeling"): a 512^3 FP32 random-ellipsoid phantom (20 ellipsoids,
0.4 mm voxels), 720 views over 2 pi given as projection matrices of a circular orbit (SID 750 mm,
SDD 1200 mm) with seeded Gaussian jitter (0.5 mm on source and detector centre, 0.2 deg detector
tilts), a 1024 x 1024 detector with 0.4 mm pixels, sampling step 0.2 mm.

One step = A x (forward projection), A^T r (matched adjoint of a standard-normal cotangent) and the
voxel-driven back-projection of the sinogram, all FP32, inputs resident in HBM. Every input is larger
than L2 (volume 512 MiB, sinograms 3 GB), so no flush is needed between steps. Every kernel is timed
with CUDA events on the launching stream.

  value            forward projection throughput, G ray-samples/s (samples inside the support box)
  bp_gupdates_per_s  voxel-driven BP throughput, G voxel-view updates/s
  fwd_adj_ms_per_iter  forward + adjoint time per iteration, ms
  e2e              forward projection through the C ABI with host buffers (copies timed)
  roofline         the step's dominant kernel against the measured peak of the unit that binds it
  cone256          the 256^3 circular cone-beam workload (360 views, 512^2 detector), same keys
  batched          16 volumes of uneven sizes and geometries in persistent launches (plans)
  precision        errors against the FP64 oracle per result and storage type (cpu_baseline leg)

`--impl reference` times the FP64 CPU oracle on bounded samples of the same workload.
With torchrun (N > 1) every rank projects its own volume (independent problems, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "cone-beam FP G ray-samples/s and BP G voxel-view updates/s; fwd+adjoint ms/iter"

WORKLOADS = {
    "cone512_jitter": dict(
        workload="arbitrary-trajectory cone beam 512^3 (0.4 mm), 720 jittered projection matrices, 1024x1024 "
                 "detector (0.4 mm)",
        volume=[512, 512, 512], voxel_mm=0.4, views=720, angular_range="2pi", sid_mm=750.0, sdd_mm=1200.0,
        detector=[1024, 1024], pixel_mm=0.4,
        trajectory="circular orbit, Gaussian jitter 0.5 mm (source, detector centre) and 0.2 deg (detector "
                   "tilts), seed 5",
        phantom="20 random ellipsoids, seed 5", dt_mm=0.2),
    "cone256": dict(
        workload="circular cone beam 256^3 (0.5 mm), 360 views, 512x512 detector (0.6 mm)",
        volume=[256, 256, 256], voxel_mm=0.5, views=360, angular_range="2pi", sid_mm=750.0, sdd_mm=1200.0,
        detector=[512, 512], pixel_mm=0.6, phantom="20 random ellipsoids, seed 3", dt_mm=0.25),
}
HEADLINE = "cone512_jitter"

# Algorithmic work per unit. FLOP: FP32 operations, an FMA counted as 2.
FP_FLOP_PER_SAMPLE = 34     # 3 position FMA (6), 3 floor + 3 frac (6), 7 lerps (21), accumulate (1)
FP_SMEM_BYTES_PER_SAMPLE = 32   # eight FP32 interpolation operands read from the staged slab
ADJ_FLOP_PER_SAMPLE = 33    # 3 position FMA (6), 3 frac (3), 1 - a (2), z split (2), 12 weight products, 8 adds
ADJ_RED_PER_SAMPLE = 8      # one shared-memory scatter-add per trilinear corner
BP_FLOP_PER_UPDATE = 18     # projection 3 FMA (6), reciprocal and 2 products (3), 3 bilinear lerps (6), weight, add
BP_LOADS_PER_UPDATE = 4     # bilinear detector operands (L1-resident global loads)


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
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(pw)) if pw else None}


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


# ------------------------------------------------------------------------------------------------
# workloads (seeded synthetic inputs)
# ------------------------------------------------------------------------------------------------

def trajectory():
    from paper_2511_08427_gb300 import inputs
    return inputs.jittered_circular_trajectory(720, 2 * math.pi, 750.0, 1200.0, 0.5, 0.2, seed=5)


def build_volume(name: str, rank: int = 0) -> np.ndarray:
    from paper_2511_08427_gb300 import inputs
    if name == "cone512_jitter":
        return inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 102.4, 5 + rank), (512, 512, 512),
                                           (0.4, 0.4, 0.4))
    return inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 64.0, 3 + rank), (256, 256, 256),
                                       (0.5, 0.5, 0.5))


def make_geometry(name: str, views: int | None = None):
    """The workload's geometry; views: keep only that many of its views, evenly spaced (profiling runs)."""
    from paper_2511_08427_gb300.operators import Geometry
    if name == "cone512_jitter":
        tr = trajectory()
        idx = np.arange(720) if views is None else np.linspace(0, 719, views).round().astype(int)
        return Geometry.cone_from_positions((512, 512, 512), (0.4, 0.4, 0.4), (1024, 1024), (0.4, 0.4), tr.src[idx],
                                            tr.det_centre[idx], tr.eu[idx], tr.ev[idx])
    n = 360 if views is None else views
    return Geometry.cone_circular((256, 256, 256), (0.5, 0.5, 0.5), (512, 512), (0.6, 0.6), n, 2 * math.pi * n / 360,
                                  750.0, 1200.0)


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline leg). Only these functions use the oracle.
# ------------------------------------------------------------------------------------------------

def oracle_geometry(name: str):
    import oracle
    if name == "cone512_jitter":
        tr = trajectory()
        return oracle.cone_from_positions((512, 512, 512), (0.4, 0.4, 0.4), (1024, 1024), (0.4, 0.4), tr.src,
                                          tr.det_centre, tr.eu, tr.ev)
    return oracle.cone_circular((256, 256, 256), (0.5, 0.5, 0.5), (512, 512), (0.6, 0.6), 360, 2 * math.pi,
                                750.0, 1200.0)


def oracle_subset(og, view_ids, rows=None):
    """The oracle geometry restricted to some views and, optionally, a band of detector rows [r0, r1): the
    rows' pixel index v becomes v - r0, i.e. P's second row minus r0 times its third (an exact change of
    pixel coordinates that keeps the matrices' normalisation)."""
    import oracle
    P = np.array(og.views[list(view_ids)], dtype=np.float64)
    det = og.det_shape
    if rows is not None:
        r0, r1 = rows
        P = P.reshape(-1, 3, 4)
        P[:, 1, :] -= r0 * P[:, 2, :]
        P = P.reshape(-1, 12)
        det = (r1 - r0, og.det_shape[1])
    return oracle.Geometry(og.vol_shape, og.vol_spacing, og.vol_offset, tuple(det), og.det_spacing, og.det_offset,
                           og.kind, P, og.dt)


def oracle_fp_views(og, vol64, view_ids):
    """Oracle forward projection of whole views: (values [n, Nv, Nu], samples, seconds)."""
    import oracle
    g = oracle_subset(og, view_ids)
    t0 = time.perf_counter()
    out = oracle.fp(g, vol64)
    dt = time.perf_counter() - t0
    return out, int(oracle.count_samples(g).sum()), dt


def oracle_single_core_rate(og, vol64, view: int):
    """The oracle on one thread: 64 detector rows of one view (a few seconds). Returns (G samples/s,
    samples, seconds)."""
    import oracle
    nv = og.det_shape[0]
    r0 = nv // 2 - 32
    g = oracle_subset(og, [view], rows=(r0, r0 + 64))
    n_all = oracle.max_threads()
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.fp(g, vol64)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(n_all)
    s = int(oracle.count_samples(g).sum())
    return s / dt / 1e9, s, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    name = args.workload
    vol64 = np.ascontiguousarray(build_volume(name), dtype=np.float64)
    og = oracle_geometry(name)
    V = og.n_views
    # one view, once, to size the per-step sample (every step times whole views of the workload)
    _, s1, t1 = oracle_fp_views(og, vol64, [1])
    per_step = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    nv = max(1, int(round(per_step / max(t1, 1e-3))))
    times, samples = [], []
    for i in range(args.warmup + args.steps):
        ids = [(7 * (i * nv + j) + 3) % V for j in range(nv)]
        _, s, dt = oracle_fp_views(og, vol64, ids)
        if i >= args.warmup:
            times.append(dt)
            samples.append(s)
    value = sum(samples) / sum(times) / 1e9
    rate1, s_1, t_1 = oracle_single_core_rate(og, vol64, 5)
    cfg = dict(WORKLOADS[name], kernel="FP64 CPU oracle, forward projection")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "G ray-samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "G ray-samples/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"forward projection of {nv} whole views per step (of {V}), full detector",
                             "single_core": {"value": rate1, "unit": "G ray-samples/s", "cores": 1,
                                             "sample": f"64 detector rows of one view on one thread ({s_1} samples, "
                                                       f"{t_1:.1f} s)"}},
            "e2e": {"value": value, "unit": "G ray-samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_leg(name, vol_np, g, dev, results):
    """The FP64 oracle on bounded samples of the workload, timed on the host cores (forward projection of
    whole views, back-projection of sampled voxels, one thread on 64 detector rows), plus the errors of
    the GPU results against those oracle values (FP32 / BF16 / FP16 storage)."""
    import torch

    import oracle
    from paper_2511_08427_gb300 import operators as ops
    og = oracle_geometry(name)
    V = og.n_views
    vol64 = np.ascontiguousarray(vol_np, dtype=np.float64)
    _, _, t1 = oracle_fp_views(og, vol64, [1])
    nv = max(1, min(64, int(10.0 / max(t1, 1e-3))))
    ids = [(7 * j + 3) % V for j in range(nv)]
    p_or, samples, dt = oracle_fp_views(og, vol64, ids)
    rate = samples / dt / 1e9
    threads = oracle.max_threads()
    rate1, s1, t1c = oracle_single_core_rate(og, vol64, 5)
    total_samples = results["samples_per_fp"]
    # voxel-driven BP of sampled voxels from the GPU's FP32 sinogram (the oracle reads it in FP64)
    sino = results["_sino"]
    rng = np.random.default_rng(11)
    n_vox = int(np.prod(og.vol_shape))
    vids = np.sort(rng.choice(n_vox, size=20000, replace=False))
    sino64 = sino.double().cpu().numpy().reshape(og.sino_shape)
    t0 = time.perf_counter()
    b_or = oracle.bp_voxels(og, sino64, vids, 0)
    bp_dt = time.perf_counter() - t0
    bp_rate = vids.size * V / bp_dt / 1e9
    # matched adjoint of a sparse cotangent (2000 rays), over the whole volume
    n_rays = V * og.det_shape[0] * og.det_shape[1]
    rids = np.sort(rng.choice(n_rays, size=2000, replace=False))
    rvals = rng.standard_normal(rids.size)
    t0 = time.perf_counter()
    a_or = oracle.adjoint_rays(og, rids, rvals)
    adj_dt = time.perf_counter() - t0

    def rel(a, b):
        """rel-L2 of a against b; None where a holds values outside the storage type's range (FP16
        back-projections of long scans exceed 65504)."""
        a = np.asarray(a, np.float64).ravel()
        b = np.asarray(b, np.float64).ravel()
        if not np.isfinite(a).all():
            return None
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    prec = {"reference": "FP64 oracle on the FP32 inputs; rel-L2 over the sampled outputs"}
    vol = results["_vol"]
    idx_dev = torch.as_tensor(ids, device=dev)
    for dtype, tag in ((torch.float32, "f32"), (torch.bfloat16, "bf16"), (torch.float16, "f16")):
        if dtype == torch.float32:
            s_dt = sino
        else:
            s_dt = ops.forward_project(vol.to(dtype), g)
        fp_err = rel(s_dt.index_select(0, idx_dev).double().cpu().numpy(), p_or)
        # BP of the sinogram in this storage type (the oracle's input is the FP32 sinogram)
        b = ops.back_project(s_dt if dtype == torch.float32 else sino.to(dtype), g, 0)
        bp_err = rel(b.reshape(-1).index_select(0, torch.as_tensor(vids, device=dev)).double().cpu().numpy(), b_or)
        del b
        y = torch.zeros(n_rays, device=dev, dtype=dtype)
        y[torch.as_tensor(rids, device=dev)] = torch.as_tensor(rvals, device=dev, dtype=torch.float32).to(dtype)
        a = ops.adjoint(y.view(og.sino_shape), g)
        adj_err = rel(a.double().cpu().numpy(), a_or)
        del a, y
        if dtype != torch.float32:
            del s_dt
        torch.cuda.empty_cache()
        prec[tag] = {"fp_rel_l2": fp_err, "bp_rel_l2": bp_err, "adjoint_rel_l2": adj_err}
    if results.get("_sino_texf") is not None:
        prec["fp_texture_filtered_f32"] = rel(results["_sino_texf"].index_select(0, idx_dev).double().cpu().numpy(),
                                              p_or)
    prec["note"] = "None: the output exceeds the storage type's range (FP16 saturates above 65504)"
    prec["samples"] = {"fp": f"{nv} whole views ({samples} samples)", "bp": f"{vids.size} random voxels",
                       "adjoint": f"sparse cotangent on {rids.size} random rays, whole volume compared"}
    base = {"value": rate, "unit": "G ray-samples/s", "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle forward projection of {nv} of {V} views, full detector ({samples} samples, "
                      f"{dt:.1f} s)",
            "bp": {"value": bp_rate, "unit": "G voxel-view updates/s", "cores": threads,
                   "sample": f"{vids.size} random voxels x {V} views ({bp_dt:.1f} s)"},
            "adjoint_sparse_s": adj_dt,
            "extrapolated": {"fp_s": total_samples / (rate * 1e9),
                             "bp_s": results["updates_per_bp"] / (bp_rate * 1e9),
                             "note": "whole-workload times at the sampled rates (extrapolated)"},
            "single_core": {"value": rate1, "unit": "G ray-samples/s", "cores": 1,
                            "sample": f"64 detector rows of one view on one thread ({s1} samples, {t1c:.1f} s)"}}
    return base, prec


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def source_digest(files) -> str:
    """SHA-1 of the concatenated bytes of a kernel's source files (its .cu and the headers it includes)."""
    h = hashlib.sha1()
    for name in files:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(kernel: str, workload: str, sources):
    """DRAM bytes per launch from the committed ncu record, if it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        digest = source_digest(sources)
    except (OSError, ValueError):
        return None
    return rec.get("dram_bytes_per_launch") if rec.get("source_sha1") == digest else None


_CSRC = "paper_2511_08427_gb300/csrc/"
SOURCES = {"fp_tma_kernel": [_CSRC + f for f in ("k_fp_tma.cu", "device_common.cuh", "tma_common.cuh")],
           "adjoint_slab_kernel": [_CSRC + f for f in ("k_adjoint_slab.cu", "device_common.cuh")],
           "bp_brick_kernel": [_CSRC + f for f in ("k_bp_brick.cu", "bp_common.cuh", "device_common.cuh")],
           "bp_tma_kernel": [_CSRC + f for f in ("k_bp_tma.cu", "bp_common.cuh", "device_common.cuh",
                                                 "tma_common.cuh")]}


def rooflines(rates, mhz, workload, n_samples, n_updates, fp_s, adj_s, bp_s, bp_kernel=2):
    """Per kernel: the unit that binds it, its algorithmic rate and the measured peak of that unit at the
    SM clock seen during the timed region; the FP32 (ALU) fraction beside it. bp_kernel: the
    back-projector that ran (2 brick kernel, L1 taps; 3 staged kernel, shared-memory taps)."""
    from paper_2511_08427_gb300 import roofline as R
    src = (f"roofline_peaks.cu probes: {rates['sms']} SMs x measured rate per SM clock x {mhz:.0f} MHz "
           f"(median SM clock sampled during the timed region)")
    alu_peak = R.peak(rates, "ffma", mhz) * 2 / 1e12

    def entry(kernel, bound, achieved, peak, unit, flop, seconds, per_unit):
        alu = flop / seconds / 1e12
        return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": kernel_traffic(kernel, workload, SOURCES[kernel]), "kernel": kernel,
                "launch_ms": seconds * 1e3, "peak_source": src, "per_unit": per_unit,
                "alu": {"achieved_tflops": alu, "peak_tflops": alu_peak, "frac": alu / alu_peak}}

    fp_ach = n_samples * FP_SMEM_BYTES_PER_SAMPLE / fp_s / 1e9
    fp_pk = R.peak(rates, "ld_shared_b32", mhz) * 4 / 1e9
    rl_fp = entry("fp_tma_kernel", "smem", fp_ach, fp_pk, "GB/s", n_samples * FP_FLOP_PER_SAMPLE, fp_s,
                  f"{FP_SMEM_BYTES_PER_SAMPLE} B of shared-memory operands and {FP_FLOP_PER_SAMPLE} FLOP per sample")
    adj_ach = n_samples * ADJ_RED_PER_SAMPLE / adj_s / 1e9
    adj_pk = R.peak(rates, "red_shared_s32", mhz) / 1e9
    rl_adj = entry("adjoint_slab_kernel", "smem_atomics", adj_ach, adj_pk, "Gop/s", n_samples * ADJ_FLOP_PER_SAMPLE,
                   adj_s, f"{ADJ_RED_PER_SAMPLE} shared-memory int32 reductions and {ADJ_FLOP_PER_SAMPLE} FLOP per sample")
    bp_ach = n_updates * BP_LOADS_PER_UPDATE / bp_s / 1e9
    if bp_kernel == 3:
        bp_pk = R.peak(rates, "ld_shared_b32", mhz) / 1e9
        rl_bp = entry("bp_tma_kernel", "smem", bp_ach, bp_pk, "Gop/s", n_updates * BP_FLOP_PER_UPDATE, bp_s,
                      f"{BP_LOADS_PER_UPDATE} shared-memory detector loads and {BP_FLOP_PER_UPDATE} FLOP per "
                      f"voxel-view update")
    else:
        bp_pk = R.peak(rates, "ld_global_l1_b32", mhz) / 1e9
        rl_bp = entry("bp_brick_kernel", "l1", bp_ach, bp_pk, "Gop/s", n_updates * BP_FLOP_PER_UPDATE, bp_s,
                      f"{BP_LOADS_PER_UPDATE} L1-hit detector loads and {BP_FLOP_PER_UPDATE} FLOP per voxel-view "
                      f"update")
    return {"fp": rl_fp, "adjoint": rl_adj, "bp": rl_bp}


def timed_steps(ops, g, vol, sino, cot, adj, bpv, steps, stream, torch, flush=None):
    """steps x (FP, adjoint, BP) with per-kernel CUDA events; returns (total ms, fp ms[], adj ms[], bp ms[])."""
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(steps):
        if flush is not None:
            flush.fill_(1.0)
        evs[i][0].record(stream)
        ops.forward_project(vol, g, out=sino)
        evs[i][1].record(stream)
        ops.adjoint(cot, g, out=adj)
        evs[i][2].record(stream)
        ops.back_project(sino, g, out=bpv)
        evs[i][3].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    fp = np.array([e[0].elapsed_time(e[1]) for e in evs])
    ad = np.array([e[1].elapsed_time(e[2]) for e in evs])
    bp = np.array([e[2].elapsed_time(e[3]) for e in evs])
    return t_start.elapsed_time(t_end), fp, ad, bp


def run_cone256(dev, steps, rates, mhz):
    """The 256^3 circular workload: FP, adjoint, BP (L2 flushed before each step: the volume fits in L2),
    a gradient-descent iteration fused and unfused, BF16-storage FP and the FBP filter."""
    import torch
    from paper_2511_08427_gb300 import operators as ops
    g = make_geometry("cone256")
    vol_np = build_volume("cone256")
    vol = torch.from_numpy(vol_np).to(dev)
    sino = torch.empty((360, 512, 512), device=dev)
    cot = torch.randn((360, 512, 512), device=dev, generator=torch.Generator(device=dev).manual_seed(22))
    adj = torch.empty_like(vol)
    bpv = torch.empty_like(vol)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)
    stream = torch.cuda.current_stream(dev)
    timed_steps(ops, g, vol, sino, cot, adj, bpv, 2, stream, torch, flush)
    total, fp, ad, bp = timed_steps(ops, g, vol, sino, cot, adj, bpv, steps, stream, torch, flush)
    n_samples = g.count_samples()
    n_updates = 256 ** 3 * 360

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
    for nm, fn in (("unfused", gd_unfused), ("fused", gd_fused)):
        x_it.copy_(vol).mul_(0.9)
        gd_ms[nm] = time_ms(fn, 3)
    del p_meas, x_it
    vol_bf, sino_bf = vol.bfloat16(), torch.empty(sino.shape, device=dev, dtype=torch.bfloat16)
    fp_bf16_ms = time_ms(lambda: ops.forward_project(vol_bf, g, out=sino_bf), 3)
    del vol_bf, sino_bf
    fbp_out = torch.empty_like(sino)
    fbp_ms = time_ms(lambda: ops.fbp_filter(sino, g, out=fbp_out), 3)
    del fbp_out
    fp_s, adj_s, bp_s = fp.mean() * 1e-3, ad.mean() * 1e-3, bp.mean() * 1e-3
    out = {"config": dict(WORKLOADS["cone256"], l2="flushed before every timed step (256 MiB write)"),
           "steps": steps, "ms_per_step": total / steps,
           "fp_gsamples_per_s": n_samples / fp_s / 1e9, "bp_gupdates_per_s": n_updates / bp_s / 1e9,
           "fwd_adj_ms_per_iter": (fp.mean() + ad.mean()),
           "kernel_ms": {"fp": float(fp.mean()), "adjoint": float(ad.mean()), "bp": float(bp.mean())},
           "samples_per_fp": n_samples, "updates_per_bp": n_updates, "gd_iteration_ms": gd_ms,
           "fp_bf16": {"ms": fp_bf16_ms, "gsamples_per_s": n_samples / (fp_bf16_ms * 1e-3) / 1e9},
           "fbp_filter_ms": fbp_ms,
           "rooflines": rooflines(rates, mhz, "cone256", n_samples, n_updates, fp_s, adj_s, bp_s,
                                  g.bp_config()["kernel"])}
    del vol, sino, cot, adj, bpv, flush
    torch.cuda.empty_cache()
    return out


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
        bps = [torch.empty(g.volume_shape, device=dev, dtype=dtype) for g in geoms]
        plan.forward_project(xs, sinos)
        plan.adjoint(sinos, adj)
        plan.back_project(sinos, bps)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        for _ in range(K):
            plan.forward_project(xs, sinos)
        ev[1].record(stream)
        for _ in range(K):
            plan.adjoint(sinos, adj)
        ev[2].record(stream)
        for _ in range(K):
            plan.back_project(sinos, bps)
        ev[3].record(stream)
        torch.cuda.synchronize()
        fp_ms = ev[0].elapsed_time(ev[1]) / K
        adj_ms = ev[1].elapsed_time(ev[2]) / K
        bp_ms = ev[2].elapsed_time(ev[3]) / K
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
        out[tag] = {"fp_ms": fp_ms, "adjoint_ms": adj_ms, "bp_ms": bp_ms,
                    "fp_gsamples_per_s": samples / (fp_ms * 1e-3) / 1e9,
                    "graph_fwd_adj_ms": ev[0].elapsed_time(ev[1]) / K, "grids": plan.info()["grids"]}
        del plan, xs, sinos, adj, bps, graph
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

    from paper_2511_08427_gb300 import _lib, operators as ops, roofline

    name = args.workload
    spec = WORKLOADS[name]
    vol_np = build_volume(name, rank)
    g = make_geometry(name)
    n_samples = g.count_samples()
    nz, ny, nx = spec["volume"]
    V = spec["views"]
    nv, nu = spec["detector"]
    n_updates = nx * ny * nz * V
    vol = torch.from_numpy(vol_np).to(dev)
    sino = torch.empty((V, nv, nu), device=dev)
    cot = torch.randn((V, nv, nu), device=dev, generator=torch.Generator(device=dev).manual_seed(22))
    adj = torch.empty_like(vol)
    bpv = torch.empty_like(vol)
    stream = torch.cuda.current_stream(dev)
    big = vol_np.nbytes > 200 * 2 ** 20
    flush = None if big else torch.empty(256 * 1024 * 1024 // 4, device=dev)

    # tile and brick shapes chosen by the library's autotuner: the projector and the adjoint on an evenly
    # spaced eighth of the views (the per-view work is the same; the whole geometry would take a minute of
    # timing), the back-projector on the whole geometry (its staged variant's pipeline start is paid once
    # per brick, so a subset of the views would understate it; it takes a few seconds)
    from paper_2511_08427_gb300 import autotune
    tuned = {}
    g_sub = make_geometry(name, views=max(1, V // 8))
    for op in ("fp", "adjoint", "bp"):
        gt = g if op == "bp" else g_sub
        r = autotune.tune(gt, op, repeats=2, use_cache=False, device=dev)
        autotune.apply(g, autotune.OPS[op], *r["params"])
        tuned[op] = {"params": r["params"], "tuned_ms": r["ms"], "candidates": r["candidates"],
                     "tuned_on_views": gt.n_views}
    del g_sub
    rates = roofline.measure()   # on-chip peaks per SM clock, measured on this GPU before the timed region
    timed_steps(ops, g, vol, sino, cot, adj, bpv, args.warmup, stream, torch, flush)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        total_ms, fp_ms, adj_ms, bp_ms = timed_steps(ops, g, vol, sino, cot, adj, bpv, args.steps, stream, torch,
                                                     flush)
    if world > 1:
        dist.barrier()
    total_ms, fp_sum, adj_sum, bp_sum = max_over_ranks([total_ms, fp_ms.sum(), adj_ms.sum(), bp_ms.sum()], world, dev)
    K = args.steps
    fp_rate = job_rate(n_samples, world, K, fp_sum * 1e-3)
    bp_rate = job_rate(n_updates, world, K, bp_sum * 1e-3)
    clk = clocks.summary()
    mhz = clk["sm_mhz"] or rates["sm_mhz"]
    fp_s, adj_s, bp_s = fp_sum / K * 1e-3, adj_sum / K * 1e-3, bp_sum / K * 1e-3
    rl = rooflines(rates, mhz, name, n_samples, n_updates, fp_s, adj_s, bp_s, g.bp_config()["kernel"])
    dominant = max(rl.values(), key=lambda r: r["launch_ms"])

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    import ctypes
    h_vol = torch.from_numpy(vol_np).pin_memory()
    h_sino = torch.empty((V, nv, nu), dtype=torch.float32).pin_memory()
    L = _lib.lib()

    def e2e_call():
        _lib.check(L.pyronn_fp_host(g.handle, ctypes.c_void_p(h_vol.data_ptr()), ctypes.c_void_p(h_sino.data_ptr()),
                                    0, 1, ctypes.c_void_p(stream.cuda_stream)))

    e2e_call()
    n_e2e = 3
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_call()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_s = max_over_ranks([e2e_s], world, dev)[0]
    e2e_rate = job_rate(n_samples, world, 1, e2e_s)
    del h_vol, h_sino

    # the hardware-filtered texture projector (opt-in variant 5: the texture unit's 8-bit trilinear
    # weights, not the FP32 operator) on the same workload; its error is measured in the CPU leg
    g.set_variant(0, 5)
    texf = None
    if g.fp_config()["kernel"] == 5:
        sino_tf = torch.empty((V, nv, nu), device=dev)
        ops.forward_project(vol, g, out=sino_tf)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            ops.forward_project(vol, g, out=sino_tf)
        e1.record(stream)
        torch.cuda.synchronize()
        tf_ms = e0.elapsed_time(e1) / 3
        texf = {"ms": tf_ms, "gsamples_per_s": n_samples / (tf_ms * 1e-3) / 1e9,
                "texture_unit": {"achieved_gfetch_per_s": n_samples / (tf_ms * 1e-3) / 1e9,
                                 "peak_gfetch_per_s": rates["tex3d_trilinear_per_clk_sm"] * rates["sms"] * mhz / 1e3,
                                 "frac": n_samples / (tf_ms * 1e-3) / (rates["tex3d_trilinear_per_clk_sm"] *
                                                                     rates["sms"] * mhz * 1e6)},
                "note": "opt-in approximation (8-bit interpolation fractions of the texture unit); includes the "
                        "copy of the volume into the 3D texture"}
    g.set_variant(0, 0)

    # kernels of one step: FP (plus the y-fastest copy it stages x-march slabs from), adjoint, BP
    fpc = g.fp_config()
    launches_per_step = 3 + (1 if fpc["kernel"] == 3 and fpc["y_fastest_x_march"] else 0)
    peaks, peak_src = measured_peaks()
    result = {
        "metric": METRIC, "value": fp_rate, "unit": "G ray-samples/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(spec, l2=("inputs larger than L2 (volume 512 MiB, sinograms 3 GB): no flush" if big else
                                 "flushed before every timed step (256 MiB write)"),
                       step="forward projection + matched adjoint + voxel-driven BP",
                       parallelism=f"{world} independent volume(s), one per GPU"),
        "bp_gupdates_per_s": bp_rate, "fwd_adj_ms_per_iter": (fp_sum + adj_sum) / K,
        "kernel_ms": {"fp": fp_sum / K, "adjoint": adj_sum / K, "bp": bp_sum / K},
        "samples_per_fp": n_samples, "updates_per_bp": n_updates,
        "e2e": {"value": e2e_rate, "unit": "G ray-samples/s", "h2d_bytes_per_step": int(vol_np.nbytes),
                "d2h_bytes_per_step": int(V * nv * nu * 4), "call": "pyronn_fp_host"},
        "gpu_launches": launches_per_step * K,
        "clocks": clk,
        "roofline": dominant,
        "rooflines": rl,
        "onchip_peaks": dict(rates, source="roofline_peaks.cu, measured in this run before the timed region"),
        "autotune": dict(tuned, params="fp: (slab depth, buffers); adjoint: (slab depth, pitch mode); bp: (brick "
                                       "depth, variant 2 L1 path / 3 staged shadows)"),
        "fp_texture_filtered": texf,
        "hbm": {"compulsory_gb_per_step": (3 * vol_np.nbytes + 3 * V * nv * nu * 4) / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"), "peak_source": peak_src},
    }
    if rank == 0 and not args.no_cpu_baseline:
        results = {"_sino": sino, "_vol": vol, "samples_per_fp": n_samples, "updates_per_bp": n_updates,
                   "_sino_texf": sino_tf if texf else None}
        base, prec = cpu_baseline_leg(name, vol_np, g, dev, results)
        result["cpu_baseline"] = base
        result["precision"] = prec
    del sino, cot, adj, bpv, vol
    if texf:
        del sino_tf
    torch.cuda.empty_cache()
    if name == HEADLINE and not args.no_secondary:
        result["cone256"] = run_cone256(dev, max(3, K // 2), rates, mhz)
    if not args.no_batched:
        result["batched"] = run_batched(dev, K=max(3, K // 4))
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """One operator of a workload, a few launches after one warm-up launch (for Nsight Compute): fp, adj
    (matched adjoint of a standard-normal cotangent), bp (voxel-driven), fbp (filter). --views keeps a
    subset of the views so that a capture of many passes stays small. --time prints the mean CUDA-event
    time per launch."""
    import torch
    from paper_2511_08427_gb300 import operators as ops
    dev = torch.device("cuda", 0)
    dt = getattr(torch, args.dtype)
    g = make_geometry(args.workload, args.views)
    if args.params:
        # the autotuner's parameters of the operator (as the bench line's "autotune" record reports them)
        from paper_2511_08427_gb300 import autotune
        a, b = (int(x) for x in args.params.split(","))
        autotune.apply(g, autotune.OPS[{"fp": "fp", "adj": "adjoint", "bp": "bp"}[args.profile]], a, b)
    if args.variant:
        g.set_variant(0 if args.profile == "fp" else (1 if args.profile == "adj" else 2), args.variant)
    vol = torch.from_numpy(build_volume(args.workload)).to(dev).to(dt)
    sshape = (g.n_views,) + tuple(g.detector_shape)
    sino = torch.empty(sshape, device=dev, dtype=dt)
    out2 = torch.empty_like(sino) if args.profile == "fbp" else None
    if args.profile != "fp":
        sino.copy_(torch.randn(sshape, device=dev, generator=torch.Generator(device=dev).manual_seed(22)))

    def run():
        if args.profile == "fp":
            ops.forward_project(vol, g, out=sino)
        elif args.profile == "adj":
            ops.adjoint(sino, g, out=vol)
        elif args.profile == "fbp":
            ops.fbp_filter(sino, g, out=out2)
        else:
            ops.back_project(sino, g, out=vol)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.repeat):
        run()
    e1.record()
    torch.cuda.synchronize()
    msg = f"{args.profile} {args.workload} views={g.n_views} {args.dtype}"
    if args.time:
        msg += f": {e0.elapsed_time(e1) / args.repeat:.3f} ms per launch"
    print(msg, "flags", g.read_flags(), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--profile", choices=["fp", "adj", "bp", "fbp"], default=None,
                    help="run one operator of --workload for a profiler instead of the benchmark")
    ap.add_argument("--views", type=int, default=None, help="--profile: keep this many of the workload's views")
    ap.add_argument("--repeat", type=int, default=2, help="--profile: launches after the warm-up launch")
    ap.add_argument("--variant", type=int, default=0, help="--profile: kernel variant of the operator (0 automatic)")
    ap.add_argument("--params", default=None,
                    help="--profile: autotuner parameters 'a,b' of fp, adj or bp to apply (as in the bench line)")
    ap.add_argument("--dtype", default="float32", choices=["float32", "bfloat16", "float16"])
    ap.add_argument("--time", action="store_true", help="--profile: print the mean time per launch")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
