"""Run one operator on a cone-beam workload a few times (for profilers such as Nsight Compute).

    python -m paper_2511_08427_gb300.profile_ops {fp,adj,bp,fbp} [N] [--repeat R] [--dtype float32|bfloat16]
                                                 [--accum 0|1|2] [--time]

N = 256: 256^3 volume (0.5 mm voxels), 360 views over 2 pi, 512 x 512 detector (0.6 mm),
SID 750 mm, SDD 1200 mm, 20 random ellipsoids (seed 3). Smaller N keeps the same field of view
and magnification with N^3 voxels, 180 views and a 2N x 2N detector. Prints the device counters;
--time also prints the mean CUDA-event time of the repeats after one warm-up launch. --accum sets
the slab adjoint's box accumulation (0 automatic, 1 FP32 only, 2 fixed point with cells).
"""
from __future__ import annotations

import argparse
import math

import torch

from . import inputs, operators as ops


def workload(n: int):
    if n == 256:
        views, det = 360, 512
    else:
        views, det = 180, 2 * n
    sp = 0.5 * 256 / n
    g = ops.Geometry.cone_circular((n, n, n), (sp,) * 3, (det, det), (0.6 * 512 / det,) * 2, views, 2 * math.pi,
                                   750.0, 1200.0)
    vol = inputs.rasterise_ellipsoids(inputs.random_ellipsoids(20, 64.0, 3), (n, n, n), (sp,) * 3)
    return g, vol, (views, det, det)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["fp", "adj", "bp", "fbp"])
    ap.add_argument("n", nargs="?", type=int, default=256)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--dtype", default="float32", choices=["float32", "bfloat16", "float16"])
    ap.add_argument("--accum", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--time", action="store_true")
    a = ap.parse_args()
    dt = getattr(torch, a.dtype)
    g, vol_np, sshape = workload(a.n)
    g.set_tuning(ops.TUNE_ADJ_ACCUM, a.accum)
    vol = torch.from_numpy(vol_np).cuda().to(dt)
    sino = torch.empty(sshape, device="cuda", dtype=dt)
    sino2 = torch.empty_like(sino) if a.op == "fbp" else None
    if a.op != "fp":
        sino.copy_(torch.randn(sshape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(22)))

    def run():
        if a.op == "fp":
            ops.forward_project(vol, g, out=sino)
        elif a.op == "adj":
            ops.adjoint(sino, g, out=vol)
        elif a.op == "fbp":
            ops.fbp_filter(sino, g, out=sino2)
        else:
            ops.back_project(sino, g, out=vol)

    if a.time:
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.repeat):
            run()
        e1.record()
        torch.cuda.synchronize()
        print(f"{a.op} N={a.n} {a.dtype} accum={a.accum}: {e0.elapsed_time(e1) / a.repeat:.3f} ms per launch")
    else:
        for _ in range(a.repeat):
            run()
        torch.cuda.synchronize()
    print("ok", a.op, a.n, a.dtype, "flags", g.read_flags())


if __name__ == "__main__":
    main()
