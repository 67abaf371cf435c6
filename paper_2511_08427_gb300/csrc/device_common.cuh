// Device helpers shared by the projector kernels: storage conversion, ray setup, clipping.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "pyronn_internal.h"

namespace pyronn {

// ---------------------------------------------------------------------------------------------
// storage types: FP32 / BF16 / FP16 in memory, FP32 arithmetic
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_f32(T x);
template <>
__device__ __forceinline__ float to_f32<float>(float x) { return x; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float to_f32<__half>(__half x) { return __half2float(x); }

template <typename T>
__device__ __forceinline__ T from_f32(float x);
template <>
__device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }

template <typename T>
__device__ __forceinline__ float ldg_f32(const T *p) { return to_f32<T>(__ldg(p)); }

// ---------------------------------------------------------------------------------------------
// packed FP32x2 arithmetic (two independent FP32 lanes in a 64-bit register pair; each lane rounds
// exactly as the scalar instruction would)
// ---------------------------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f32x2 splat2(float x) { return pack2(x, x); }
__device__ __forceinline__ float lo2(f32x2 v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo;
}
__device__ __forceinline__ float hi2(f32x2 v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return hi;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// rounded toward minus infinity (the floor-by-magic-number addition)
__device__ __forceinline__ f32x2 add2_rd(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a + t (b - a) per lane: one packed subtraction and one packed FMA
__device__ __forceinline__ f32x2 lerp2(f32x2 t, f32x2 a, f32x2 b) {
    f32x2 d, r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b), "l"(a));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(t), "l"(d), "l"(a));
    return r;
}

// 1 / x by the hardware's approximate reciprocal (one instruction, relative error of the order of
// 2^-23; subnormal x gives infinity): for voxel-driven depth weights, whose positions on the detector
// are offsets of at most a few tens of pixels times 1 / w, so the error stays near 1e-5 pixel
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------------------------
// rays
// ---------------------------------------------------------------------------------------------

// A ray in index coordinates: sample k sits at c + ((k + 1/2) dt) d, where c is the ray's point
// closest to the volume centre and d the unit world direction divided by the voxel spacing.
struct RayIdx {
    float cx, cy, cz;
    float dx, dy, dz;
};

__device__ __forceinline__ RayIdx ray_setup(const FpRec &r, const VolDims &v, float u, float w) {
    float Y0 = fmaf(w, r.Rv[0], fmaf(u, r.Ru[0], r.R0[0]));
    float Y1 = fmaf(w, r.Rv[1], fmaf(u, r.Ru[1], r.R0[1]));
    float Y2 = fmaf(w, r.Rv[2], fmaf(u, r.Ru[2], r.R0[2]));
    float D0 = fmaf(w, r.Bv[0], fmaf(u, r.Bu[0], r.B0[0]));
    float D1 = fmaf(w, r.Bv[1], fmaf(u, r.Bu[1], r.B0[1]));
    float D2 = fmaf(w, r.Bv[2], fmaf(u, r.Bu[2], r.B0[2]));
    float inv = rsqrtf(fmaf(D0, D0, fmaf(D1, D1, D2 * D2)));
    D0 *= inv; D1 *= inv; D2 *= inv;
    float tau = -fmaf(Y0, D0, fmaf(Y1, D1, Y2 * D2));
    RayIdx o;
    o.cx = fmaf(fmaf(tau, D0, Y0), v.isx, v.hx);
    o.cy = fmaf(fmaf(tau, D1, Y1), v.isy, v.hy);
    o.cz = fmaf(fmaf(tau, D2, Y2), v.isz, v.hz);
    o.dx = D0 * v.isx;
    o.dy = D1 * v.isy;
    o.dz = D2 * v.isz;
    return o;
}

__device__ __forceinline__ void clip_axis(float c, float d, int n, float &lo, float &hi, bool &empty) {
    if (fabsf(d) > 1e-30f) {
        float id = 1.0f / d;
        float t1 = (-1.0f - c) * id, t2 = ((float)n - c) * id;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
    } else if (!(c > -1.0f && c < (float)n)) {
        empty = true;
    }
}

// Sample index range [k0, k1] covering every sample inside the open support box (-1, N_a) on all
// axes (plus possibly a zero-weight sample at each end). Returns false if the ray misses.
__device__ __forceinline__ bool ray_k_range(const RayIdx &r, const VolDims &v, float dt, int &k0, int &k1) {
    float lo = -3.0e38f, hi = 3.0e38f;
    bool empty = false;
    clip_axis(r.cx, r.dx, v.nx, lo, hi, empty);
    clip_axis(r.cy, r.dy, v.ny, lo, hi, empty);
    clip_axis(r.cz, r.dz, v.nz, lo, hi, empty);
    if (empty || !(hi > lo)) return false;
    float idt = 1.0f / dt;
    k0 = (int)floorf(fmaf(lo, idt, -0.5f));
    k1 = (int)ceilf(fmaf(hi, idt, -0.5f));
    return k1 >= k0;
}

// Trilinear hat interpolant at index position q, zero outside the grid (read-only-cache loads).
template <typename T>
__device__ __forceinline__ float trilerp_zero(const T *__restrict__ vol, const VolDims &v, float qx, float qy,
                                              float qz) {
    float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
    float ax = qx - fx, ay = qy - fy, az = qz - fz;
    int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    bool x0 = (unsigned)ix < (unsigned)v.nx, x1 = (unsigned)(ix + 1) < (unsigned)v.nx;
    bool y0 = (unsigned)iy < (unsigned)v.ny, y1 = (unsigned)(iy + 1) < (unsigned)v.ny;
    bool z0 = (unsigned)iz < (unsigned)v.nz, z1 = (unsigned)(iz + 1) < (unsigned)v.nz;
    const int sy = v.nx, sz = v.nx * v.ny;
    const int base = iz * sz + iy * sy + ix;
    float v000 = (z0 && y0 && x0) ? ldg_f32(vol + base) : 0.0f;
    float v001 = (z0 && y0 && x1) ? ldg_f32(vol + base + 1) : 0.0f;
    float v010 = (z0 && y1 && x0) ? ldg_f32(vol + base + sy) : 0.0f;
    float v011 = (z0 && y1 && x1) ? ldg_f32(vol + base + sy + 1) : 0.0f;
    float v100 = (z1 && y0 && x0) ? ldg_f32(vol + base + sz) : 0.0f;
    float v101 = (z1 && y0 && x1) ? ldg_f32(vol + base + sz + 1) : 0.0f;
    float v110 = (z1 && y1 && x0) ? ldg_f32(vol + base + sz + sy) : 0.0f;
    float v111 = (z1 && y1 && x1) ? ldg_f32(vol + base + sz + sy + 1) : 0.0f;
    float c00 = fmaf(ax, v001 - v000, v000);
    float c01 = fmaf(ax, v011 - v010, v010);
    float c10 = fmaf(ax, v101 - v100, v100);
    float c11 = fmaf(ax, v111 - v110, v110);
    float c0 = fmaf(ay, c01 - c00, c00);
    float c1 = fmaf(ay, c11 - c10, c10);
    return fmaf(az, c1 - c0, c0);
}

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace pyronn
