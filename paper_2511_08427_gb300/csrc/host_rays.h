// FP64 host versions of the device ray set-up, used to bound shared-memory boxes on the host.
#pragma once

#include <cmath>

#include "pyronn_internal.h"

namespace pyronn {

struct RayD {
    double c[3], d[3];
};

// Same construction as ray_setup (device_common.cuh), unrounded.
inline RayD ray_setup_d(const FpRec &r, const pyronn_geom *g, double u, double v) {
    double Y[3], D[3];
    for (int i = 0; i < 3; ++i) {
        Y[i] = (double)r.R0[i] + u * r.Ru[i] + v * r.Rv[i];
        D[i] = (double)r.B0[i] + u * r.Bu[i] + v * r.Bv[i];
    }
    const double inv = 1.0 / std::sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    for (int i = 0; i < 3; ++i) D[i] *= inv;
    const double tau = -(Y[0] * D[0] + Y[1] * D[1] + Y[2] * D[2]);
    const double is[3] = {1.0 / g->sx, 1.0 / g->sy, 1.0 / g->sz};
    const double h[3] = {0.5 * (g->nx - 1), 0.5 * (g->ny - 1), 0.5 * (g->nz - 1)};
    RayD o;
    for (int i = 0; i < 3; ++i) {
        o.c[i] = (Y[i] + tau * D[i]) * is[i] + h[i];
        o.d[i] = D[i] * is[i];
    }
    return o;
}

}  // namespace pyronn
