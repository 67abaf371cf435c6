"""FP64 reference of the acquisition-artifact simulations of Sec. 2.4 (numpy, plain loops where they
keep the definition readable). TEST INFRASTRUCTURE ONLY, like the rest of this package.

Every random quantity (shifts, noise samples, the defective columns) is an input; the functions are
the deterministic transforms the paper describes:
  * detector jitter: every detector row (axis 0) or column (axis 1) of every view shifted by an
    integer number of pixels, zero-filled;
  * Gaussian noise: a normal sample scaled by std plus mean added to each pixel;
  * ring artifacts: selected detector columns scaled by a gain (0: dead element) over a segment of
    views;
  * gantry motion blur: each projection convolved with a line kernel of L samples, unit total weight,
    rotated to the view's angle (bilinear sampling, zero outside the detector).
Sinograms are [V, Nv, Nu] (u fastest).
"""
from __future__ import annotations

import math

import numpy as np


def detector_jitter(sino, shifts, axis: int = 0) -> np.ndarray:
    """out[n, v, u] = sino[n, v, u - s[n, v]] (axis 0: rows shift along u) or
    sino[n, v - s[n, u], u] (axis 1: columns shift along v); zero where the source is outside."""
    p = np.asarray(sino, dtype=np.float64)
    V, Nv, Nu = p.shape
    s = np.asarray(shifts).reshape(V, Nv if axis == 0 else Nu)
    out = np.zeros_like(p)
    for n in range(V):
        if axis == 0:
            for v in range(Nv):
                for u in range(Nu):
                    src = u - int(s[n, v])
                    if 0 <= src < Nu:
                        out[n, v, u] = p[n, v, src]
        else:
            for u in range(Nu):
                for v in range(Nv):
                    src = v - int(s[n, u])
                    if 0 <= src < Nv:
                        out[n, v, u] = p[n, src, u]
    return out


def gaussian_noise(sino, noise, mean: float, std: float) -> np.ndarray:
    return np.asarray(sino, dtype=np.float64) + mean + std * np.asarray(noise, dtype=np.float64)


def ring_artifacts(sino, columns, gains, view_begin: int, view_end: int) -> np.ndarray:
    out = np.array(sino, dtype=np.float64)
    for c, gain in zip(columns, gains):
        out[view_begin:view_end, :, int(c)] *= float(gain)
    return out


def motion_blur(sino, angles, length: int) -> np.ndarray:
    """out[n](u, v) = (1 / L) sum_j bilinear(sino[n], u + t_j cos a_n, v + t_j sin a_n),
    t_j = j - (L - 1) / 2, j = 0 .. L - 1, zero outside the detector."""
    p = np.asarray(sino, dtype=np.float64)
    V, Nv, Nu = p.shape
    out = np.zeros_like(p)

    def sample(img, x, y):
        x0, y0 = math.floor(x), math.floor(y)
        fx, fy = x - x0, y - y0
        acc = 0.0
        for dy, wy in ((0, 1.0 - fy), (1, fy)):
            for dx, wx in ((0, 1.0 - fx), (1, fx)):
                xx, yy = x0 + dx, y0 + dy
                if 0 <= xx < Nu and 0 <= yy < Nv:
                    acc += wx * wy * img[yy, xx]
        return acc

    for n in range(V):
        ca, sa = math.cos(float(angles[n])), math.sin(float(angles[n]))
        for v in range(Nv):
            for u in range(Nu):
                acc = 0.0
                for j in range(length):
                    t = j - 0.5 * (length - 1)
                    acc += sample(p[n], u + t * ca, v + t * sa)
                out[n, v, u] = acc / length
    return out
