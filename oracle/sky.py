"""FP64 oracle of the sky composite (Sec. 3.2 "Sky Modeling", Eq. 2).  Test infrastructure only:
only the test suite, smoke() and the CPU-baseline leg of bench.py may import it; it shares
nothing with the CUDA path.

    C = C_voxels + T_final * C_sky(d)

with d the unit world direction of the pixel's ray and C_sky a bilinear lookup of a 2-D
spherical environment map.  The paper names the map and the bilinear lookup but not the map's
parameterisation; the reading used here (and by the GPU path) is the equirectangular map of
the world frame with z up:

  * column coordinate  x = (atan2(d_y, d_x) + pi) / (2 pi) * W   (longitude, -pi at x = 0)
  * row coordinate     y = acos(d_z) / pi * H                    (polar angle, +z at y = 0)
  * texel (i, j) covers [i, i+1) x [j, j+1); its value sits at its centre (i + 1/2, j + 1/2);
  * bilinear interpolation between the four nearest centres, wrapping around in longitude and
    clamping to the first / last row in latitude.

Everything is written per pixel with Python loops over the four texels (slow, small images only).
"""
from __future__ import annotations

import math

import numpy as np


def pixel_directions(cam):
    """Unit world directions of every pixel centre ([H*W, 3]), OpenCV camera axes."""
    R = np.asarray(cam.pose.R, np.float64).reshape(3, 3)
    v, u = np.meshgrid(np.arange(cam.H), np.arange(cam.W), indexing="ij")
    dc = np.stack([(u.ravel() + 0.5 - float(np.float32(cam.cx))) / float(np.float32(cam.fx)),
                   (v.ravel() + 0.5 - float(np.float32(cam.cy))) / float(np.float32(cam.fy)),
                   np.ones(cam.W * cam.H)], 1)
    d = dc @ R.T
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _taps(d, H, W):
    """The four (row, column, weight) taps of the bilinear lookup for direction d."""
    lon = math.atan2(d[1], d[0])
    polar = math.acos(max(-1.0, min(1.0, d[2])))
    x = (lon + math.pi) / (2.0 * math.pi) * W - 0.5
    y = polar / math.pi * H - 0.5
    i0, j0 = math.floor(x), math.floor(y)
    fx, fy = x - i0, y - j0
    taps = []
    for dj, wy in ((0, 1.0 - fy), (1, fy)):
        j = min(max(j0 + dj, 0), H - 1)
        for di, wx in ((0, 1.0 - fx), (1, fx)):
            taps.append((j, (i0 + di) % W, wx * wy))
    return taps


def sky_color(env, d):
    env = np.asarray(env, np.float64)
    H, W = env.shape[:2]
    return sum(w * env[j, i] for j, i, w in _taps(d, H, W))


def composite(rgb, alpha, dirs, env):
    """C = rgb + (1 - alpha) * C_sky(d) per pixel ([n,3], [n], [n,3] -> [n,3])."""
    rgb = np.asarray(rgb, np.float64).reshape(-1, 3)
    alpha = np.asarray(alpha, np.float64).reshape(-1)
    out = np.empty_like(rgb)
    for p in range(rgb.shape[0]):
        out[p] = rgb[p] + (1.0 - alpha[p]) * sky_color(env, dirs[p])
    return out


def backward(alpha, dirs, env, g_out):
    """Given dL/dC ([n,3]): dL/d env ([H,W,3]), dL/d alpha ([n]) and dL/d rgb (= dL/dC)."""
    env = np.asarray(env, np.float64)
    H, W = env.shape[:2]
    alpha = np.asarray(alpha, np.float64).reshape(-1)
    g_out = np.asarray(g_out, np.float64).reshape(-1, 3)
    d_env = np.zeros_like(env)
    d_alpha = np.zeros(alpha.shape[0])
    for p in range(alpha.shape[0]):
        sky = np.zeros(3)
        for j, i, w in _taps(dirs[p], H, W):
            d_env[j, i] += w * (1.0 - alpha[p]) * g_out[p]
            sky += w * env[j, i]
        d_alpha[p] = -float(np.dot(g_out[p], sky))
    return d_env, d_alpha, g_out.copy()
