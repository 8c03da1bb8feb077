"""FP64 oracle of the LiDAR-guided initialisation of the background octree (Sec. 3.3).  Test
infrastructure only: only the test suite, smoke() and the CPU-baseline leg of bench.py may import
it; it shares nothing with the CUDA path (nor with the scene generators, which use the same prior
only to shape their synthetic densities).

* Shared corners: a leaf (level l, index (i, j, k)) of an octree with finest level L has its corner
  c = (c_x, c_y, c_z) (c = c_x + 2 c_y + 4 c_z, the corner order of the density arrays) at grid point
  ((i + c_x) 2^(L-l), (j + c_y) 2^(L-l), (k + c_z) 2^(L-l)) of the finest level; leaves touching the
  same grid point share that corner's density (one value per grid point).
* Proximity subdivision (step 2): in one round, every leaf whose box lies within `threshold` of a
  LiDAR point (Euclidean distance from the point to the closed box) is replaced by its eight
  children; the other leaves are kept.
* Soft density prior (step 3, Eq. 1): a corner at distance d from the nearest LiDAR point gets
  v_far + (v_close - v_far) exp(-2 d^2 / s^2), s the minimum voxel size (v_close = -2, v_far = -10).

Everything is brute force (every query against every point) in float64.
"""
from __future__ import annotations

import numpy as np

V_CLOSE, V_FAR = -2.0, -10.0


def _unpack(keys):
    keys = np.asarray(keys, np.uint64)
    m = np.uint64((1 << 19) - 1)
    i = (keys & m).astype(np.int64)
    j = ((keys >> np.uint64(19)) & m).astype(np.int64)
    k = ((keys >> np.uint64(38)) & m).astype(np.int64)
    lev = ((keys >> np.uint64(57)) & np.uint64(31)).astype(np.int64)
    return lev, i, j, k


def _pack(lev, i, j, k):
    return ((np.asarray(lev, np.uint64) << np.uint64(57)) | (np.asarray(k, np.uint64) << np.uint64(38)) |
            (np.asarray(j, np.uint64) << np.uint64(19)) | np.asarray(i, np.uint64))


def corner_grid_points(keys, max_level):
    """[V, 8, 3] integer grid coordinates (finest level) of every leaf corner."""
    lev, i, j, k = _unpack(keys)
    sc = np.left_shift(1, max_level - lev)
    out = np.empty((len(lev), 8, 3), np.int64)
    for c in range(8):
        out[:, c, 0] = (i + (c & 1)) * sc
        out[:, c, 1] = (j + ((c >> 1) & 1)) * sc
        out[:, c, 2] = (k + ((c >> 2) & 1)) * sc
    return out


def shared_corners(keys, max_level):
    """(unique grid points [N, 3] in lexicographic (z, y, x) order, per-leaf corner index [V, 8])."""
    pts = corner_grid_points(keys, max_level)
    flat = pts.reshape(-1, 3)
    order = np.lexsort((flat[:, 0], flat[:, 1], flat[:, 2]))
    uniq, inv = [], np.empty(len(flat), np.int64)
    last = None
    for idx in order:
        p = tuple(flat[idx])
        if p != last:
            uniq.append(p)
            last = p
        inv[idx] = len(uniq) - 1
    return np.array(uniq, np.int64).reshape(-1, 3), inv.reshape(-1, 8)


def grid_to_world(grid, center, root_size, max_level):
    root_min = np.asarray(center, np.float64) - 0.5 * root_size
    return root_min + np.asarray(grid, np.float64) * (root_size / 2.0 ** max_level)


def nearest_distance(q, cloud):
    """Distance from every query point to its nearest cloud point (brute force; inf if no points)."""
    q = np.asarray(q, np.float64).reshape(-1, 3)
    cloud = np.asarray(cloud, np.float64).reshape(-1, 3)
    out = np.full(len(q), np.inf)
    for a in range(len(q)):
        if len(cloud):
            out[a] = np.sqrt(np.min(np.sum((cloud - q[a]) ** 2, axis=1)))
    return out


def soft_prior(d, s, v_close=V_CLOSE, v_far=V_FAR):
    """Eq. 1."""
    d = np.asarray(d, np.float64)
    return v_far + (v_close - v_far) * np.exp(-2.0 * d * d / (s * s))


def box_distance(lo, hi, p):
    """Distance from point p to the closed box [lo, hi]."""
    g = np.maximum(np.maximum(lo - p, 0.0), p - hi)
    return float(np.sqrt(np.sum(g * g)))


def subdivide_round(keys, center, root_size, cloud, threshold):
    """One proximity-subdivision round: (new keys, mask of the input leaves that were split)."""
    lev, i, j, k = _unpack(keys)
    root_min = np.asarray(center, np.float64) - 0.5 * root_size
    cloud = np.asarray(cloud, np.float64).reshape(-1, 3)
    split = np.zeros(len(lev), bool)
    for v in range(len(lev)):
        s = root_size / 2.0 ** lev[v]
        lo = root_min + np.array([i[v], j[v], k[v]], np.float64) * s
        hi = lo + s
        split[v] = any(box_distance(lo, hi, p) <= threshold for p in cloud)
    out = [keys[~split]]
    for c in range(8):
        out.append(_pack(lev[split] + 1, 2 * i[split] + (c & 1), 2 * j[split] + ((c >> 1) & 1),
                         2 * k[split] + ((c >> 2) & 1)))
    return np.concatenate(out).astype(np.uint64), split


def visible_from(keys, center, root_size, cams, z_min):
    """Step 1 (visibility and height pruning), as read here: a leaf is kept if its box's top is at
    or above ``z_min`` (world z) and some camera sees it, i.e. its 8 corners (camera frame,
    OpenCV axes) are not all behind the near plane or all beyond the far plane, and either some
    corners lie on each side of the near plane (the box straddles it: kept) or the bounding
    rectangle of the projected corners overlaps the image [0, W] x [0, H]."""
    lev, i, j, k = _unpack(keys)
    root_min = np.asarray(center, np.float64) - 0.5 * root_size
    keep = np.zeros(len(lev), bool)
    offs = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.float64)
    for v in range(len(lev)):
        s = root_size / 2.0 ** lev[v]
        lo = root_min + np.array([i[v], j[v], k[v]], np.float64) * s
        if lo[2] + s < z_min:
            continue
        corners = lo + offs * s
        for cam in cams:
            R = np.asarray(cam.pose.R, np.float64).reshape(3, 3)
            t = np.asarray(cam.pose.t, np.float64)
            pc = (corners - t) @ R          # camera-frame coordinates (R^T (p - t))
            z = pc[:, 2]
            near, far = float(np.float32(cam.near)), float(np.float32(cam.far))
            if np.all(z < near) or np.all(z > far):
                continue
            if np.any(z < near):
                keep[v] = True
                break
            fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
            cx, cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
            u = fx * pc[:, 0] / z + cx
            w = fy * pc[:, 1] / z + cy
            if u.max() >= 0.0 and u.min() <= cam.W and w.max() >= 0.0 and w.min() <= cam.H:
                keep[v] = True
                break
    return keep


ASSET_MARGIN = 1.2   # an asset's cubic bound: its largest box dimension scaled outward by 20% (Sec. 3.3, assets)
V_INIT_ASSET = -10.0  # every corner of a new asset grid starts empty, whatever its size or category


def asset_init(box_dims, level, v_init=V_INIT_ASSET):
    """Initial octree of a dynamic asset (Sec. 3.3, "Assets"): a uniform voxel grid in the asset's
    canonical frame (origin at the box centre, axes along the box's), bounded by a cube whose edge is
    the largest box dimension scaled by 1.2, every corner density at v_init.  Leaves are listed with
    i fastest, then j, then k.  Returns (keys uint64 [8^level], dens float64 [8^level, 8], root_size,
    center)."""
    dims = [float(x) for x in box_dims]
    root_size = ASSET_MARGIN * max(dims)
    n = 1 << int(level)
    keys = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                keys.append(int(_pack(level, i, j, k)))
    keys = np.array(keys, np.uint64)
    dens = np.full((len(keys), 8), float(v_init))
    return keys, dens, root_size, (0.0, 0.0, 0.0)
