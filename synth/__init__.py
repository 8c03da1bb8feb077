"""Seeded synthetic inputs for the compositional sparse-voxel renderer.

This module only *builds inputs*: octree leaf sets, per-corner raw densities,
SH coefficients, SE(3) poses, pinhole cameras, target images and request
streams.  It contains none of the rendering arithmetic (no ray casting, no
interpolation, no compositing), so both the FP64 oracle and the CUDA path can
draw their inputs from it without sharing any of the method's code.

Scene layout follows the representation of DrivingVoxels (Sec. 3.1-3.2):
a background octree in world frame and one octree per rigid actor in its
canonical local frame (origin at the box centre, axes along the box axes),
each storing only leaf voxels as (level, integer grid index) with eight raw
corner densities and SH colour coefficients.

Leaf key packing (uint64): bits [0,19) = i (x index), [19,38) = j (y),
[38,57) = k (z), [57,62) = level.  A leaf at level ``l`` with index (i,j,k)
spans ``min = center - root/2 + (i,j,k) * s`` to ``min + s`` with
``s = root / 2**l``.  Corner ``c`` of the eight densities sits at offset
``(c & 1, (c >> 1) & 1, (c >> 2) & 1)`` (x is bit 0, z is bit 2).

The background generator mimics the LiDAR-guided initialisation of Sec. 3.3:
a coarse grid over the scene volume, proximity-based subdivision near
Gaussian-jittered LiDAR-like points (deeper levels nearer the sensor), and
corner densities from the soft prior of Eq. 1 (v_far = -10).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

V_FAR = -10.0      # empty density of Eq. 1
V_CLOSE = -2.0     # Eq. 1 close density (used by the 'init' density mode)
ASSET_MARGIN = 1.2 # Sec. 3.3, assets: largest box dimension scaled by 20%
SH_C0 = 0.28209479177387814  # 1 / (2 sqrt(pi)); only used to encode a DC colour

BG, ACTOR = 0, 1

_IMASK = (1 << 19) - 1


def pack_keys(level, i, j, k) -> np.ndarray:
    level = np.asarray(level, dtype=np.uint64)
    i = np.asarray(i, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    k = np.asarray(k, dtype=np.uint64)
    return (level << np.uint64(57)) | (k << np.uint64(38)) | (j << np.uint64(19)) | i


def unpack_keys(key: np.ndarray):
    key = np.asarray(key, dtype=np.uint64)
    m = np.uint64(_IMASK)
    i = (key & m).astype(np.int64)
    j = ((key >> np.uint64(19)) & m).astype(np.int64)
    k = ((key >> np.uint64(38)) & m).astype(np.int64)
    level = ((key >> np.uint64(57)) & np.uint64(31)).astype(np.int64)
    return level, i, j, k


@dataclass
class Octree:
    key: np.ndarray            # uint64 [V]
    dens: np.ndarray           # float32 [V, 8]
    sh: np.ndarray             # float32 [V, n_sh, 3]
    sh_degree: int
    center: tuple              # 3 floats (float64)
    root_size: float
    role: int = BG
    clip_half: tuple = (0.0, 0.0, 0.0)  # actor clip box half extents (local frame)

    @property
    def n(self) -> int:
        return int(self.key.shape[0])

    def voxel_bounds(self):
        """(min corner [V,3], size [V]) in float64 -- a convenience for generators/tests."""
        level, i, j, k = unpack_keys(self.key)
        s = self.root_size / np.exp2(level.astype(np.float64))
        base = np.asarray(self.center, np.float64) - self.root_size / 2
        mn = base[None, :] + np.stack([i, j, k], 1).astype(np.float64) * s[:, None]
        return mn, s


@dataclass
class Pose:
    """Rigid transform local -> world: p_world = R @ p_local + t."""
    R: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    t: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))

    def __post_init__(self):
        self.R = np.asarray(self.R, np.float32).reshape(3, 3)
        self.t = np.asarray(self.t, np.float32).reshape(3)

    def matrix(self) -> np.ndarray:
        m = np.eye(4)
        m[:3, :3] = self.R
        m[:3, 3] = self.t
        return m

    @staticmethod
    def from_matrix(m) -> "Pose":
        m = np.asarray(m, np.float64)
        return Pose(m[:3, :3], m[:3, 3])


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward), pose = camera -> world."""
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    pose: Pose
    near: float = 0.05
    far: float = 1000.0


@dataclass
class Scene:
    octrees: list              # [Octree], index 0 = background
    poses: list                # [Pose] per octree (background: identity unless stated)


# ---------------------------------------------------------------------------
# rotations / cameras
# ---------------------------------------------------------------------------

def rot_z(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> Pose:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return Pose(np.stack([r, d, f], 1), eye)


def pinhole(W, H, fov_deg, pose: Pose, near=0.05, far=1000.0) -> Camera:
    """fov is horizontal; fx = fy; principal point at the image centre."""
    fx = (W / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return Camera(int(W), int(H), float(np.float32(fx)), float(np.float32(fx)),
                  W / 2.0, H / 2.0, pose, float(near), float(far))


def orbit_camera(W, H, fov_deg, dist, az_deg, el_deg, target=(0.0, 0.0, 0.0), near=0.05, far=100.0):
    az, el = math.radians(az_deg), math.radians(el_deg)
    t = np.asarray(target, np.float64)
    eye = t + dist * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return pinhole(W, H, fov_deg, look_at(eye, t), near, far)


def vehicle_camera(W, H, fov_deg, yaw_deg, position=(0.0, 0.0, 1.8), pitch_deg=0.0, near=0.1, far=400.0):
    """A roof camera looking along heading yaw (world z up)."""
    yaw, pitch = math.radians(yaw_deg), math.radians(pitch_deg)
    p = np.asarray(position, np.float64)
    f = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), -math.sin(pitch)])
    return pinhole(W, H, fov_deg, look_at(p, p + f), near, far)


def surround_cameras(W, H, n=6, fov_deg=60.0, position=(0.0, 0.0, 1.8), far=400.0):
    return [vehicle_camera(W, H, fov_deg, i * 360.0 / n, position, far=far) for i in range(n)]


# ---------------------------------------------------------------------------
# colour / density helpers (inputs only)
# ---------------------------------------------------------------------------

def n_sh(degree: int) -> int:
    return (degree + 1) ** 2


def sh_from_rgb(rgb: np.ndarray, degree: int = 0) -> np.ndarray:
    """SH coefficients whose DC term encodes ``rgb`` under colour = SH + 0.5 (higher bands zero)."""
    rgb = np.asarray(rgb, np.float64)
    sh = np.zeros((rgb.shape[0], n_sh(degree), 3), np.float64)
    sh[:, 0, :] = (rgb - 0.5) / SH_C0
    return sh.astype(np.float32)


def _box_surface_distance(p: np.ndarray, c: np.ndarray, h: np.ndarray) -> np.ndarray:
    q = np.abs(p - c) - h
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return np.abs(outside + inside)


def _corner_offsets() -> np.ndarray:
    c = np.arange(8)
    return np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], 1).astype(np.float64)


def soft_prior_density(dist: np.ndarray, s: np.ndarray, v_hi: np.ndarray) -> np.ndarray:
    """Eq. 1 form: v_far + (v_hi - v_far) * exp(-2 d^2 / s^2)."""
    return V_FAR + (v_hi - V_FAR) * np.exp(-2.0 * dist * dist / (s * s))


# ---------------------------------------------------------------------------
# small scenes
# ---------------------------------------------------------------------------

def grid_octree(level: int, center=(0.0, 0.0, 0.0), root_size=2.0, rng=None, dens=None, rgb=None,
                sh_degree=0, role=BG, clip_half=(0.0, 0.0, 0.0), ijk=None) -> Octree:
    """Uniform grid of leaves at one level (all 8**level cells unless ``ijk`` is given)."""
    n = 1 << level
    if ijk is None:
        k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    ijk = np.asarray(ijk, np.int64).reshape(-1, 3)
    V = ijk.shape[0]
    if dens is None:
        dens = rng.lognormal(0.0, 1.0, (V, 8))
    if rgb is None:
        rgb = rng.uniform(0.0, 1.0, (V, 3))
    key = pack_keys(np.full(V, level), ijk[:, 0], ijk[:, 1], ijk[:, 2])
    return Octree(key, np.asarray(dens, np.float32).reshape(V, 8), sh_from_rgb(rgb, sh_degree), sh_degree,
                  tuple(float(x) for x in center), float(root_size), role, tuple(float(x) for x in clip_half))


def config1(seed: int = 0):
    """Plain static scene: 16^3 leaves at level 4 of [-1,1]^3, LogNormal(0,1) corner densities,
    SH degree 0 from RGB ~ U(0,1); one 64x64 camera, fov 60, distance 2.5 (generic direction);
    plus a U(0,1) target image for an L2 loss."""
    rng = np.random.default_rng(seed)
    oc = grid_octree(4, rng=rng)
    cam = orbit_camera(64, 64, 60.0, 2.5, 30.0, 20.0, near=0.1, far=100.0)
    target = rng.uniform(0.0, 1.0, (64, 64, 3)).astype(np.float32)
    return Scene([oc], [Pose()]), [cam], target


# ---------------------------------------------------------------------------
# LiDAR-shaped background
# ---------------------------------------------------------------------------

@dataclass
class CityLayout:
    half_xy: float
    height: float
    buildings_c: np.ndarray   # [B,3]
    buildings_h: np.ndarray   # [B,3] half extents


def city_layout(rng, half_xy: float, height: float, n_buildings: int, road_half=12.0) -> CityLayout:
    cs, hs = [], []
    tries = 0
    while len(cs) < n_buildings and tries < 10000:
        tries += 1
        size = rng.uniform(5.0, 30.0, 3)
        size[2] = min(size[2], height - 1.0)
        c = np.array([rng.uniform(-half_xy + size[0] / 2, half_xy - size[0] / 2),
                      rng.uniform(-half_xy + size[1] / 2, half_xy - size[1] / 2), size[2] / 2])
        h = size / 2
        if abs(c[1]) - h[1] < road_half:          # keep the road corridor along x free
            continue
        ok = all(np.any(np.abs(c - c2) > h + h2 + 1.0) for c2, h2 in zip(cs, hs))
        if ok:
            cs.append(c)
            hs.append(h)
    return CityLayout(half_xy, height, np.array(cs).reshape(-1, 3), np.array(hs).reshape(-1, 3))


def lidar_points(rng, lay: CityLayout, n_ground: int, n_building: int, sigma=0.05, r0=1.5):
    """LiDAR-like points: ground hits with density ~ 1/r^2 around the sensor, building faces
    weighted by area / distance^2; every point Gaussian-jittered with std ``sigma``."""
    R = lay.half_xy * math.sqrt(2.0)
    r = r0 * (R / r0) ** rng.uniform(0.0, 1.0, n_ground)
    a = rng.uniform(0.0, 2 * math.pi, n_ground)
    g = np.stack([r * np.cos(a), r * np.sin(a), np.zeros(n_ground)], 1)
    g = g[(np.abs(g[:, 0]) < lay.half_xy) & (np.abs(g[:, 1]) < lay.half_xy)]
    pts = [g]
    if lay.buildings_c.shape[0] and n_building > 0:
        faces = []   # (centre, u-axis half vec, v-axis half vec, weight)
        for c, h in zip(lay.buildings_c, lay.buildings_h):
            for ax in range(3):
                for sgn in ((1.0,) if ax == 2 else (-1.0, 1.0)):
                    fc = c.copy()
                    fc[ax] += sgn * h[ax]
                    u, v = [x for x in range(3) if x != ax]
                    area = 4 * h[u] * h[v]
                    d2 = max(float(np.dot(fc, fc)), 25.0)
                    faces.append((fc, u, v, h[u], h[v], area / d2))
        w = np.array([f[5] for f in faces])
        cnt = rng.multinomial(n_building, w / w.sum())
        for f, m in zip(faces, cnt):
            if m == 0:
                continue
            fc, u, v, hu, hv, _ = f
            p = np.repeat(fc[None, :], m, 0)
            p[:, u] += rng.uniform(-hu, hu, m)
            p[:, v] += rng.uniform(-hv, hv, m)
            pts.append(p)
    p = np.concatenate(pts, 0)
    p += rng.normal(0.0, sigma, p.shape)
    return p


def _surface_distance(corners: np.ndarray, mn: np.ndarray, s: np.ndarray, lay: CityLayout) -> np.ndarray:
    """Distance of each voxel corner [V,8,3] to the nearest surface (ground plane or building box).
    Buildings are only visited for voxels within three voxel sizes of them; beyond that the Eq. 1
    prior is already at v_far, so the ground distance is kept there."""
    d = np.abs(corners[..., 2])
    cc = mn + 0.5 * s[:, None]
    for c, h in zip(lay.buildings_c, lay.buildings_h):
        near = np.all(np.abs(cc - c) < h + 3.5 * s[:, None], axis=1)
        idx = np.nonzero(near)[0]
        if idx.size:
            d[idx] = np.minimum(d[idx], _box_surface_distance(corners[idx], c, h))
    return d


def _unique_sorted(x: np.ndarray) -> np.ndarray:
    x = np.sort(x)
    if x.size == 0:
        return x
    return x[np.concatenate([[True], x[1:] != x[:-1]])]


def _in_sorted(x: np.ndarray, table: np.ndarray) -> np.ndarray:
    if table.size == 0:
        return np.zeros(x.shape, bool)
    pos = np.minimum(np.searchsorted(table, x), table.size - 1)
    return table[pos] == x


def lidar_background(n_target: int, seed: int, root_size=200.0, center=(0.0, 0.0, 15.0), level_min=6,
                     level_max=12, half_xy=100.0, height=30.0, n_buildings=20, sh_degree=3,
                     n_ground=1_000_000, n_building=400_000, fine_radius=6.0,
                     transparent=False):
    """Background octree shaped by a synthetic LiDAR sweep (Sec. 3.3 steps 1-3, synthetic analogue).

    1. a coarse grid of level ``level_min`` cells over the scene box (height-filtered to [0, height]);
    2. proximity subdivision: a cell containing a point is split while its level is below the
       distance-dependent maximum (``level_max`` within ``fine_radius`` of the sensor, one level
       less per doubling of the distance);
    3. corner densities from the Eq. 1 form with the distance to the nearest surface, v_far = -10
       and a close value chosen so that a surface voxel has optical depth about 3 (x LogNormal(0,.25));
       ``transparent=True`` draws LogNormal(0,1) raw densities instead (worst case for early stop).
    Leaves are trimmed to ``n_target`` (seeded), dropping empty-space leaves first."""
    rng = np.random.default_rng(seed)
    lay = city_layout(rng, half_xy, height, n_buildings)
    pts = lidar_points(rng, lay, n_ground, n_building)
    center = np.asarray(center, np.float64)
    rmin = center - root_size / 2

    def cell_max_level(lv, ijk):
        s = root_size / (1 << lv)
        cx = rmin[0] + (ijk[:, 0] + 0.5) * s
        cy = rmin[1] + (ijk[:, 1] + 0.5) * s
        r2 = cx * cx + cy * cy
        edges = (fine_radius * np.exp2(np.arange(0, level_max - level_min + 1))) ** 2
        return np.maximum(level_max - np.searchsorted(edges, r2, side="right"), level_min)

    def pack(ijk):
        return (ijk[:, 2] << 42) | (ijk[:, 1] << 21) | ijk[:, 0]

    # occupied cells per level, derived from the finest level by integer halving of the packed keys
    # (each 21-bit field shifted right by one: the bit that crosses into the next field is cleared)
    sf = root_size / (1 << level_max)
    pc = np.floor((pts - rmin) / sf).astype(np.int64)
    pc = pc[(pc >= 0).all(1) & (pc < (1 << level_max)).all(1)]
    occ_keys = {level_max: _unique_sorted(pack(pc))}
    halve = ~np.int64((1 << 20) | (1 << 41))
    for lv in range(level_max - 1, level_min - 1, -1):
        occ_keys[lv] = _unique_sorted((occ_keys[lv + 1] >> 1) & halve)

    s0 = root_size / (1 << level_min)
    n0 = 1 << level_min
    ix = np.arange(n0)
    xs = rmin[0] + (ix + 0.5) * s0
    ys = rmin[1] + (ix + 0.5) * s0
    zs = rmin[2] + (ix + 0.5) * s0
    ii = ix[np.abs(xs) < half_xy]
    jj = ix[np.abs(ys) < half_xy]
    kk = ix[(zs > -s0) & (zs < height + s0)]
    K, J, I = np.meshgrid(kk, jj, ii, indexing="ij")
    cur = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.int64)
    leaves, occ_flags = [], []
    off = _corner_offsets().astype(np.int64)
    for lv in range(level_min, level_max + 1):
        is_occ = _in_sorted(pack(cur), occ_keys[lv])
        if lv == level_max:
            split = np.zeros(cur.shape[0], bool)
        else:
            split = is_occ & (lv < cell_max_level(lv, cur))
        leaves.append((lv, cur[~split]))
        occ_flags.append(is_occ[~split])
        par = cur[split]
        if par.shape[0] == 0:
            break
        cur = (2 * par[:, None, :] + off[None, :, :]).reshape(-1, 3)
    lv_all = np.concatenate([np.full(k.shape[0], lv) for lv, k in leaves])
    ijk_all = np.concatenate([k for _, k in leaves], 0)
    occ_all = np.concatenate(occ_flags)
    V = lv_all.shape[0]
    if V > n_target:
        pri = rng.uniform(0.0, 1.0, V) + np.where(occ_all, 1.0, 0.0)   # empty leaves go first
        keep = np.sort(np.argpartition(-pri, n_target - 1)[:n_target])
        lv_all, ijk_all = lv_all[keep], ijk_all[keep]
        V = n_target
    key = pack_keys(lv_all, ijk_all[:, 0], ijk_all[:, 1], ijk_all[:, 2])
    order = np.argsort(key, kind="stable")
    key, lv_all, ijk_all = key[order], lv_all[order], ijk_all[order]
    s = (root_size / np.exp2(lv_all.astype(np.float64))).astype(np.float32)
    mn = (rmin[None, :] + ijk_all * s[:, None].astype(np.float64)).astype(np.float32)
    if transparent:
        dens = rng.lognormal(0.0, 1.0, (V, 8)).astype(np.float32)
    else:
        corners = mn[:, None, :] + _corner_offsets().astype(np.float32)[None, :, :] * s[:, None, None]
        dist = _surface_distance(corners, mn, s, lay)
        v_hi = (3.0 / s)[:, None] * rng.lognormal(0.0, 0.25, (V, 8)).astype(np.float32)
        dens = soft_prior_density(dist, s[:, None], v_hi)
    sh = rng.standard_normal((V, n_sh(sh_degree), 3), dtype=np.float32) * np.float32(0.1)
    oc = Octree(key, dens.astype(np.float32), sh, sh_degree,
                tuple(float(x) for x in center), float(root_size), BG)
    return oc, lay


# ---------------------------------------------------------------------------
# actors
# ---------------------------------------------------------------------------

def actor_octree(n_target: int, seed: int, dims=(4.5, 1.9, 1.6), sh_degree=3, level=None) -> Octree:
    """Actor in its canonical frame (Sec. 3.2): origin at the box centre, root = 1.2 x largest
    box dimension (Sec. 3.3, assets), clip box = annotated box x 1.2 per axis.  Leaves are the
    ``n_target`` grid cells inside the clip box nearest to the body surface; corner densities
    follow the Eq. 1 form of the distance to the body (optical depth ~3 at the surface)."""
    rng = np.random.default_rng(seed)
    dims = np.asarray(dims, np.float64)
    root = ASSET_MARGIN * float(dims.max())
    clip_half = ASSET_MARGIN * dims / 2
    if level is None:
        level = 6 if n_target <= 30_000 else 7
    s = root / (1 << level)
    n = 1 << level
    lo = np.ceil((root / 2 - clip_half) / s - 1e-9).astype(np.int64)
    hi = np.floor((root / 2 + clip_half) / s + 1e-9).astype(np.int64)   # exclusive upper cell
    I, J, K = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]), np.arange(lo[2], hi[2]),
                          indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    ijk = ijk[(ijk >= 0).all(1) & (ijk < n).all(1)]
    mn = -root / 2 + ijk * s
    cc = mn + s / 2
    body_h = dims / 2 * np.array([0.95, 0.9, 0.9])
    d = _box_surface_distance(cc, np.zeros(3), body_h) + rng.uniform(0, 1e-3 * s, ijk.shape[0])
    order = np.argsort(d, kind="stable")[:n_target]
    ijk = ijk[np.sort(order)]
    V = ijk.shape[0]
    key = pack_keys(np.full(V, level), ijk[:, 0], ijk[:, 1], ijk[:, 2])
    mn = -root / 2 + ijk * s
    corners = mn[:, None, :] + _corner_offsets()[None, :, :] * s
    dist = _box_surface_distance(corners, np.zeros(3), body_h)
    v_hi = (3.0 / s) * rng.lognormal(0.0, 0.25, (V, 8))
    dens = soft_prior_density(dist, s, v_hi)
    sh = rng.normal(0.0, 0.1, (V, n_sh(sh_degree), 3))
    return Octree(key, dens.astype(np.float32), sh.astype(np.float32), sh_degree, (0.0, 0.0, 0.0), root,
                  ACTOR, tuple(float(x) for x in clip_half))


@dataclass
class Lane:
    p0: np.ndarray     # start position (x, y, z)
    yaw: float         # heading
    speed: float

    def pose(self, t: float) -> Pose:
        h = np.array([math.cos(self.yaw), math.sin(self.yaw), 0.0])
        return Pose(rot_z(self.yaw), self.p0 + self.speed * t * h)


def lanes(n: int, seed: int, x_range=(8.0, 45.0), y_range=(-9.0, 9.0), z=0.8, box_half=(2.7, 1.14, 0.96),
          min_gap=0.5):
    """Straight-line tracks with yaw ~ U(-pi, pi) and speed ~ U(5, 15) m/s; boxes disjoint at t = 0."""
    rng = np.random.default_rng(seed)
    out = []
    rad = float(np.hypot(box_half[0], box_half[1])) + min_gap
    tries = 0
    while len(out) < n:
        tries += 1
        p = np.array([rng.uniform(*x_range), rng.uniform(*y_range), z])
        if tries < 100000 and any(np.hypot(*(p[:2] - l.p0[:2])) < 2 * rad for l in out):
            continue
        out.append(Lane(p, float(rng.uniform(-math.pi, math.pi)), float(rng.uniform(5.0, 15.0))))
    return out


def street_scene(n_bg: int, actor_sizes, seed: int, t: float = 0.0, sh_degree=3, transparent=False, **bg_kw):
    bg, lay = lidar_background(n_bg, seed, sh_degree=sh_degree, transparent=transparent, **bg_kw)
    octs, poses = [bg], [Pose()]
    tracks = lanes(len(actor_sizes), seed + 1000,
                   x_range=(8.0, 8.0 + 6.0 * max(len(actor_sizes), 6)) if len(actor_sizes) > 8 else (8.0, 45.0),
                   y_range=(-9.0, 9.0))
    for a, n in enumerate(actor_sizes):
        octs.append(actor_octree(int(n), seed + 2000 + a, sh_degree=sh_degree))
        poses.append(tracks[a].pose(t))
    sc = Scene(octs, poses)
    sc.layout = lay
    sc.tracks = tracks
    return sc


def config2(seed: int = 0, transparent=False):
    """Compositional forward+backward: 500k-leaf LiDAR-shaped background (levels 6-12, 200 m root),
    3 actors of 20k leaves fit to 4.5 x 1.9 x 1.6 m boxes on straight lanes, SH degree 3 ~ N(0, 0.1);
    one 1920x1080 front camera."""
    sc = street_scene(500_000, [20_000] * 3, seed, transparent=transparent)
    cam = vehicle_camera(1920, 1080, 60.0, 0.0)
    rng = np.random.default_rng(seed + 7)
    target = rng.uniform(0.0, 1.0, (1080, 1920, 3)).astype(np.float32)
    return sc, [cam], target


def config3(seed: int = 0):
    """Full frame: 8M-leaf background (levels 6-14, 200 x 200 x 30 m), 20 actors of 20k-60k leaves,
    6 surround 1920x1080 cameras at 60 degree yaw spacing."""
    rng = np.random.default_rng(seed + 11)
    sizes = rng.integers(20_000, 60_001, 20)
    sc = street_scene(8_000_000, sizes, seed, level_max=14, n_ground=12_000_000, n_building=5_000_000,
                      fine_radius=6.0)
    cams = surround_cameras(1920, 1080)
    return sc, cams


def config4(seed: int = 0):
    """Serving scene: the config-2 background with 20 actors of 20k leaves on straight lanes (their
    poses follow the request timestamp)."""
    return street_scene(500_000, [20_000] * 20, seed)


def config5(seed: int = 0):
    """Stress: 32M-leaf background (levels 6-16, 500 x 500 x 40 m), 64 actors of 40k leaves,
    6 cameras at 3840x2160."""
    sc = street_scene(32_000_000, [40_000] * 64, seed, root_size=500.0, center=(0.0, 0.0, 20.0), level_max=16,
                      half_xy=250.0, height=40.0, n_ground=40_000_000, n_building=16_000_000, fine_radius=4.0)
    cams = surround_cameras(3840, 2160, far=800.0)
    return sc, cams


# ---------------------------------------------------------------------------
# serving request stream
# ---------------------------------------------------------------------------

RESOLUTIONS = ((480, 270), (960, 540), (1920, 1080))


@dataclass
class Request:
    rid: int
    arrival_s: float
    camera: Camera
    t: float                 # timestamp setting every actor pose


def request_stream(n: int, rate_hz: float, seed: int, resolutions=RESOLUTIONS, track_len=100.0):
    """Poisson arrivals; camera at u ~ U(0,1) along a 100 m straight trajectory (x axis),
    timestamp ~ U(0, 10) s (it sets every actor pose), resolution uniform over ``resolutions``."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n)
    arr = np.cumsum(gaps)
    out = []
    for r in range(n):
        u = rng.uniform(0.0, 1.0)
        W, H = resolutions[int(rng.integers(0, len(resolutions)))]
        cam = vehicle_camera(W, H, 60.0, 0.0, position=(-50.0 + track_len * u, 0.0, 1.8))
        out.append(Request(r, float(arr[r]), cam, float(rng.uniform(0.0, 10.0))))
    return out


def request_poses(scene, t: float):
    """Octree poses at timestamp t: background fixed, every actor on its lane."""
    return [scene.poses[0]] + [tr.pose(t) for tr in scene.tracks]
