"""Pins of the initialisation oracle (oracle/init.py, Sec. 3.3):

- Eq. 1: v_close at d = 0, v_far far away, v_far + (v_close - v_far)/e at d = s/sqrt(2);
- shared corners: a full n^3 grid of leaves has (n+1)^3 corners; every corner index of a leaf
  points at the grid point of that corner; two face neighbours share exactly four corners;
  a coarse leaf next to fine ones shares only the grid points the fine ones touch;
- nearest distance == scipy's k-d tree query;
- subdivision: the children exactly tile the parent, untouched leaves are kept, and a leaf is
  split iff some point lies within the threshold of its box (checked against a dense sampling
  of the box).
"""
import math

import numpy as np
import pytest

import oracle.init as oi
import synth


def test_eq1_closed_forms():
    s = 0.3
    assert oi.soft_prior(0.0, s) == pytest.approx(-2.0, abs=1e-15)
    assert oi.soft_prior(100.0, s) == pytest.approx(-10.0, abs=1e-15)
    assert oi.soft_prior(s / math.sqrt(2.0), s) == pytest.approx(-10.0 + 8.0 / math.e, rel=1e-14)
    d = np.linspace(0, 1, 11)
    assert np.all(np.diff(oi.soft_prior(d, s)) < 0)


def test_full_grid_has_n_plus_one_cubed_corners():
    n, L = 4, 2
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    keys = synth.pack_keys(np.full(n ** 3, L), i.ravel(), j.ravel(), k.ravel())
    pts, idx = oi.shared_corners(keys, L)
    assert len(pts) == (n + 1) ** 3
    grid = oi.corner_grid_points(keys, L)
    np.testing.assert_array_equal(pts[idx], grid)
    # face neighbours along x share the 4 corners of their common face
    a = int(np.where((i.ravel() == 1) & (j.ravel() == 2) & (k.ravel() == 0))[0][0])
    b = int(np.where((i.ravel() == 2) & (j.ravel() == 2) & (k.ravel() == 0))[0][0])
    assert len(set(idx[a]) & set(idx[b])) == 4
    assert set(idx[a][[1, 3, 5, 7]]) == set(idx[b][[0, 2, 4, 6]])


def test_mixed_levels_share_grid_points_only():
    # one level-1 leaf and the 8 level-2 leaves of its +x neighbour: the coarse leaf's +x face has
    # 4 corners; the fine leaves touch 9 points of that face, 4 of which are the coarse corners
    keys = [synth.pack_keys([1], [0], [0], [0])[0]]
    for c in range(8):
        keys.append(synth.pack_keys([2], [2 + (c & 1)], [(c >> 1) & 1], [(c >> 2) & 1])[0])
    keys = np.array(keys, np.uint64)
    pts, idx = oi.shared_corners(keys, 2)
    coarse_face = set(idx[0][[1, 3, 5, 7]])
    fine_pts = set(idx[1:].ravel())
    assert coarse_face <= fine_pts
    assert len(pts) == 8 + 27 - 4


def test_nearest_distance_matches_kdtree():
    sp = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(0)
    cloud = rng.normal(size=(300, 3))
    q = rng.normal(size=(50, 3)) * 1.5
    np.testing.assert_allclose(oi.nearest_distance(q, cloud), sp.cKDTree(cloud).query(q)[0], rtol=1e-12)


def test_subdivision_round():
    rng = np.random.default_rng(1)
    L = 2
    i, j, k = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    keys = synth.pack_keys(np.full(64, L), i.ravel(), j.ravel(), k.ravel())
    cloud = rng.uniform(-1.0, 1.0, size=(6, 3))
    center, root, thr = (0.0, 0.0, 0.0), 2.0, 0.12
    new, split = oi.subdivide_round(keys, center, root, cloud, thr)
    assert 0 < split.sum() < 64
    assert len(new) == 64 + 7 * split.sum()
    # volumes: children tile their parents
    lev, *_ = oi._unpack(new)
    assert np.sum(8.0 ** -lev) == pytest.approx(1.0)
    # dense sampling of each box: split iff some point is within the threshold of a sample
    root_min = -1.0
    for v in range(64):
        s = root / 4
        lo = root_min + np.array([i.ravel()[v], j.ravel()[v], k.ravel()[v]]) * s
        g = np.stack(np.meshgrid(*[np.linspace(0, 1, 21)] * 3, indexing="ij"), -1).reshape(-1, 3) * s + lo
        dmin = np.min(np.linalg.norm(g[:, None, :] - cloud[None], axis=2))
        if dmin <= thr - 0.06:
            assert split[v]
        if dmin > thr + 1e-9:
            assert not split[v]


def test_visibility_pruning_reading():
    # a camera at (0.5, 0.5, 0.5) looking along +x, far plane 2: leaves behind it, outside its field of
    # view, beyond its far plane or below the height threshold are pruned; leaves in view or around
    # the camera are kept
    from types import SimpleNamespace
    eye = np.array([0.5, 0.5, 0.5])
    cam_pose = synth.look_at(eye, eye + np.array([1.0, 0.0, 0.0]))
    cam = SimpleNamespace(W=64, H=48, fx=40.0, fy=40.0, cx=32.0, cy=24.0, near=0.1, far=2.0,
                          pose=SimpleNamespace(R=np.asarray(cam_pose.R, np.float64), t=eye))
    L = 3   # root 8 m centred at 0: 1 m leaves
    n = 8
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    keys = synth.pack_keys(np.full(n ** 3, L), i.ravel(), j.ravel(), k.ravel())
    keep = oi.visible_from(keys, (0.0, 0.0, 0.0), 8.0, [cam], z_min=-2.5)
    lo = np.stack([i.ravel(), j.ravel(), k.ravel()], 1) - 4.0       # leaf min corners (1 m leaves)
    at = lambda x, y, z: int(np.where((lo[:, 0] == x) & (lo[:, 1] == y) & (lo[:, 2] == z))[0][0])
    assert keep[at(2, 0, 0)]            # ahead on the axis, partly within the far plane
    assert keep[at(0, 0, 0)]            # contains the camera (straddles the near plane)
    assert not keep[at(-4, 0, 0)]       # behind
    assert not keep[at(3, 0, 0)]        # entirely beyond the far plane
    assert not keep[at(2, 0, -4)]       # top at z = -3, below the height threshold
    # the horizontal field of view is 2 atan(32/40) ~ 77 deg: a leaf far to the side of the axis is pruned
    assert not keep[at(2, 3, 0)]
    assert 0 < keep.sum() < len(keys)


# ---------------------------------------------------------------------------
# asset initialisation (Sec. 3.3, "Assets")
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,level", [((4.5, 1.9, 1.6), 3), ((1.0, 2.5, 0.8), 2), ((3.0, 3.0, 3.0), 0)])
def test_asset_grid_tiles_its_cubic_bound(dims, level):
    keys, dens, root, center = oi.asset_init(dims, level)
    n = 1 << level
    assert len(keys) == n ** 3 and dens.shape == (n ** 3, 8)
    lev, i, j, k = synth.unpack_keys(keys)
    assert np.all(lev == level)
    # every cell of the n^3 grid appears exactly once: the leaves tile the cube without gaps or overlaps
    cells = np.unique(np.stack([i, j, k], 1), axis=0)
    assert cells.shape[0] == n ** 3 and cells.min() == 0 and cells.max() == n - 1
    # the box grown by 20% fits inside the cube centred on the box, and touches it along its largest axis
    assert center == (0.0, 0.0, 0.0)
    grown = 0.5 * 1.2 * np.asarray(dims, np.float64)
    assert np.all(grown <= 0.5 * root + 1e-12)
    assert grown.max() == pytest.approx(0.5 * root, rel=1e-15)
    # one empty density everywhere, whatever the size
    assert np.all(dens == -10.0)


def test_asset_grid_renders_as_a_uniform_empty_medium():
    """A fresh asset placed by a rigid pose renders, through the compositing oracle, exactly like one
    homogeneous medium of density explin(-10) filling its clip box: alpha = 1 - exp(-sigma l) with l the
    ray's chord through the clip box within the grid's cube (found by bisection of a point-in-box test).  A missing or doubled
    leaf would change l; alpha stays far below visible (the paper's 'empty' initial density)."""
    import oracle
    from helpers import pose64
    from test_oracle_pins import cam_looking, chord_bisect, ray_of

    dims = (4.5, 1.9, 1.6)
    keys, dens, root, _ = oi.asset_init(dims, 3)
    clip = tuple(0.6 * d for d in dims)
    act = synth.Octree(keys, np.float32(dens), np.zeros((len(keys), 1, 3), np.float32), 0, (0.0, 0.0, 0.0), root,
                       role=synth.ACTOR, clip_half=clip)
    bg = synth.Octree(np.zeros(0, np.uint64), np.zeros((0, 8), np.float32), np.zeros((0, 1, 3), np.float32), 0,
                      (0.0, 0.0, 0.0), 8.0)
    # the pose as the renderers receive it (float32)
    R = np.float32(synth.rot_z(0.7)).astype(np.float64)
    t = np.float32([0.3, -0.2, 0.1]).astype(np.float64)
    cam = cam_looking((7.0, 3.0, 2.0), (0.2, -0.1, 0.0), W=12, H=9, fov=40.0)
    rgb, depth, alpha, nseg = oracle.render([bg, act], [pose64(), pose64(R, t)], cam, oracle.Opts(K=1, eps_stop=0.0))
    sigma = 1.1 * math.exp(-10.0 / 1.1 - 1.0)
    hits = 0
    for v in range(cam.H):
        for u in range(cam.W):
            o, d = ray_of(cam, u, v)
            # the medium fills the clip box (as the renderers receive it, float32) within the grid's cube
            c32 = np.minimum(np.float32(clip).astype(np.float64), 0.5 * root)
            ch = chord_bisect(R.T @ (o - t), R.T @ d, -c32, c32, tmax=20.0)
            if ch is None:
                assert alpha[v, u] == 0.0
                continue
            hits += 1
            a = 1.0 - math.exp(-sigma * (ch[1] - ch[0]))
            assert alpha[v, u] == pytest.approx(a, rel=1e-9)
            assert alpha[v, u] < 1e-3
    assert hits >= 20
