"""LiDAR-guided initialisation (Sec. 3.3) on the GPU vs the FP64 oracle (oracle/init.py):
shared corners and the subdivision round bit for bit, the Eq. 1 prior within float32 rounding
(|v| <= 10, so 1e-5 absolute), and the corner gather / scatter."""
import numpy as np
import pytest

import oracle.init as oi
import synth

pytestmark = pytest.mark.gpu


def _keys_t(keys):
    import torch
    return torch.as_tensor(np.asarray(keys, np.uint64).view(np.int64), device="cuda")


def _surface_cloud(rng, n):
    # points on a tilted plane and a sphere inside the unit root box centred at 0
    a = rng.uniform(-0.9, 0.9, size=(n // 2, 2))
    plane = np.stack([a[:, 0], a[:, 1], 0.2 * a[:, 0] - 0.1 * a[:, 1] - 0.3], 1)
    u = rng.normal(size=(n - n // 2, 3))
    sphere = 0.35 * u / np.linalg.norm(u, axis=1, keepdims=True) + np.array([0.2, -0.1, 0.25])
    return np.float32(np.concatenate([plane, sphere]))


def _grid_keys(level):
    n = 1 << level
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return synth.pack_keys(np.full(n ** 3, level), i.ravel(), j.ravel(), k.ravel())


def test_subdivision_rounds_and_shared_corners(dv):
    import torch
    import paper_2606_23031_gb300 as m
    rng = np.random.default_rng(70)
    cloud = _surface_cloud(rng, 400)
    center, root = (0.0, 0.0, 0.0), 2.0
    keys = _grid_keys(2)
    kt = _keys_t(keys)
    ct = torch.as_tensor(cloud, device="cuda")
    lev = 2
    for thr in (0.15, 0.08):
        gpu = m.dv_subdivide_round(kt, lev, center, root, ct, thr)
        ref, split = oi.subdivide_round(keys, center, root, cloud, thr)
        got = gpu.cpu().numpy().view(np.uint64)
        assert 0 < split.sum() < len(keys)
        np.testing.assert_array_equal(got, ref)
        keys, kt, lev = ref, gpu, lev + 1
    grid_g, index_g = m.dv_shared_corners(kt, lev)
    pts, idx = oi.shared_corners(keys, lev)
    g = grid_g.cpu().numpy().view(np.uint64)
    mask = np.uint64((1 << 21) - 1)
    unpacked = np.stack([(g & mask), (g >> np.uint64(21)) & mask, (g >> np.uint64(42)) & mask], 1).astype(np.int64)
    np.testing.assert_array_equal(unpacked, pts)
    np.testing.assert_array_equal(index_g.cpu().numpy().astype(np.int64), idx)


def test_soft_prior_matches_eq1_from_nearest_points(dv):
    import torch
    import paper_2606_23031_gb300 as m
    rng = np.random.default_rng(71)
    cloud = _surface_cloud(rng, 600)
    center, root, L = (0.0, 0.0, 0.0), 2.0, 4
    keys = _grid_keys(L)
    grid_g, index_g = m.dv_shared_corners(_keys_t(keys), L)
    s_min = root / 2 ** L
    dens = m.dv_soft_prior(grid_g, center, root, L, torch.as_tensor(cloud, device="cuda"), s_min).cpu().numpy()
    pts, _ = oi.shared_corners(keys, L)
    world = oi.grid_to_world(pts, center, root, L)
    ref = oi.soft_prior(oi.nearest_distance(world, np.float64(cloud)), s_min)
    assert (ref > -9.0).sum() > 50 and (ref < -9.99).sum() > 50
    np.testing.assert_allclose(dens, ref, rtol=0, atol=1e-5)
    # no points at all: every corner is empty space
    empty = m.dv_soft_prior(grid_g, center, root, L, torch.zeros((0, 3), device="cuda"), s_min).cpu().numpy()
    assert np.all(empty == np.float32(-10.0))


def test_soft_prior_with_dense_clusters(dv):
    # Dense blobs put hundreds of points into a few cells, so the search's row pruning decides
    # most corners near them; corners on every third grid line sit exactly on cell boundaries
    # (cell = 3 finest voxels).  Still the brute-force nearest point of the oracle.
    import torch
    import paper_2606_23031_gb300 as m
    rng = np.random.default_rng(73)
    centres = rng.uniform(-0.7, 0.7, size=(6, 3))
    blobs = centres[rng.integers(0, 6, size=3000)] + 0.02 * rng.normal(size=(3000, 3))
    cloud = np.float32(np.concatenate([blobs, _surface_cloud(rng, 400)]))
    center, root, L = (0.0, 0.0, 0.0), 2.0, 5
    keys = _grid_keys(L)
    grid_g, _ = m.dv_shared_corners(_keys_t(keys), L)
    s_min = root / 2 ** L
    dens = m.dv_soft_prior(grid_g, center, root, L, torch.as_tensor(cloud, device="cuda"), s_min).cpu().numpy()
    pts, _ = oi.shared_corners(keys, L)
    world = oi.grid_to_world(pts, center, root, L)
    ref = oi.soft_prior(oi.nearest_distance(world, np.float64(cloud)), s_min)
    assert (ref > -5.0).sum() > 100
    np.testing.assert_allclose(dens, ref, rtol=0, atol=1e-5)


def test_corner_gather_and_scatter(dv):
    import torch
    import paper_2606_23031_gb300 as m
    rng = np.random.default_rng(72)
    keys = _grid_keys(3)
    grid_g, index_g = m.dv_shared_corners(_keys_t(keys), 3)
    nc = int(grid_g.numel())
    corner = torch.as_tensor(np.float32(rng.normal(size=nc)), device="cuda")
    dens = m.dv_corner_gather(index_g, corner).cpu().numpy()
    idx = index_g.cpu().numpy()
    np.testing.assert_array_equal(dens, corner.cpu().numpy()[idx])
    g = np.float32(rng.normal(size=(len(keys), 8)))
    d_corner = torch.zeros(nc, device="cuda")
    m.dv_corner_scatter(index_g, torch.as_tensor(g, device="cuda"), d_corner)
    ref = np.zeros(nc)
    np.add.at(ref, idx.ravel(), np.float64(g.ravel()))
    np.testing.assert_allclose(d_corner.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


def test_level_above_max_level_is_rejected(dv):
    import paper_2606_23031_gb300 as m
    keys = synth.pack_keys([3], [1], [2], [3])
    with pytest.raises(RuntimeError):
        m.dv_shared_corners(_keys_t(keys), 2)


def test_visibility_pruning(dv):
    import paper_2606_23031_gb300 as m
    rng = np.random.default_rng(73)
    L = 4   # 16^3 leaves of a 16 m root centred at (0, 0, 4)
    keys = _grid_keys(L)
    center, root = (0.0, 0.0, 4.0), 16.0
    cams = [synth.vehicle_camera(64, 48, 70.0, yaw, position=(0.3, -0.2, 1.8), pitch_deg=5.0, near=0.2, far=9.0)
            for yaw in (0.0, 130.0)]
    gpu = m.dv_visibility_prune(_keys_t(keys), L, center, root, cams, z_min=-1.0).cpu().numpy().view(np.uint64)
    keep = oi.visible_from(keys, center, root, cams, -1.0)
    assert 0 < keep.sum() < len(keys)
    np.testing.assert_array_equal(gpu, keys[keep])


@pytest.mark.parametrize("dims,level", [((4.5, 1.9, 1.6), 4), ((0.7, 3.1, 1.2), 5), ((2.0, 2.0, 2.0), 0)])
def test_asset_init_bit_exact(dv, dims, level):
    keys, dens, root = dv.dv_asset_init(dims, level)
    ok, od, oroot, _ = oi.asset_init(np.float32(dims).astype(np.float64), level)  # the ABI carries float32 dims
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), ok)
    np.testing.assert_array_equal(dens.cpu().numpy(), np.float32(od))
    assert root == oroot


def test_asset_init_capacity_and_arguments(dv):
    import ctypes as C
    import torch
    lib = dv.load()
    ctx = dv.default_context()
    keys = torch.empty(64, dtype=torch.int64, device="cuda")
    dens = torch.empty((64, 8), dtype=torch.float32, device="cuda")
    dims = (C.c_float * 3)(4.5, 1.9, 1.6)
    root, n = C.c_double(), C.c_int64()
    launches = dv.dv_launch_count()
    st = lib.dv_asset_init(ctx.handle, dims, 3, -10.0, 64, C.c_void_p(keys.data_ptr()), C.c_void_p(dens.data_ptr()),
                           C.byref(root), C.byref(n), None)
    assert st == dv.DV_ERR_CAPACITY and n.value == 0 and dv.dv_launch_count() == launches
    bad = (C.c_float * 3)(4.5, 0.0, 1.6)
    st = lib.dv_asset_init(ctx.handle, bad, 2, -10.0, 64, C.c_void_p(keys.data_ptr()), C.c_void_p(dens.data_ptr()),
                           C.byref(root), C.byref(n), None)
    assert st == dv.DV_ERR_INVALID_ARG
    st = lib.dv_asset_init(ctx.handle, dims, 2, -10.0, 64, C.c_void_p(keys.data_ptr()), C.c_void_p(dens.data_ptr()),
                           C.byref(root), C.byref(n), None)
    assert st == dv.DV_OK and n.value == 64


def test_asset_init_renders_like_the_oracle(dv):
    """A GPU-initialised asset placed in a scene renders (GPU) as the oracle renders the oracle's grid."""
    import oracle
    from helpers import check_forward, device_scene, gpu_render, orbit, pose64, split_images
    dims = (4.5, 1.9, 1.6)
    keys, dens, root = dv.dv_asset_init(dims, 4, v_init=-2.0)   # denser than -10 so the render is visible
    rng = np.random.default_rng(5)
    k_np = keys.cpu().numpy().view(np.uint64)
    sh = np.float32(rng.normal(0.0, 0.1, size=(len(k_np), 16, 3)))
    act = synth.Octree(k_np, dens.cpu().numpy(), sh, 3, (0.0, 0.0, 0.0), root, role=synth.ACTOR,
                       clip_half=tuple(0.6 * d for d in dims))
    bg = synth.grid_octree(3, center=(0.0, 0.0, -4.0), root_size=4.0, rng=rng)
    scene = synth.Scene([bg, act], [synth.Pose(), synth.Pose(synth.rot_z(0.4), (0.5, 0.2, 0.3))])
    cam = orbit(48, 40, 50.0, 30.0, dist=9.0)
    ds = device_scene(scene)
    rgb, depth, alpha, _ = gpu_render(ds, scene.poses, [cam])
    o_rgb, o_d, o_a, _ = oracle.render(scene.octrees, scene.poses, cam, oracle.Opts(1, 1e-4))
    check_forward(split_images(rgb.cpu().numpy(), [cam], 3)[0], split_images(depth.cpu().numpy(), [cam])[0],
                  split_images(alpha.cpu().numpy(), [cam])[0], o_rgb, o_d, o_a, "asset init render")
    assert o_a.max() > 0.05
