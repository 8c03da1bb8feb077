"""Forward parity: CUDA path (through the C ABI) vs the FP64 oracle, element by element.

Tolerances are those of tests/helpers.py (RGB/alpha 1e-4 absolute, depth 1e-3 relative)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import (check_forward, device_scene, gpu_render, orbit, sample_pixels, small_comp_scene,
                     split_images)

pytestmark = pytest.mark.gpu


def _compare_full(sc, cams, K=1, eps=1e-4, act=0, what=""):
    ds = device_scene(sc)
    rgb, depth, alpha, _ = gpu_render(ds, sc.poses, cams, K, eps, act)
    gr = split_images(rgb.cpu().numpy(), cams, 3)
    gd = split_images(depth.cpu().numpy(), cams)
    ga = split_images(alpha.cpu().numpy(), cams)
    for c, cam in enumerate(cams):
        o = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(K, eps, act))
        check_forward(gr[c], gd[c], ga[c], o[0], o[1], o[2], f"{what} cam{c}")
    return gr, ga


@pytest.mark.parametrize("K,eps", [(1, 1e-4), (2, 0.0), (4, 1e-4)])
def test_config1_full_image(dv, K, eps):
    sc, cams, _ = synth.config1()
    _, ga = _compare_full(sc, cams, K, eps, what=f"cfg1 K={K}")
    assert (ga[0] > 0.5).mean() > 0.3


def test_config1_identity_activation(dv):
    sc, cams, _ = synth.config1()
    _compare_full(sc, cams, 1, 0.0, act=1, what="cfg1 identity")


@pytest.mark.parametrize("seed,W,H", [(0, 64, 48), (1, 37, 23), (2, 100, 70), (3, 17, 16), (4, 1, 1)])
def test_compositional_small_scenes_ragged_sizes(dv, seed, W, H):
    sc = small_comp_scene(seed=seed, n_actors=3)
    cams = [orbit(W, H, 25.0 + 40 * seed, 15.0 + 5 * seed)]
    for K, eps in ((1, 1e-4), (3, 0.0)):
        _compare_full(sc, cams, K, eps, what=f"comp seed={seed} {W}x{H} K={K}")


def test_multiple_cameras_concatenated(dv):
    sc = small_comp_scene(seed=5, n_actors=2)
    cams = [orbit(40, 30, 10.0, 20.0), orbit(33, 41, 130.0, -10.0), orbit(16, 16, 250.0, 35.0)]
    _compare_full(sc, cams, 2, 1e-4, what="3 cameras")


def test_dense_opaque_scene_early_stop(dv):
    sc = small_comp_scene(seed=6, n_actors=2, density_scale=30.0)
    cams = [orbit(48, 40, 60.0, 25.0)]
    for eps in (1e-4, 1e-2, 0.3):
        _compare_full(sc, cams, 1, eps, what=f"opaque eps={eps}")


def test_empty_background_and_off_screen_actor(dv):
    sc = small_comp_scene(seed=7, n_actors=2, empty_bg=True)
    sc.poses[2] = synth.Pose(np.eye(3), np.array([0.0, 0.0, 40.0]))   # far outside the view
    _compare_full(sc, [orbit(32, 24, 45.0, 30.0)], 1, 1e-4, what="empty bg")


def test_zero_size_image_and_no_voxels(dv):
    sc = small_comp_scene(seed=8, n_actors=1, empty_bg=True)
    sc.octrees[1].key = sc.octrees[1].key[:0]
    sc.octrees[1].dens = sc.octrees[1].dens[:0]
    sc.octrees[1].sh = sc.octrees[1].sh[:0]
    ds = device_scene(sc)
    empty = orbit(16, 16, 0.0, 0.0)
    empty.W = empty.H = 0
    rgb, depth, alpha, _ = gpu_render(ds, sc.poses, [empty])
    assert rgb.numel() == 0
    _compare_full(sc, [orbit(20, 20, 0.0, 0.0)], 1, 1e-4, what="no voxels")


def test_camera_inside_the_grid_near_plane_crossings(dv):
    sc = small_comp_scene(seed=9, n_actors=2)
    cam = synth.pinhole(48, 36, 90.0, synth.look_at((0.2, 0.1, 0.05), (1.0, 0.4, 0.2)), near=0.05, far=20.0)
    _compare_full(sc, [cam], 2, 1e-4, what="inside grid")


def test_actor_box_containing_the_camera(dv):
    sc = small_comp_scene(seed=10, n_actors=2)
    cam = synth.pinhole(40, 30, 70.0, synth.look_at(sc.poses[1].t + np.array([0.05, 0.0, 0.02]), (0.0, 0.0, 0.0)),
                        near=0.02, far=20.0)
    _compare_full(sc, [cam], 1, 1e-4, what="camera in actor box")


def test_overlapping_actor_boxes(dv):
    sc = small_comp_scene(seed=11, n_actors=3)
    sc.poses[2] = synth.Pose(sc.poses[1].R, sc.poses[1].t + np.array([0.15, 0.1, 0.0], np.float32))
    sc.poses[3] = synth.Pose(sc.poses[1].R, sc.poses[1].t + np.array([-0.1, 0.12, 0.05], np.float32))
    _compare_full(sc, [orbit(56, 44, 75.0, 20.0)], 2, 1e-4, what="overlapping boxes")


def test_config2_full_frame_sampled_pixels(dv, config2_scene):
    sc, cams, _ = config2_scene
    ds = device_scene(sc)
    rgb, depth, alpha, st = gpu_render(ds, sc.poses, cams, 1, 1e-4, save_state=True)
    stats = st.stats(0)
    assert stats["n_pairs"] > 100_000 and stats["n_visible"] > 20_000
    cam = cams[0]
    # uniform sample plus a block around the image centre, where the actors are
    pix = sample_pixels(cam, 768, seed=1)
    cy, cx = cam.H // 2, cam.W // 2
    extra = np.array([(cy + dy) * cam.W + cx + dx for dy in range(-40, 60, 7) for dx in range(-400, 400, 37)])
    pix = np.unique(np.concatenate([pix, extra]))
    o = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(1, 1e-4), pixels=pix)
    g_rgb = rgb.cpu().numpy()[pix]
    g_d = depth.cpu().numpy()[pix]
    g_a = alpha.cpu().numpy()[pix]
    check_forward(g_rgb, g_d, g_a, o[0], o[1], o[2], "cfg2 sampled")
    assert (o[2] > 0.5).mean() > 0.2
    st.free()


def test_batched_views_with_their_own_poses(dv):
    """dv_render_views: every view has its own camera and actor poses; each view matches the oracle
    rendered with that view's poses, and equals the same view rendered alone."""
    import torch
    sc = small_comp_scene(seed=12, n_actors=3)
    rng = np.random.default_rng(12)
    views = []
    for k in range(4):
        poses = [sc.poses[0]] + [synth.Pose(synth.random_rotation(rng), rng.uniform(-0.7, 0.7, 3))
                                 for _ in sc.poses[1:]]
        W, H = [(40, 30), (17, 23), (64, 48), (33, 33)][k]
        views.append((orbit(W, H, 30.0 + 70 * k, 10.0 + 8 * k), poses))
    ds = device_scene(sc)
    opts = dv.make_opts(2, 1e-4)
    rgb, depth, alpha, _ = dv.dv_render_views(ds, views, opts)
    torch.cuda.synchronize()
    cams = [c for c, _ in views]
    gr = split_images(rgb.cpu().numpy(), cams, 3)
    gd = split_images(depth.cpu().numpy(), cams)
    ga = split_images(alpha.cpu().numpy(), cams)
    for k, (cam, poses) in enumerate(views):
        o = oracle.render(sc.octrees, poses, cam, oracle.Opts(2, 1e-4))
        check_forward(gr[k], gd[k], ga[k], o[0], o[1], o[2], f"batched view {k}")
        r1, d1, a1, _ = dv.dv_render_views(ds, [(cam, poses)], opts)
        torch.cuda.synchronize()
        np.testing.assert_allclose(r1.cpu().numpy().reshape(cam.H, cam.W, 3), gr[k], atol=1e-6)
        np.testing.assert_allclose(a1.cpu().numpy().reshape(cam.H, cam.W), ga[k], atol=1e-6)


def test_maximum_octree_count_many_actors_per_tile(dv):
    # 1 background + 127 actors (the most one call takes): most tiles see more actor boxes than
    # the lockstep slots, so the per-lane actor walk runs as well
    sc = small_comp_scene(seed=21, n_actors=127)
    assert len(sc.octrees) == 128
    cams = [orbit(48, 40, 35.0, 25.0)]
    _compare_full(sc, cams, 1, 1e-4, what="128 octrees")


def test_axis_parallel_rays(dv):
    # camera axes exactly along the grid axes (x right = +x, y down = +y, z forward = +z) with the
    # principal point on a pixel centre: the middle row and column of pixels have ray direction
    # components that are exactly zero, i.e. rays parallel to voxel slabs, some starting inside
    # a slab (the camera sits inside the grid's x and y extent)
    sc = small_comp_scene(seed=23, n_actors=0)
    W = H = 33
    fx = 20.0
    pose = synth.Pose(np.eye(3), np.array([0.13, -0.21, -1.9]))
    cam = synth.Camera(W, H, fx, fx, 16.5, 16.5, pose, 0.05, 20.0)
    gr, ga = _compare_full(sc, [cam], 2, 1e-4, what="axis-parallel rays")
    assert ga[0][16, :].max() > 0.5 and ga[0][:, 16].max() > 0.5
