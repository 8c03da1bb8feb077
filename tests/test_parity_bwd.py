"""Backward parity: gradients from the CUDA replay (through the C ABI and through the
autograd Function) vs the oracle's analytic FP64 gradients on the same inputs.
The oracle's analytic gradient is itself pinned to central differences in test_oracle_pins."""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_grad, check_grads, device_scene, gpu_render, orbit, sample_pixels, small_comp_scene

pytestmark = pytest.mark.gpu


def _gpu_grads(sc, cams, g_rgb, g_depth, g_alpha, K=1, eps=1e-4):
    import torch
    import paper_2606_23031_gb300 as dv
    ds = device_scene(sc)
    rgb, depth, alpha, st = gpu_render(ds, sc.poses, cams, K, eps, save_state=True)
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    t = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    dv.dv_render_backward(st, t(g_rgb), t(g_depth), t(g_alpha), d_dens, d_sh)
    torch.cuda.synchronize()
    st.free()
    return [x.cpu().numpy() for x in d_dens], [x.cpu().numpy() for x in d_sh], (rgb, depth, alpha)


def _compare(sc, cams, g_rgb, g_depth, g_alpha, K=1, eps=1e-4, what="", pixels=None):
    gd, gs, _ = _gpu_grads(sc, cams, g_rgb, g_depth, g_alpha, K, eps)
    cam = cams[0]
    if pixels is None:
        od, os_ = oracle.backward(sc.octrees, sc.poses, cam, np.float64(np.float32(g_rgb)).reshape(-1, 3),
                                  np.float64(np.float32(g_depth)).reshape(-1), np.float64(np.float32(g_alpha)).reshape(-1),
                                  oracle.Opts(K, eps))
    else:
        od, os_ = oracle.backward(sc.octrees, sc.poses, cam, np.float64(np.float32(g_rgb)).reshape(-1, 3)[pixels],
                                  np.float64(np.float32(g_depth)).reshape(-1)[pixels],
                                  np.float64(np.float32(g_alpha)).reshape(-1)[pixels], oracle.Opts(K, eps),
                                  pixels=pixels)
    check_grads(gd, od, f"{what} d_dens")
    check_grads(gs, os_, f"{what} d_sh")
    return gd, od


@pytest.mark.parametrize("K,eps", [(1, 1e-4), (2, 0.0)])
def test_config1_l2_loss_gradients(dv, K, eps):
    sc, cams, target = synth.config1()
    ds = device_scene(sc)
    rgb, _, _, _ = gpu_render(ds, sc.poses, cams, K, eps)
    C = rgb.cpu().numpy().reshape(64, 64, 3)
    g_rgb = 2.0 * (C - target)
    zeros = np.zeros((64, 64), np.float32)
    gd, od = _compare(sc, cams, g_rgb, zeros, zeros, K, eps, what=f"cfg1 L2 K={K}")
    assert np.count_nonzero(od[0]) > 1000


def test_config1_mixed_upstream(dv):
    sc, cams, _ = synth.config1()
    rng = np.random.default_rng(2)
    _compare(sc, cams, rng.normal(size=(64, 64, 3)), rng.normal(size=(64, 64)) * 0.2, rng.normal(size=(64, 64)),
             2, 1e-4, what="cfg1 mixed")


@pytest.mark.parametrize("seed,W,H", [(0, 48, 40), (1, 37, 23), (6, 30, 30)])
def test_compositional_gradients(dv, seed, W, H):
    sc = small_comp_scene(seed=seed, n_actors=3, density_scale=3.0 if seed == 6 else 1.0)
    cams = [orbit(W, H, 30.0 + 50 * seed, 20.0)]
    rng = np.random.default_rng(seed)
    _compare(sc, cams, rng.normal(size=(H, W, 3)), rng.normal(size=(H, W)) * 0.2, rng.normal(size=(H, W)), 2, 1e-4,
             what=f"comp seed={seed}")


def test_autograd_function_matches_oracle(dv):
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=3, n_actors=2)
    cam = orbit(40, 32, 70.0, 25.0)
    ds = device_scene(sc)
    dens = [o.dens.clone().requires_grad_(True) for o in ds]
    sh = [o.sh.clone().requires_grad_(True) for o in ds]
    target = torch.rand((40 * 32, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    rgb, depth, alpha = m.render(ds, sc.poses, [cam], m.make_opts(2, 1e-4), dens=dens, sh=sh)
    loss = ((rgb - target) ** 2).sum() + 0.1 * depth.sum() + alpha.sum()
    loss.backward()
    g_rgb = (2.0 * (rgb - target)).detach().cpu().numpy().astype(np.float64)
    od, os_ = oracle.backward(sc.octrees, sc.poses, cam, g_rgb, np.full(40 * 32, np.float64(np.float32(0.1))),
                              np.ones(40 * 32), oracle.Opts(2, 1e-4))
    check_grads([d.grad.cpu().numpy() for d in dens], od, "autograd dens")
    check_grads([s.grad.cpu().numpy() for s in sh], os_, "autograd sh")


def test_config2_sampled_pixel_gradients(dv, config2_scene):
    sc, cams, target = config2_scene
    cam = cams[0]
    pix = sample_pixels(cam, 256, seed=3)
    cy, cx = cam.H // 2, cam.W // 2
    extra = np.array([(cy + dy) * cam.W + cx + dx for dy in range(-30, 40, 13) for dx in range(-300, 300, 41)])
    pix = np.unique(np.concatenate([pix, extra]))
    rng = np.random.default_rng(4)
    P = cam.W * cam.H
    g_rgb = np.zeros((P, 3), np.float32)
    g_d = np.zeros(P, np.float32)
    g_a = np.zeros(P, np.float32)
    g_rgb[pix] = rng.normal(size=(pix.size, 3))
    g_d[pix] = rng.normal(size=pix.size) * 0.01
    g_a[pix] = rng.normal(size=pix.size)
    _compare(sc, cams, g_rgb, g_d, g_a, 1, 1e-4, what="cfg2 sampled", pixels=pix)


def test_batched_views_backward(dv):
    """Backward of a batched call over views with different poses == the sum of the oracle's
    gradients of every view."""
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=13, n_actors=2)
    rng = np.random.default_rng(13)
    views = []
    for k in range(3):
        poses = [sc.poses[0]] + [synth.Pose(synth.random_rotation(rng), rng.uniform(-0.6, 0.6, 3))
                                 for _ in sc.poses[1:]]
        views.append((orbit(30 + 7 * k, 26, 50.0 + 90 * k, 15.0), poses))
    ds = device_scene(sc)
    rgb, depth, alpha, st = m.dv_render_views(ds, views, m.make_opts(1, 1e-4), save_state=True)
    P = rgb.shape[0]
    g = [rng.normal(size=(P, 3)), rng.normal(size=P) * 0.1, rng.normal(size=P)]
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    m.dv_render_backward(st, t(g[0]), t(g[1]), t(g[2]), d_dens, d_sh)
    torch.cuda.synchronize()
    st.free()
    ref_d = [np.zeros(o.dens.shape) for o in sc.octrees]
    ref_s = [np.zeros(o.sh.shape) for o in sc.octrees]
    off = 0
    for cam, poses in views:
        n = cam.W * cam.H
        sl = slice(off, off + n)
        od, os_ = oracle.backward(sc.octrees, poses, cam, np.float64(np.float32(g[0][sl])),
                                  np.float64(np.float32(g[1][sl])), np.float64(np.float32(g[2][sl])),
                                  oracle.Opts(1, 1e-4))
        for i in range(len(ref_d)):
            ref_d[i] += od[i]
            ref_s[i] += os_[i]
        off += n
    check_grads([x.cpu().numpy() for x in d_dens], ref_d, "batched d_dens")
    check_grads([x.cpu().numpy() for x in d_sh], ref_s, "batched d_sh")


def test_maximum_octree_count_gradients(dv):
    sc = small_comp_scene(seed=22, n_actors=127)
    cams = [orbit(40, 32, 120.0, 20.0)]
    rng = np.random.default_rng(22)
    _compare(sc, cams, rng.normal(size=(32, 40, 3)), rng.normal(size=(32, 40)) * 0.2, rng.normal(size=(32, 40)), 1,
             1e-4, what="128 octrees")
