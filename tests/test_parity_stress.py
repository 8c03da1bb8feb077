"""Stress configuration at full size (config 5): 32M-leaf background (levels 6-16, 500 x 500 x 40 m),
64 actors of 40k leaves with overlapping screen footprints, 6 cameras at 3840x2160 rendered in one
call.  Sampled pixels of every camera against the oracle; the backward of one camera (upstream
gradient on sampled pixels only) against the oracle's analytic gradient on the voxels those rays hit
(see test_parity_large for why that reduced scene is exact)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_forward, check_grads, device_scene, split_images
from test_parity_large import _actor_pixels, _reduced_scene

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def config5():
    return synth.config5(0)


def _sample(scene, cam, n, seed):
    rng = np.random.default_rng(seed)
    pix = rng.choice(cam.W * cam.H, size=n, replace=False)
    return np.unique(np.concatenate([pix, _actor_pixels(scene, cam, per_actor=2, seed=seed)]))


def test_config5_six_4k_cameras_sampled_pixels(dv, config5):
    import torch
    sc, cams = config5
    ds = device_scene(sc)
    rgb, depth, alpha, st = dv.dv_render(ds, sc.poses, cams, dv.make_opts(1, 1e-4), save_state=True)
    torch.cuda.synchronize()
    stats = st.stats()
    assert stats["n_visible"] > 5_000_000 and stats["n_tiles"] == 6 * 240 * 135
    gr = split_images(rgb.cpu().numpy(), cams, 3)
    gd = split_images(depth.cpu().numpy(), cams)
    ga = split_images(alpha.cpu().numpy(), cams)
    st.free()
    for c, cam in enumerate(cams):
        pix = _sample(sc, cam, 24, seed=100 + c)
        o = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(1, 1e-4), pixels=pix)
        v, u = pix // cam.W, pix % cam.W
        check_forward(gr[c][v, u], gd[c][v, u], ga[c][v, u], o[0], o[1], o[2], f"cfg5 camera {c}")


def test_config5_backward_on_sampled_pixels(dv, config5):
    import torch
    sc, cams = config5
    cam = cams[0]
    pix = _sample(sc, cam, 24, seed=7)
    P = cam.W * cam.H
    rng = np.random.default_rng(8)
    g_rgb = np.zeros((P, 3), np.float32)
    g_d = np.zeros(P, np.float32)
    g_a = np.zeros(P, np.float32)
    g_rgb[pix] = rng.normal(size=(pix.size, 3))
    g_d[pix] = 0.01 * rng.normal(size=pix.size)
    g_a[pix] = rng.normal(size=pix.size)
    ds = device_scene(sc)
    rgb, depth, alpha, st = dv.dv_render(ds, sc.poses, [cam], dv.make_opts(1, 1e-4), save_state=True)
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    t = lambda a: torch.as_tensor(a, device="cuda")
    dv.dv_render_backward(st, t(g_rgb), t(g_d), t(g_a), d_dens, d_sh)
    torch.cuda.synchronize()
    st.free()
    red, maps = _reduced_scene(sc, cam, pix)
    od, os_ = oracle.backward(red, sc.poses, cam, np.float64(g_rgb[pix]), np.float64(g_d[pix]),
                              np.float64(g_a[pix]), oracle.Opts(1, 1e-4), pixels=pix)
    check_grads([d_dens[i].cpu().numpy()[maps[i]] for i in range(len(red))], od, "cfg5 d_dens on hit voxels")
    check_grads([d_sh[i].cpu().numpy()[maps[i]] for i in range(len(red))], os_, "cfg5 d_sh on hit voxels")
