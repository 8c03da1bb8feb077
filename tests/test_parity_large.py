"""Full-size parity on the large configurations, in the launch configuration bench.py uses
(all cameras of a frame in one call).

* config 3: 8M-leaf background, 20 actors of 20k-60k leaves, 6 surround 1920x1080 cameras:
  sampled pixels of every camera vs the oracle, and the backward checked by central finite
  differences in FP64 on 256 sampled voxel parameters.
* The finite differences run on a reduced scene: the voxels hit by the sampled pixels' rays
  (from the oracle's segment lists).  Voxels a ray does not hit do not change its result, and
  the interval partition depends only on the actor boxes, so the reduced scene renders those
  pixels exactly like the full one (asserted below before it is used).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_forward, check_grad, check_grads, device_scene, split_images

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def config3():
    return synth.config3(0)


def _actor_pixels(scene, cam, per_actor=6, seed=0):
    rng = np.random.default_rng(seed)
    Rc = np.asarray(cam.pose.R, np.float64)
    tc = np.asarray(cam.pose.t, np.float64)
    out = []
    for p in scene.poses[1:]:
        q = Rc.T @ (np.asarray(p.t, np.float64) - tc)
        if q[2] <= 1.0:
            continue
        u, v = cam.fx * q[0] / q[2] + cam.cx, cam.fy * q[1] / q[2] + cam.cy
        for _ in range(per_actor):
            uu, vv = int(u + rng.normal(0, 25)), int(v + rng.normal(0, 15))
            if 0 <= uu < cam.W and 0 <= vv < cam.H:
                out.append(vv * cam.W + uu)
    return np.array(out, np.int64)


def _sample(scene, cam, n, seed):
    rng = np.random.default_rng(seed)
    pix = rng.choice(cam.W * cam.H, size=n, replace=False)
    return np.unique(np.concatenate([pix, _actor_pixels(scene, cam, seed=seed)]))


def test_config3_six_cameras_sampled_pixels(dv, config3):
    sc, cams = config3
    ds = device_scene(sc)
    rgb, depth, alpha, st = dv.dv_render(ds, sc.poses, cams, dv.make_opts(1, 1e-4), save_state=True)
    import torch
    torch.cuda.synchronize()
    assert st.stats()["n_visible"] > 1_000_000
    gr = split_images(rgb.cpu().numpy(), cams, 3)
    gd = split_images(depth.cpu().numpy(), cams)
    ga = split_images(alpha.cpu().numpy(), cams)
    hit_actor = 0
    for c, cam in enumerate(cams):
        pix = _sample(sc, cam, 48, seed=c)
        o = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(1, 1e-4), pixels=pix)
        v, u = pix // cam.W, pix % cam.W
        check_forward(gr[c][v, u], gd[c][v, u], ga[c][v, u], o[0], o[1], o[2], f"cfg3 camera {c}")
        hit_actor += len(_actor_pixels(sc, cam, seed=c))
    assert hit_actor > 20
    st.free()


def _reduced_scene(scene, cam, pixels):
    """Voxels hit by the given pixels' rays, per octree (original order kept), plus index maps."""
    keep = [set() for _ in scene.octrees]
    for p in pixels:
        _, _, oi, vi = oracle.pixel_segments(scene.octrees, scene.poses, cam, int(p % cam.W), int(p // cam.W),
                                             cap=100000)
        for o, v in zip(oi, vi):
            keep[int(o)].add(int(v))
    red, maps = [], []
    for oc, k in zip(scene.octrees, keep):
        idx = np.array(sorted(k), np.int64)
        maps.append(idx)
        red.append(synth.Octree(oc.key[idx], oc.dens[idx], oc.sh[idx], oc.sh_degree, oc.center, oc.root_size,
                                oc.role, oc.clip_half))
    return red, maps


def test_config3_backward_central_differences_256_params(dv, config3):
    import torch
    sc, cams = config3
    cam = cams[0]
    pix = _sample(sc, cam, 40, seed=11)
    P = cam.W * cam.H
    rng = np.random.default_rng(5)
    g_rgb = np.zeros((P, 3), np.float32)
    g_d = np.zeros(P, np.float32)
    g_a = np.zeros(P, np.float32)
    g_rgb[pix] = rng.normal(size=(pix.size, 3))
    g_d[pix] = 0.05 * rng.normal(size=pix.size)
    g_a[pix] = rng.normal(size=pix.size)
    eps = 0.0   # no early stop, so the loss is smooth in every parameter
    ds = device_scene(sc)
    rgb, depth, alpha, st = dv.dv_render(ds, sc.poses, [cam], dv.make_opts(1, eps), save_state=True)
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    t = lambda a: torch.as_tensor(a, device="cuda")
    dv.dv_render_backward(st, t(g_rgb), t(g_d), t(g_a), d_dens, d_sh)
    torch.cuda.synchronize()
    st.free()
    gd = [x.cpu().numpy() for x in d_dens]
    gs = [x.cpu().numpy() for x in d_sh]

    red, maps = _reduced_scene(sc, cam, pix)
    opts = oracle.Opts(1, eps)
    full = oracle.render(sc.octrees, sc.poses, cam, opts, pixels=pix)
    part = oracle.render(red, sc.poses, cam, opts, pixels=pix)
    for a, b in zip(full[:3], part[:3]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)
    gr64, gd64, ga64 = (np.float64(x[pix]) for x in (g_rgb, g_d, g_a))
    od, os_ = oracle.backward(red, sc.poses, cam, gr64, gd64, ga64, opts, pixels=pix)
    f64 = [(o.dens.astype(np.float64), o.sh.astype(np.float64)) for o in red]

    def loss():
        r, d, a, _ = oracle.render(red, sc.poses, cam, opts, pixels=pix, f64_arrays=f64)
        return float(np.sum(gr64 * r) + np.sum(gd64 * d) + np.sum(ga64 * a))

    cand = []
    for oi in range(len(red)):
        for idx in np.argwhere(np.abs(od[oi]) > 0):
            cand.append(("d", oi, tuple(idx)))
        for idx in np.argwhere(np.abs(os_[oi]) > 0):
            cand.append(("s", oi, tuple(idx)))
    assert len(cand) >= 256
    pick = [cand[i] for i in rng.choice(len(cand), size=256, replace=False)]
    fd, gpu, ana = [], [], []
    for kind, oi, idx in pick:
        arr = f64[oi][0] if kind == "d" else f64[oi][1]
        x0 = arr[idx]
        h = 1e-6 * max(1.0, abs(x0))
        arr[idx] = x0 + h
        lp = loss()
        arr[idx] = x0 - h
        lm = loss()
        arr[idx] = x0
        fd.append((lp - lm) / (2 * h))
        full_v = maps[oi][idx[0]]
        gpu.append(gd[oi][(full_v,) + idx[1:]] if kind == "d" else gs[oi][(full_v,) + idx[1:]])
        ana.append(od[oi][idx] if kind == "d" else os_[oi][idx])
    fd, gpu, ana = np.array(fd), np.array(gpu), np.array(ana)
    check_grad(ana, fd, "cfg3 oracle analytic vs central differences")
    check_grad(gpu, fd, "cfg3 GPU vs central differences (256 parameters)")
    # and the GPU gradient of every parameter the sampled rays touch vs the oracle's analytic one
    check_grads([gd[oi][maps[oi]] for oi in range(len(red))], od, "cfg3 d_dens on hit voxels")
    check_grads([gs[oi][maps[oi]] for oi in range(len(red))], os_, "cfg3 d_sh on hit voxels")
    # parameters the oracle's rays do not touch get (next to) no gradient: at most a grazing hit
    # that fp32 geometry resolves as a sliver, far below the gradient's scale
    scale = max(np.abs(x).max(initial=0.0) for x in od + os_)
    for oi in range(len(red)):
        mask = np.ones(gd[oi].shape[0], bool)
        mask[maps[oi]] = False
        assert np.abs(gd[oi][mask]).max(initial=0.0) <= 1e-3 * scale
        assert np.abs(gs[oi][mask]).max(initial=0.0) <= 1e-3 * scale
