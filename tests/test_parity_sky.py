"""Sky composite (Eq. 2) on the GPU vs the FP64 oracle (oracle/sky.py): forward on rendered
images, the backward (map gradient by atomics, alpha gradient added to what the caller passes),
the chain into dv_render_backward, and a 1080p frame with a 512 x 1024 map on sampled pixels.
Cameras include one looking at the zenith and one looking across the longitude seam.

Tolerances: colours 1e-4 absolute, the RGB target of every parity test.  The inputs are the GPU's
own fp32 images, so only the lookup differs: the fp32 ray direction, atan2 and acos carry a few
1e-7 rad, i.e. up to ~1e-4 texel at 1024 columns, and a noise map changes by up to 1 between
neighbouring texels.  Map and alpha gradients: 1e-5 (|ref| + max|ref|) on small maps."""
import math

import numpy as np
import pytest

import oracle
import oracle.sky as osky
import synth
from helpers import check_grads, device_scene, orbit, small_comp_scene

pytestmark = pytest.mark.gpu


def _rel_close(a, b, what, rtol=1e-5):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    lim = rtol * (np.abs(b) + np.abs(b).max(initial=0.0)) + 1e-7
    err = np.abs(a - b)
    assert (err <= lim).all(), f"{what}: max err {err.max():.3g} (limit {lim[np.argmax(err - lim)]:.3g})"


def _cams():
    up = synth.pinhole(24, 20, 80.0, synth.look_at((0.0, 0.0, 0.5), (0.001, 0.0, 5.0), up=(1.0, 0.0, 0.0)), 0.05, 50.0)
    seam = synth.pinhole(30, 18, 90.0, synth.look_at((0.0, 0.0, 0.0), (-1.0, 0.0, 0.1)), 0.05, 50.0)
    return [orbit(40, 32, 30.0, 20.0), up, seam]


def _env(H=32, W=64, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(H, W, 3)).astype(np.float32)


def test_sky_composite_forward(dv):
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=50, n_actors=2)
    cams = _cams()
    ds = device_scene(sc)
    rgb, depth, alpha, _ = m.dv_render(ds, sc.poses, cams, m.make_opts(1, 1e-4))
    env = _env()
    out = m.dv_sky_composite(cams, torch.as_tensor(env, device="cuda"), rgb, alpha)
    torch.cuda.synchronize()
    r, a, o = rgb.cpu().numpy(), alpha.cpu().numpy(), out.cpu().numpy()
    off = 0
    for cam in cams:
        n = cam.W * cam.H
        ref = osky.composite(r[off:off + n], a[off:off + n], osky.pixel_directions(cam), env)
        err = np.abs(o[off:off + n] - ref).max()
        assert err <= 1e-4, f"sky forward {cam.W}x{cam.H}: {err:.3g}"
        off += n
    assert (a < 0.5).any(), "some pixels should see the sky"


def test_sky_backward_and_chain_into_render_backward(dv):
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=51, n_actors=2)
    cam = orbit(36, 28, 150.0, 10.0)
    ds = device_scene(sc)
    rgb, depth, alpha, st = m.dv_render(ds, sc.poses, [cam], m.make_opts(1, 1e-4), save_state=True)
    env = _env(16, 48, seed=1)
    env_d = torch.as_tensor(env, device="cuda")
    P = cam.W * cam.H
    rng = np.random.default_rng(51)
    g = np.float32(rng.normal(size=(P, 3)))
    g_a0 = np.float32(rng.normal(size=P))
    d_env = torch.zeros_like(env_d)
    d_alpha = torch.as_tensor(g_a0, device="cuda").clone()
    g_t = torch.as_tensor(g, device="cuda")
    m.dv_sky_backward([cam], env_d, alpha, g_t, d_env, d_alpha)
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    m.dv_render_backward(st, g_t, None, d_alpha, d_dens, d_sh)
    torch.cuda.synchronize()
    st.free()
    dirs = osky.pixel_directions(cam)
    a = alpha.cpu().numpy()
    ref_env, ref_alpha, _ = osky.backward(a, dirs, env, np.float64(g))
    _rel_close(d_env.cpu().numpy(), ref_env, "d_env")
    _rel_close(d_alpha.cpu().numpy() - g_a0, ref_alpha, "d_alpha (added)")
    # the chain: render gradient for dL/dC = g and dL/dalpha = g_a0 + sky term
    od, os_ = oracle.backward(sc.octrees, sc.poses, cam, np.float64(g), np.zeros(P),
                              np.float64(g_a0) + ref_alpha, oracle.Opts(1, 1e-4))
    check_grads([x.cpu().numpy() for x in d_dens], od, "sky chain d_dens")
    check_grads([x.cpu().numpy() for x in d_sh], os_, "sky chain d_sh")


def test_sky_1080p_frame_sampled(dv, config2_scene):
    import torch
    import paper_2606_23031_gb300 as m
    sc, cams, _ = config2_scene
    cam = cams[0]
    ds = device_scene(sc)
    rgb, depth, alpha, _ = m.dv_render(ds, sc.poses, [cam], m.make_opts(1, 1e-4))
    env = _env(512, 1024, seed=2)
    out = m.dv_sky_composite([cam], torch.as_tensor(env, device="cuda"), rgb, alpha)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    pix = rng.choice(cam.W * cam.H, size=2000, replace=False)
    dirs = osky.pixel_directions(cam)[pix]
    ref = osky.composite(rgb.cpu().numpy()[pix], alpha.cpu().numpy()[pix], dirs, env)
    err = np.abs(out.cpu().numpy()[pix] - ref).max()
    assert err <= 1e-4, f"1080p sky: {err:.3g}"


def test_sky_rejects_bad_arguments(dv):
    import torch
    import paper_2606_23031_gb300 as m
    cam = orbit(8, 8, 0.0, 0.0)
    x = torch.zeros((64, 3), device="cuda")
    a = torch.zeros(64, device="cuda")
    with pytest.raises(RuntimeError):
        m.dv_sky_composite([cam], torch.zeros((0, 4, 3), device="cuda"), x, a)
