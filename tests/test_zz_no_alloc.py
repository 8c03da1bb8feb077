"""The allocation-free backward (dv_render_backward_static) against the allocating one.

Callers that may not allocate device memory while the backward runs (graph capture without
allocation nodes, real-time loops, a device whose memory belongs to another allocator) use the
static-scratch variant.  This file runs last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest
import ctypes as C

import synth
from helpers import check_grad, check_grads, device_scene, orbit, small_comp_scene

pytestmark = pytest.mark.gpu


def _grads(fn, st, ds, g):
    import torch
    d_dens = [torch.zeros_like(o.dens) for o in ds]
    d_sh = [torch.zeros_like(o.sh) for o in ds]
    fn(st, g[0], g[1], g[2], d_dens, d_sh)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in d_dens], [x.cpu().numpy() for x in d_sh]


def test_static_backward_matches_allocating_backward_twice(dv):
    import torch
    sc = small_comp_scene(seed=21, n_actors=3)
    cams = [orbit(61, 47, 40.0, 20.0), orbit(33, 29, 200.0, -5.0)]
    ds = device_scene(sc)
    rgb, depth, alpha, st = dv.dv_render(ds, sc.poses, cams, dv.make_opts(2, 1e-4), save_state=True)
    gen = torch.Generator(device="cuda").manual_seed(3)
    P = rgb.shape[0]
    g = (torch.randn((P, 3), device="cuda", generator=gen), 0.1 * torch.randn((P,), device="cuda", generator=gen),
         torch.randn((P,), device="cuda", generator=gen))
    ref_d, ref_s = _grads(dv.dv_render_backward, st, ds, g)
    assert sum(np.count_nonzero(x) for x in ref_d) > 100
    for call in range(2):
        got_d, got_s = _grads(dv.dv_render_backward_static, st, ds, g)
        check_grads(got_d, ref_d, f"static call {call} d_dens")
        check_grads(got_s, ref_s, f"static call {call} d_sh")
    st.free()


def test_static_backward_rejects_cameras_above_the_limit(dv):
    import torch
    # a dense level-6 grid (262144 leaves) seen whole: more visible voxels than the static scratch holds
    rng = np.random.default_rng(0)
    oc = synth.grid_octree(6, rng=rng)
    ds = device_scene(synth.Scene([oc], [synth.Pose()]))
    cam = orbit(64, 64, 30.0, 20.0, dist=4.0)
    rgb, depth, alpha, st = dv.dv_render(ds, [synth.Pose()], [cam], dv.make_opts(1, 1e-4), save_state=True)
    assert st.stats(0)["n_visible"] > dv.STATIC_MAX_VISIBLE
    d_dens = [torch.zeros_like(ds[0].dens)]
    d_sh = [torch.zeros_like(ds[0].sh)]
    with pytest.raises(dv.DVError) as ei:
        dv.dv_render_backward_static(st, torch.ones_like(rgb), None, None, d_dens, d_sh)
    assert ei.value.status == dv.DV_ERR_CAPACITY
    assert "static limit" in str(ei.value)
    st.free()
