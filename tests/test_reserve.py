"""The workspace reservation and the CAPACITY contract (dv_reserve, dv_workspace_need).

A render limited to a workspace it cannot fit fails with DV_ERR_CAPACITY: before any work is
enqueued when the part known from the octree, camera and tile counts is already too large, after the
projection (outputs untouched) when the visible-voxel and pair counts push it over.  The caller
reserves what dv_workspace_need reports and retries; the retried render matches the oracle."""
import numpy as np
import pytest

import oracle
from helpers import check_forward, device_scene, orbit, small_comp_scene, split_images

pytestmark = pytest.mark.gpu


def test_capacity_then_reserve_and_retry(dv):
    import torch
    sc = small_comp_scene(seed=31, n_actors=2)
    ds = device_scene(sc)
    cam = orbit(40, 32, 70.0, 25.0)
    opts = dv.make_opts(1, 1e-4)
    ctx = dv.Context(0)
    P = cam.W * cam.H
    out = (torch.full((P, 3), float("nan"), device="cuda"), torch.full((P,), float("nan"), device="cuda"),
           torch.full((P,), float("nan"), device="cuda"))

    # 1. far too small: refused before anything is enqueued
    ctx.reserve(4096)
    n0 = dv.dv_launch_count()
    with pytest.raises(dv.DVError) as ei:
        dv.dv_render(ds, sc.poses, [cam], opts, ctx=ctx, out=out)
    assert ei.value.status == dv.DV_ERR_CAPACITY
    assert dv.dv_launch_count() == n0
    need0 = ctx.workspace_need()
    assert need0 > 4096

    # 2. the part known up front fits, the sized part does not: refused after the projection, outputs untouched
    ctx.reserve(need0)
    with pytest.raises(dv.DVError) as ei:
        dv.dv_render(ds, sc.poses, [cam], opts, ctx=ctx, out=out)
    assert ei.value.status == dv.DV_ERR_CAPACITY and "no output was written" in str(ei.value)
    assert dv.dv_launch_count() > n0
    torch.cuda.synchronize()
    assert all(torch.isnan(t).all().item() for t in out)
    need = ctx.workspace_need()
    assert need > need0

    # 3. reserve the whole need and retry: the render goes through and matches the oracle
    ctx.reserve(need)
    rgb, depth, alpha, st = dv.dv_render(ds, sc.poses, [cam], opts, ctx=ctx, out=out, save_state=True)
    st.check(wait=True)
    st.free()
    o_rgb, o_d, o_a, _ = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(1, 1e-4))
    check_forward(split_images(rgb.cpu().numpy(), [cam], 3)[0], split_images(depth.cpu().numpy(), [cam])[0],
                  split_images(alpha.cpu().numpy(), [cam])[0], o_rgb, o_d, o_a, "render after reserve")
    assert ctx.workspace_need() == need

    # 4. no limit again
    ctx.reserve(0)
    dv.dv_render(ds, sc.poses, [cam], opts, ctx=ctx)
    torch.cuda.synchronize()
    ctx.close()
