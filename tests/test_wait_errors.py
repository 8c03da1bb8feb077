"""Bounded waits report on the host.  A one-sweep sort pass whose look-back runs out of its bound sets
the device's wait-error word; the next render takes it in its size read-back and fails with
DV_ERR_TIMEOUT, and the word is then clear.  Here the word is set from the host through the
library's test hook: no kernel is made to wait."""
import numpy as np
import pytest

from helpers import device_scene, orbit, small_comp_scene

pytestmark = pytest.mark.gpu


def test_sort_wait_error_is_reported_by_the_next_render(dv):
    sc = small_comp_scene(seed=41, n_actors=1)
    ds = device_scene(sc)
    cams = [orbit(20, 14, 35.0, 15.0)]
    opts = dv.make_opts(1, 1e-4)
    ctx = dv.Context(0)
    rgb0 = dv.dv_render(ds, sc.poses, cams, opts, ctx=ctx)[0].cpu().numpy()
    ctx.debug_flag_spin_timeout()
    with pytest.raises(dv.DVError) as ei:
        dv.dv_render(ds, sc.poses, cams, opts, ctx=ctx)
    assert ei.value.status == dv.DV_ERR_TIMEOUT
    assert "look-back" in str(ei.value)
    rgb1 = dv.dv_render(ds, sc.poses, cams, opts, ctx=ctx)[0].cpu().numpy()  # reported once, then clear
    np.testing.assert_array_equal(rgb1, rgb0)
    ctx.close()
