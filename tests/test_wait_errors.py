"""Bounded waits report on the host.  A one-sweep sort pass whose look-back runs out of its bound sets
the call's own flag and the device's wait-error word.  The first test runs one real sort tile whose
predecessor never publishes, with a short bound, and reads both flags; the others check the two
report paths: a render's state (dv_state_check) and the device word taken by the next render (set
here from the host through the library's test hook)."""
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


def test_sort_look_back_runs_out_sets_both_flags(dv):
    ctx = dv.Context(0)
    call, device = ctx.debug_sort_timeout(spin_limit=1000)
    assert call == 1 and device == 1
    # the hook cleared the device word again: renders on the device go on working
    sc = small_comp_scene(seed=43, n_actors=1)
    ds = device_scene(sc)
    _, _, _, st = dv.dv_render(ds, sc.poses, [orbit(16, 12, 20.0, 10.0)], dv.make_opts(1, 1e-4), ctx=ctx,
                               save_state=True)
    st.check(wait=True)
    st.free()
    ctx.close()


def test_state_check_of_a_clean_render(dv):
    sc = small_comp_scene(seed=44, n_actors=2)
    ds = device_scene(sc)
    ctx = dv.Context(0)
    _, _, _, st = dv.dv_render(ds, sc.poses, [orbit(24, 20, 60.0, 20.0)], dv.make_opts(1, 1e-4), ctx=ctx,
                               save_state=True)
    st.check(wait=False)    # unknown or clean: no error either way
    st.check(wait=True)
    st.free()
    ctx.close()
