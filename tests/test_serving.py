"""Serving loop (continuous batching): results in the mix equal results alone, batches really form,
waits are bounded, and the memory budget admits requests without losing any."""
import numpy as np
import pytest

import oracle
import synth
from helpers import check_forward, device_scene, small_comp_scene

pytestmark = pytest.mark.gpu


def _requests(sc, n, seed, sizes=((48, 27), (96, 54), (64, 64), (31, 17))):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        W, H = sizes[int(rng.integers(0, len(sizes)))]
        cam = synth.orbit_camera(W, H, 55.0, 2.8, float(rng.uniform(0, 360)), float(rng.uniform(-10, 40)), near=0.1,
                                 far=50.0)
        poses = [sc.poses[0]] + [synth.Pose(synth.random_rotation(rng), rng.uniform(-0.7, 0.7, 3))
                                 for _ in sc.poses[1:]]
        out.append((cam, poses))
    return out


def _outputs(cam):
    import torch
    n = cam.W * cam.H
    return (torch.empty((n, 3), device="cuda"), torch.empty((n,), device="cuda"), torch.empty((n,), device="cuda"))


def test_results_in_the_mix_equal_results_alone(dv):
    import torch
    sc = small_comp_scene(seed=30, n_actors=3)
    ds = device_scene(sc)
    reqs = _requests(sc, 40, seed=1)
    opts = dv.make_opts(1, 1e-4)
    srv = dv.Server(ds, max_views=8, n_workers=2, max_batch_pixels=10 ** 7, max_inflight_pixels=10 ** 8, opts=opts)
    outs, tickets = [], []
    for cam, poses in reqs:
        o = _outputs(cam)
        outs.append(o)
        tickets.append(srv.submit(cam, poses, o))
    lat = [srv.wait(t, 60000.0) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs)
    assert st["batches"] < len(reqs), st          # requests were batched
    assert st["max_batch"] > 1
    assert all(x >= 0 for x in lat)
    for (cam, poses), (rgb, depth, alpha) in zip(reqs, outs):
        r1, d1, a1, _ = dv.dv_render_views(ds, [(cam, poses)], opts)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(rgb.cpu().numpy(), r1.cpu().numpy())
        np.testing.assert_array_equal(depth.cpu().numpy(), d1.cpu().numpy())
        np.testing.assert_array_equal(alpha.cpu().numpy(), a1.cpu().numpy())
    # and one request of the mix against the oracle
    cam, poses = reqs[3]
    o = oracle.render(sc.octrees, poses, cam, oracle.Opts(1, 1e-4))
    rgb, depth, alpha = outs[3]
    check_forward(rgb.cpu().numpy().reshape(cam.H, cam.W, 3), depth.cpu().numpy().reshape(cam.H, cam.W),
                  alpha.cpu().numpy().reshape(cam.H, cam.W), o[0], o[1], o[2], "served request")


def test_bounded_wait_times_out_and_budget_admits_everything(dv):
    sc = small_comp_scene(seed=31, n_actors=2)
    ds = device_scene(sc)
    reqs = _requests(sc, 12, seed=2)
    # a budget smaller than one request: requests then run one at a time, none is lost
    srv = dv.Server(ds, max_views=4, n_workers=2, max_batch_pixels=10 ** 6, max_inflight_pixels=100,
                    opts=dv.make_opts(1, 1e-4))
    tickets = [srv.submit(cam, poses, _outputs(cam)) for cam, poses in reqs]
    with pytest.raises(dv.DVError) as ei:
        srv.wait(tickets[-1], 0.0)                 # nothing is done in zero time
    assert ei.value.status == dv.DV_ERR_TIMEOUT
    for t in tickets:
        srv.wait(t, 60000.0)
        srv.release(t)
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs)
    assert st["max_batch"] == 1


def test_poisoned_request_is_rejected_at_admission(dv):
    # a non-finite or non-rigid actor pose is refused by submit itself, so it cannot join a batch and
    # fail the requests batched with it; the others are served as usual
    sc = small_comp_scene(seed=31, n_actors=2)
    ds = device_scene(sc)
    reqs = _requests(sc, 6, seed=2)
    srv = dv.Server(ds, max_views=8, n_workers=1, max_batch_pixels=10 ** 7, max_inflight_pixels=10 ** 8,
                    opts=dv.make_opts(1, 1e-4))
    tickets = [srv.submit(cam, poses, _outputs(cam)) for cam, poses in reqs[:3]]
    cam, poses = reqs[3]
    bad_nan = [poses[0], synth.Pose(poses[1].R, np.array([np.nan, 0.0, 0.0])), poses[2]]
    bad_scale = [poses[0], synth.Pose(2.0 * np.asarray(poses[1].R), poses[1].t), poses[2]]
    for bad in (bad_nan, bad_scale):
        with pytest.raises(RuntimeError):
            srv.submit(cam, bad, _outputs(cam))
    tickets += [srv.submit(c, p, _outputs(c)) for c, p in reqs[4:]]
    lat = [srv.wait(t, 60000.0) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(x >= 0 for x in lat)
    assert st["requests"] == 5


def test_byte_budget_serialises_large_requests_and_batches_small_ones(dv):
    """Admission by device memory: with a byte budget below two large requests' charges, two large
    requests never render at once; small requests still share a batch under the same budget."""
    sc = small_comp_scene(seed=32, n_actors=2)
    ds = device_scene(sc)
    big = synth.orbit_camera(640, 480, 55.0, 2.8, 40.0, 20.0, near=0.1, far=50.0)
    small = synth.orbit_camera(32, 24, 55.0, 2.8, 40.0, 20.0, near=0.1, far=50.0)
    opts = dv.make_opts(1, 1e-4)
    # learn one large request's charge (the first batch also calibrates the memory model)
    probe = dv.Server(ds, max_views=8, n_workers=2, max_batch_pixels=10 ** 8, max_inflight_pixels=10 ** 9, opts=opts)
    t = probe.submit(big, sc.poses, _outputs(big))
    probe.wait(t, 60000.0)
    t = probe.submit(big, sc.poses, _outputs(big))
    probe.wait(t, 60000.0)
    b_big = probe.memory()["last_request_bytes"]
    t = probe.submit(small, sc.poses, _outputs(small))
    probe.wait(t, 60000.0)
    b_small = probe.memory()["last_request_bytes"]
    probe.close()
    assert b_big > 4 * b_small > 0
    budget = int(1.5 * b_big)
    srv = dv.Server(ds, max_views=8, n_workers=2, max_batch_pixels=10 ** 8, max_inflight_pixels=10 ** 9, opts=opts,
                    max_inflight_bytes=budget)
    # calibrate the fresh server's model, then queue everything while admission is held
    t = srv.submit(big, sc.poses, _outputs(big))
    srv.wait(t, 60000.0)
    srv.memory(reset_peak=True)           # the calibration request ran alone, charged by the starting model
    srv.pause(True)
    tickets = [srv.submit(big, sc.poses, _outputs(big)) for _ in range(3)]
    srv.pause(False)
    for t in tickets:
        srv.wait(t, 60000.0)
    mem = srv.memory()
    assert mem["peak_inflight_bytes"] <= budget               # two large requests were never in flight together
    b0 = srv.stats()["batches"]
    srv.pause(True)
    tickets = [srv.submit(small, sc.poses, _outputs(small)) for _ in range(6)]
    srv.pause(False)
    for t in tickets:
        srv.wait(t, 60000.0)
    st = srv.stats()
    srv.close()
    assert st["max_batch"] >= 2                               # the small requests shared batches
    assert st["batches"] - b0 < 6
