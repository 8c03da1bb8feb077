"""Compositing weights and feature fields on the GPU vs the FP64 oracle's per-pixel weights
(oracle.pixel_weights): the weights export of a saved render, a C-channel feature render over
it, and the fusion of 2-D features into voxels.

Tolerances: per voxel and pixel the summed weight within 1e-4 (the alpha target: the weights
of a pixel sum to its alpha); features within 1e-4 * max|feature| (a weighted sum of features
with weights summing to alpha <= 1); fused sums with the gradient rule of helpers.py (they are
sums over many pixels, like a gradient)."""
from collections import defaultdict

import numpy as np
import pytest

import oracle
from helpers import check_grad, device_scene, orbit, small_comp_scene

pytestmark = pytest.mark.gpu


def _offsets(sc):
    return np.concatenate([[0], np.cumsum([o.n for o in sc.octrees])]).astype(np.int64)


def _oracle_weights(sc, cams, opts):
    off = _offsets(sc)
    rows = []
    for cam in cams:
        for v in range(cam.H):
            for u in range(cam.W):
                oi, vi, w = oracle.pixel_weights(sc.octrees, sc.poses, cam, u, v, opts)
                rows.append((off[oi] + vi, w))
    return rows


def _gpu_weights(sc, cams, K, eps):
    import torch
    import paper_2606_23031_gb300 as m
    ds = device_scene(sc)
    rgb, depth, alpha, st = m.dv_render(ds, sc.poses, cams, m.make_opts(K, eps), save_state=True)
    W = m.dv_state_weights(st)
    torch.cuda.synchronize()
    return ds, st, W, (rgb, alpha)


def _per_pixel(W):
    off = W.offsets.cpu().numpy()
    vox = W.voxel.cpu().numpy().astype(np.int64)
    w = W.weight.cpu().numpy().astype(np.float64)
    return [(vox[off[p]:off[p + 1]], w[off[p]:off[p + 1]]) for p in range(len(off) - 1)]


@pytest.mark.parametrize("K,eps,seed", [(1, 1e-4, 60), (2, 0.0, 61), (1, 1e-2, 62)])
def test_weights_export_matches_oracle(dv, K, eps, seed):
    sc = small_comp_scene(seed=seed, n_actors=3, density_scale=4.0 if eps > 1e-3 else 1.0)
    cams = [orbit(30, 24, 40.0 + seed, 20.0), orbit(17, 13, 200.0, 5.0)]
    ds, st, W, (rgb, alpha) = _gpu_weights(sc, cams, K, eps)
    gpu = _per_pixel(W)
    ref = _oracle_weights(sc, cams, oracle.Opts(K, eps))
    a = alpha.cpu().numpy()
    worst = 0.0
    for p, ((gv, gw), (ov, ow)) in enumerate(zip(gpu, ref)):
        gs, os_ = defaultdict(float), defaultdict(float)
        for v_, w_ in zip(gv, gw):
            gs[int(v_)] += w_
        for v_, w_ in zip(ov, ow):
            os_[int(v_)] += w_
        for k in set(gs) | set(os_):
            worst = max(worst, abs(gs[k] - os_[k]))
        assert abs(gw.sum() - a[p]) <= 1e-5, f"pixel {p}: weights sum {gw.sum()} vs alpha {a[p]}"
    assert worst <= 1e-4, f"max per-voxel weight difference {worst:.3g}"
    assert sum(len(g[0]) for g in gpu) > 500
    st.free()


def test_feature_render_and_fusion(dv):
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=63, n_actors=2)
    cams = [orbit(28, 22, 75.0, 25.0)]
    ds, st, W, _ = _gpu_weights(sc, cams, 1, 1e-4)
    nv = int(_offsets(sc)[-1])
    Cc = 40
    rng = np.random.default_rng(63)
    feat = np.float32(rng.normal(size=(nv, Cc)))
    F = m.dv_features_render(W, torch.as_tensor(feat, device="cuda")).cpu().numpy()
    P = cams[0].W * cams[0].H
    f2d = np.float32(rng.normal(size=(P, Cc)))
    acc = torch.zeros((nv, Cc), device="cuda")
    wsum = torch.zeros(nv, device="cuda")
    m.dv_features_fuse(W, torch.as_tensor(f2d, device="cuda"), acc, wsum)
    torch.cuda.synchronize()
    st.free()
    ref = _oracle_weights(sc, cams, oracle.Opts(1, 1e-4))
    F_ref = np.stack([w @ np.float64(feat[v]) if len(w) else np.zeros(Cc) for v, w in ref])
    err = np.abs(F - F_ref).max()
    assert err <= 1e-4 * np.abs(feat).max(), f"feature render: {err:.3g}"
    acc_ref = np.zeros((nv, Cc))
    ws_ref = np.zeros(nv)
    for p, (v, w) in enumerate(ref):
        np.add.at(acc_ref, v, w[:, None] * np.float64(f2d[p])[None, :])
        np.add.at(ws_ref, v, w)
    check_grad(acc.cpu().numpy(), acc_ref, "fused features")
    check_grad(wsum.cpu().numpy(), ws_ref, "fused weights")


def test_colour_features_reproduce_the_render(dv):
    # degree-0 SH: a voxel's colour is view independent; as a 3-channel feature it must give the RGB
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=64, n_actors=2, sh_degree=0)
    cams = [orbit(26, 20, 110.0, 15.0), orbit(19, 15, 300.0, 35.0)]
    ds, st, W, (rgb, alpha) = _gpu_weights(sc, cams, 1, 1e-4)
    cols = np.concatenate([np.maximum(o.sh[:, 0, :].astype(np.float64) * 0.28209479177387814 + 0.5, 0.0)
                           for o in sc.octrees])
    F = m.dv_features_render(W, torch.as_tensor(np.float32(cols), device="cuda")).cpu().numpy()
    st.free()
    err = np.abs(F - rgb.cpu().numpy()).max()
    assert err <= 1e-5, f"colour features vs RGB: {err:.3g}"
