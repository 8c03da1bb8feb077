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


@pytest.mark.parametrize("Cc,shift", [(1, 0), (4, 0), (8, 0), (16, 0), (32, 0), (40, 0), (64, 0), (64, 1), (100, 0),
                                      (128, 0), (300, 0)])
def test_feature_kernels_on_synthetic_slots(dv, Cc, shift):
    # Slot lists with the export's layout but chosen to reach every kernel path: a skewed voxel
    # mix (a few voxels own thousands of slots; the rest are spread over 5,000 voxels, so a
    # 128-pixel chunk of the fusion holds about 2,200 slots over more distinct voxels than its
    # 1,023-row table, and the overflow row is used; the first chunk holds about 5,700 slots, more
    # than one 3,072-slot piece), empty pixels, zero weights, and
    # channel counts for the 16-byte and the scalar paths of both kernels (300: five 64-channel
    # slices of the fusion; shift 1: 64 channels in rows that are only 4-byte aligned, which the
    # fusion must take through its scalar path).  The sums are plain definitions, compared with
    # FP64 numpy.
    import torch
    import paper_2606_23031_gb300 as m
    rng = np.random.default_rng(70 + Cc)
    P, nv = 3000, 5000
    cnt = rng.integers(0, 40, size=P)
    cnt[rng.random(P) < 0.1] = 0
    cnt[:128] = rng.integers(30, 60, size=128)  # the first 128-pixel chunk of the fusion: two pieces
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    n = int(off[-1])
    heavy = rng.integers(0, nv, size=4)
    vox = np.where(rng.random(n) < 0.3, heavy[rng.integers(0, 4, size=n)], rng.integers(0, nv, size=n))
    w = np.float32(rng.random(n))
    w[rng.random(n) < 0.05] = 0.0
    feat = np.float32(rng.normal(size=(nv, Cc)))
    f2d = np.float32(rng.normal(size=(P, Cc)))
    dev = lambda a: torch.as_tensor(a, device="cuda")
    W = m.Weights(dev(off), dev(vox.astype(np.int32)), dev(w))
    F = m.dv_features_render(W, dev(feat)).cpu().numpy()
    acc = torch.zeros((nv, Cc), device="cuda")
    wsum = torch.zeros(nv, device="cuda")
    if shift:
        # rows 4-byte aligned only (a view one float into a buffer): the fusion's scalar loads and atomics
        buf = torch.zeros(P * Cc + shift, device="cuda")
        f2d_d = buf[shift:].view(P, Cc)
        f2d_d.copy_(dev(f2d))
        acc_buf = torch.zeros(nv * Cc + shift, device="cuda")
        acc = acc_buf[shift:].view(nv, Cc)
    else:
        f2d_d = dev(f2d)
    m.dv_features_fuse(W, f2d_d, acc, wsum)
    torch.cuda.synchronize()
    w64 = np.float64(w)
    F_ref = np.zeros((P, Cc))
    for p in range(P):
        s = slice(off[p], off[p + 1])
        F_ref[p] = w64[s] @ np.float64(feat[vox[s]])
    pix = np.repeat(np.arange(P), cnt)
    acc_ref = np.zeros((nv, Cc))
    np.add.at(acc_ref, vox, w64[:, None] * np.float64(f2d[pix]))
    ws_ref = np.bincount(vox, weights=w64, minlength=nv)
    assert np.bincount(vox).max() > 1000
    err = np.abs(F - F_ref).max()
    assert err <= 1e-5 * max(1.0, np.abs(F_ref).max()), f"feature render, C={Cc}: {err:.3g}"
    check_grad(acc.cpu().numpy(), acc_ref, f"fused features, C={Cc}")
    check_grad(wsum.cpu().numpy(), ws_ref, f"fused weights, C={Cc}")


def test_feature_fusion_without_slots(dv):
    # every pixel empty: nothing is added, and a NULL weight sum is accepted
    import torch
    import paper_2606_23031_gb300 as m
    W = m.Weights(torch.zeros(101, dtype=torch.int64, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"),
                  torch.zeros(0, device="cuda"))
    acc = torch.zeros((10, 64), device="cuda")
    m.dv_features_fuse(W, torch.ones((100, 64), device="cuda"), acc)
    assert float(acc.abs().sum()) == 0.0
    F = m.dv_features_render(W, torch.ones((10, 64), device="cuda"))
    assert F.shape == (100, 64) and float(F.abs().sum()) == 0.0
