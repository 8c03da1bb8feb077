"""Shared test utilities: device scenes from synth inputs, the GPU call through the C ABI,
the oracle call, and the comparison rules with their tolerances.

Tolerances (stated once, used by every parity test):
  RGB and alpha: max |gpu - oracle| <= 1e-4 (absolute);
  depth: |gpu - oracle| <= 1e-3 |D| + 1e-4 (D / alpha): the relative bound plus the alpha bound carried
         through the pixel's mean hit distance D / alpha (D = alpha x mean distance, so an alpha
         error inside its own bound moves D by up to that much); and, for pixels with alpha > 0.5,
         the mean hit distance D / alpha itself within 1e-3 relative;
  gradients (the whole gradient vector, all octrees together): per element
             |gpu - oracle| <= 1e-3 (|oracle| + max|oracle|), and ||gpu - oracle||_2 <= 1e-3 ||oracle||_2.
The gradient bound is relative to the gradient's scale: an element fed by one sliver segment
(a voxel grazed by the ray or cut by an actor box) carries the fp32 relative error of that
segment's length, which is ~1e-7 t / l and can exceed 1e-3 of the element itself.

Both relaxed terms are watched.  Every forward comparison counts the pixels whose depth passes only
through the alpha term (at most RELAXED_DEPTH_FRAC of the pixels, or 2).  Every gradient comparison
counts the nonzero elements that pass only through the 1e-3 max|g| floor and requires (a) that they
carry at most FLOOR_NORM_FRAC of the reference gradient's L2 norm (the floor only ever excuses
elements that do not matter to the gradient), and (b) that every element of at least BIG x max|g|
meets the strict 1e-3 relative bound within BIG_RTOL.  With DV_TOL_LOG set to a file name, each
comparison appends its figures there as one JSON line.
"""
import json
import math
import os
from types import SimpleNamespace

import numpy as np

import oracle
import synth

RGB_ATOL = 1e-4
DEPTH_RTOL, DEPTH_ATOL = 1e-3, 1e-5
G_RTOL, G_FLOOR, G_NORM = 1e-3, 1e-3, 1e-3
RELAXED_DEPTH_FRAC = 1e-3   # pixels whose depth needs the alpha term, at most this fraction of the pixels
FLOOR_NORM_FRAC = 0.05     # the elements that need the scale floor carry at most this share of ||g_ref||
BIG, BIG_RTOL = 1e-2, 5e-3  # elements of at least BIG max|g| must be within BIG_RTOL relative, element by element


def _log_tolerance(kind, what, **fig):
    path = os.environ.get("DV_TOL_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"kind": kind, "what": what, **fig}) + "\n")


def device_scene(scene, device="cuda"):
    import paper_2606_23031_gb300 as dv
    return [dv.DeviceOctree.from_host(o, device) for o in scene.octrees]


def gpu_render(dscene, poses, cams, K=1, eps=1e-4, act=0, save_state=False):
    import paper_2606_23031_gb300 as dv
    import torch
    rgb, depth, alpha, st = dv.dv_render(dscene, poses, cams, dv.make_opts(K, eps, act), save_state=save_state)
    torch.cuda.synchronize()
    return rgb, depth, alpha, st


def split_images(t, cams, ch=None):
    out, o = [], 0
    for c in cams:
        n = c.W * c.H
        x = t[o:o + n]
        out.append(x.reshape(c.H, c.W, ch) if ch else x.reshape(c.H, c.W))
        o += n
    return out


def check_forward(g_rgb, g_depth, g_alpha, o_rgb, o_depth, o_alpha, what=""):
    g_rgb, g_depth, g_alpha = (np.asarray(x, np.float64) for x in (g_rgb, g_depth, g_alpha))
    o_depth, o_alpha = np.asarray(o_depth, np.float64), np.asarray(o_alpha, np.float64)
    e_rgb = np.abs(g_rgb - o_rgb).max(initial=0.0)
    e_a = np.abs(g_alpha - o_alpha).max(initial=0.0)
    tbar = np.where(o_alpha > 0, np.abs(o_depth) / np.maximum(o_alpha, 1e-300), 0.0)
    lim_d = DEPTH_RTOL * np.abs(o_depth) + RGB_ATOL * tbar + DEPTH_ATOL
    ex_d = np.abs(g_depth - o_depth) - lim_d
    e_d = ex_d.max(initial=-1.0)
    op = o_alpha > 0.5
    e_m = 0.0
    if op.any():
        mg = g_depth[op] / np.maximum(g_alpha[op], 1e-30)
        mo = o_depth[op] / o_alpha[op]
        e_m = (np.abs(mg - mo) / np.abs(mo)).max()
    worst = np.unravel_index(int(np.argmax(ex_d)), ex_d.shape) if ex_d.size else ()
    # the strict depth bound alone (without the alpha term): how many pixels need the relaxation
    strict_d = np.abs(g_depth - o_depth) <= DEPTH_RTOL * np.abs(o_depth) + DEPTH_ATOL
    n_relaxed = int(np.count_nonzero(~strict_d))
    rel_d = np.abs(g_depth - o_depth) / np.maximum(np.abs(o_depth), 1e-30)
    worst_strict = float(rel_d[o_depth > 0].max(initial=0.0))
    _log_tolerance("forward", what, pixels=int(o_depth.size), max_drgb=float(e_rgb), max_dalpha=float(e_a),
                   depth_relaxed_pixels=n_relaxed, worst_depth_rel=worst_strict, mean_distance_rel=float(e_m))
    msg = (f"{what}: max|drgb|={e_rgb:.3g} max|dalpha|={e_a:.3g} depth excess={e_d:.3g} "
           f"(worst {worst}: gpu D={g_depth[worst] if ex_d.size else 0:.6g} oracle D={o_depth[worst] if ex_d.size else 0:.6g} "
           f"alpha={o_alpha[worst] if ex_d.size else 0:.4g}) mean-distance rel err (alpha>0.5)={e_m:.3g}; "
           f"{n_relaxed} of {o_depth.size} pixels pass only through the alpha term (worst strict rel {worst_strict:.3g})")
    assert e_rgb <= RGB_ATOL and e_a <= RGB_ATOL and e_d <= 0.0 and e_m <= DEPTH_RTOL, msg
    assert n_relaxed <= max(2, RELAXED_DEPTH_FRAC * o_depth.size), msg
    return e_rgb, e_a


def check_grads(gs, refs, what=""):
    """Compare a gradient given as several arrays (one per octree) as one vector."""
    return check_grad(np.concatenate([np.asarray(x, np.float64).ravel() for x in gs]),
                      np.concatenate([np.asarray(x, np.float64).ravel() for x in refs]), what)


def check_grad(g, ref, what=""):
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    scale = np.abs(ref).max(initial=0.0)
    err = np.abs(g - ref)
    lim = G_RTOL * np.abs(ref) + G_FLOOR * scale
    worst = int(np.argmax(err - lim)) if err.size else 0
    nrm = np.linalg.norm(ref)
    rel = np.linalg.norm(g - ref) / nrm if nrm > 0 else np.linalg.norm(g)
    # the strict per-element bound alone (no scale floor): the nonzero elements that need the floor, the
    # share of the gradient's norm they carry, and the worst strict error among the large elements
    nz = ref != 0.0
    n_nz = int(np.count_nonzero(nz))
    floor = nz & (err > G_RTOL * np.abs(ref))
    n_floor = int(np.count_nonzero(floor))
    n_zero_err = int(np.count_nonzero(~nz & (err > 0.0)))
    floor_norm = float(np.linalg.norm(ref[floor]) / nrm) if nrm > 0 else 0.0
    big = np.abs(ref) >= BIG * scale
    worst_big = float((err[big] / np.abs(ref[big])).max(initial=0.0)) if big.any() else 0.0
    _log_tolerance("gradient", what, elements=int(ref.size), nonzero=n_nz, floor_elements=n_floor,
                   floor_norm_frac=floor_norm, zero_ref_with_error=n_zero_err, worst_rel_big=worst_big,
                   norm_rel=float(rel))
    msg = (f"{what}: worst element {worst}: gpu={g[worst] if g.size else 0:.6g} ref={ref[worst] if ref.size else 0:.6g}"
           f" (limit {lim[worst] if lim.size else 0:.3g}); norm rel err {rel:.3g}; scale {scale:.3g}; "
           f"{n_floor} of {n_nz} nonzero elements pass only through the floor, carrying {floor_norm:.3g} of the "
           f"norm; worst strict rel among elements >= {BIG:g} max|g|: {worst_big:.3g}")
    assert (err <= lim).all() and rel <= G_NORM, msg
    assert floor_norm <= FLOOR_NORM_FRAC and worst_big <= BIG_RTOL, msg
    return rel


def pose64(R=None, t=None):
    return SimpleNamespace(R=np.eye(3) if R is None else np.asarray(R, np.float64),
                           t=np.zeros(3) if t is None else np.asarray(t, np.float64))


def small_comp_scene(seed=0, n_actors=2, level=4, sh_degree=2, hole=False, empty_bg=False, density_scale=1.0):
    """A few-thousand-voxel background grid plus actors with random rigid poses."""
    rng = np.random.default_rng(seed)
    n = 1 << level
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    ijk = ijk[rng.uniform(size=ijk.shape[0]) < 0.5]
    if empty_bg:
        ijk = ijk[:0]
    V = ijk.shape[0]
    key = synth.pack_keys(np.full(V, level), ijk[:, 0], ijk[:, 1], ijk[:, 2])
    dens = (rng.lognormal(-0.5, 1.0, (V, 8)) * density_scale).astype(np.float32)
    sh = rng.normal(0, 0.3, (V, (sh_degree + 1) ** 2, 3)).astype(np.float32)
    bg = synth.Octree(key, dens, sh, sh_degree, (0.1, -0.05, 0.02), 2.0, synth.BG)
    octs, poses = [bg], [synth.Pose()]
    for a in range(n_actors):
        la = 3
        m = 1 << la
        k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
        aijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
        aijk = aijk[rng.uniform(size=aijk.shape[0]) < 0.6]
        Va = aijk.shape[0]
        akey = synth.pack_keys(np.full(Va, la), aijk[:, 0], aijk[:, 1], aijk[:, 2])
        root = 0.7
        half = (0.33, 0.28, 0.3)
        octs.append(synth.Octree(akey, (rng.lognormal(0.8, 0.8, (Va, 8)) * density_scale).astype(np.float32),
                                 rng.normal(0, 0.3, (Va, (sh_degree + 1) ** 2, 3)).astype(np.float32), sh_degree,
                                 (0.0, 0.0, 0.0), root, synth.ACTOR, half))
        poses.append(synth.Pose(synth.random_rotation(rng), rng.uniform(-0.7, 0.7, 3)))
    return synth.Scene(octs, poses)


def orbit(W, H, az, el, dist=2.8, fov=55.0, near=0.1, far=50.0):
    return synth.orbit_camera(W, H, fov, dist, az, el, near=near, far=far)


def sample_pixels(cam, n, seed):
    rng = np.random.default_rng(seed)
    tot = cam.W * cam.H
    return np.sort(rng.choice(tot, size=min(n, tot), replace=False))
