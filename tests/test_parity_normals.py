"""Normal state N (Alg. 1: the pixel state sums voxel normals) on the GPU vs the FP64
oracle: forward values and the backward through N, on scenes that exercise every compositing
path (lockstep actor partials, stops inside an actor, more actors per tile than lockstep slots,
the 1080p compositional frame).

Tolerance for N: max |gpu - oracle| <= 1e-4 per component, as for RGB (|N| <= alpha <= 1 and each
voxel normal is a unit vector computed in fp32).  Gradients use the shared rule of helpers.py."""
import numpy as np
import pytest

import oracle
import synth
from helpers import (check_forward, check_grads, device_scene, orbit, sample_pixels, small_comp_scene,
                     split_images)

pytestmark = pytest.mark.gpu

N_ATOL = 1e-4


def _gpu(sc, cams, K, eps, g=None):
    import torch
    import paper_2606_23031_gb300 as dv
    ds = device_scene(sc)
    rgb, depth, alpha, nrm, st = dv.dv_render(ds, sc.poses, cams, dv.make_opts(K, eps), save_state=True,
                                              normals=True)
    grads = None
    if g is not None:
        d_dens = [torch.zeros_like(o.dens) for o in ds]
        d_sh = [torch.zeros_like(o.sh) for o in ds]
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
        dv.dv_render_backward(st, t(g[0]), t(g[1]), t(g[2]), d_dens, d_sh, d_normal=t(g[3]))
        grads = ([x.cpu().numpy() for x in d_dens], [x.cpu().numpy() for x in d_sh])
    torch.cuda.synchronize()
    st.free()
    return [x.cpu().numpy() for x in (rgb, depth, alpha, nrm)], grads


def _check_full(sc, cams, K=1, eps=1e-4, what=""):
    (rgb, depth, alpha, nrm), _ = _gpu(sc, cams, K, eps)
    gr, gd, ga, gn = (split_images(rgb, cams, 3), split_images(depth, cams), split_images(alpha, cams),
                      split_images(nrm, cams, 3))
    worst = 0.0
    for c, cam in enumerate(cams):
        o = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(K, eps), normals=True)
        check_forward(gr[c], gd[c], ga[c], o[0], o[1], o[2], f"{what} cam{c}")
        e = np.abs(gn[c] - o[4]).max(initial=0.0)
        assert e <= N_ATOL, f"{what} cam{c}: max|dN|={e:.3g}"
        worst = max(worst, np.abs(o[4]).max(initial=0.0))
    assert worst > 0.3, "the scene should carry normals"


@pytest.mark.parametrize("K,eps", [(1, 1e-4), (2, 0.0)])
def test_normals_compositional_scene(dv, K, eps):
    sc = small_comp_scene(seed=40, n_actors=3)
    _check_full(sc, [orbit(56, 44, 40.0, 25.0), orbit(33, 27, 200.0, 10.0)], K, eps, what=f"normals K={K}")


def test_normals_with_stops_inside_actors(dv):
    sc = small_comp_scene(seed=41, n_actors=3, density_scale=30.0)
    for eps in (1e-4, 1e-2):
        _check_full(sc, [orbit(48, 40, 75.0, 20.0)], 1, eps, what=f"opaque normals eps={eps}")


def test_normals_more_actors_than_lockstep_slots(dv):
    sc = small_comp_scene(seed=42, n_actors=24)
    _check_full(sc, [orbit(48, 40, 15.0, 30.0)], 1, 1e-4, what="24 actors normals")


def test_normals_config2_sampled_pixels(dv, config2_scene):
    sc, cams, _ = config2_scene
    cam = cams[0]
    (rgb, depth, alpha, nrm), _ = _gpu(sc, [cam], 1, 1e-4)
    pix = sample_pixels(cam, 384, seed=9)
    o = oracle.render(sc.octrees, sc.poses, cam, oracle.Opts(1, 1e-4), pixels=pix, normals=True)
    check_forward(rgb[pix], depth[pix], alpha[pix], o[0], o[1], o[2], "cfg2 normals")
    e = np.abs(nrm[pix] - o[4]).max()
    assert e <= N_ATOL, f"cfg2 max|dN|={e:.3g}"


@pytest.mark.parametrize("seed,density", [(43, 1.0), (44, 20.0)])
def test_normals_backward(dv, seed, density):
    sc = small_comp_scene(seed=seed, n_actors=3, density_scale=density)
    cam = orbit(40, 34, 35.0 + seed, 20.0)
    P = cam.W * cam.H
    rng = np.random.default_rng(seed)
    g = [rng.normal(size=(P, 3)), 0.1 * rng.normal(size=P), rng.normal(size=P), rng.normal(size=(P, 3))]
    g = [np.float64(np.float32(x)) for x in g]
    _, (gd, gs) = _gpu(sc, [cam], 1, 1e-4, g)
    od, os_ = oracle.backward(sc.octrees, sc.poses, cam, g[0], g[1], g[2], oracle.Opts(1, 1e-4), g_normal=g[3])
    check_grads(gd, od, f"normals seed={seed} d_dens")
    check_grads(gs, os_, f"normals seed={seed} d_sh")


def test_normals_backward_only_through_n(dv):
    # upstream gradient on N alone: d_sh is zero and d_dens comes from N's weights and normals
    sc = small_comp_scene(seed=45, n_actors=2)
    cam = orbit(36, 30, 120.0, 15.0)
    P = cam.W * cam.H
    rng = np.random.default_rng(45)
    z3, z1 = np.zeros((P, 3)), np.zeros(P)
    gN = np.float64(np.float32(rng.normal(size=(P, 3))))
    _, (gd, gs) = _gpu(sc, [cam], 2, 0.0, (z3, z1, z1, gN))
    od, _ = oracle.backward(sc.octrees, sc.poses, cam, z3, z1, z1, oracle.Opts(2, 0.0), g_normal=gN)
    check_grads(gd, od, "N-only d_dens")
    assert all(np.all(x == 0.0) for x in gs)


def test_normals_autograd_cosine_loss(dv):
    import torch
    import paper_2606_23031_gb300 as m
    sc = small_comp_scene(seed=46, n_actors=2)
    cam = orbit(32, 28, 60.0, 25.0)
    ds = device_scene(sc)
    dens = [o.dens.clone().requires_grad_(True) for o in ds]
    sh = [o.sh.clone().requires_grad_(True) for o in ds]
    rgb, depth, alpha, nrm = m.render(ds, sc.poses, [cam], m.make_opts(1, 1e-4), dens=dens, sh=sh, normals=True)
    ref = torch.nn.functional.normalize(torch.randn((cam.W * cam.H, 3), device="cuda",
                                                    generator=torch.Generator("cuda").manual_seed(1)), dim=1)
    # the paper's normal loss: 1 - cos(N, N_pseudo), on pixels with a surface
    mask = alpha.detach() > 0.05
    cos = (nrm * ref).sum(1) / (nrm.norm(dim=1) + 1e-12)
    loss = (1.0 - cos)[mask].sum()
    loss.backward()
    # the same gradient from the oracle: dL/dN of the cosine loss, evaluated on the GPU's N
    n = nrm.detach().double()
    nn_ = n.norm(dim=1, keepdim=True) + 1e-12
    r = ref.double()
    gN = -(r / nn_ - (n * r).sum(1, keepdim=True) * n / nn_ ** 3)
    gN[~mask] = 0.0
    z = np.zeros(cam.W * cam.H)
    od, os_ = oracle.backward(sc.octrees, sc.poses, cam, np.zeros((cam.W * cam.H, 3)), z, z, oracle.Opts(1, 1e-4),
                              g_normal=np.float64(np.float32(gN.cpu().numpy())))
    check_grads([d.grad.cpu().numpy() for d in dens], od, "cosine-loss d_dens")
    assert all(float(s.grad.abs().max()) == 0.0 for s in sh)
