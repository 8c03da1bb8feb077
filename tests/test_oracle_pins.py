"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test fixes a part of the oracle against a closed form, an invariant of
the method, a library routine, or finite differences, chosen so that a
plausible slip (a dropped term, a wrong sign or index, a transposed operand)
breaks at least one of them:

- single constant voxel (Sec. 3.4 compositing): alpha = 1 - exp(-sigma l) with the
  chord l found by bisection of the point-in-box test, C = alpha c, D = alpha (t_in + t_out)/2;
- stacked voxels: C = c1 a1 + (1 - a1) a2 c2, alpha = 1 - (1-a1)(1-a2);
- multilinear corner field: trilinear interpolation reproduces any multilinear
  function exactly, so tau equals the midpoint rule of that function (corner indexing);
- linear field: midpoint rule is the exact integral for every K;
- exponential-linear activation: C1 at 1.1, identity above, v_far = -10 is empty (Sec. 3.3);
- subdivision invariance of colour and alpha;
- Alg. 1 interval walk: background before, actor inside, background after the box,
  with the background voxel straddling the box clipped on both sides;
- overlapping boxes: the box entered first owns the overlap;
- early stop once T < eps_stop (Alg. 1);
- identity-pose actor == the same voxels merged into the static octree;
- rigid equivariance: moving every octree and the camera by G leaves the image unchanged;
- actor permutation invariance;
- SH basis == scipy's spherical harmonics (real form) and orthonormal on the sphere;
- view direction sign (camera -> voxel centre, local frame);
- analytic backward == central finite differences of the oracle (FP64 arrays).
"""
import math
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import synth

EXPLIN = oracle.ACT_EXPLIN
IDENT = oracle.ACT_IDENTITY


def pose64(R=None, t=None):
    return SimpleNamespace(R=np.eye(3) if R is None else np.asarray(R, np.float64),
                           t=np.zeros(3) if t is None else np.asarray(t, np.float64))


def cam_looking(eye, target, W=5, H=5, fov=20.0, near=0.01, far=100.0, up=(0.0, 0.0, 1.0)):
    p = synth.look_at(eye, target, up)
    fx = float(np.float32((W / 2.0) / math.tan(math.radians(fov) / 2.0)))   # the ABI carries float32
    return SimpleNamespace(W=W, H=H, fx=fx, fy=fx, cx=W / 2.0, cy=H / 2.0,
                           pose=pose64(np.asarray(p.R, np.float64), np.asarray(eye, np.float64)), near=near, far=far)


def ray_of(cam, u, v):
    dc = np.array([(u + 0.5 - cam.cx) / cam.fx, (v + 0.5 - cam.cy) / cam.fy, 1.0])
    d = cam.pose.R @ dc
    return np.asarray(cam.pose.t, np.float64), d / np.linalg.norm(d)


def chord_bisect(o, d, lo, hi, tmax=50.0, n=200001):
    """Entry/exit distances of the ray in the closed box, from a dense point-in-box scan refined by
    bisection (independent of any slab arithmetic)."""
    inside = lambda t: bool(np.all(o + t * d >= lo) and np.all(o + t * d <= hi))
    ts = np.linspace(0.0, tmax, n)
    pts = o[None, :] + ts[:, None] * d[None, :]
    ins = np.all((pts >= lo) & (pts <= hi), axis=1)
    idx = np.nonzero(ins)[0]
    if idx.size == 0:
        return None
    a_out, a_in = ts[idx[0] - 1], ts[idx[0]]
    b_in, b_out = ts[idx[-1]], ts[idx[-1] + 1]
    for _ in range(80):
        m = 0.5 * (a_out + a_in)
        a_out, a_in = (a_out, m) if inside(m) else (m, a_in)
        m = 0.5 * (b_in + b_out)
        b_in, b_out = (m, b_out) if inside(m) else (b_in, m)
    return 0.5 * (a_out + a_in), 0.5 * (b_in + b_out)


def one_voxel(level, ijk, dens, rgb, center=(0.0, 0.0, 0.0), root=1.0, role=synth.BG, clip_half=(0, 0, 0),
              sh_degree=0):
    ijk = np.asarray(ijk).reshape(-1, 3)
    V = ijk.shape[0]
    dens = np.broadcast_to(np.asarray(dens, np.float64).reshape(-1, 8) if np.ndim(dens) else np.full((1, 8), dens),
                           (V, 8))
    rgb = np.broadcast_to(np.asarray(rgb, np.float64).reshape(-1, 3), (V, 3))
    return synth.grid_octree(level, center, root, dens=dens, rgb=rgb, ijk=ijk, role=role, clip_half=clip_half,
                             sh_degree=sh_degree)


def explin(x):
    return x if x > 1.1 else 1.1 * math.exp(x / 1.1 - 1.0)


def colour_of(rgb):
    # the DC encoding of synth.sh_from_rgb rounds through float32
    sh0 = np.float32((np.asarray(rgb, np.float64) - 0.5) / synth.SH_C0).astype(np.float64)
    return np.maximum(sh0 * (0.5 / math.sqrt(math.pi)) + 0.5, 0.0)


# ---------------------------------------------------------------------------
# single voxel / stacks / fields
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rho,K", [(2.0, 1), (2.0, 3), (0.3, 1), (-1.5, 4)])
def test_single_constant_voxel_closed_form(rho, K):
    oc = one_voxel(0, [0, 0, 0], rho, [0.9, 0.4, 0.2])           # box [-0.5, 0.5]^3
    cam = cam_looking((3.0, 0.7, 0.4), (0.05, 0.02, -0.03), W=7, H=5, fov=30.0)
    rgb, depth, alpha, nseg = oracle.render([oc], [pose64()], cam, oracle.Opts(K=K, eps_stop=0.0))
    sigma = float(np.float32(rho)) if rho > 1.1 else explin(float(np.float32(rho)))
    c = colour_of([0.9, 0.4, 0.2])
    hits = 0
    for v in range(cam.H):
        for u in range(cam.W):
            o, d = ray_of(cam, u, v)
            ch = chord_bisect(o, d, -0.5 * np.ones(3), 0.5 * np.ones(3))
            if ch is None:
                assert alpha[v, u] == 0.0 and nseg[v, u] == 0
                continue
            hits += 1
            t0, t1 = ch
            a = 1.0 - math.exp(-sigma * (t1 - t0))
            assert alpha[v, u] == pytest.approx(a, rel=1e-9, abs=1e-12)
            np.testing.assert_allclose(rgb[v, u], a * c, rtol=1e-9, atol=1e-12)
            assert depth[v, u] == pytest.approx(a * 0.5 * (t0 + t1), rel=1e-9)
    assert hits >= 10


def test_axial_ray_exact_chord():
    # odd image: the centre pixel's ray is the optical axis; chord through a unit voxel = 1
    oc = one_voxel(0, [0, 0, 0], 2.0, [0.25, 0.5, 0.75])
    cam = cam_looking((4.0, 0.0, 0.0), (0.0, 0.0, 0.0), W=5, H=5)
    rgb, depth, alpha, _ = oracle.render([oc], [pose64()], cam, oracle.Opts(K=1, eps_stop=0.0))
    a = 1.0 - math.exp(-2.0)
    assert alpha[2, 2] == pytest.approx(a, rel=1e-12)
    assert depth[2, 2] == pytest.approx(a * 4.0, rel=1e-12)
    np.testing.assert_allclose(rgb[2, 2], a * colour_of([0.25, 0.5, 0.75]), rtol=1e-12)


def test_two_stacked_voxels_closed_form():
    # two unit voxels along x: [-1,0] then [0,1] as seen from +x: front voxel is ijk (1,0,0)
    dens = np.stack([np.full(8, 1.7), np.full(8, 3.1)])
    rgbs = np.array([[0.9, 0.1, 0.3], [0.2, 0.8, 0.6]])
    oc = one_voxel(1, [[0, 0, 1], [1, 0, 1]], dens, rgbs, center=(0.0, 0.5, -0.5), root=2.0)
    # voxel 0 spans x in [-1,0], voxel 1 spans x in [0,1]; y in [-0.5,0.5]; z in [-0.5,0.5]
    cam = cam_looking((5.0, 0.0, 0.0), (0.0, 0.0, 0.0), W=5, H=5)
    rgb, depth, alpha, nseg = oracle.render([oc], [pose64()], cam, oracle.Opts(K=2, eps_stop=0.0))
    a_front = 1 - math.exp(-float(np.float32(3.1)) * 1.0)   # x in [0,1], t in [4,5]
    a_back = 1 - math.exp(-float(np.float32(1.7)) * 1.0)    # x in [-1,0], t in [5,6]
    c_f, c_b = colour_of(rgbs[1]), colour_of(rgbs[0])
    np.testing.assert_allclose(rgb[2, 2], a_front * c_f + (1 - a_front) * a_back * c_b, rtol=1e-12)
    assert alpha[2, 2] == pytest.approx(1 - (1 - a_front) * (1 - a_back), rel=1e-12)
    assert depth[2, 2] == pytest.approx(a_front * 4.5 + (1 - a_front) * a_back * 5.5, rel=1e-12)
    assert nseg[2, 2] == 2


def _field(coef, x, y, z):
    a, b, c, d, e, f, g, h = coef
    return a + b * x + c * y + d * z + e * x * y + f * y * z + g * x * z + h * x * y * z


@pytest.mark.parametrize("K", [1, 2, 5])
def test_multilinear_field_matches_midpoint_rule(K):
    # corner c at offsets (c&1, c>>1&1, c>>2&1); the field is a non-symmetric multilinear polynomial
    coef = [0.9, 0.31, -0.17, 0.53, 0.23, -0.41, 0.13, 0.37]
    corners = [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]
    dens = np.array([_field(coef, *xyz) for xyz in corners], np.float32)
    coef = [float(x) for x in coef]
    oc = one_voxel(0, [0, 0, 0], dens, [0.5, 0.5, 0.5], center=(0.5, 0.5, 0.5), root=1.0)  # box [0,1]^3
    cam = cam_looking((2.7, 1.9, 1.4), (0.45, 0.55, 0.5), W=9, H=7, fov=25.0)
    _, _, alpha, _ = oracle.render([oc], [pose64()], cam, oracle.Opts(K=K, eps_stop=0.0, activation=IDENT))
    dens64 = dens.astype(np.float64)
    # exact multilinear interpolant of the float32 corner values
    fit = np.linalg.solve(np.array([[1, x, y, z, x * y, y * z, x * z, x * y * z] for x, y, z in corners], float),
                          dens64)
    checked = 0
    for v in range(cam.H):
        for u in range(cam.W):
            o, d = ray_of(cam, u, v)
            ch = chord_bisect(o, d, np.zeros(3), np.ones(3))
            if ch is None:
                continue
            t0, t1 = ch
            l = t1 - t0
            tau = l / K * sum(_field(fit, *(o + (t0 + (k + 0.5) * l / K) * d)) for k in range(K))
            assert alpha[v, u] == pytest.approx(1 - math.exp(-tau), rel=1e-8, abs=1e-12)
            checked += 1
    assert checked >= 20


@pytest.mark.parametrize("K", [1, 2, 4])
def test_linear_field_integral_exact(K):
    # sigma linear along the ray and > 1.1 everywhere (explin = identity): tau = exact integral
    corners = np.array([(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)], float)
    dens = (3.0 + 2.0 * corners[:, 0] + 1.0 * corners[:, 1] + 4.0 * corners[:, 2]).astype(np.float32)
    oc = one_voxel(0, [0, 0, 0], dens, [0.5, 0.5, 0.5], center=(0.5, 0.5, 0.5), root=1.0)
    cam = cam_looking((2.2, -1.3, 1.7), (0.5, 0.5, 0.5), W=6, H=6, fov=20.0)
    _, _, alpha, _ = oracle.render([oc], [pose64()], cam, oracle.Opts(K=K, eps_stop=0.0, activation=EXPLIN))
    for v in range(cam.H):
        for u in range(cam.W):
            o, d = ray_of(cam, u, v)
            ch = chord_bisect(o, d, np.zeros(3), np.ones(3))
            if ch is None:
                continue
            t0, t1 = ch
            p0, p1 = o + t0 * d, o + t1 * d
            f = lambda p: 3.0 + 2.0 * p[0] + p[1] + 4.0 * p[2]
            integral = (t1 - t0) * 0.5 * (f(p0) + f(p1))     # trapezoid = exact for linear
            assert alpha[v, u] == pytest.approx(1 - math.exp(-integral), rel=1e-9)


def test_explin_properties():
    # identity above 1.1, C1 at 1.1, and the Eq. 1 empty density v_far = -10 is (near) transparent
    cam = cam_looking((4.0, 0.0, 0.0), (0.0, 0.0, 0.0), W=5, H=5)
    vals = {}
    for rho in (1.1 - 1e-7, 1.1, 1.1 + 1e-7, 2.5, -10.0):
        oc = one_voxel(0, [0, 0, 0], rho, [0.5, 0.5, 0.5])
        _, _, alpha, _ = oracle.render([oc], [pose64()], cam, oracle.Opts(K=1, eps_stop=0.0))
        vals[rho] = -math.log(1.0 - alpha[2, 2])   # sigma * chord(=1)
    r32 = lambda x: float(np.float32(x))
    assert vals[2.5] == pytest.approx(r32(2.5), rel=1e-12)
    slope = (vals[1.1 + 1e-7] - vals[1.1 - 1e-7]) / (r32(1.1 + 1e-7) - r32(1.1 - 1e-7))
    assert slope == pytest.approx(1.0, abs=1e-3)
    assert vals[1.1] == pytest.approx(r32(1.1), rel=1e-6)
    assert 0.0 < vals[-10.0] < 1e-4          # v_far renders as empty space


def test_subdivision_invariance_of_colour_and_alpha():
    rng = np.random.default_rng(3)
    parent = one_voxel(0, [0, 0, 0], 1.9, [0.3, 0.6, 0.9], root=1.0)
    kids = one_voxel(1, [[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], 1.9, [0.3, 0.6, 0.9], root=1.0)
    cam = cam_looking((2.3, 1.1, -0.8), (0.0, 0.1, 0.0), W=11, H=9, fov=40.0)
    for K in (1, 3):
        r1, d1, a1, _ = oracle.render([parent], [pose64()], cam, oracle.Opts(K=K, eps_stop=0.0))
        r2, d2, a2, _ = oracle.render([kids], [pose64()], cam, oracle.Opts(K=K, eps_stop=0.0))
        np.testing.assert_allclose(r1, r2, atol=1e-12)
        np.testing.assert_allclose(a1, a2, atol=1e-12)
    assert rng is not None


# ---------------------------------------------------------------------------
# Alg. 1 interval walk
# ---------------------------------------------------------------------------

def test_background_voxel_straddling_an_actor_box():
    # background: one voxel [-2,2]^3 (sigma 0.4, colour A); actor box half 0.5 at x = 0.7 holding one
    # voxel filling it (sigma 2.2, colour B).  Axial ray from +x: bg [t_in, a), actor [a, b), bg [b, t_out)
    bg = one_voxel(0, [0, 0, 0], 0.4, [0.8, 0.2, 0.1], root=4.0)
    act = one_voxel(0, [0, 0, 0], 2.2, [0.1, 0.7, 0.9], root=1.0, role=synth.ACTOR, clip_half=(0.5, 0.5, 0.5))
    pose_a = pose64(synth.rot_z(0.3), (0.7, 0.0, 0.0))
    cam = cam_looking((6.0, 0.0, 0.0), (0.0, 0.0, 0.0), W=5, H=5)
    rgb, depth, alpha, nseg = oracle.render([bg, act], [pose64(), pose_a], cam, oracle.Opts(K=2, eps_stop=0.0))
    # rotated box: along x the half-chord is the slab of a square rotated by 0.3 rad through its centre
    half = 0.5 / math.cos(0.3)
    t_in, t_out = 4.0, 8.0
    a, b = 6.0 - 0.7 - half, 6.0 - 0.7 + half
    s_bg, s_act = explin(float(np.float32(0.4))), float(np.float32(2.2))
    cA, cB = colour_of([0.8, 0.2, 0.1]), colour_of([0.1, 0.7, 0.9])
    segs = [(t_in, a, s_bg, cA), (a, b, s_act, cB), (b, t_out, s_bg, cA)]
    T, C, D = 1.0, np.zeros(3), 0.0
    for t0, t1, s, c in segs:
        al = 1 - math.exp(-s * (t1 - t0))
        C += T * al * c
        D += T * al * 0.5 * (t0 + t1)
        T *= 1 - al
    np.testing.assert_allclose(rgb[2, 2], C, rtol=1e-10)
    assert depth[2, 2] == pytest.approx(D, rel=1e-10)
    assert alpha[2, 2] == pytest.approx(1 - T, rel=1e-10)
    assert nseg[2, 2] == 3


def test_overlapping_boxes_first_entered_owns_overlap():
    # two actors along the optical axis; boxes [x in 0.5..2.5] and [x in -0.5..1.5] overlap in x in [0.5, 1.5]
    A = one_voxel(0, [0, 0, 0], 1.3, [0.9, 0.1, 0.1], root=2.0, role=synth.ACTOR, clip_half=(1.0, 1.0, 1.0))
    B = one_voxel(0, [0, 0, 0], 2.6, [0.1, 0.1, 0.9], root=2.0, role=synth.ACTOR, clip_half=(1.0, 1.0, 1.0))
    bg = synth.Octree(np.zeros(0, np.uint64), np.zeros((0, 8), np.float32), np.zeros((0, 1, 3), np.float32), 0,
                      (0.0, 0.0, 0.0), 1.0, synth.BG)
    cam = cam_looking((6.0, 0.0, 0.0), (0.0, 0.0, 0.0), W=5, H=5)
    pa, pb = pose64(t=(1.5, 0, 0)), pose64(t=(0.5, 0, 0))
    for order in ([bg, A, B], [bg, B, A]):
        poses = [pose64(), pa, pb] if order[1] is A else [pose64(), pb, pa]
        rgb, depth, alpha, _ = oracle.render(order, poses, cam, oracle.Opts(K=1, eps_stop=0.0))
        # A (front box) owns t in [3.5, 5.5]; B owns only its remainder t in [5.5, 6.5]
        aA = 1 - math.exp(-float(np.float32(1.3)) * 2.0)
        aB = 1 - math.exp(-float(np.float32(2.6)) * 1.0)
        C = aA * colour_of([0.9, 0.1, 0.1]) + (1 - aA) * aB * colour_of([0.1, 0.1, 0.9])
        np.testing.assert_allclose(rgb[2, 2], C, rtol=1e-10)
        assert depth[2, 2] == pytest.approx(aA * 4.5 + (1 - aA) * aB * 6.0, rel=1e-10)


def test_early_stop_after_the_segment_that_crosses_eps():
    dens = np.stack([np.full(8, 0.9), np.full(8, 1.2), np.full(8, 1.5), np.full(8, 2.0)])
    rgbs = np.array([[0.9, 0.1, 0.1], [0.1, 0.9, 0.1], [0.1, 0.1, 0.9], [0.5, 0.5, 0.5]])
    ijk = [[3, 0, 0], [2, 0, 0], [1, 0, 0], [0, 0, 0]]   # front to back as seen from +x
    oc = one_voxel(2, ijk, dens, rgbs, center=(0.0, 1.5, 1.5), root=4.0)   # unit voxels x in [-2..2]
    cam = cam_looking((6.0, 0.0, 0.0), (0.0, 0.0, 0.0), W=5, H=5)
    eps = 0.2
    rgb, depth, alpha, nseg = oracle.render([oc], [pose64()], cam, oracle.Opts(K=1, eps_stop=eps))
    T, C, n = 1.0, np.zeros(3), 0
    for r, c in zip([0.9, 1.2, 1.5, 2.0], rgbs):
        s = explin(float(np.float32(r)))
        a = 1 - math.exp(-s)
        C += T * a * colour_of(c)
        T *= 1 - a
        n += 1
        if T < eps:
            break
    assert n == 2
    assert nseg[2, 2] == n
    np.testing.assert_allclose(rgb[2, 2], C, rtol=1e-12)
    assert alpha[2, 2] == pytest.approx(1 - T, rel=1e-12)


# ---------------------------------------------------------------------------
# composition invariants (the ones the method is built on)
# ---------------------------------------------------------------------------

def _small_bg(level=3, hole=True, seed=0, sh_degree=2):
    rng = np.random.default_rng(seed)
    n = 1 << level
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    if hole:   # leave [-0.5, 0.5]^3 empty (cells 2..5 at level 3 of [-1,1]^3)
        inner = np.all((ijk >= n // 4) & (ijk < 3 * n // 4), axis=1)
        ijk = ijk[~inner]
    V = ijk.shape[0]
    keep = rng.uniform(size=V) < 0.6
    ijk = ijk[keep]
    V = ijk.shape[0]
    key = synth.pack_keys(np.full(V, level), ijk[:, 0], ijk[:, 1], ijk[:, 2])
    dens = rng.lognormal(-0.5, 1.0, (V, 8)).astype(np.float32)
    sh = rng.normal(0, 0.3, (V, (sh_degree + 1) ** 2, 3)).astype(np.float32)
    return synth.Octree(key, dens, sh, sh_degree, (0.0, 0.0, 0.0), 2.0, synth.BG), ijk


def test_identity_pose_actor_equals_merged_octree():
    bg, _ = _small_bg()
    rng = np.random.default_rng(1)
    # actor: level 2 of a unit root at the origin = the level-3 cells of the hole
    n = 4
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    aijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    aijk = aijk[rng.uniform(size=64) < 0.7]
    Va = aijk.shape[0]
    akey = synth.pack_keys(np.full(Va, 2), aijk[:, 0], aijk[:, 1], aijk[:, 2])
    adens = rng.lognormal(0.0, 1.0, (Va, 8)).astype(np.float32)
    ash = rng.normal(0, 0.3, (Va, 9, 3)).astype(np.float32)
    act = synth.Octree(akey, adens, ash, 2, (0.0, 0.0, 0.0), 1.0, synth.ACTOR, (0.5, 0.5, 0.5))
    mijk = aijk + 2
    merged = synth.Octree(np.concatenate([bg.key, synth.pack_keys(np.full(Va, 3), mijk[:, 0], mijk[:, 1], mijk[:, 2])]),
                          np.concatenate([bg.dens, adens]), np.concatenate([bg.sh, ash]), 2, (0.0, 0.0, 0.0), 2.0,
                          synth.BG)
    cam = cam_looking((2.6, 1.3, 0.9), (0.0, 0.0, 0.0), W=24, H=20, fov=55.0)
    for K, eps in ((1, 0.0), (2, 1e-4)):
        a = oracle.render([bg, act], [pose64(), pose64()], cam, oracle.Opts(K=K, eps_stop=eps))
        b = oracle.render([merged], [pose64()], cam, oracle.Opts(K=K, eps_stop=eps))
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-13)


def _comp_scene(seed=4):
    bg, _ = _small_bg(seed=seed, hole=False)
    rng = np.random.default_rng(seed + 1)
    acts, poses = [], [pose64()]
    for a in range(2):
        n = 4
        k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
        ijk = ijk[rng.uniform(size=64) < 0.5]
        V = ijk.shape[0]
        key = synth.pack_keys(np.full(V, 2), ijk[:, 0], ijk[:, 1], ijk[:, 2])
        acts.append(synth.Octree(key, rng.lognormal(0.5, 0.7, (V, 8)).astype(np.float32),
                                 rng.normal(0, 0.3, (V, 9, 3)).astype(np.float32), 2, (0.0, 0.0, 0.0), 0.6,
                                 synth.ACTOR, (0.31, 0.27, 0.3)))
        poses.append(pose64(synth.random_rotation(rng), rng.uniform(-0.6, 0.6, 3)))
    return [bg] + acts, poses


def test_rigid_equivariance():
    octs, poses = _comp_scene()
    cam = cam_looking((2.4, -1.5, 1.1), (0.0, 0.0, 0.0), W=20, H=16, fov=50.0)
    rng = np.random.default_rng(9)
    G = np.eye(4)
    G[:3, :3] = synth.random_rotation(rng)
    G[:3, 3] = rng.uniform(-3, 3, 3)
    mv = lambda p: (lambda m: pose64(m[:3, :3], m[:3, 3]))(G @ np.block([[p.R, p.t[:, None]], [np.zeros((1, 3)), 1]]))
    poses2 = [mv(p) for p in poses]
    cam2 = SimpleNamespace(**{**cam.__dict__, "pose": mv(cam.pose)})
    a = oracle.render(octs, poses, cam, oracle.Opts(K=2, eps_stop=1e-4))
    b = oracle.render(octs, poses2, cam2, oracle.Opts(K=2, eps_stop=1e-4))
    assert np.count_nonzero(a[2] > 0.05) > 50
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-11)


def test_actor_permutation_invariance():
    octs, poses = _comp_scene(seed=7)
    cam = cam_looking((2.4, 1.5, 1.1), (0.0, 0.0, 0.0), W=16, H=16, fov=50.0)
    a = oracle.render(octs, poses, cam, oracle.Opts(K=1))
    b = oracle.render([octs[0], octs[2], octs[1]], [poses[0], poses[2], poses[1]], cam, oracle.Opts(K=1))
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-13)


def test_output_bounds_on_config1():
    sc, cams, _ = synth.config1()
    rgb, depth, alpha, nseg = oracle.render(sc.octrees, sc.poses, cams[0], oracle.Opts(K=1, eps_stop=0.0))
    assert np.all(alpha >= 0) and np.all(alpha <= 1)
    # colours are in [0, 1] here, so C <= alpha componentwise; depth lies in [near, far] * alpha
    assert np.all(rgb <= alpha[..., None] + 1e-12)
    assert np.all(depth >= cams[0].near * alpha - 1e-12) and np.all(depth <= cams[0].far * alpha + 1e-12)
    assert (alpha > 0.5).mean() > 0.3


# ---------------------------------------------------------------------------
# spherical harmonics and view direction
# ---------------------------------------------------------------------------

def _scipy_real_sh(l, m, x, y, z):
    sp = pytest.importorskip("scipy.special")
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if hasattr(sp, "sph_harm_y"):
        Y = lambda mm: complex(sp.sph_harm_y(l, mm, theta, phi))
    else:
        Y = lambda mm: complex(sp.sph_harm(mm, l, phi, theta))
    if m == 0:
        return Y(0).real
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * Y(m).real
    return math.sqrt(2.0) * (-1) ** m * Y(-m).imag


def test_sh_basis_matches_scipy_with_odd_m_sign():
    # Reading: the real SH of the SH-coloured voxel lineage (degree-1 terms -k*y, k*z, -k*x): scipy's
    # real SH (built below from the complex ones with the Condon-Shortley phase cancelled) times
    # (-1)^m, term for term.
    rng = np.random.default_rng(0)
    dirs = rng.normal(size=(25, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    lm = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    sign = np.array([(-1.0) ** m for _, m in lm])
    for x, y, z in dirs:
        Y = oracle.sh_basis(3, x, y, z)
        ref = np.array([_scipy_real_sh(l, m, x, y, z) for l, m in lm])
        np.testing.assert_allclose(Y, sign * ref, rtol=1e-10, atol=1e-12)


def test_sh_basis_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 polynomials exactly
    xg, wg = np.polynomial.legendre.leggauss(8)
    phis = np.arange(16) * 2 * math.pi / 16
    G = np.zeros((16, 16))
    for z, w in zip(xg, wg):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            Y = oracle.sh_basis(3, r * math.cos(ph), r * math.sin(ph), z)
            G += np.outer(Y, Y) * w * (2 * math.pi / 16)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_view_direction_is_camera_to_voxel_centre_in_local_frame():
    # degree-1 SH with only the (1,0) ~ z coefficient: colour = 0.5 + k1 * g_z * coef
    k1 = math.sqrt(3.0 / (4.0 * math.pi))
    coef = 0.4
    key = synth.pack_keys([0], [0], [0], [0])
    sh = np.zeros((1, 4, 3), np.float32)
    sh[0, 2, :] = coef
    oc = synth.Octree(key, np.full((1, 8), 30.0, np.float32), sh, 1, (0.0, 0.0, 0.0), 1.0, synth.BG)
    for zc, gz in ((6.0, -1.0), (-6.0, 1.0)):
        cam = cam_looking((0.0, 0.0, zc), (0.0, 0.0, 0.0), W=5, H=5, up=(0.0, 1.0, 0.0))
        rgb, _, alpha, _ = oracle.render([oc], [pose64()], cam, oracle.Opts(K=1, eps_stop=0.0))
        expect = 0.5 + k1 * gz * float(np.float32(coef))
        np.testing.assert_allclose(rgb[2, 2] / alpha[2, 2], expect, rtol=1e-12)
    # rotating the octree (pose) by 180 deg about x flips the local view direction
    cam = cam_looking((0.0, 0.0, 6.0), (0.0, 0.0, 0.0), W=5, H=5, up=(0.0, 1.0, 0.0))
    Rx = np.diag([1.0, -1.0, -1.0])
    rgb, _, alpha, _ = oracle.render([oc], [pose64(Rx)], cam, oracle.Opts(K=1, eps_stop=0.0))
    np.testing.assert_allclose(rgb[2, 2] / alpha[2, 2], 0.5 + k1 * float(np.float32(coef)), rtol=1e-12)


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

def _loss(octs, poses, cam, f64, g, opts):
    rgb, depth, alpha, _ = oracle.render(octs, poses, cam, opts, f64_arrays=f64)
    return float(np.sum(g[0] * rgb) + np.sum(g[1] * depth) + np.sum(g[2] * alpha))


@pytest.mark.parametrize("K", [1, 3])
def test_backward_matches_central_differences(K):
    octs, poses = _comp_scene(seed=11)
    cam = cam_looking((2.2, 1.7, 0.9), (0.0, 0.0, 0.0), W=13, H=10, fov=45.0)
    opts = oracle.Opts(K=K, eps_stop=0.0)
    rng = np.random.default_rng(5)
    g = (rng.normal(size=(cam.H, cam.W, 3)), rng.normal(size=(cam.H, cam.W)) * 0.1, rng.normal(size=(cam.H, cam.W)))
    f64 = [(o.dens.astype(np.float64), o.sh.astype(np.float64)) for o in octs]
    dd, ds = oracle.backward(octs, poses, cam, g[0].reshape(-1, 3), g[1].reshape(-1), g[2].reshape(-1), opts,
                             f64_arrays=f64)
    checked = 0
    for oi in range(len(octs)):
        nz = np.argwhere(np.abs(dd[oi]) > 1e-4)
        for idx in nz[rng.permutation(len(nz))[:6]]:
            v, c = idx
            x0 = f64[oi][0][v, c]
            if abs(x0 - 1.1) < 1e-3:
                continue
            h = 1e-6 * max(1.0, abs(x0))
            f64[oi][0][v, c] = x0 + h
            lp = _loss(octs, poses, cam, f64, g, opts)
            f64[oi][0][v, c] = x0 - h
            lm = _loss(octs, poses, cam, f64, g, opts)
            f64[oi][0][v, c] = x0
            fd = (lp - lm) / (2 * h)
            assert dd[oi][v, c] == pytest.approx(fd, rel=2e-5, abs=1e-8)
            checked += 1
        nz = np.argwhere(np.abs(ds[oi]) > 1e-4)
        for idx in nz[rng.permutation(len(nz))[:6]]:
            v, lm_, ch = idx
            x0 = f64[oi][1][v, lm_, ch]
            h = 1e-6
            f64[oi][1][v, lm_, ch] = x0 + h
            lp = _loss(octs, poses, cam, f64, g, opts)
            f64[oi][1][v, lm_, ch] = x0 - h
            lmv = _loss(octs, poses, cam, f64, g, opts)
            f64[oi][1][v, lm_, ch] = x0
            fd = (lp - lmv) / (2 * h)
            assert ds[oi][v, lm_, ch] == pytest.approx(fd, rel=2e-5, abs=1e-8)
            checked += 1
    assert checked >= 20


def test_backward_through_the_colour_clamp():
    # colour = max(0, sum Y k + 0.5): a channel clamped at zero gets no SH gradient, the others get
    # the full one; both checked against central differences of the whole image's loss
    key = synth.pack_keys([1], [0], [0], [0])
    sh = np.zeros((1, 4, 3), np.float32)
    sh[0, 0, :] = (-3.0, 0.7, 0.1)       # red clamped: 0.5 - 3 * 0.282 < 0
    sh[0, 1:, :] = 0.05
    oc = synth.Octree(key, np.full((1, 8), 1.5, np.float32), sh, 1, (0.0, 0.0, 0.0), 2.0, synth.BG)
    cam = cam_looking((1.3, 0.8, 3.0), (0.0, 0.0, 0.0), W=9, H=7, fov=40.0)
    opts = oracle.Opts(K=2, eps_stop=0.0)
    rng = np.random.default_rng(2)
    g = (rng.normal(size=(cam.H, cam.W, 3)), np.zeros((cam.H, cam.W)), np.zeros((cam.H, cam.W)))
    f64 = [(oc.dens.astype(np.float64), oc.sh.astype(np.float64))]
    _, ds = oracle.backward([oc], [pose64()], cam, g[0].reshape(-1, 3), g[1].reshape(-1), g[2].reshape(-1), opts,
                            f64_arrays=f64)
    rgb, _, alpha, _ = oracle.render([oc], [pose64()], cam, opts)
    assert alpha.max() > 0.1 and np.all(rgb[..., 0] == 0.0)
    assert np.all(ds[0][0, :, 0] == 0.0) and np.abs(ds[0][0, :, 1]).max() > 1e-3
    for lm_ in range(4):
        for ch in range(3):
            x0 = f64[0][1][0, lm_, ch]
            h = 1e-6
            f64[0][1][0, lm_, ch] = x0 + h
            lp = _loss([oc], [pose64()], cam, f64, g, opts)
            f64[0][1][0, lm_, ch] = x0 - h
            lmv = _loss([oc], [pose64()], cam, f64, g, opts)
            f64[0][1][0, lm_, ch] = x0
            assert ds[0][0, lm_, ch] == pytest.approx((lp - lmv) / (2 * h), rel=2e-5, abs=1e-8)


# ---------------------------------------------------------------------------
# normal state N (Alg. 1: the pixel state sums voxel normals)
# ---------------------------------------------------------------------------

def _linear_field(u, k0=3.0, scale=0.7):
    # corner densities k0 - scale * (u . corner bits): the trilinear field decreases along u, so the
    # voxel normal (minus the normalised density gradient) is u / |u|
    bits = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.float64)
    return k0 - scale * bits @ np.asarray(u, np.float64)


def test_normal_of_a_linear_field_is_its_descent_direction():
    rng = np.random.default_rng(31)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    dens = np.float32(_linear_field(u)).astype(np.float64)
    oc = one_voxel(0, (0, 0, 0), dens, (0.4, 0.5, 0.6))
    cam = cam_looking((2.0, 1.4, 1.1), (0.0, 0.0, 0.0), W=9, H=9, fov=40.0)
    # the float32-stored corners give the exact field direction up to float32 rounding of the inputs
    bits = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.float64)
    g = np.array([np.sum(np.where(bits[:, a] == 1, dens, -dens)) for a in range(3)])
    n_exp = -g / np.linalg.norm(g)
    assert np.allclose(n_exp, u, atol=1e-6)
    rgb, _, alpha, _, N = oracle.render([oc], [pose64()], cam, oracle.Opts(K=1, eps_stop=0.0), normals=True)
    hit = alpha > 1e-3
    assert hit.sum() > 20
    np.testing.assert_allclose(N[hit] / alpha[hit, None], np.broadcast_to(n_exp, (hit.sum(), 3)), rtol=1e-10,
                               atol=1e-12)
    # the same voxel as an actor under a rotation: the normal turns with the pose
    R = synth.random_rotation(rng).astype(np.float64)
    t = np.array([0.1, -0.2, 0.05])
    act = one_voxel(0, (0, 0, 0), dens, (0.4, 0.5, 0.6), role=synth.ACTOR, clip_half=(0.6, 0.6, 0.6))
    empty = one_voxel(0, np.zeros((0, 3), int), 1.0, (0.5, 0.5, 0.5))
    _, _, a2, _, N2 = oracle.render([empty, act], [pose64(), pose64(R, t)], cam, oracle.Opts(K=1, eps_stop=0.0),
                                    normals=True)
    hit = a2 > 1e-3
    assert hit.sum() > 20
    np.testing.assert_allclose(N2[hit] / a2[hit, None], np.broadcast_to(R @ n_exp, (hit.sum(), 3)), rtol=1e-10,
                               atol=1e-12)


def test_normal_of_a_constant_voxel_is_zero():
    oc = one_voxel(0, (0, 0, 0), 2.0, (0.4, 0.5, 0.6))
    cam = cam_looking((2.0, 1.4, 1.1), (0.0, 0.0, 0.0), W=7, H=7, fov=40.0)
    _, _, alpha, _, N = oracle.render([oc], [pose64()], cam, oracle.Opts(K=2, eps_stop=0.0), normals=True)
    assert alpha.max() > 0.5 and np.all(N == 0.0)


def test_normals_of_stacked_voxels_are_weighted_front_to_back():
    # two voxels on the optical axis with different normals: N = a1 n1 + (1 - a1) a2 n2, with each
    # voxel's own alpha taken from a render of that voxel alone
    rng = np.random.default_rng(32)
    u1, u2 = rng.normal(size=3), rng.normal(size=3)
    u1 /= np.linalg.norm(u1)
    u2 /= np.linalg.norm(u2)
    d1 = np.float32(_linear_field(u1, k0=1.6, scale=0.5)).astype(np.float64)
    d2 = np.float32(_linear_field(u2, k0=2.4, scale=0.9)).astype(np.float64)
    both = one_voxel(1, [(0, 0, 0), (1, 0, 0)], np.stack([d1, d2]), (0.5, 0.5, 0.5), center=(0.5, 0.5, 0.5),
                     root=2.0)
    front = one_voxel(1, [(0, 0, 0)], d1, (0.5, 0.5, 0.5), center=(0.5, 0.5, 0.5), root=2.0)
    back = one_voxel(1, [(1, 0, 0)], d2, (0.5, 0.5, 0.5), center=(0.5, 0.5, 0.5), root=2.0)
    cam = cam_looking((-3.0, 0.0, 0.0), (1.0, 0.0, 0.0), W=1, H=1, fov=1.0, up=(0.0, 0.0, 1.0))
    opts = oracle.Opts(K=1, eps_stop=0.0)
    _, _, a1, _ = oracle.render([front], [pose64()], cam, opts)
    _, _, a2, _ = oracle.render([back], [pose64()], cam, opts)
    _, _, a, _, N = oracle.render([both], [pose64()], cam, opts, normals=True)
    a1, a2 = float(a1[0, 0]), float(a2[0, 0])
    assert 0.05 < a1 < 0.95 and 0.05 < a2 < 0.99
    n = lambda d: (lambda g: -g / np.linalg.norm(g))(
        np.array([np.sum([d[c] if (c >> ax) & 1 else -d[c] for c in range(8)]) for ax in range(3)]))
    np.testing.assert_allclose(N[0, 0], a1 * n(d1) + (1 - a1) * a2 * n(d2), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(a[0, 0], 1 - (1 - a1) * (1 - a2), rtol=1e-12)


def test_normals_turn_with_a_rigid_motion_of_scene_and_camera():
    octs, poses = _comp_scene()
    cam = cam_looking((2.4, -1.5, 1.1), (0.0, 0.0, 0.0), W=20, H=16, fov=50.0)
    rng = np.random.default_rng(33)
    G = np.eye(4)
    G[:3, :3] = synth.random_rotation(rng)
    G[:3, 3] = rng.uniform(-3, 3, 3)
    mv = lambda p: (lambda m: pose64(m[:3, :3], m[:3, 3]))(G @ np.block([[p.R, p.t[:, None]], [np.zeros((1, 3)), 1]]))
    cam2 = SimpleNamespace(**{**cam.__dict__, "pose": mv(cam.pose)})
    a = oracle.render(octs, poses, cam, oracle.Opts(K=2, eps_stop=1e-4), normals=True)
    b = oracle.render(octs, [mv(p) for p in poses], cam2, oracle.Opts(K=2, eps_stop=1e-4), normals=True)
    assert np.abs(a[4]).max() > 0.3
    np.testing.assert_allclose(b[4], a[4] @ G[:3, :3].T, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("K", [1, 2])
def test_backward_through_normals_matches_central_differences(K):
    octs, poses = _comp_scene(seed=12)
    cam = cam_looking((2.2, 1.7, 0.9), (0.0, 0.0, 0.0), W=11, H=9, fov=45.0)
    opts = oracle.Opts(K=K, eps_stop=0.0)
    rng = np.random.default_rng(34)
    gN = rng.normal(size=(cam.H * cam.W, 3))
    gC = 0.3 * rng.normal(size=(cam.H * cam.W, 3))
    z = np.zeros(cam.H * cam.W)
    f64 = [(o.dens.astype(np.float64), o.sh.astype(np.float64)) for o in octs]
    dd, _ = oracle.backward(octs, poses, cam, gC, z, z, opts, f64_arrays=f64, g_normal=gN)

    def loss():
        r = oracle.render(octs, poses, cam, opts, f64_arrays=f64, normals=True)
        return float(np.sum(gC * r[0].reshape(-1, 3)) + np.sum(gN * r[4].reshape(-1, 3)))

    checked = 0
    for oi in range(len(octs)):
        nz = np.argwhere(np.abs(dd[oi]) > 1e-4)
        for v, c in nz[rng.permutation(len(nz))[:8]]:
            x0 = f64[oi][0][v, c]
            if abs(x0 - 1.1) < 1e-3:
                continue
            h = 1e-6 * max(1.0, abs(x0))
            f64[oi][0][v, c] = x0 + h
            lp = loss()
            f64[oi][0][v, c] = x0 - h
            lm = loss()
            f64[oi][0][v, c] = x0
            assert dd[oi][v, c] == pytest.approx((lp - lm) / (2 * h), rel=2e-5, abs=1e-8)
            checked += 1
    assert checked >= 16


# ---------------------------------------------------------------------------
# compositing weights (feature fields: RGB replaced by a per-voxel feature)
# ---------------------------------------------------------------------------

def test_pixel_weights_reproduce_colour_alpha_and_depth():
    octs, poses = _comp_scene(seed=13)
    cam = cam_looking((2.2, -1.2, 1.0), (0.0, 0.0, 0.0), W=9, H=7, fov=50.0)
    opts = oracle.Opts(K=2, eps_stop=1e-3)
    rgb, depth, alpha, nseg = oracle.render(octs, poses, cam, opts)
    seen = 0
    for v in range(cam.H):
        for u in range(cam.W):
            oi, vi, w = oracle.pixel_weights(octs, poses, cam, u, v, opts)
            assert len(w) == nseg[v, u]
            assert np.all(w >= 0)
            np.testing.assert_allclose(w.sum(), alpha[v, u], rtol=1e-12, atol=1e-14)
            seen += len(w) > 0
    assert seen > 20


def test_feature_of_a_constant_colour_scene_equals_its_render():
    # degree-0 SH: every voxel's colour is its feature; F = sum w f must equal the rendered RGB
    rng = np.random.default_rng(14)
    ijk = np.argwhere(rng.uniform(size=(4, 4, 4)) < 0.6)
    cols = rng.uniform(0.1, 0.9, size=(len(ijk), 3))
    oc = one_voxel(2, ijk, rng.lognormal(0.0, 0.7, size=(len(ijk), 8)), cols)
    cam = cam_looking((2.0, 1.1, 0.8), (0.0, 0.0, 0.0), W=8, H=6, fov=55.0)
    opts = oracle.Opts(K=1, eps_stop=1e-4)
    rgb, _, _, _ = oracle.render([oc], [pose64()], cam, opts)
    feat = colour_of(cols)   # the colour each voxel actually renders with
    for v in range(cam.H):
        for u in range(cam.W):
            _, vi, w = oracle.pixel_weights([oc], [pose64()], cam, u, v, opts)
            np.testing.assert_allclose(w @ feat[vi] if len(w) else np.zeros(3), rgb[v, u], rtol=1e-12, atol=1e-14)
