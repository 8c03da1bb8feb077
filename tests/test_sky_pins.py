"""Pins of the sky-composite oracle (Eq. 2, equirectangular reading; see oracle/sky.py):

- a constant map adds T_final * constant to every pixel;
- yaw equivariance: turning the camera about the world z axis by k texel widths equals rolling
  the map by k columns (pins the longitude direction, its origin and the wrap-around);
- the zenith samples the first row, the nadir the last, the horizon the mean of the two middle
  rows (pins the latitude mapping and the clamp);
- bilinear weights equal scipy's linear grid interpolation away from the seam and the poles;
- the backward equals central differences in FP64 (map texels and alpha).
"""
import math
from types import SimpleNamespace

import numpy as np
import pytest

import oracle.sky as sky
import synth


def _cam(W=12, H=9, yaw=0.3, pitch=0.2, fov=70.0):
    f = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch)])
    p = synth.look_at((0.0, 0.0, 0.0), f)
    fx = float(np.float32((W / 2.0) / math.tan(math.radians(fov) / 2.0)))
    return SimpleNamespace(W=W, H=H, fx=fx, fy=fx, cx=W / 2.0, cy=H / 2.0,
                           pose=SimpleNamespace(R=np.asarray(p.R, np.float64), t=np.zeros(3)))


def test_constant_map_adds_transmittance_times_colour():
    rng = np.random.default_rng(0)
    cam = _cam()
    n = cam.W * cam.H
    rgb, alpha = rng.uniform(size=(n, 3)), rng.uniform(size=n)
    env = np.broadcast_to(np.array([0.2, 0.5, 0.9]), (8, 16, 3))
    out = sky.composite(rgb, alpha, sky.pixel_directions(cam), env)
    np.testing.assert_allclose(out, rgb + (1 - alpha)[:, None] * np.array([0.2, 0.5, 0.9]), rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("k", [1, 5, -3])
def test_yaw_by_whole_texels_rolls_the_map(k):
    rng = np.random.default_rng(1)
    H, W = 8, 24
    env = rng.uniform(size=(H, W, 3))
    dirs = sky.pixel_directions(_cam(yaw=0.37, pitch=0.15))
    th = 2 * math.pi * k / W
    Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    n = dirs.shape[0]
    a = sky.composite(np.zeros((n, 3)), np.zeros(n), dirs @ Rz.T, env)
    b = sky.composite(np.zeros((n, 3)), np.zeros(n), dirs, np.roll(env, -k, axis=1))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_zenith_nadir_and_horizon_rows():
    H, W = 6, 10
    rows = np.arange(H, dtype=np.float64)[:, None, None] * np.array([1.0, 10.0, 100.0])
    env = np.broadcast_to(rows, (H, W, 3))
    np.testing.assert_allclose(sky.sky_color(env, np.array([0.0, 0.0, 1.0])), env[0, 0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(sky.sky_color(env, np.array([0.0, 0.0, -1.0])), env[H - 1, 0], rtol=0, atol=1e-12)
    for lon in np.linspace(-3.0, 3.0, 7):
        d = np.array([math.cos(lon), math.sin(lon), 0.0])
        np.testing.assert_allclose(sky.sky_color(env, d), 0.5 * (env[H // 2 - 1, 0] + env[H // 2, 0]), atol=1e-12)


def test_bilinear_weights_match_scipy_linear_interpolation():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(2)
    H, W = 10, 20
    env = rng.uniform(size=(H, W, 3))
    f = interp.RegularGridInterpolator((np.arange(H) + 0.5, np.arange(W) + 0.5), env, method="linear")
    for _ in range(50):
        # directions whose lookup stays between texel centres (no seam, no pole clamp)
        lon = rng.uniform(-math.pi + 2 * math.pi / W, math.pi - 2 * math.pi / W)
        polar = rng.uniform(math.pi / H, math.pi - math.pi / H)
        d = np.array([math.sin(polar) * math.cos(lon), math.sin(polar) * math.sin(lon), math.cos(polar)])
        y = polar / math.pi * H
        x = (lon + math.pi) / (2 * math.pi) * W
        np.testing.assert_allclose(sky.sky_color(env, d), f([[y, x]])[0], rtol=1e-12, atol=1e-12)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    cam = _cam(W=7, H=5)
    dirs = sky.pixel_directions(cam)
    n = dirs.shape[0]
    env = rng.uniform(size=(6, 12, 3))
    rgb, alpha = rng.uniform(size=(n, 3)), rng.uniform(size=n)
    g = rng.normal(size=(n, 3))
    d_env, d_alpha, d_rgb = sky.backward(alpha, dirs, env, g)
    loss = lambda e, a: float(np.sum(g * sky.composite(rgb, a, dirs, e)))
    h = 1e-6
    for j, i, c in [tuple(x) for x in np.argwhere(np.abs(d_env) > 1e-3)[:25]]:
        e1, e2 = env.copy(), env.copy()
        e1[j, i, c] += h
        e2[j, i, c] -= h
        assert d_env[j, i, c] == pytest.approx((loss(e1, alpha) - loss(e2, alpha)) / (2 * h), rel=1e-6, abs=1e-9)
    for p in range(0, n, 3):
        a1, a2 = alpha.copy(), alpha.copy()
        a1[p] += h
        a2[p] -= h
        assert d_alpha[p] == pytest.approx((loss(env, a1) - loss(env, a2)) / (2 * h), rel=1e-6, abs=1e-9)
    np.testing.assert_array_equal(d_rgb, g)
