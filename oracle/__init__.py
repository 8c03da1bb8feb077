"""FP64 brute-force oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
pthreads) through ctypes and shares no code with the CUDA path.  Inputs come
from :mod:`synth`; the oracle reads the same float32 arrays the GPU reads and
computes in double precision.

Pins (closed forms, invariants, finite differences, the SH basis against
scipy) live in ``tests/test_oracle_pins.py``; see that file's docstring.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ROLE_BG, ROLE_ACTOR = 0, 1
ACT_EXPLIN, ACT_IDENTITY = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, so x86 and Arm agree bit for bit)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Octree(C.Structure):
    _fields_ = [("n_vox", C.c_int64), ("sh_degree", C.c_int), ("role", C.c_int), ("f64", C.c_int),
                ("center", C.c_double * 3), ("root_size", C.c_double), ("clip_half", C.c_double * 3),
                ("key", C.c_void_p), ("dens", C.c_void_p), ("sh", C.c_void_p)]


class _Pose(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3)]


class _Camera(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("c2w", _Pose), ("near_", C.c_double), ("far_", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("K", C.c_int), ("eps_stop", C.c_double), ("activation", C.c_int)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        override = os.environ.get("DV_ORACLE_LIB")   # a separately built oracle (mutation tests)
        lib = C.CDLL(override if override else build())
        lib.orc_render.restype = C.c_int
        lib.orc_backward.restype = C.c_int
        lib.orc_pixel_segments.restype = C.c_int64
        lib.orc_pixel_weights.restype = C.c_int64
        lib.orc_sh_basis.restype = None
        _lib = lib
    return _lib


@dataclass
class Opts:
    K: int = 1
    eps_stop: float = 1e-4
    activation: int = ACT_EXPLIN


def _pose(p) -> _Pose:
    P = _Pose()
    R = np.asarray(p.R, np.float64).reshape(9)   # float32 values promoted exactly
    t = np.asarray(p.t, np.float64).reshape(3)
    for i in range(9):
        P.R[i] = float(R[i])
    for i in range(3):
        P.t[i] = float(t[i])
    return P


class _Marshal:
    """Keeps the numpy buffers alive while the C call runs."""

    def __init__(self, octrees, poses, cam, opts, f64_arrays=None):
        self.keep = []
        n = len(octrees)
        self.oct = (_Octree * max(n, 1))()
        for i, oc in enumerate(octrees):
            key = np.ascontiguousarray(oc.key, np.uint64)
            if f64_arrays is not None and f64_arrays[i] is not None:
                dens, sh = f64_arrays[i]
                f64 = 1
            else:
                dens = np.ascontiguousarray(oc.dens, np.float32)
                sh = np.ascontiguousarray(oc.sh, np.float32)
                f64 = 0
            self.keep += [key, dens, sh]
            o = self.oct[i]
            o.n_vox = oc.n
            o.sh_degree = oc.sh_degree
            o.role = oc.role
            o.f64 = f64
            for a in range(3):
                o.center[a] = float(oc.center[a])
                o.clip_half[a] = float(np.float32(oc.clip_half[a]))
            o.root_size = float(oc.root_size)
            o.key = key.ctypes.data
            o.dens = dens.ctypes.data
            o.sh = sh.ctypes.data
        self.n = n
        self.poses = (_Pose * max(n, 1))(*[_pose(p) for p in poses])
        c = _Camera()
        c.W, c.H = int(cam.W), int(cam.H)
        c.fx, c.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
        c.cx, c.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
        c.c2w = _pose(cam.pose)
        c.near_, c.far_ = float(np.float32(cam.near)), float(np.float32(cam.far))
        self.cam = c
        o = _Opts()
        o.K, o.eps_stop, o.activation = int(opts.K), float(np.float32(opts.eps_stop)), int(opts.activation)
        self.opts = o


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def render(octrees, poses, cam, opts: Opts = Opts(), pixels=None, n_threads=None, f64_arrays=None, normals=False):
    """Returns (rgb [n,3], depth [n], alpha [n], n_seg [n]) in float64 for the given linear pixel
    indices (v*W+u), or the whole image ([H,W,...]) when ``pixels`` is None; with ``normals`` the
    normal state N [n,3] (world frame) is appended."""
    lib = _load()
    m = _Marshal(octrees, poses, cam, opts, f64_arrays)
    if pixels is None:
        n = cam.W * cam.H
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        n = pix.shape[0]
        pix_ptr = pix.ctypes.data
    rgb = np.zeros((n, 3))
    depth = np.zeros(n)
    alpha = np.zeros(n)
    nseg = np.zeros(n, np.int32)
    nrm = np.zeros((n, 3)) if normals else None
    st = lib.orc_render(m.oct, C.c_int(m.n), m.poses, C.byref(m.cam), C.byref(m.opts), C.c_int64(n),
                        C.c_void_p(pix_ptr), rgb.ctypes.data_as(C.c_void_p), depth.ctypes.data_as(C.c_void_p),
                        alpha.ctypes.data_as(C.c_void_p), nseg.ctypes.data_as(C.c_void_p),
                        C.c_int(_threads(n_threads)), C.c_void_p(nrm.ctypes.data if normals else None))
    if st != 0:
        raise RuntimeError(f"orc_render failed with status {st}")
    if pixels is None:
        out = (rgb.reshape(cam.H, cam.W, 3), depth.reshape(cam.H, cam.W), alpha.reshape(cam.H, cam.W),
               nseg.reshape(cam.H, cam.W))
        return out + (nrm.reshape(cam.H, cam.W, 3),) if normals else out
    return (rgb, depth, alpha, nseg, nrm) if normals else (rgb, depth, alpha, nseg)


def backward(octrees, poses, cam, g_rgb, g_depth, g_alpha, opts: Opts = Opts(), pixels=None, n_threads=None,
             f64_arrays=None, g_normal=None):
    """Analytic FP64 gradients (list of d_dens [V,8], list of d_sh [V,nsh,3]) for upstream
    gradients given per pixel (same pixel convention as :func:`render`); ``g_normal`` [n,3] is
    dL/dN (None: zero)."""
    lib = _load()
    m = _Marshal(octrees, poses, cam, opts, f64_arrays)
    if pixels is None:
        n = cam.W * cam.H
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        n = pix.shape[0]
        pix_ptr = pix.ctypes.data
    g_rgb = np.ascontiguousarray(np.asarray(g_rgb, np.float64).reshape(n, 3))
    g_depth = np.ascontiguousarray(np.asarray(g_depth, np.float64).reshape(n))
    g_alpha = np.ascontiguousarray(np.asarray(g_alpha, np.float64).reshape(n))
    g_nrm = None if g_normal is None else np.ascontiguousarray(np.asarray(g_normal, np.float64).reshape(n, 3))
    d_dens = [np.zeros((oc.n, 8)) for oc in octrees]
    d_sh = [np.zeros((oc.n, (oc.sh_degree + 1) ** 2, 3)) for oc in octrees]
    pd = (C.c_void_p * max(len(octrees), 1))(*[a.ctypes.data for a in d_dens])
    ps = (C.c_void_p * max(len(octrees), 1))(*[a.ctypes.data for a in d_sh])
    st = lib.orc_backward(m.oct, C.c_int(m.n), m.poses, C.byref(m.cam), C.byref(m.opts), C.c_int64(n),
                          C.c_void_p(pix_ptr), g_rgb.ctypes.data_as(C.c_void_p),
                          g_depth.ctypes.data_as(C.c_void_p), g_alpha.ctypes.data_as(C.c_void_p), pd, ps,
                          C.c_int(_threads(n_threads)), C.c_void_p(None if g_nrm is None else g_nrm.ctypes.data))
    if st != 0:
        raise RuntimeError(f"orc_backward failed with status {st}")
    return d_dens, d_sh


def pixel_segments(octrees, poses, cam, u, v, cap=4096):
    """Sorted (t0, t1, octree, voxel) sub-segments along pixel (u, v)'s ray."""
    lib = _load()
    m = _Marshal(octrees, poses, cam, Opts())
    t0 = np.zeros(cap)
    t1 = np.zeros(cap)
    oi = np.zeros(cap, np.int32)
    vi = np.zeros(cap, np.int64)
    n = lib.orc_pixel_segments(m.oct, C.c_int(m.n), m.poses, C.byref(m.cam), C.c_int(u), C.c_int(v),
                               C.c_int64(cap), t0.ctypes.data_as(C.c_void_p), t1.ctypes.data_as(C.c_void_p),
                               oi.ctypes.data_as(C.c_void_p), vi.ctypes.data_as(C.c_void_p))
    if n < 0:
        raise RuntimeError("orc_pixel_segments failed")
    n = min(n, cap)
    return t0[:n], t1[:n], oi[:n], vi[:n]


def pixel_weights(octrees, poses, cam, u, v, opts: Opts = Opts(), cap=65536):
    """Composited segments of pixel (u, v) in front-to-back order: (octree [n], voxel [n],
    weight T_k alpha_k [n]), ending at the early stop."""
    lib = _load()
    m = _Marshal(octrees, poses, cam, opts)
    oi = np.zeros(cap, np.int32)
    vi = np.zeros(cap, np.int64)
    w = np.zeros(cap)
    n = lib.orc_pixel_weights(m.oct, C.c_int(m.n), m.poses, C.byref(m.cam), C.byref(m.opts), C.c_int(u), C.c_int(v),
                              C.c_int64(cap), oi.ctypes.data_as(C.c_void_p), vi.ctypes.data_as(C.c_void_p),
                              w.ctypes.data_as(C.c_void_p))
    if n < 0:
        raise RuntimeError("orc_pixel_weights failed")
    n = min(n, cap)
    return oi[:n], vi[:n], w[:n]


def sh_basis(deg, x, y, z):
    lib = _load()
    Y = np.zeros(16)
    lib.orc_sh_basis(C.c_int(deg), C.c_double(x), C.c_double(y), C.c_double(z), Y.ctypes.data_as(C.c_void_p))
    return Y[: (deg + 1) ** 2]
