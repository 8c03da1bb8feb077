"""GB300-native compositional sparse-voxel rasterizer (DrivingVoxels hot path).

A thin Python layer over the C ABI in ``include/dv.h`` (``libdv.so``, built
in-tree from ``csrc/`` for sm_103a).  Everything that renders or
differentiates runs inside that library's CUDA kernels; this module only
marshals torch device tensors into the ABI structs and passes the current
CUDA stream.  There is no fallback: if the library cannot be loaded, every
entry point raises.

Names follow the ABI: :func:`dv_render`, :func:`dv_render_backward`,
:func:`dv_state_free`, plus :class:`RenderFn` (a ``torch.autograd.Function``
whose backward replays the compositing through ``dv_render_backward``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_INC = os.path.join(_ROOT, "include")
LIB_PATH = os.path.join(_HERE, "libdv.so")
SOURCES = ["dv_api.cu", "dv_scan_sort.cu", "dv_project.cu", "dv_composite.cu", "dv_serve.cu", "dv_sky.cu", "dv_features.cu",
           "dv_init.cu", "dv_measure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

DV_OK, DV_ERR_INVALID_ARG, DV_ERR_INVALID_POSE, DV_ERR_CAPACITY, DV_ERR_CUDA, DV_ERR_TIMEOUT, DV_ERR_NOMEM = range(7)
DV_ROLE_BG, DV_ROLE_ACTOR = 0, 1
DV_ACT_EXPLIN, DV_ACT_IDENTITY = 0, 1
DV_MAX_OCTREES = 128
KERNELS = ("project", "sort_vox", "records", "sort_pairs", "ranges", "composite_fwd", "composite_bwd", "sh_bwd")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a (in parallel) and link libdv.so in-tree."""
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, "dv_internal.cuh"), os.path.join(_INC, "dv.h")]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB_PATH
    bdir = os.path.join(_HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + _INC, "-I" + _CSRC]

    def one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ---------------------------------------------------------------------------
# ABI structs
# ---------------------------------------------------------------------------

class dv_octree(C.Structure):
    _fields_ = [("n_vox", C.c_int64), ("sh_degree", C.c_int32), ("role", C.c_int32), ("max_level", C.c_int32),
                ("reserved", C.c_int32), ("center", C.c_double * 3), ("root_size", C.c_double),
                ("clip_half", C.c_float * 3), ("key", C.c_void_p), ("dens", C.c_void_p), ("sh", C.c_void_p)]


class dv_pose(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3)]


class dv_camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("cam_to_world", dv_pose), ("near_", C.c_float), ("far_", C.c_float)]


class dv_view(C.Structure):
    _fields_ = [("camera", dv_camera), ("poses", C.c_void_p)]


class dv_opts(C.Structure):
    _fields_ = [("K", C.c_int32), ("eps_stop", C.c_float), ("activation", C.c_int32), ("reserved", C.c_int32)]


class dv_serve_config(C.Structure):
    _fields_ = [("max_views", C.c_int32), ("n_workers", C.c_int32), ("max_batch_pixels", C.c_int64),
                ("max_inflight_pixels", C.c_int64), ("opts", dv_opts), ("max_inflight_bytes", C.c_int64)]


_lib = None


def load(path: str | None = None):
    """Load libdv.so (building it first if it is missing or stale).  Raises if that fails:
    there is no CPU or eager fallback for any entry point."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if path is None:
        build()
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA extension {p} is missing; run build()")
    lib = C.CDLL(p)
    lib.dv_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32]
    lib.dv_create.restype = C.c_int
    lib.dv_destroy.argtypes = [C.c_void_p]
    lib.dv_destroy.restype = None
    lib.dv_last_error.argtypes = [C.c_void_p]
    lib.dv_last_error.restype = C.c_char_p
    lib.dv_profile_enable_stages.argtypes = [C.c_void_p, C.c_uint32]
    lib.dv_profile_enable_stages.restype = C.c_int
    lib.dv_debug_flag_spin_timeout.argtypes = [C.c_void_p]
    lib.dv_debug_flag_spin_timeout.restype = C.c_int
    lib.dv_debug_sort_timeout.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    lib.dv_debug_sort_timeout.restype = C.c_int
    lib.dv_measure_fp32_fma.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
    lib.dv_measure_fp32_fma.restype = C.c_int
    lib.dv_reserve.argtypes = [C.c_void_p, C.c_int64]
    lib.dv_reserve.restype = C.c_int
    lib.dv_workspace_need.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    lib.dv_workspace_need.restype = C.c_int
    lib.dv_state_check.argtypes = [C.c_void_p, C.c_int32]
    lib.dv_state_check.restype = C.c_int
    lib.dv_asset_init.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int32, C.c_float, C.c_int64, C.c_void_p,
                                  C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_void_p]
    lib.dv_asset_init.restype = C.c_int
    lib.dv_render_backward_static.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]
    lib.dv_render_backward_static.restype = C.c_int
    lib.dv_version.restype = C.c_char_p
    lib.dv_render.argtypes = [C.c_void_p, C.POINTER(dv_octree), C.c_int32, C.POINTER(dv_pose), C.POINTER(dv_camera),
                              C.c_int32, C.POINTER(dv_opts), C.c_void_p, C.c_void_p, C.c_void_p,
                              C.POINTER(C.c_void_p), C.c_void_p]
    lib.dv_render.restype = C.c_int
    lib.dv_render_views.argtypes = [C.c_void_p, C.POINTER(dv_octree), C.c_int32, C.POINTER(dv_view), C.c_int32,
                                    C.POINTER(dv_opts), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p),
                                    C.c_void_p]
    lib.dv_render_views.restype = C.c_int
    lib.dv_render_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]
    lib.dv_render_backward.restype = C.c_int
    lib.dv_render_normals.argtypes = [C.c_void_p, C.POINTER(dv_octree), C.c_int32, C.POINTER(dv_pose),
                                      C.POINTER(dv_camera), C.c_int32, C.POINTER(dv_opts), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p]
    lib.dv_render_normals.restype = C.c_int
    lib.dv_render_backward_normals.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                               C.c_void_p]
    lib.dv_render_backward_normals.restype = C.c_int
    lib.dv_state_weight_offsets.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]
    lib.dv_state_weight_offsets.restype = C.c_int
    lib.dv_state_weights.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dv_state_weights.restype = C.c_int
    lib.dv_features_render.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int32, C.c_void_p, C.c_void_p]
    lib.dv_features_render.restype = C.c_int
    lib.dv_features_fuse.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dv_features_fuse.restype = C.c_int
    lib.dv_shared_corners.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.POINTER(C.c_int64), C.c_void_p]
    lib.dv_shared_corners.restype = C.c_int
    lib.dv_soft_prior.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.c_double, C.c_int32,
                                  C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_void_p, C.c_void_p]
    lib.dv_soft_prior.restype = C.c_int
    lib.dv_subdivide_round.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double),
                                       C.c_double, C.c_void_p, C.c_int64, C.c_float, C.c_void_p,
                                       C.POINTER(C.c_int64), C.c_void_p]
    lib.dv_subdivide_round.restype = C.c_int
    lib.dv_visibility_prune.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double),
                                        C.c_double, C.POINTER(dv_camera), C.c_int32, C.c_double, C.c_void_p,
                                        C.POINTER(C.c_int64), C.c_void_p]
    lib.dv_visibility_prune.restype = C.c_int
    lib.dv_corner_gather.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dv_corner_gather.restype = C.c_int
    lib.dv_corner_scatter.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dv_corner_scatter.restype = C.c_int
    lib.dv_sky_composite.argtypes = [C.c_void_p, C.POINTER(dv_camera), C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dv_sky_composite.restype = C.c_int
    lib.dv_sky_backward.argtypes = [C.c_void_p, C.POINTER(dv_camera), C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dv_sky_backward.restype = C.c_int
    lib.dv_state_free.argtypes = [C.c_void_p]
    lib.dv_state_free.restype = None
    lib.dv_state_stats.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]
    lib.dv_state_stats.restype = C.c_int
    lib.dv_state_work.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                  C.POINTER(C.c_uint64)]
    lib.dv_state_work.restype = C.c_int
    lib.dv_launch_count.argtypes = [C.c_int32]
    lib.dv_launch_count.restype = C.c_longlong
    lib.dv_serve_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(dv_octree), C.c_int32,
                                    C.POINTER(dv_serve_config)]
    lib.dv_serve_create.restype = C.c_int
    lib.dv_serve_submit.argtypes = [C.c_void_p, C.POINTER(dv_camera), C.POINTER(dv_pose), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_int64)]
    lib.dv_serve_submit.restype = C.c_int
    lib.dv_serve_poll.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.dv_serve_poll.restype = C.c_int
    lib.dv_serve_wait.argtypes = [C.c_void_p, C.c_int64, C.c_double, C.POINTER(C.c_double)]
    lib.dv_serve_wait.restype = C.c_int
    lib.dv_serve_release.argtypes = [C.c_void_p, C.c_int64]
    lib.dv_serve_release.restype = C.c_int
    lib.dv_serve_stats.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.dv_serve_stats.restype = C.c_int
    lib.dv_serve_memory.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)]
    lib.dv_serve_memory.restype = C.c_int
    lib.dv_serve_pause.argtypes = [C.c_void_p, C.c_int32]
    lib.dv_serve_pause.restype = C.c_int
    lib.dv_serve_last_error.argtypes = [C.c_void_p]
    lib.dv_serve_last_error.restype = C.c_char_p
    lib.dv_serve_destroy.argtypes = [C.c_void_p]
    lib.dv_serve_destroy.restype = None
    lib.dv_profile_enable.argtypes = [C.c_void_p, C.c_int32]
    lib.dv_profile_enable.restype = C.c_int
    lib.dv_profile_read.argtypes = [C.c_void_p, C.POINTER(C.c_char_p), C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64)]
    lib.dv_profile_read.restype = C.c_int
    _lib = lib
    return lib


class DVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"dv status {status}: {msg}")
        self.status = status


# ---------------------------------------------------------------------------
# context / scene marshalling
# ---------------------------------------------------------------------------

class Context:
    """Owns a dv_ctx (one per device and host thread)."""

    def __init__(self, device: int = 0):
        lib = load()
        h = C.c_void_p()
        st = lib.dv_create(C.byref(h), int(device))
        if st != DV_OK:
            raise DVError(st, "dv_create failed")
        self.handle = h
        self.device = device

    def check(self, st):
        if st != DV_OK:
            raise DVError(st, load().dv_last_error(self.handle).decode())

    def debug_flag_spin_timeout(self):
        """Test hook: marks this device's wait-error word, so the next render reports DV_ERR_TIMEOUT."""
        self.check(load().dv_debug_flag_spin_timeout(self.handle))

    def debug_sort_timeout(self, spin_limit=1000):
        """Test hook: one sort tile whose predecessor never publishes; returns (call flag, device flag)
        as the kernel left them after its bounded waits ran out."""
        a, b = C.c_uint32(), C.c_uint32()
        self.check(load().dv_debug_sort_timeout(self.handle, int(spin_limit), C.byref(a), C.byref(b)))
        return a.value, b.value

    def reserve(self, nbytes: int):
        """Limit each render call's workspace to ``nbytes`` and grow the pool to it (0: no limit)."""
        self.check(load().dv_reserve(self.handle, int(nbytes)))

    def workspace_need(self) -> int:
        """Bytes the last render call needed (or the part known when it failed with DV_ERR_CAPACITY)."""
        n = C.c_int64()
        self.check(load().dv_workspace_need(self.handle, C.byref(n)))
        return n.value

    def close(self):
        if self.handle:
            load().dv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, on: bool, stages=None):
        """Per-stage event timing on (all stages, or only the named ones) or off."""
        if stages is None or not on:
            self.check(load().dv_profile_enable(self.handle, 1 if on else 0))
        else:
            mask = 0
            for name in stages:
                mask |= 1 << KERNELS.index(name)
            self.check(load().dv_profile_enable_stages(self.handle, mask))

    def profile_read(self, names=KERNELS):
        n = len(names)
        arr = (C.c_char_p * n)(*[s.encode() for s in names])
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        self.check(load().dv_profile_read(self.handle, arr, n, ms, cnt))
        return {names[i]: (ms[i], cnt[i]) for i in range(n)}


_ctx_cache = {}


def default_context(device: int | None = None) -> Context:
    import torch
    d = torch.cuda.current_device() if device is None else device
    if d not in _ctx_cache:
        _ctx_cache[d] = Context(d)
    return _ctx_cache[d]


class DeviceOctree:
    """Device-resident octree tensors (torch) plus the metadata of dv_octree."""

    def __init__(self, key, dens, sh, sh_degree, center, root_size, role, clip_half=(0.0, 0.0, 0.0), max_level=None):
        self.key, self.dens, self.sh = key, dens, sh
        self.sh_degree, self.center, self.root_size = int(sh_degree), tuple(center), float(root_size)
        self.role, self.clip_half = int(role), tuple(clip_half)
        if max_level is None:
            max_level = 16
        self.max_level = int(max_level)

    @property
    def n(self):
        return int(self.key.shape[0])

    @staticmethod
    def from_host(oc, device="cuda"):
        import numpy as np
        import torch
        key = torch.from_numpy(np.ascontiguousarray(oc.key).view(np.int64)).to(device)
        dens = torch.from_numpy(np.ascontiguousarray(oc.dens, np.float32)).to(device)
        sh = torch.from_numpy(np.ascontiguousarray(oc.sh, np.float32)).to(device)
        lv = (np.asarray(oc.key, np.uint64) >> np.uint64(57)) & np.uint64(31)
        ml = int(lv.max()) if lv.size else 0
        return DeviceOctree(key, dens, sh, oc.sh_degree, oc.center, oc.root_size, oc.role, oc.clip_half, ml)

    def struct(self, dens=None, sh=None) -> dv_octree:
        d = self.dens if dens is None else dens
        s = self.sh if sh is None else sh
        # the struct of the octree's own tensors is kept (with the tensors, so their ids stay theirs)
        own = dens is None and sh is None
        if own:
            c = getattr(self, "_struct", None)
            if c is not None and c[0] is self.key and c[1] is d and c[2] is s:
                return c[3]
        o = dv_octree()
        for t in (self.key, d, s):
            if t.numel() and (not t.is_cuda or not t.is_contiguous()):
                raise ValueError("octree tensors must be contiguous CUDA tensors")
        o.n_vox = self.n
        o.sh_degree = self.sh_degree
        o.role = self.role
        o.max_level = self.max_level
        for k in range(3):
            o.center[k] = float(self.center[k])
            o.clip_half[k] = float(self.clip_half[k])
        o.root_size = self.root_size
        o.key = self.key.data_ptr() if self.n else None
        o.dens = d.data_ptr() if self.n else None
        o.sh = s.data_ptr() if self.n else None
        if own:
            self._struct = (self.key, d, s, o)
        return o


def make_pose(p) -> dv_pose:
    import numpy as np
    buf = np.empty(12, np.float32)
    buf[:9] = np.asarray(p.R, np.float32).reshape(9)
    buf[9:] = np.asarray(p.t, np.float32).reshape(3)
    return dv_pose.from_buffer_copy(buf)


def make_camera(cam) -> dv_camera:
    c = dv_camera()
    c.W, c.H = int(cam.W), int(cam.H)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.cam_to_world = make_pose(cam.pose)
    c.near_, c.far_ = float(cam.near), float(cam.far)
    return c


def make_opts(K=1, eps_stop=1e-4, activation=DV_ACT_EXPLIN) -> dv_opts:
    o = dv_opts()
    o.K, o.eps_stop, o.activation, o.reserved = int(K), float(eps_stop), int(activation), 0
    return o


def _stream_ptr(stream=None):
    import torch
    if stream is None:
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)  # the current stream's handle, cheaply
        if raw is not None:
            return C.c_void_p(raw(torch.cuda.current_device()))
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------
# ABI-named entry points
# ---------------------------------------------------------------------------

class State:
    """Owning wrapper of a dv_state*; freed stream-ordered on its render stream."""

    def __init__(self, ctx: Context, handle, n_cam: int, keep):
        self.ctx, self.handle, self.n_cam, self.keep = ctx, handle, n_cam, keep

    def stats(self, view=-1):
        """Sizes of view ``view`` (-1: the whole call)."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self.ctx.check(load().dv_state_stats(self.handle, view, C.byref(a), C.byref(b), C.byref(c)))
        return {"n_visible": a.value, "n_pairs": b.value, "n_tiles": c.value}

    def check(self, wait=True):
        """Raises DVError(DV_ERR_TIMEOUT) if a sort of this state's render ran out of its bounded wait;
        ``wait`` first synchronises the render's stream (else an unfinished render passes)."""
        self.ctx.check(load().dv_state_check(self.handle, 1 if wait else 0))

    def work(self, view=-1):
        a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
        self.ctx.check(load().dv_state_work(self.handle, view, C.byref(a), C.byref(b), C.byref(c)))
        return {"tests": a.value, "box_tests": b.value, "segments": c.value}

    def free(self):
        if self.handle:
            load().dv_state_free(self.handle)
            self.handle = None
            self.keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dv_render(octrees, poses, cams, opts=None, *, ctx: Context | None = None, save_state=False, out=None,
              dens=None, sh=None, stream=None, normals=False):
    """Forward render; returns (rgb [P,3], depth [P], alpha [P], state or None) with P = sum of H*W
    over the cameras (images concatenated in camera order).  With ``normals`` the normal state
    N [P,3] (world frame) is rendered too and returned before the state:
    (rgb, depth, alpha, normal, state)."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = len(octrees)
    oct_arr = (dv_octree * n)(*[o.struct(None if dens is None else dens[i], None if sh is None else sh[i])
                                for i, o in enumerate(octrees)])
    pose_arr = (dv_pose * n)(*[make_pose(p) for p in poses])
    cam_arr = (dv_camera * max(len(cams), 1))(*[make_camera(c) for c in cams])
    opts = opts or make_opts()
    P = sum(int(c.W) * int(c.H) for c in cams)
    dev = torch.device("cuda", ctx.device)
    if out is None:
        # one allocation, viewed as the output images
        buf = torch.empty((P * (8 if normals else 5),), device=dev, dtype=torch.float32)
        rgb = buf[:3 * P].view(P, 3)
        depth = buf[3 * P:4 * P]
        alpha = buf[4 * P:5 * P]
        normal = buf[5 * P:].view(P, 3) if normals else None
    else:
        rgb, depth, alpha = out[:3]
        normal = out[3] if normals else None
    st = C.c_void_p()
    ptr = lambda t: C.c_void_p(t.data_ptr() if P else None)
    if normals:
        status = lib.dv_render_normals(ctx.handle, oct_arr, n, pose_arr, cam_arr, len(cams), C.byref(opts), ptr(rgb),
                                       ptr(depth), ptr(alpha), ptr(normal), C.byref(st) if save_state else None,
                                       _stream_ptr(stream))
    else:
        status = lib.dv_render(ctx.handle, oct_arr, n, pose_arr, cam_arr, len(cams), C.byref(opts), ptr(rgb),
                               ptr(depth), ptr(alpha), C.byref(st) if save_state else None, _stream_ptr(stream))
    ctx.check(status)
    state = State(ctx, st, len(cams), (octrees, dens, sh, rgb, depth, alpha, normal)) if save_state else None
    return (rgb, depth, alpha, normal, state) if normals else (rgb, depth, alpha, state)


def dv_render_views(octrees, views, opts=None, *, ctx: Context | None = None, save_state=False, out=None,
                    dens=None, sh=None, stream=None):
    """Batched render of independent views, each a (camera, per-octree poses) pair; one launch per
    stage for all of them.  Returns (rgb, depth, alpha, state) with the images concatenated in view order."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = len(octrees)
    oct_arr = (dv_octree * n)(*[o.struct(None if dens is None else dens[i], None if sh is None else sh[i])
                                for i, o in enumerate(octrees)])
    pose_arrs = [(dv_pose * n)(*[make_pose(p) for p in poses]) for _, poses in views]
    varr = (dv_view * max(len(views), 1))()
    for i, ((cam, _), pa) in enumerate(zip(views, pose_arrs)):
        varr[i].camera = make_camera(cam)
        varr[i].poses = C.cast(pa, C.c_void_p)
    opts = opts or make_opts()
    P = sum(int(c.W) * int(c.H) for c, _ in views)
    dev = torch.device("cuda", ctx.device)
    if out is None:
        rgb = torch.empty((P, 3), device=dev, dtype=torch.float32)
        depth = torch.empty((P,), device=dev, dtype=torch.float32)
        alpha = torch.empty((P,), device=dev, dtype=torch.float32)
    else:
        rgb, depth, alpha = out
    st = C.c_void_p()
    status = lib.dv_render_views(ctx.handle, oct_arr, n, varr, len(views), C.byref(opts),
                                 C.c_void_p(rgb.data_ptr() if P else None),
                                 C.c_void_p(depth.data_ptr() if P else None),
                                 C.c_void_p(alpha.data_ptr() if P else None), C.byref(st) if save_state else None,
                                 _stream_ptr(stream))
    ctx.check(status)
    state = State(ctx, st, len(views), (octrees, dens, sh, rgb, depth, alpha)) if save_state else None
    return rgb, depth, alpha, state


def dv_render_backward(state: State, d_rgb=None, d_depth=None, d_alpha=None, d_dens=None, d_sh=None, stream=None,
                       d_normal=None):
    """Adds dL/d dens and dL/d sh into the given per-octree tensors (lists; None entries skipped).
    ``d_normal`` [P,3] is dL/dN of a render with normals."""
    lib = load()
    if d_dens is None and d_sh is None:
        raise DVError(DV_ERR_INVALID_ARG, "give d_dens or d_sh (per-octree lists; None entries skip an octree)")
    n = len(d_dens) if d_dens is not None else len(d_sh)
    pd = (C.c_void_p * n)(*[(t.data_ptr() if t is not None and t.numel() else None) for t in (d_dens or [None] * n)])
    ps = (C.c_void_p * n)(*[(t.data_ptr() if t is not None and t.numel() else None) for t in (d_sh or [None] * n)])
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    if d_normal is not None:
        status = lib.dv_render_backward_normals(state.ctx.handle, state.handle, ptr(d_rgb), ptr(d_depth),
                                                ptr(d_alpha), ptr(d_normal), pd, ps, _stream_ptr(stream))
    else:
        status = lib.dv_render_backward(state.ctx.handle, state.handle, ptr(d_rgb), ptr(d_depth), ptr(d_alpha), pd,
                                        ps, _stream_ptr(stream))
    state.ctx.check(status)


def dv_state_free(state: State):
    state.free()


def dv_measure_fp32_fma(device=0, iters=4096, reps=10):
    """(FP32 operations, milliseconds) of the library's FMA-rate kernel on ``device`` (FMA = 2 operations)."""
    f, ms = C.c_double(), C.c_double()
    st = load().dv_measure_fp32_fma(int(device), int(iters), int(reps), C.byref(f), C.byref(ms))
    if st != DV_OK:
        raise DVError(st, "dv_measure_fp32_fma failed")
    return f.value, ms.value


# ---------------------------------------------------------------------------
# cameras split across ranks (the one exchange of a multi-GPU forward + backward)
# ---------------------------------------------------------------------------

def camera_shard(cams, rank: int, world: int):
    """The cameras rank ``rank`` of ``world`` renders: every world-th camera from ``rank`` (the octrees
    are replicated on every rank, so cameras are independent units of the forward)."""
    return list(cams)[rank::world]


def allreduce_gradients(tensors, group=None):
    """Sums per-octree gradient tensors (d_dens, d_sh, ...) over the ranks of ``group`` in place, as one
    collective over a flat buffer: the exchange a forward + backward over cameras split across ranks
    needs, each rank having added the gradients of its own cameras.  CUDA tensors are reduced on the
    device with NCCL; with a CPU backend (gloo) they travel through host memory."""
    import torch
    import torch.distributed as dist
    ts = [t for t in tensors if t is not None and t.numel()]
    if not ts or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return
    flat = torch.cat([t.reshape(-1) for t in ts])
    on_host = dist.get_backend(group) == "gloo" and flat.is_cuda
    buf = flat.cpu() if on_host else flat
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    if on_host:
        flat.copy_(buf)
    off = 0
    for t in ts:
        n = t.numel()
        t.copy_(flat[off:off + n].view_as(t))
        off += n


def dv_launch_count(reset: bool = False) -> int:
    """Kernel launches issued by the library in this process."""
    return int(load().dv_launch_count(1 if reset else 0))


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

def _autograd_fn():
    import torch

    class RenderFn(torch.autograd.Function):
        """Differentiable render w.r.t. every octree's corner densities and SH coefficients.
        forward(meta, *tensors) with tensors = dens_0..dens_{n-1}, sh_0..sh_{n-1}."""

        @staticmethod
        def forward(ctx_, meta, *tensors):
            octrees, poses, cams, opts, normals = meta
            n = len(octrees)
            dens, sh = list(tensors[:n]), list(tensors[n:])
            out = dv_render(octrees, poses, cams, opts, save_state=True, dens=[d.detach() for d in dens],
                            sh=[s.detach() for s in sh], normals=normals)
            ctx_.state = out[-1]
            ctx_.n = n
            ctx_.normals = normals
            ctx_.shapes = [(d.shape, s.shape) for d, s in zip(dens, sh)]
            return out[:-1]

        @staticmethod
        def backward(ctx_, g_rgb, g_depth, g_alpha, g_normal=None):
            import torch as T
            n = ctx_.n
            st = ctx_.state
            dev = next(g.device for g in (g_rgb, g_depth, g_alpha, g_normal) if g is not None)
            d_dens = [T.zeros(s[0], device=dev, dtype=T.float32) for s in ctx_.shapes]
            d_sh = [T.zeros(s[1], device=dev, dtype=T.float32) for s in ctx_.shapes]
            c = lambda t: None if t is None else t.contiguous()
            dv_render_backward(st, c(g_rgb), c(g_depth), c(g_alpha), d_dens, d_sh,
                               d_normal=c(g_normal) if ctx_.normals else None)
            st.free()
            ctx_.state = None
            return (None, *d_dens, *d_sh)

    return RenderFn


_RenderFn = None


def __getattr__(name):
    global _RenderFn
    if name == "RenderFn":
        if _RenderFn is None:
            _RenderFn = _autograd_fn()
        return _RenderFn
    raise AttributeError(name)


def render(octrees, poses, cams, opts=None, dens=None, sh=None, normals=False):
    """Autograd entry: gradients flow to ``dens``/``sh`` (lists of per-octree tensors; defaults
    to the octrees' own tensors).  Returns (rgb, depth, alpha), plus the normal state N with
    ``normals``."""
    global _RenderFn
    if _RenderFn is None:
        _RenderFn = _autograd_fn()
    dens = [o.dens for o in octrees] if dens is None else dens
    sh = [o.sh for o in octrees] if sh is None else sh
    return _RenderFn.apply((octrees, poses, cams, opts or make_opts(), normals), *dens, *sh)


class Weights:
    """Compositing weights of a saved render: pixel p's (voxel, weight) slots are
    [offsets[p], offsets[p+1]) of ``voxel`` (int32 view of uint32 indices) and ``weight``."""

    def __init__(self, offsets, voxel, weight):
        self.offsets, self.voxel, self.weight = offsets, voxel, weight

    @property
    def n_pix(self):
        return self.offsets.numel() - 1


def dv_state_weights(state: State, stream=None, out: Weights | None = None) -> Weights:
    """The weights export of a saved render (two calls through the C ABI: offsets, then slots);
    ``out``, a previous export of the same state, is refilled in place (slots only)."""
    import torch
    lib = load()
    if out is not None:
        state.ctx.check(lib.dv_state_weights(state.ctx.handle, state.handle, C.c_void_p(out.offsets.data_ptr()),
                                             C.c_void_p(out.voxel.data_ptr()), C.c_void_p(out.weight.data_ptr()),
                                             _stream_ptr(stream)))
        return out
    P = _state_pixels(state)
    dev = torch.device("cuda", state.ctx.device)
    offsets = torch.empty(P + 1, dtype=torch.int64, device=dev)
    total = C.c_int64()
    state.ctx.check(lib.dv_state_weight_offsets(state.ctx.handle, state.handle, C.c_void_p(offsets.data_ptr()),
                                                C.byref(total), _stream_ptr(stream)))
    if P == 0:
        offsets.zero_()
    n = int(total.value)
    voxel = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    weight = torch.zeros(max(n, 1), dtype=torch.float32, device=dev)
    state.ctx.check(lib.dv_state_weights(state.ctx.handle, state.handle, C.c_void_p(offsets.data_ptr()),
                                         C.c_void_p(voxel.data_ptr()), C.c_void_p(weight.data_ptr()),
                                         _stream_ptr(stream)))
    return Weights(offsets, voxel[:n], weight[:n])


def _state_pixels(state: State) -> int:
    keep = state.keep
    return int(keep[3].shape[0]) if keep is not None else 0


def dv_features_render(w: Weights, feat, *, ctx: Context | None = None, out=None, stream=None):
    """F [P, C] = sum over each pixel's slots of weight * feat[voxel] (feat [n_voxels, C], device)."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    Cc = int(feat.shape[1])
    out = torch.empty((w.n_pix, Cc), dtype=torch.float32, device=feat.device) if out is None else out
    ctx.check(lib.dv_features_render(ctx.handle, w.n_pix, C.c_void_p(w.offsets.data_ptr()),
                                     C.c_void_p(w.voxel.data_ptr()), C.c_void_p(w.weight.data_ptr()),
                                     C.c_void_p(feat.data_ptr()), Cc, C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def dv_features_fuse(w: Weights, feat2d, accum, wsum=None, *, ctx: Context | None = None, stream=None):
    """Adds weight * feat2d[p] into accum[voxel] and weight into wsum[voxel] for every slot."""
    lib = load()
    ctx = ctx or default_context()
    Cc = int(feat2d.shape[1])
    ctx.check(lib.dv_features_fuse(ctx.handle, w.n_pix, C.c_void_p(w.offsets.data_ptr()),
                                   C.c_void_p(w.voxel.data_ptr()), C.c_void_p(w.weight.data_ptr()),
                                   C.c_void_p(feat2d.data_ptr()), Cc, C.c_void_p(accum.data_ptr()),
                                   C.c_void_p(wsum.data_ptr()) if wsum is not None else None, _stream_ptr(stream)))


def _u64(t):
    """uint64 keys held in an int64 tensor (same bits)."""
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def dv_shared_corners(keys, max_level, *, ctx: Context | None = None, stream=None):
    """(grid [N] int64 tensor of packed points z<<42|y<<21|x, index [n, 8] int32 tensor) for leaf keys
    (int64 tensor of the uint64 key bits)."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = int(keys.numel())
    grid = torch.empty(max(8 * n, 1), dtype=torch.int64, device=keys.device)
    index = torch.empty((max(n, 1), 8), dtype=torch.int32, device=keys.device)
    nc = C.c_int64()
    ctx.check(lib.dv_shared_corners(ctx.handle, _u64(keys), n, int(max_level), C.c_void_p(grid.data_ptr()),
                                    C.c_void_p(index.data_ptr()), C.byref(nc), _stream_ptr(stream)))
    return grid[:nc.value], index[:n]


def dv_soft_prior(grid, center, root_size, max_level, cloud, s_min, v_close=-2.0, v_far=-10.0, *,
                  ctx: Context | None = None, stream=None):
    """Eq. 1 densities [N] for the shared corners ``grid`` from the LiDAR points ``cloud`` [m, 3]."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    dens = torch.empty(max(int(grid.numel()), 1), dtype=torch.float32, device=grid.device)
    c3 = (C.c_double * 3)(*[float(x) for x in center])
    ctx.check(lib.dv_soft_prior(ctx.handle, _u64(grid), int(grid.numel()), c3, float(root_size), int(max_level),
                                C.c_void_p(cloud.data_ptr()) if cloud.numel() else None, int(cloud.shape[0]),
                                float(s_min), float(v_close), float(v_far), C.c_void_p(dens.data_ptr()),
                                _stream_ptr(stream)))
    return dens[:grid.numel()]


def dv_subdivide_round(keys, max_level, center, root_size, cloud, threshold, *, ctx: Context | None = None,
                       stream=None):
    """New leaf keys (int64 tensor of uint64 bits) after one proximity-subdivision round."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = int(keys.numel())
    out = torch.empty(max(8 * n, 1), dtype=torch.int64, device=keys.device)
    n_out = C.c_int64()
    c3 = (C.c_double * 3)(*[float(x) for x in center])
    ctx.check(lib.dv_subdivide_round(ctx.handle, _u64(keys), n, int(max_level), c3, float(root_size),
                                     C.c_void_p(cloud.data_ptr()) if cloud.numel() else None, int(cloud.shape[0]),
                                     float(threshold), C.c_void_p(out.data_ptr()), C.byref(n_out),
                                     _stream_ptr(stream)))
    return out[:n_out.value]


def dv_visibility_prune(keys, max_level, center, root_size, cams, z_min, *, ctx: Context | None = None,
                        stream=None):
    """Kept leaf keys (int64 tensor of uint64 bits) after visibility and height pruning."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = int(keys.numel())
    out = torch.empty(max(n, 1), dtype=torch.int64, device=keys.device)
    n_out = C.c_int64()
    c3 = (C.c_double * 3)(*[float(x) for x in center])
    cam_arr = (dv_camera * max(len(cams), 1))(*[make_camera(c) for c in cams])
    ctx.check(lib.dv_visibility_prune(ctx.handle, _u64(keys), n, int(max_level), c3, float(root_size), cam_arr,
                                      len(cams), float(z_min), C.c_void_p(out.data_ptr()), C.byref(n_out),
                                      _stream_ptr(stream)))
    return out[:n_out.value]


def dv_asset_init(box_dims, level, v_init=-10.0, *, ctx: Context | None = None, stream=None, device=None):
    """Initial octree of an actor (Sec. 3.3, assets): a uniform grid of 8^level leaves in the actor's
    canonical frame whose cubic bound is 1.2 x the largest box dimension, every corner density at
    ``v_init``.  Returns (keys int64 tensor of the uint64 key bits [8^level], dens [8^level, 8],
    root_size); the grid's centre is the local origin."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = 1 << (3 * int(level)) if 0 <= int(level) <= 10 else 0
    dev = torch.device("cuda", ctx.device if device is None else device)
    keys = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    dens = torch.empty((max(n, 1), 8), dtype=torch.float32, device=dev)
    dims = (C.c_float * 3)(*[float(x) for x in box_dims])
    root = C.c_double()
    n_out = C.c_int64()
    ctx.check(lib.dv_asset_init(ctx.handle, dims, int(level), float(v_init), n, C.c_void_p(keys.data_ptr()),
                                C.c_void_p(dens.data_ptr()), C.byref(root), C.byref(n_out), _stream_ptr(stream)))
    return keys[:n_out.value], dens[:n_out.value], root.value


def dv_corner_gather(index, corner, *, ctx: Context | None = None, stream=None):
    import torch
    lib = load()
    ctx = ctx or default_context()
    n = int(index.shape[0])
    dens = torch.empty((n, 8), dtype=torch.float32, device=corner.device)
    ctx.check(lib.dv_corner_gather(ctx.handle, C.c_void_p(index.data_ptr()), n, C.c_void_p(corner.data_ptr()),
                                   C.c_void_p(dens.data_ptr()), _stream_ptr(stream)))
    return dens


def dv_corner_scatter(index, d_dens, d_corner, *, ctx: Context | None = None, stream=None):
    lib = load()
    ctx = ctx or default_context()
    ctx.check(lib.dv_corner_scatter(ctx.handle, C.c_void_p(index.data_ptr()), int(index.shape[0]),
                                    C.c_void_p(d_dens.data_ptr()), C.c_void_p(d_corner.data_ptr()),
                                    _stream_ptr(stream)))


def dv_sky_composite(cams, env, rgb, alpha, *, ctx: Context | None = None, out=None, stream=None):
    """Sky composite of Eq. 2: returns rgb + (1 - alpha) * C_sky(d) ([P,3]) for an equirectangular
    world-frame map ``env`` ([He, We, 3], device)."""
    import torch
    lib = load()
    ctx = ctx or default_context()
    cam_arr = (dv_camera * max(len(cams), 1))(*[make_camera(c) for c in cams])
    He, We = int(env.shape[0]), int(env.shape[1])
    out = torch.empty_like(rgb) if out is None else out
    P = rgb.shape[0]
    p = lambda t: C.c_void_p(t.data_ptr() if P else None)
    ctx.check(lib.dv_sky_composite(ctx.handle, cam_arr, len(cams), C.c_void_p(env.data_ptr()), He, We, p(rgb),
                                   p(alpha), p(out), _stream_ptr(stream)))
    return out


def dv_sky_backward(cams, env, alpha, d_out, d_env=None, d_alpha=None, *, ctx: Context | None = None, stream=None):
    """Adds dL/d env into ``d_env`` and -dL/d out . C_sky into ``d_alpha`` (either may be None)."""
    lib = load()
    ctx = ctx or default_context()
    cam_arr = (dv_camera * max(len(cams), 1))(*[make_camera(c) for c in cams])
    He, We = int(env.shape[0]), int(env.shape[1])
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    ctx.check(lib.dv_sky_backward(ctx.handle, cam_arr, len(cams), ptr(env), He, We, ptr(alpha), ptr(d_out),
                                  ptr(d_env), ptr(d_alpha), _stream_ptr(stream)))


STATIC_MAX_VISIBLE = 1 << 17  # visible voxels per render call, summed over its views


def dv_render_backward_static(state: State, d_rgb=None, d_depth=None, d_alpha=None, d_dens=None, d_sh=None,
                              stream=None):
    """Allocation-free variant of :func:`dv_render_backward` for callers that may not allocate device
    memory while the backward runs (graph capture without allocation nodes, real-time loops, a device
    whose memory belongs to another allocator).  Its scratch is a static device array for at most
    ``STATIC_MAX_VISIBLE`` visible voxels per render call, summed over its views; calls that overlap on
    the GPU race on it, and the first call on a device should precede any stream capture."""
    lib = load()
    fn = lib.dv_render_backward_static
    if d_dens is None and d_sh is None:
        raise DVError(DV_ERR_INVALID_ARG, "give d_dens or d_sh (per-octree lists; None entries skip an octree)")
    n = len(d_dens) if d_dens is not None else len(d_sh)
    pd = (C.c_void_p * n)(*[(t.data_ptr() if t is not None and t.numel() else None) for t in (d_dens or [None] * n)])
    ps = (C.c_void_p * n)(*[(t.data_ptr() if t is not None and t.numel() else None) for t in (d_sh or [None] * n)])
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    status = fn(state.ctx.handle, state.handle, ptr(d_rgb), ptr(d_depth), ptr(d_alpha), pd, ps, _stream_ptr(stream))
    state.ctx.check(status)


class Server:
    """Continuous-batching render server over resident octrees (``dv_serve_*``).

    ``submit`` queues a request (camera, per-octree poses, device output tensors) and returns a
    ticket; ``wait`` blocks at most ``timeout_ms``; results are written into the given tensors."""

    def __init__(self, octrees, max_views=16, n_workers=2, max_batch_pixels=8 * 1920 * 1080,
                 max_inflight_pixels=16 * 1920 * 1080, opts=None, device=None, max_inflight_bytes=0):
        import torch
        lib = load()
        self.octrees = octrees  # keep the device buffers alive
        self.n_oct = len(octrees)
        arr = (dv_octree * self.n_oct)(*[o.struct() for o in octrees])
        cfg = dv_serve_config()
        cfg.max_views, cfg.n_workers = int(max_views), int(n_workers)
        cfg.max_batch_pixels, cfg.max_inflight_pixels = int(max_batch_pixels), int(max_inflight_pixels)
        cfg.opts = opts or make_opts()
        cfg.max_inflight_bytes = int(max_inflight_bytes)
        h = C.c_void_p()
        dev = torch.cuda.current_device() if device is None else device
        st = lib.dv_serve_create(C.byref(h), int(dev), arr, self.n_oct, C.byref(cfg))
        if st != DV_OK:
            raise DVError(st, "dv_serve_create failed")
        self.handle = h
        self.keep = {}

    def _check(self, st):
        if st != DV_OK:
            raise DVError(st, load().dv_serve_last_error(self.handle).decode())

    def submit(self, cam, poses, out):
        rgb, depth, alpha = out
        c = make_camera(cam)
        pa = (dv_pose * self.n_oct)(*[make_pose(p) for p in poses])
        t = C.c_int64()
        self._check(load().dv_serve_submit(self.handle, C.byref(c), pa, C.c_void_p(rgb.data_ptr()),
                                           C.c_void_p(depth.data_ptr()), C.c_void_p(alpha.data_ptr()), C.byref(t)))
        self.keep[t.value] = out
        return t.value

    def poll(self, ticket):
        d = C.c_int32()
        lat = C.c_double()
        self._check(load().dv_serve_poll(self.handle, int(ticket), C.byref(d), C.byref(lat)))
        return (lat.value if d.value else None)

    def wait(self, ticket, timeout_ms=60000.0):
        lat = C.c_double()
        self._check(load().dv_serve_wait(self.handle, int(ticket), float(timeout_ms), C.byref(lat)))
        return lat.value

    def release(self, ticket):
        self._check(load().dv_serve_release(self.handle, int(ticket)))
        self.keep.pop(ticket, None)

    def stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(load().dv_serve_stats(self.handle, C.byref(a), C.byref(b), C.byref(c)))
        return {"batches": a.value, "requests": b.value, "max_batch": c.value}

    def memory(self, reset_peak=False):
        """Device memory charged to the requests in flight, its peak since the start or the last reset, and
        the last request's charge; ``reset_peak`` restarts the peak from now."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(load().dv_serve_memory(self.handle, 1 if reset_peak else 0, C.byref(a), C.byref(b),
                                           C.byref(c)))
        return {"inflight_bytes": a.value, "peak_inflight_bytes": b.value, "last_request_bytes": c.value}

    def pause(self, paused=True):
        """Hold (or resume) admission of queued requests."""
        self._check(load().dv_serve_pause(self.handle, 1 if paused else 0))

    def close(self):
        if self.handle:
            load().dv_serve_destroy(self.handle)
            self.handle = None
            self.keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
