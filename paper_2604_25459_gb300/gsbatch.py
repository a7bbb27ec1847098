"""Thin Python binding of libgsbatch (ctypes).

Argument marshalling only: every step of the render runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams; host inputs may be
numpy arrays.  If the compiled library is missing this module raises -- there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .synth import CAMERA_DTYPE

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgsbatch.so")

GS_OK, GS_ERR_INVALID, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED, GS_ERR_DEVICE = (
    0, -1, -2, -3, -4, -5, -6)
DTYPES = {"f32": 0, "bf16": 1, "f16": 2}
STATUS_NAMES = {0: "GS_OK", -1: "GS_ERR_INVALID", -2: "GS_ERR_OOM", -3: "GS_ERR_CUDA", -4: "GS_ERR_TIMEOUT",
                -5: "GS_ERR_UNSUPPORTED", -6: "GS_ERR_DEVICE"}


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GsGaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean", C.c_void_p), ("quat", C.c_void_p), ("log_scale", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p), ("sh_degree", C.c_int), ("dtype", C.c_int),
                ("on_device", C.c_int)]


class GsStats(C.Structure):
    _fields_ = [("waves", C.c_int64), ("kernel_launches", C.c_int64), ("intersections", C.c_int64),
                ("scratch_bytes", C.c_int64), ("n_gaussians", C.c_int64), ("composited", C.c_int64),
                ("visible", C.c_int64), ("fp64_conics", C.c_int64)]


PHASES = ("link", "project", "count", "scan", "scatter", "composite")


class GsTimings(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("launches", C.c_int64 * 6)]


class GsPlanInfo(C.Structure):
    _fields_ = [("tile_w", C.c_int), ("tile_h", C.c_int), ("chunk", C.c_int), ("waves", C.c_int),
                ("graph", C.c_int), ("tuned_candidates", C.c_int), ("tuned_ms", C.c_double), ("regrows", C.c_int),
                ("key_capacity", C.c_int64), ("scratch_bytes", C.c_int64), ("quad", C.c_int)]


# gs_env in include/gsbatch.h: camera, link range, pose offset, pixel offset (80 bytes)
ENV_DTYPE = np.dtype([("cam", CAMERA_DTYPE), ("link_begin", "<i4"), ("link_end", "<i4"), ("pose_offset", "<i8"),
                      ("pixel_offset", "<i8")])
assert ENV_DTYPE.itemsize == 80
PLAN_AUTOTUNE, PLAN_GRAPH = 1, 2

# gs_lidar in include/gsbatch.h (48 bytes)
LIDAR_DTYPE = np.dtype([("q_ws", "<f4", (4,)), ("t_ws", "<f4", (3,)), ("rows", "<i4"), ("cols", "<i4"),
                        ("elev_min", "<f4"), ("elev_max", "<f4"), ("near_range", "<f4"), ("az_min", "<f4"),
                        ("az_max", "<f4")])
assert LIDAR_DTYPE.itemsize == 56


class GsServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("max_inflight", C.c_int), ("max_batch_envs", C.c_int),
                ("tile_w", C.c_int), ("tile_h", C.c_int)]


class GsRequestResult(C.Structure):
    _fields_ = [("request_id", C.c_int64), ("env_id", C.c_int), ("status", C.c_int), ("arrival_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double)]


class GsServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("cancelled", C.c_int64),
                ("batches", C.c_int64), ("peak_inflight_bytes", C.c_int64), ("max_concurrent", C.c_int32),
                ("max_batch", C.c_int32), ("retried", C.c_int64)]


_lib = None

# name -> (restype, argtypes); the exported C ABI declared in include/gsbatch.h
_SIGS = {
    "gs_scene_create": (C.c_int, [C.POINTER(GsGaussians), C.POINTER(C.c_void_p)]),
    "gs_scene_attach_links": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(GsGaussians)]),
    "gs_render_batch": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "gs_render_batch_host": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "gs_render_batch_noalloc": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "gs_render_batch_v": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "gs_render_batch_obs": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "gs_scene_contribution": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 4),
    "gs_render_lidar": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 5),
    "gs_render_rays": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int] + [C.c_void_p] * 4),
    "gs_scene_prune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.POINTER(C.c_void_p), C.c_void_p,
                                 C.c_int64]),
    "gs_render_batch_obs_host": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "gs_plan_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "gs_plan_launch": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5),
    "gs_plan_get_info": (C.c_int, [C.c_void_p, C.POINTER(GsPlanInfo)]),
    "gs_plan_destroy": (None, [C.c_void_p]),
    "gs_scene_set_tile": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "gs_scene_set_budget": (C.c_int, [C.c_void_p, C.c_int64]),
    "gs_scene_set_wave": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_scene_set_debug": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_scene_sync_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gs_scene_get_stats": (C.c_int, [C.c_void_p, C.POINTER(GsStats)]),
    "gs_scene_set_counters": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_scene_set_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "gs_scene_get_timings": (C.c_int, [C.c_void_p, C.POINTER(GsTimings), C.c_int]),
    "gs_debug_copy_records": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 10),
    "gs_debug_copy_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]),
    "gs_scene_get_order": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "gs_scene_destroy": (None, [C.c_void_p]),
    "gs_server_create": (C.c_int, [C.POINTER(GsServerConfig), C.POINTER(C.c_void_p)]),
    "gs_server_add_scene": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "gs_server_add_env": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "gs_server_start": (C.c_int, [C.c_void_p]),
    "gs_server_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.POINTER(C.c_int64)]),
    "gs_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "gs_server_poll": (C.c_int, [C.c_void_p, C.POINTER(GsRequestResult), C.c_int, C.POINTER(C.c_int)]),
    "gs_server_drain": (C.c_int, [C.c_void_p, C.c_double]),
    "gs_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(GsServerStats)]),
    "gs_server_env_output": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "gs_server_now": (C.c_double, [C.c_void_p]),
    "gs_server_destroy": (None, [C.c_void_p]),
    "gs_measure_alu_peak": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "gs_last_error": (C.c_char_p, []),
    "gs_version": (C.c_char_p, []),
}


def lib():
    """Load libgsbatch.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2604_25459_gb300.build.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != GS_OK:
        raise GsError(status, lib().gs_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(C.c_void_p)
    raise TypeError(type(x))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _view(mean, quat, log_scale, opacity, sh, sh_degree: int, dtype: str):
    arrs = [mean, quat, log_scale, opacity, sh]
    on_dev = any(_is_torch(a) and a.is_cuda for a in arrs)
    n = int(mean.shape[0])
    v = GsGaussians(n, _ptr(mean), _ptr(quat), _ptr(log_scale), _ptr(opacity), _ptr(sh), sh_degree, DTYPES[dtype],
                    1 if on_dev else 0)
    return v, arrs


def _host_f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Scene:
    """A device-resident scene: shared background + link-attached Gaussians.

    ``background``/``links`` expose mean, quat, log_scale, opacity, sh (numpy
    or torch); with ``stored`` (dict of log_scale/opacity/sh arrays) the
    precision form passes those bf16/f16 arrays instead."""

    def __init__(self, background, dtype: str = "f32", sh_degree: int = 3, stored=None):
        self._h = C.c_void_p()
        self.dtype = dtype
        self.sh_degree = sh_degree
        v, keep = self._make_view(background, dtype, sh_degree, stored)
        _check(lib().gs_scene_create(C.byref(v), C.byref(self._h)))
        self.n_background = int(v.n)
        self.n_links = 0
        self._alive = True

    @classmethod
    def _adopt(cls, handle, dtype: str, sh_degree: int, n_background: int, n_links: int) -> "Scene":
        """Wrap a scene handle the library created (gs_scene_prune)."""
        self = cls.__new__(cls)
        self._h = handle
        self.dtype = dtype
        self.sh_degree = sh_degree
        self.n_background = n_background
        self.n_links = n_links
        self._alive = True
        return self

    def prune(self, scores, keep_bg: float = 0.3, keep_links: float = 0.1):
        """Pruning as a scene transform (gs_scene_prune, selection and the new
        scene on the device): scores CUDA float32 [n Gaussians], the caller's
        order.  Returns (the pruned Scene, kept int64 numpy: each kept
        Gaussian's index in this scene, new order)."""
        import torch

        if not (torch.is_tensor(scores) and scores.is_cuda and scores.dtype == torch.float32):
            scores = torch.as_tensor(np.ascontiguousarray(scores, dtype=np.float32)).cuda()
        n = int(scores.numel())
        kept = np.zeros(max(n, 1), np.int64)
        h = C.c_void_p()
        _check(lib().gs_scene_prune(self._h, _ptr(scores), float(keep_bg), float(keep_links), C.byref(h),
                                    _ptr(kept), n))
        sub = Scene._adopt(h, self.dtype, self.sh_degree, 0, self.n_links)
        n_kept = sub.stats()["n_gaussians"]
        kept = kept[:n_kept]
        sub.n_background = int((kept < self.n_background).sum())
        return sub, kept

    @staticmethod
    def _make_view(g, dtype, sh_degree, stored):
        if g is None:
            z = np.zeros((0, 3), np.float32)
            return GsGaussians(0, None, None, None, None, None, sh_degree, DTYPES[dtype], 0), [z]
        mean, quat = g.mean, g.quat
        if stored is not None:
            ls, op, sh = stored["log_scale"], stored["opacity"], stored["sh"]
        else:
            ls, op, sh = g.log_scale, g.opacity, g.sh
        if not _is_torch(mean):
            mean, quat = _host_f32(mean), _host_f32(quat)
            if dtype == "f32":
                ls, op, sh = _host_f32(ls), _host_f32(op), _host_f32(sh)
            else:
                ls, op, sh = (np.ascontiguousarray(a) for a in (ls, op, sh))
            nk = (sh_degree + 1) ** 2
            if sh.ndim == 3 and sh.shape[1] != nk:
                sh = np.ascontiguousarray(sh[:, :nk, :])
        return _view(mean, quat, ls, op, sh, sh_degree, dtype)

    def attach_links(self, link_offsets, links, stored=None):
        offs = np.ascontiguousarray(link_offsets, dtype=np.int64)
        v, keep = self._make_view(links, self.dtype, self.sh_degree, stored)
        _check(lib().gs_scene_attach_links(self._h, len(offs) - 1, _ptr(offs), C.byref(v)))
        self.n_links = len(offs) - 1

    def set_tile(self, tw: int, th: int):
        _check(lib().gs_scene_set_tile(self._h, tw, th))

    def set_budget(self, nbytes: int):
        _check(lib().gs_scene_set_budget(self._h, int(nbytes)))

    def set_wave(self, max_envs: int):
        _check(lib().gs_scene_set_wave(self._h, int(max_envs)))

    def set_debug(self, on: bool):
        _check(lib().gs_scene_set_debug(self._h, 1 if on else 0))

    def stats(self) -> dict:
        s = GsStats()
        _check(lib().gs_scene_get_stats(self._h, C.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in GsStats._fields_}

    def set_counters(self, on: bool):
        _check(lib().gs_scene_set_counters(self._h, 1 if on else 0))

    def set_profile(self, on: bool):
        _check(lib().gs_scene_set_profile(self._h, 1 if on else 0))

    def timings(self, reset: bool = False) -> dict:
        """Per-phase device milliseconds and kernel launches (profiling on)."""
        t = GsTimings()
        _check(lib().gs_scene_get_timings(self._h, C.byref(t), 1 if reset else 0))
        return {p: (float(t.ms[i]), int(t.launches[i])) for i, p in enumerate(PHASES)}

    def sync_status(self, stream=None):
        _check(lib().gs_scene_sync_status(self._h, _stream_handle(stream)))

    def render(self, link_poses, cams: np.ndarray, rgb=None, depth=None, alpha=None, want_alpha: bool = True,
               stream=None):
        """Device render.  link_poses: CUDA float32 [E][L][7] (or None when the
        scene has no links); cams: numpy CAMERA_DTYPE [E].  Returns (rgb, depth,
        alpha) CUDA tensors [E,H,W,3], [E,H,W], [E,H,W] (alpha None if not wanted)."""
        import torch

        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        E = int(cams.shape[0])
        H, W = (int(cams["height"][0]), int(cams["width"][0])) if E else (0, 0)
        dev = torch.device("cuda", torch.cuda.current_device())
        if rgb is None:
            rgb = torch.empty((E, H, W, 3), dtype=torch.float32, device=dev)
        if depth is None:
            depth = torch.empty((E, H, W), dtype=torch.float32, device=dev)
        if alpha is None and want_alpha:
            alpha = torch.empty((E, H, W), dtype=torch.float32, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(lib().gs_render_batch(self._h, E, _ptr(link_poses), _ptr(cams), _ptr(rgb), _ptr(depth), _ptr(alpha),
                                     _stream_handle(stream)))
        return rgb, depth, alpha

    def render_noalloc(self, link_poses, cams: np.ndarray, rgb, depth, alpha=None, stream=None):
        """gs_render_batch_noalloc: same render into caller-provided CUDA
        tensors, with the library's working memory in its fixed device array
        (no allocation by the library)."""
        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        _check(lib().gs_render_batch_noalloc(self._h, int(cams.shape[0]), _ptr(link_poses), _ptr(cams), _ptr(rgb),
                                             _ptr(depth), _ptr(alpha), _stream_handle(stream)))
        return rgb, depth, alpha

    def render_host(self, link_poses: np.ndarray, cams: np.ndarray, rgb: np.ndarray, depth: np.ndarray,
                    alpha=None, stream=None):
        """Host-buffer render (copies inside the call); returns when done."""
        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        E = int(cams.shape[0])
        _check(lib().gs_render_batch_host(self._h, E, _ptr(link_poses), _ptr(cams), _ptr(rgb), _ptr(depth),
                                          _ptr(alpha), _stream_handle(stream)))
        return rgb, depth, alpha

    def render_obs(self, link_poses, cams: np.ndarray, appearance=None, rgb8=None, depth16=None,
                   want_depth: bool = True, stream=None):
        """Observation form on the device (gs_render_batch_obs): appearance is a
        CUDA float32 [E][3] (exposure, contrast, brightness) or None; returns
        (rgb8 uint8 [E,H,W,3], depth16 float16 [E,H,W] or None)."""
        import torch

        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        E = int(cams.shape[0])
        H, W = (int(cams["height"][0]), int(cams["width"][0])) if E else (0, 0)
        dev = torch.device("cuda", torch.cuda.current_device())
        if rgb8 is None:
            rgb8 = torch.empty((E, H, W, 3), dtype=torch.uint8, device=dev)
        if depth16 is None and want_depth:
            depth16 = torch.empty((E, H, W), dtype=torch.float16, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(lib().gs_render_batch_obs(self._h, E, _ptr(link_poses), _ptr(cams), _ptr(appearance), _ptr(rgb8),
                                         _ptr(depth16), _stream_handle(stream)))
        return rgb8, depth16

    def render_obs_host(self, link_poses: np.ndarray, cams: np.ndarray, appearance, rgb8: np.ndarray, depth16=None,
                        stream=None):
        """Observation form with host buffers (gs_render_batch_obs_host):
        appearance numpy float32 [E][3] or None, rgb8 uint8 [E,H,W,3], depth16
        float16 [E,H,W] or None.  Returns when the images are on the host."""
        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        E = int(cams.shape[0])
        if appearance is not None:
            appearance = np.ascontiguousarray(appearance, dtype=np.float32)
        _check(lib().gs_render_batch_obs_host(self._h, E, _ptr(link_poses), _ptr(cams), _ptr(appearance), _ptr(rgb8),
                                              _ptr(depth16), _stream_handle(stream)))
        return rgb8, depth16

    def render_lidar(self, link_poses, sensors: np.ndarray, rng=None, hit=None, want_hit: bool = True, stream=None):
        """Batch-LiDAR scan (gs_render_lidar): sensors numpy LIDAR_DTYPE [E];
        returns (range [E, rows, cols], hit [E, rows, cols] or None) CUDA tensors."""
        import torch

        sensors = np.ascontiguousarray(sensors, dtype=LIDAR_DTYPE)
        E = int(sensors.shape[0])
        R, Cc = (int(sensors["rows"][0]), int(sensors["cols"][0])) if E else (0, 0)
        if rng is None:
            rng = torch.empty((E, R, Cc), dtype=torch.float32, device="cuda")
        if hit is None and want_hit:
            hit = torch.empty((E, R, Cc), dtype=torch.float32, device="cuda")
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(lib().gs_render_lidar(self._h, E, _ptr(link_poses), _ptr(sensors), _ptr(rng), _ptr(hit),
                                     _stream_handle(stream)))
        return rng, hit

    def render_rays(self, link_poses, sensors: np.ndarray, ray_dirs, rng=None, hit=None, want_hit: bool = True,
                    stream=None):
        """Batch-LiDAR along arbitrary rays (gs_render_rays): sensors numpy
        LIDAR_DTYPE [E] (pose, near range, binning grid); ray_dirs CUDA float32
        [E, R, 3] in the sensor frame; returns (range [E, R], hit [E, R] or
        None) CUDA tensors."""
        import torch

        sensors = np.ascontiguousarray(sensors, dtype=LIDAR_DTYPE)
        E, R = int(ray_dirs.shape[0]), int(ray_dirs.shape[1])
        if E != int(sensors.shape[0]) or tuple(ray_dirs.shape[2:]) != (3,):
            raise ValueError("ray_dirs must be [n_envs, n_rays, 3] with one sensor per env")
        if rng is None:
            rng = torch.empty((E, R), dtype=torch.float32, device="cuda")
        if hit is None and want_hit:
            hit = torch.empty((E, R), dtype=torch.float32, device="cuda")
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(lib().gs_render_rays(self._h, E, _ptr(link_poses), _ptr(sensors), R, _ptr(ray_dirs), _ptr(rng),
                                    _ptr(hit), _stream_handle(stream)))
        return rng, hit

    def contribution(self, link_poses, cams: np.ndarray, scores=None, stream=None):
        """Add each Gaussian's summed blending weight over the envs' pixels to
        scores (CUDA float32 [n_gaussians], zeros if None); returns scores."""
        import torch

        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        if scores is None:
            st = self.stats()
            scores = torch.zeros(st["n_gaussians"], dtype=torch.float32, device="cuda")
        if stream is None:
            stream = torch.cuda.current_stream()
        _check(lib().gs_scene_contribution(self._h, int(cams.shape[0]), _ptr(link_poses), _ptr(cams), _ptr(scores),
                                           _stream_handle(stream)))
        return scores

    def render_v(self, envs: np.ndarray, link_poses, rgb, depth, alpha=None, stream=None):
        """Uneven batch (gs_render_batch_v): envs is a numpy ENV_DTYPE array (host);
        outputs are flat CUDA tensors addressed by each env's pixel_offset."""
        envs = np.ascontiguousarray(envs, dtype=ENV_DTYPE)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        _check(lib().gs_render_batch_v(self._h, int(envs.shape[0]), _ptr(envs), _ptr(link_poses), _ptr(rgb),
                                       _ptr(depth), _ptr(alpha), _stream_handle(stream)))
        return rgb, depth, alpha

    def plan(self, envs: np.ndarray, autotune: bool = True, graph: bool = True) -> "Plan":
        return Plan(self, envs, (PLAN_AUTOTUNE if autotune else 0) | (PLAN_GRAPH if graph else 0))

    def storage_order(self) -> np.ndarray:
        """order[k] = the caller's index of the background Gaussian stored at
        position k (the scene's Morton order of the means)."""
        order = np.zeros(max(self.n_background, 1), np.int64)
        _check(lib().gs_scene_get_order(self._h, _ptr(order), len(order)))
        return order[:self.n_background]

    def debug_records(self, env: int, n: int) -> dict:
        out = dict(visible=np.zeros(n, np.uint8), u=np.zeros(n, np.float32), v=np.zeros(n, np.float32),
                   hx=np.zeros(n, np.float32), hy=np.zeros(n, np.float32), z=np.zeros(n, np.float32),
                   opacity=np.zeros(n, np.float32), conic=np.zeros((n, 3), np.float32),
                   rgb=np.zeros((n, 3), np.float32), range=np.zeros((n, 4), np.int32))
        _check(lib().gs_debug_copy_records(self._h, env, *[_ptr(out[k]) for k in (
            "visible", "u", "v", "hx", "hy", "z", "opacity", "conic", "rgb", "range")]))
        return out

    def debug_tiles(self, env: int, n_tiles: int, with_lists: bool = True):
        counts = np.zeros(n_tiles, np.uint32)
        _check(lib().gs_debug_copy_tiles(self._h, env, _ptr(counts), n_tiles, None, 0))
        if not with_lists:
            return counts, None
        total = int(counts.astype(np.int64).sum())
        lists = np.zeros(max(total, 1), np.uint32)
        _check(lib().gs_debug_copy_tiles(self._h, env, _ptr(counts), n_tiles, _ptr(lists), total))
        return counts, lists[:total]

    def close(self):
        if getattr(self, "_alive", False):
            lib().gs_scene_destroy(self._h)
            self._alive = False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Plan:
    """A fixed uneven batch rendered repeatedly (gs_plan_*): autotuned on the
    first launch, then replayed from a captured CUDA graph."""

    def __init__(self, scene: Scene, envs: np.ndarray, flags: int):
        self.scene = scene
        self.envs = np.ascontiguousarray(envs, dtype=ENV_DTYPE)
        self._h = C.c_void_p()
        _check(lib().gs_plan_create(scene._h, int(self.envs.shape[0]), _ptr(self.envs), flags, C.byref(self._h)))
        self._alive = True

    def launch(self, link_poses, rgb, depth, alpha=None, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        _check(lib().gs_plan_launch(self._h, _ptr(link_poses), _ptr(rgb), _ptr(depth), _ptr(alpha),
                                    _stream_handle(stream)))

    def info(self) -> dict:
        i = GsPlanInfo()
        _check(lib().gs_plan_get_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in GsPlanInfo._fields_}

    def close(self):
        if getattr(self, "_alive", False):
            lib().gs_plan_destroy(self._h)
            self._alive = False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevView:
    """A borrowed device array exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3, "strides": None}


class Server:
    """The request loop (gs_server_*): resident scenes and env instances,
    requests batched continuously on a pool of CUDA streams under an HBM
    budget."""

    def __init__(self, budget_bytes: int, max_inflight: int = 4, max_batch_envs: int = 512, tile=(16, 16)):
        cfg = GsServerConfig(int(budget_bytes), int(max_inflight), int(max_batch_envs), int(tile[0]), int(tile[1]))
        self._h = C.c_void_p()
        _check(lib().gs_server_create(C.byref(cfg), C.byref(self._h)))
        self._alive = True
        self._scenes = []
        self._env_shape = []
        self._env_links = []

    def add_scene(self, scene: Scene) -> int:
        sid = C.c_int()
        _check(lib().gs_server_add_scene(self._h, scene._h, C.byref(sid)))
        self._scenes.append(scene)  # the scene must outlive the server
        return sid.value

    def add_env(self, scene_id: int, cam, link_begin: int = 0, link_end: int = 0) -> int:
        cam = np.ascontiguousarray(np.asarray(cam, dtype=CAMERA_DTYPE).reshape(1))
        eid = C.c_int()
        _check(lib().gs_server_add_env(self._h, int(scene_id), _ptr(cam), int(link_begin), int(link_end),
                                       C.byref(eid)))
        self._env_shape.append((int(cam["height"][0]), int(cam["width"][0])))
        self._env_links.append(int(link_end) - int(link_begin))
        return eid.value

    def start(self):
        _check(lib().gs_server_start(self._h))

    def submit(self, env_id: int, link_poses=None, arrival_s: float = -1.0) -> int:
        p = None
        nl = self._env_links[env_id] if 0 <= env_id < len(self._env_links) else 0  # the library checks env_id
        if nl > 0:
            link_poses = np.ascontiguousarray(link_poses, dtype=np.float32)
            if link_poses.size != nl * 7:
                raise ValueError("link_poses must hold 7 floats per link of the env")
            p = _ptr(link_poses)
        rid = C.c_int64()
        _check(lib().gs_server_submit(self._h, int(env_id), p, float(arrival_s), C.byref(rid)))
        return rid.value

    def cancel(self, request_id: int):
        _check(lib().gs_server_cancel(self._h, int(request_id)))

    def poll(self, max_results: int = 4096) -> list:
        buf = (GsRequestResult * max_results)()
        n = C.c_int()
        _check(lib().gs_server_poll(self._h, buf, max_results, C.byref(n)))
        return [{k: getattr(buf[i], k) for k, _ in GsRequestResult._fields_} for i in range(n.value)]

    def drain(self, timeout_s: float = 600.0):
        _check(lib().gs_server_drain(self._h, float(timeout_s)))

    def now(self) -> float:
        """Seconds since start: the clock of arrival times."""
        return float(lib().gs_server_now(self._h))

    def stats(self) -> dict:
        st = GsServerStats()
        _check(lib().gs_server_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in GsServerStats._fields_}

    def env_output(self, env_id: int):
        """(rgb [H,W,3], depth [H,W]) torch views of the env's resident outputs."""
        import torch
        rgb, depth = C.c_void_p(), C.c_void_p()
        _check(lib().gs_server_env_output(self._h, int(env_id), C.byref(rgb), C.byref(depth)))
        H, W = self._env_shape[env_id]
        return (torch.as_tensor(_DevView(rgb.value, (H, W, 3)), device="cuda"),
                torch.as_tensor(_DevView(depth.value, (H, W)), device="cuda"))

    def close(self):
        if getattr(self, "_alive", False):
            lib().gs_server_destroy(self._h)
            self._alive = False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def measure_alu_peak(stream=None) -> dict:
    """Measured FP32 FMA and MUFU ex2 lane-op rates of the current device."""
    f, e = C.c_double(), C.c_double()
    _check(lib().gs_measure_alu_peak(C.byref(f), C.byref(e), _stream_handle(stream)))
    return {"fma_lane_ops_per_s": f.value, "ex2_lane_ops_per_s": e.value}


def prune_workload(w, scores, keep_bg: float = 0.3, keep_links: float = 0.1, scene=None):
    """The pruned workload of gs_scene_prune (the selection runs in the
    library): the Gaussians it keeps from w, in their original order, with the
    same poses and cameras.  scores: per Gaussian, the caller's order (numpy or
    CUDA); scene: w's scene (built here when None).  Returns (workload, pruned
    Scene); the caller closes the scene."""
    from . import synth

    own = scene is None
    if own:
        scene = scene_from_workload(w)
    sub, kept = scene.prune(scores, keep_bg, keep_links)
    if own:
        scene.close()
    nb = w.background.n
    bg_idx, link_idx = kept[kept < nb], kept[kept >= nb] - nb
    old = np.asarray(w.link_offsets, dtype=np.int64)
    counts = [int(((link_idx >= old[l]) & (link_idx < old[l + 1])).sum()) for l in range(len(old) - 1)]
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)

    def take(g, idx):
        return synth.Gaussians(g.mean[idx], g.quat[idx], g.log_scale[idx], g.opacity[idx], g.sh[idx])

    return synth.Workload(w.name + "_pruned", take(w.background, bg_idx), offs, take(w.links, link_idx),
                          w.link_poses, w.cams), sub


def make_envs(cams: np.ndarray, link_ranges=None, pose_offsets=None) -> np.ndarray:
    """ENV_DTYPE array for cameras of any resolutions, packed back to back in
    the outputs; link_ranges [E,2] (default: no links), pose_offsets [E]."""
    cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
    E = len(cams)
    envs = np.zeros(E, dtype=ENV_DTYPE)
    envs["cam"] = cams
    if link_ranges is not None:
        lr = np.asarray(link_ranges, dtype=np.int64).reshape(E, 2)
        envs["link_begin"], envs["link_end"] = lr[:, 0], lr[:, 1]
    if pose_offsets is not None:
        envs["pose_offset"] = np.asarray(pose_offsets, dtype=np.int64)
    px = cams["width"].astype(np.int64) * cams["height"].astype(np.int64)
    envs["pixel_offset"] = np.concatenate([[0], np.cumsum(px)[:-1]])
    return envs


def scene_from_workload(w, dtype: str = "f32", sh_degree: int = 3) -> Scene:
    """Build a Scene from a synth.Workload (quantising SH/scales/opacity for bf16/f16)."""
    from . import synth
    if dtype == "f32":
        s = Scene(w.background, "f32", sh_degree)
        if w.n_links > 0:
            s.attach_links(w.link_offsets, w.links)
        return s
    st_bg, _ = synth.quantize(w.background, dtype)
    s = Scene(w.background, dtype, sh_degree, stored=st_bg)
    if w.n_links > 0:
        st_l, _ = synth.quantize(w.links, dtype)
        s.attach_links(w.link_offsets, w.links, stored=st_l)
    return s
