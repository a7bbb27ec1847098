"""Python side of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this module.  It loads
``liboracle.so`` built from ``gs_oracle.c`` (plain C, OpenMP over pixel rows)
and never touches the CUDA library.

What it computes is the forward pass of 3D Gaussian Splatting with rigid-link
Gaussian kinematics and an RGB plus depth output (paper Sec. II-B, Sec. III-A
"Data Flow", Sec. III-C "Throughput Scaling" and "RLGK"); the step-by-step
definition is in ``gs_oracle_impl.inc``.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, an independent SH
library, brute force); parity with the paper's own renderer is unpinned
because the paper prints no pixel values.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction, so results do not
    depend on the host ISA's fused multiply-add)."""
    src = [os.path.join(_HERE, "gs_oracle.c")]
    deps = src + [os.path.join(_HERE, "gs_oracle_impl.inc")]
    if not force and os.path.exists(_LIB_PATH):
        if all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(d) for d in deps):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp] + src + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_bg", C.c_int64), ("n_links", C.c_int), ("link_offsets", C.c_void_p),
                ("mean", C.c_void_p), ("quat", C.c_void_p), ("log_scale", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("sh_stride", C.c_int), ("sh_degree", C.c_int)]


class _Camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int),
                ("height", C.c_int), ("q_cw", C.c_float * 4), ("t_cw", C.c_float * 3), ("near_plane", C.c_float)]


class _Proj(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("valid", "proj_ok", "u", "v", "z", "cov2d", "conic", "hx", "hy", "rgb",
                                          "opacity", "range")]


class _Image(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("rgb", "depth", "alpha", "amb", "neval", "contrib", "wbound")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            for sfx in ("f64", "f32"):
                f = getattr(L, f"or_project_{sfx}")
                f.argtypes = [C.POINTER(_Scene), C.c_void_p, C.POINTER(_Camera), C.POINTER(_Proj)]
                f.restype = C.c_int
                f = getattr(L, f"or_render_{sfx}")
                f.argtypes = [C.POINTER(_Proj), C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                              C.POINTER(_Image)]
                f.restype = C.c_int
                f = getattr(L, f"or_sh_basis_{sfx}")
                f.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
                f.restype = None
            L.or_bin.argtypes = [C.c_int64] + [C.c_void_p] * 6 + [C.c_int] * 4 + [C.c_void_p, C.c_void_p]
            L.or_bin.restype = C.c_int64
            L.or_num_threads.restype = C.c_int
            L.or_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(n)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def sh_basis(d, degree: int = 3, precision: str = "f64") -> np.ndarray:
    """The oracle's real SH basis Y_k(d), k < (degree+1)^2, for one direction."""
    dt = np.float64 if precision == "f64" else np.float32
    d = np.ascontiguousarray(d, dtype=dt)
    Y = np.zeros(16, dtype=dt)
    getattr(lib(), f"or_sh_basis_{precision}")(degree, _ptr(d), _ptr(Y))
    return Y[: (degree + 1) ** 2]


class SceneArrays:
    """Concatenated (background, then link-major) float32 arrays of a workload."""

    def __init__(self, background, link_offsets, links, sh_degree: int = 3):
        self.n_bg = background.n
        self.n = background.n + links.n
        self.n_links = int(len(link_offsets) - 1)
        self.link_offsets = np.ascontiguousarray(link_offsets, dtype=np.int64)
        cat = lambda f: _f32(np.concatenate([getattr(background, f), getattr(links, f)]))
        self.mean, self.quat, self.log_scale = cat("mean"), cat("quat"), cat("log_scale")
        self.opacity, self.sh = cat("opacity"), cat("sh")
        self.sh_stride = int(self.sh.shape[1]) if self.sh.ndim == 3 else 1
        self.sh_degree = sh_degree

    def cstruct(self) -> _Scene:
        return _Scene(self.n, self.n_bg, self.n_links, _ptr(self.link_offsets), _ptr(self.mean), _ptr(self.quat),
                      _ptr(self.log_scale), _ptr(self.opacity), _ptr(self.sh), self.sh_stride, self.sh_degree)


def scene_arrays(w, sh_degree: int = 3) -> SceneArrays:
    return SceneArrays(w.background, w.link_offsets, w.links, sh_degree)


def _camera(cam) -> _Camera:
    c = _Camera()
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    for i in range(4):
        c.q_cw[i] = float(cam["q_cw"][i])
    for i in range(3):
        c.t_cw[i] = float(cam["t_cw"][i])
    c.near_plane = float(cam["near_plane"])
    return c


def project(S: SceneArrays, link_poses_env, cam, precision: str = "f64") -> dict:
    """Per-Gaussian projection of one env (steps 1-7 of the definition)."""
    dt = np.float64 if precision == "f64" else np.float32
    n = S.n
    out = dict(valid=np.zeros(n, np.uint8), proj_ok=np.zeros(n, np.uint8), u=np.zeros(n, dt), v=np.zeros(n, dt),
               z=np.zeros(n, dt), cov2d=np.zeros((n, 3), dt), conic=np.zeros((n, 3), dt), hx=np.zeros(n, dt),
               hy=np.zeros(n, dt), rgb=np.zeros((n, 3), dt), opacity=np.zeros(n, dt),
               range=np.zeros((n, 4), np.int32))
    P = _Proj(*[_ptr(out[k]) for k in ("valid", "proj_ok", "u", "v", "z", "cov2d", "conic", "hx", "hy", "rgb",
                                      "opacity", "range")])
    lp = _f32(np.asarray(link_poses_env).reshape(-1, 7)) if S.n_links > 0 else np.zeros((1, 7), np.float32)
    sc = S.cstruct()
    cc = _camera(cam)
    rc = getattr(lib(), f"or_project_{precision}")(C.byref(sc), _ptr(lp), C.byref(cc), C.byref(P))
    if rc != 0:
        raise ValueError(f"oracle projection rejected the input (code {rc}): zero quaternion")
    out["_P"] = P
    return out


def render_projected(proj: dict, width: int, height: int, mode: str = "plain", precision: str = "f64",
                     zkey=None, contrib: bool = False, rank=None) -> dict:
    """Composite projected Gaussians; with ``contrib`` also each Gaussian's
    summed blending weight sum_p alpha T over the pixels where it was added
    (the contribution that ranks Gaussians for pruning).  Gaussians of equal
    depth composite in global-index order, or in ascending ``rank`` [n] when
    given (the tie order of a renderer that stores the scene in another order)."""
    img = dict(rgb=np.zeros((height, width, 3), np.float32), depth=np.zeros((height, width), np.float32),
               alpha=np.zeros((height, width), np.float32), amb=np.zeros((height, width), np.uint8),
               neval=np.zeros((height, width), np.int32), wbound=np.zeros((height, width), np.float32))
    n = len(proj["u"])
    if contrib:
        img["contrib"] = np.zeros(n, np.float64)
    I = _Image(*[_ptr(img[k]) for k in ("rgb", "depth", "alpha", "amb", "neval")],
               _ptr(img["contrib"]) if contrib else None, _ptr(img["wbound"]))
    zk = _f32(zkey) if zkey is not None else None
    rk = np.ascontiguousarray(rank, dtype=np.int64) if rank is not None else None
    if rk is not None and rk.shape != (n,):
        raise ValueError(f"rank must hold one entry per Gaussian ({n})")
    rc = getattr(lib(), f"or_render_{precision}")(C.byref(proj["_P"]), n, _ptr(zk), _ptr(rk), width, height,
                                                   1 if mode == "brute" else 0, C.byref(I))
    assert rc == 0
    return img


def render_env(w, e: int = 0, mode: str = "plain", precision: str = "f64", sh_degree: int = 3, S=None,
               zkey=None, contrib: bool = False, rank=None) -> dict:
    """Render env ``e`` of workload ``w``: rgb [H,W,3], depth, alpha, amb (ambiguous-pixel mask), neval."""
    S = S or scene_arrays(w, sh_degree)
    cam = w.cams[e]
    proj = project(S, w.link_poses[e], cam, precision)
    img = render_projected(proj, int(cam["width"]), int(cam["height"]), mode, precision, zkey, contrib, rank)
    img["proj"] = proj
    return img


def bin_records(u, v, hx, hy, zbits, gidx, width: int, height: int, tile_w: int, tile_h: int):
    """Binning oracle (keyed mode): per-tile counts and per-tile global-index
    lists in (depth bits, global index) order, from a renderer's records."""
    u, v, hx, hy = _f32(u), _f32(v), _f32(hx), _f32(hy)
    zb = np.ascontiguousarray(zbits, dtype=np.uint32)
    gi = np.ascontiguousarray(gidx, dtype=np.uint32)
    ntiles = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    counts = np.zeros(ntiles, np.int64)
    L = lib()
    total = L.or_bin(len(u), _ptr(u), _ptr(v), _ptr(hx), _ptr(hy), _ptr(zb), _ptr(gi), width, height, tile_w,
                     tile_h, _ptr(counts), None)
    lists = np.zeros(max(total, 1), np.uint32)
    L.or_bin(len(u), _ptr(u), _ptr(v), _ptr(hx), _ptr(hy), _ptr(zb), _ptr(gi), width, height, tile_w, tile_h,
             _ptr(counts), _ptr(lists))
    return counts, lists[:total]


def observation(rgb, depth, appearance=None):
    """Observation form of a rendered image: the paper's manipulation
    experiments randomise image-level brightness, contrast and exposure
    (Sec. IV-E); policies take 8-bit colour.  Reading (the paper gives no
    formula): per channel c = clamp(colour, 0, 1), v = clamp((c 2^exposure -
    0.5) contrast + 0.5 + brightness, 0, 1), u8 = round half to even of 255 v;
    depth as IEEE half.  ``appearance`` = (exposure, contrast, brightness) or
    None for the identity.  Computed in FP64 (depth rounded from FP64)."""
    c = np.clip(np.asarray(rgb, dtype=np.float64), 0.0, 1.0)
    if appearance is not None:
        e, k, b = (float(x) for x in appearance)
        c = np.clip((c * 2.0 ** e - 0.5) * k + 0.5 + b, 0.0, 1.0)
    u8 = np.rint(c * 255.0).astype(np.uint8)
    d16 = np.asarray(depth, dtype=np.float64).astype(np.float16)
    return u8, d16
