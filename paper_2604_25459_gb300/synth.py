"""Seeded synthetic inputs for the batched 3DGS RGB-D renderer.

This module samples scenes, link poses and cameras and nothing else: it holds
none of the rendering arithmetic (no projection, no SH evaluation, no
compositing).  Both the CUDA path and the CPU oracle consume the exact float32
arrays it returns, so the two always see the same input bytes.

Workloads (shapes follow the paper's rendering benchmark, Sec. III-C
"Throughput Scaling": 2048 environments at 640x480, each a static 3DGS
background plus robot links that carry their own Gaussians, Sec. III-C
"RLGK").  The paper's scenes are real captures that are not available, so
these seeded synthetic scenes stand in for them:

* ``tiny``   -- a few Gaussians, for brute-force checks.
* ``c0``     -- 1 env, 128x96, f=110, camera at (0,0,-3) looking at the
  origin, 16,384 Gaussians (means U[-1,1]^3, log-scales N(-4,0.5), uniform
  unit quaternions, opacity sigmoid(N(0,1)), SH degree 3 ~ N(0,0.3) with the
  DC term +0.5).
* ``c1``     -- E envs (2048 by default) at 640x480, f=500: a 500k-Gaussian
  room-shell background plus a 20-link robot with 5k Gaussians per link,
  per-env joint angles U(-1,1) on a fixed chain and a jittered head camera.
* ``c2``     -- ``c1`` at another resolution (128x128 with f=100, or 640x480).

Conventions: world z up; camera axes x right, y down, z forward; a pose is a
unit quaternion (w,x,y,z) plus a translation; link poses map link->world,
camera poses map world->camera.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# gs_camera in include/gsbatch.h: 14 four-byte fields, 56 bytes.
CAMERA_DTYPE = np.dtype(
    [
        ("fx", "<f4"),
        ("fy", "<f4"),
        ("cx", "<f4"),
        ("cy", "<f4"),
        ("width", "<i4"),
        ("height", "<i4"),
        ("q_cw", "<f4", (4,)),
        ("t_cw", "<f4", (3,)),
        ("near_plane", "<f4"),
    ]
)
assert CAMERA_DTYPE.itemsize == 56

SH_COEFFS = 16  # degree 3
NEAR_PLANE = 0.01


@dataclasses.dataclass
class Gaussians:
    """Structure-of-arrays Gaussian set (float32)."""

    mean: np.ndarray  # [n,3]
    quat: np.ndarray  # [n,4] (w,x,y,z), unit
    log_scale: np.ndarray  # [n,3]
    opacity: np.ndarray  # [n] activated, in (0,1)
    sh: np.ndarray  # [n,16,3] coefficient-major, channel-minor

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def slice(self, a: int, b: int) -> "Gaussians":
        return Gaussians(self.mean[a:b], self.quat[a:b], self.log_scale[a:b],
                         self.opacity[a:b], self.sh[a:b])

    @staticmethod
    def concat(parts) -> "Gaussians":
        return Gaussians(*[np.ascontiguousarray(np.concatenate([getattr(p, f) for p in parts]))
                           for f in ("mean", "quat", "log_scale", "opacity", "sh")])


@dataclasses.dataclass
class Workload:
    """One batch: shared background, link-attached Gaussians, per-env state."""

    name: str
    background: Gaussians
    link_offsets: np.ndarray  # int64 [L+1]
    links: Gaussians  # link-frame Gaussians, link-major
    link_poses: np.ndarray  # f32 [E][L][7]  (qw,qx,qy,qz,tx,ty,tz), link->world
    cams: np.ndarray  # CAMERA_DTYPE [E]

    @property
    def n_envs(self) -> int:
        return int(self.cams.shape[0])

    @property
    def n_links(self) -> int:
        return int(self.link_offsets.shape[0] - 1)

    def env(self, e: int) -> "Workload":
        return dataclasses.replace(self, link_poses=self.link_poses[e:e + 1].copy(),
                                   cams=self.cams[e:e + 1].copy(), name=f"{self.name}[{e}]")

    def envs(self, idx) -> "Workload":
        idx = np.asarray(idx, dtype=np.int64)
        return dataclasses.replace(self, link_poses=np.ascontiguousarray(self.link_poses[idx]),
                                   cams=np.ascontiguousarray(self.cams[idx]), name=f"{self.name}{list(idx)}")


def _rng(*key: int) -> np.random.Generator:
    """Independent seeded stream per (seed, purpose[, index])."""
    return np.random.default_rng([int(k) for k in key])


_STREAM = {"bg": 1, "robot": 2, "joints": 3, "cams": 4, "tiny": 5, "c0": 6, "rays": 11}


def _attributes(rng: np.random.Generator, n: int) -> tuple:
    """The per-Gaussian appearance distributions shared by every workload."""
    log_scale = rng.normal(-4.0, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, size=n)))
    sh = rng.normal(0.0, 0.3, size=(n, SH_COEFFS, 3))
    sh[:, 0, :] += 0.5
    return q, log_scale, opacity, sh


def _gaussians(mean, q, log_scale, opacity, sh) -> Gaussians:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Gaussians(f(mean), f(q), f(log_scale), f(opacity), f(sh))


def make_gaussians_uniform_cube(n: int, seed: int, stream: str = "c0", half: float = 1.0) -> Gaussians:
    rng = _rng(seed, _STREAM[stream])
    mean = rng.uniform(-half, half, size=(n, 3))
    return _gaussians(mean, *_attributes(rng, n))


def make_room_shell(n: int, seed: int, extent=(10.0, 10.0, 3.0), jitter=0.02) -> Gaussians:
    """n Gaussians area-uniform on the six faces of the box
    [-X/2,X/2]x[-Y/2,Y/2]x[0,Z] with N(0, jitter) displacement along the face normal."""
    rng = _rng(seed, _STREAM["bg"])
    X, Y, Z = extent
    # faces: floor, ceiling, x-, x+, y-, y+
    areas = np.array([X * Y, X * Y, Y * Z, Y * Z, X * Z, X * Z])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    a = rng.uniform(0.0, 1.0, size=n)
    b = rng.uniform(0.0, 1.0, size=n)
    off = rng.normal(0.0, jitter, size=n)
    mean = np.empty((n, 3))
    x = (a - 0.5) * X
    y = (b - 0.5) * Y
    for f in range(6):
        m = face == f
        if f < 2:
            mean[m] = np.stack([x[m], y[m], np.full(m.sum(), 0.0 if f == 0 else Z) + off[m]], 1)
        elif f < 4:
            mean[m] = np.stack([np.full(m.sum(), -X / 2 if f == 2 else X / 2) + off[m],
                                (a[m] - 0.5) * Y, b[m] * Z], 1)
        else:
            mean[m] = np.stack([(a[m] - 0.5) * X, np.full(m.sum(), -Y / 2 if f == 4 else Y / 2) + off[m],
                                b[m] * Z], 1)
    return _gaussians(mean, *_attributes(rng, n))


def make_robot(n_links: int, per_link: int, seed: int, sigma: float = 0.05) -> tuple:
    rng = _rng(seed, _STREAM["robot"])
    n = n_links * per_link
    mean = rng.normal(0.0, sigma, size=(n, 3))
    offsets = np.arange(n_links + 1, dtype=np.int64) * per_link
    return offsets, _gaussians(mean, *_attributes(rng, n))


# ---------------------------------------------------------------- rotations (input sampling only)

def _rot_axis(axis: int, ang: np.ndarray) -> np.ndarray:
    c, s = np.cos(ang), np.sin(ang)
    R = np.zeros(ang.shape + (3, 3))
    i, j = [(1, 2), (2, 0), (0, 1)][axis]
    R[..., axis, axis] = 1.0
    R[..., i, i] = c
    R[..., j, j] = c
    R[..., i, j] = -s
    R[..., j, i] = s
    return R


def matrix_to_quat(R: np.ndarray) -> np.ndarray:
    """Rotation matrices [...,3,3] -> unit quaternions [...,4] (w,x,y,z), w >= 0.

    Shepperd's method: pick the largest of (trace, R00, R11, R22) as pivot."""
    R = np.asarray(R, dtype=np.float64)
    shp = R.shape[:-2]
    R = R.reshape(-1, 3, 3)
    q = np.empty((R.shape[0], 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    piv = np.argmax(np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1), axis=1)
    for k in range(4):
        m = piv == k
        r = R[m]
        if k == 0:
            s = np.sqrt(1.0 + tr[m]) * 2
            q[m] = np.stack([0.25 * s, (r[:, 2, 1] - r[:, 1, 2]) / s, (r[:, 0, 2] - r[:, 2, 0]) / s,
                             (r[:, 1, 0] - r[:, 0, 1]) / s], 1)
        else:
            i = k - 1
            j, l = (i + 1) % 3, (i + 2) % 3
            s = np.sqrt(1.0 + r[:, i, i] - r[:, j, j] - r[:, l, l]) * 2
            qq = np.empty((m.sum(), 4))
            qq[:, 0] = (r[:, l, j] - r[:, j, l]) / s
            qq[:, 1 + i] = 0.25 * s
            qq[:, 1 + j] = (r[:, j, i] + r[:, i, j]) / s
            qq[:, 1 + l] = (r[:, l, i] + r[:, i, l]) / s
            q[m] = qq
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.reshape(shp + (4,))


def chain_link_poses(joint_angles: np.ndarray, base=(0.0, 0.0, 0.8), link_len: float = 0.08) -> np.ndarray:
    """Forward kinematics of the fixed chain used by the c1 robot.

    Joint k is revolute about the local z axis (k even) or local y axis (k odd);
    consecutive links are 0.08 m apart along the parent's local x axis; the base
    sits at (0,0,0.8).  Returns f32 [E][L][7] (qw,qx,qy,qz,tx,ty,tz), link->world."""
    E, L = joint_angles.shape
    R = np.broadcast_to(np.eye(3), (E, 3, 3)).copy()
    t = np.broadcast_to(np.asarray(base, dtype=np.float64), (E, 3)).copy()
    out = np.zeros((E, L, 7))
    for k in range(L):
        if k > 0:
            t = t + R @ np.array([link_len, 0.0, 0.0])
        R = R @ _rot_axis(2 if k % 2 == 0 else 1, joint_angles[:, k])
        out[:, k, :4] = matrix_to_quat(R)
        out[:, k, 4:] = t
    return out.astype(np.float32)


def look_camera(pos: np.ndarray, yaw: np.ndarray, pitch: np.ndarray, roll: np.ndarray):
    """World->camera poses for cameras at ``pos`` [E,3] with the given yaw (about
    world z), pitch (positive looks down) and roll (about the optical axis).
    Returns (q_cw [E,4], t_cw [E,3]) in float64."""
    cp, sp = np.cos(pitch), np.sin(pitch)
    cy, sy = np.cos(yaw), np.sin(yaw)
    fwd = np.stack([cp * cy, cp * sy, -sp], 1)
    right0 = np.stack([sy, -cy, np.zeros_like(yaw)], 1)
    down0 = np.cross(fwd, right0)
    cr, sr = np.cos(roll)[:, None], np.sin(roll)[:, None]
    right = cr * right0 + sr * down0
    down = -sr * right0 + cr * down0
    R_wc = np.stack([right, down, fwd], 2)  # columns = camera axes in world
    R_cw = np.transpose(R_wc, (0, 2, 1))
    t_cw = -np.einsum("eij,ej->ei", R_cw, pos)
    return matrix_to_quat(R_cw), t_cw


def make_cameras(n: int, fx, fy, cx, cy, width, height, q_cw, t_cw, near=NEAR_PLANE) -> np.ndarray:
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    cams["fx"], cams["fy"], cams["cx"], cams["cy"] = fx, fy, cx, cy
    cams["width"], cams["height"] = width, height
    cams["q_cw"] = np.asarray(q_cw, dtype=np.float32).reshape(n, 4)
    cams["t_cw"] = np.asarray(t_cw, dtype=np.float32).reshape(n, 3)
    cams["near_plane"] = near
    return cams


def head_cameras(n_envs: int, seed: int, width: int, height: int, f: float) -> np.ndarray:
    """Per-env head cameras: nominal position (-1,0,1.4) looking along +x pitched
    25 deg down, jittered U(+-0.2 m) per axis and U(+-10 deg) in yaw, pitch, roll."""
    rng = _rng(seed, _STREAM["cams"])
    pos = np.array([-1.0, 0.0, 1.4]) + rng.uniform(-0.2, 0.2, size=(n_envs, 3))
    d = math.radians(10.0)
    yaw = rng.uniform(-d, d, n_envs)
    pitch = math.radians(25.0) + rng.uniform(-d, d, n_envs)
    roll = rng.uniform(-d, d, n_envs)
    q, t = look_camera(pos, yaw, pitch, roll)
    return make_cameras(n_envs, f, f, width / 2.0, height / 2.0, width, height, q, t)


# ---------------------------------------------------------------- workloads

def make_c0(seed: int = 0, n: int = 16384, width: int = 128, height: int = 96, f: float = 110.0) -> Workload:
    bg = make_gaussians_uniform_cube(n, seed, "c0")
    cams = make_cameras(1, f, f, width / 2.0, height / 2.0, width, height, [1, 0, 0, 0], [0, 0, 3.0])
    empty = bg.slice(0, 0)
    return Workload("c0", bg, np.zeros(1, np.int64), empty, np.zeros((1, 0, 7), np.float32), cams)


def make_c1(n_envs: int = 2048, seed: int = 0, width: int = 640, height: int = 480, f: float = 500.0,
            n_bg: int = 500_000, n_links: int = 20, per_link: int = 5000, name: str = "c1") -> Workload:
    bg = make_room_shell(n_bg, seed)
    offsets, robot = make_robot(n_links, per_link, seed)
    jrng = _rng(seed, _STREAM["joints"])
    angles = jrng.uniform(-1.0, 1.0, size=(n_envs, n_links))
    poses = chain_link_poses(angles)
    cams = head_cameras(n_envs, seed, width, height, f)
    return Workload(name, bg, offsets, robot, poses, cams)


def make_c2(n_envs: int = 2048, seed: int = 0, res: str = "128x128") -> Workload:
    if res == "128x128":
        return make_c1(n_envs, seed, 128, 128, 100.0, name="c2_128")
    return make_c1(n_envs, seed, 640, 480, 500.0, name="c2_640")


def make_tiny(seed: int = 0, n: int = 48, width: int = 32, height: int = 24, f: float = 30.0,
              n_links: int = 2, per_link: int = 8, n_envs: int = 2) -> Workload:
    """A few Gaussians in front of the camera plus two small links, for brute-force checks."""
    rng = _rng(seed, _STREAM["tiny"])
    mean = rng.uniform(-0.6, 0.6, size=(n, 3))
    q, ls, o, sh = _attributes(rng, n)
    ls = ls + 1.5  # larger footprints so that a 32x24 image has overlaps
    bg = _gaussians(mean, q, ls, o, sh)
    lm = rng.normal(0.0, 0.1, size=(n_links * per_link, 3))
    q2, ls2, o2, sh2 = _attributes(rng, n_links * per_link)
    links = _gaussians(lm, q2, ls2 + 1.5, o2, sh2)
    offsets = np.arange(n_links + 1, dtype=np.int64) * per_link
    ang = rng.uniform(-1.0, 1.0, size=(n_envs, n_links))
    poses = chain_link_poses(ang, base=(0.0, 0.0, -0.3), link_len=0.2)
    pos = np.array([0.0, 0.0, -3.0]) + rng.uniform(-0.1, 0.1, size=(n_envs, 3))
    # cameras looking along +z (world), small jitter
    R = np.broadcast_to(np.eye(3), (n_envs, 3, 3))
    q_cw = matrix_to_quat(R)
    t_cw = -pos
    cams = make_cameras(n_envs, f, f, width / 2.0, height / 2.0, width, height, q_cw, t_cw)
    return Workload("tiny", bg, offsets, links, poses, cams)


def rosette_rays(n_envs: int, n_rays: int, seed: int = 0, half_fov: float = 0.6, turns: float = 37.0,
                 petals: float = 7.3) -> np.ndarray:
    """Ray directions of a non-repetitive scan pattern, float32 [E][R][3] in
    the sensor frame (x forward, y left, z up): a rosette inside a cone of
    half-angle half_fov about +x, ray k at polar angle
    half_fov |sin(petals u)| and azimuth about the axis 2 pi u, u = turns
    (k + phase_e) / R, with a seeded phase per env so that frames differ (the
    pattern does not repeat; densest near the axis, as such sensors are)."""
    rng = _rng(seed, _STREAM["rays"])
    phase = rng.uniform(0.0, float(n_rays), size=(n_envs, 1))
    u = turns * (np.arange(n_rays)[None, :] + phase) / n_rays
    rho = half_fov * np.abs(np.sin(petals * u))
    psi = 2.0 * np.pi * u
    # direction at polar angle rho from +x, rotated by psi about +x
    d = np.stack([np.cos(rho), np.sin(rho) * np.cos(psi), np.sin(rho) * np.sin(psi)], -1)
    return np.ascontiguousarray(d, dtype=np.float32)


def to_half(a: np.ndarray, dtype: str) -> np.ndarray:
    """float32 -> bfloat16 (as uint16, round to nearest even) or float16."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    if dtype == "f16":
        return a.astype(np.float16)
    if dtype != "bf16":
        raise ValueError(dtype)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def from_half(h: np.ndarray, dtype: str) -> np.ndarray:
    """Exact widening of bf16 (uint16 storage) or f16 to float32."""
    if dtype == "f16":
        return np.asarray(h, dtype=np.float16).astype(np.float32)
    return (np.asarray(h, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def quantize(g: Gaussians, dtype: str) -> tuple:
    """Storage form of the precision variant: SH, log-scales and opacities in
    bf16/f16 (means and quaternions stay f32).  Returns (stored_arrays, widened
    Gaussians) -- the widened set is what the stored bytes represent exactly."""
    stored = dict(log_scale=to_half(g.log_scale, dtype), opacity=to_half(g.opacity, dtype),
                  sh=to_half(g.sh, dtype))
    widened = Gaussians(g.mean, g.quat, from_half(stored["log_scale"], dtype),
                        from_half(stored["opacity"], dtype), from_half(stored["sh"], dtype))
    return stored, widened


# ---------------------------------------------------------------- batched uneven workload (c3)

C3_RESOLUTIONS = ((64, 64), (128, 128), (320, 240), (640, 480))
C3_PROBS = (0.3, 0.3, 0.2, 0.2)


def focal_for(width: int, height: int) -> float:
    """Focal length keeping the c1/c2 field of view: f = 500 at 640 px width for
    4:3 images, f = 100 at 128 px for square ones."""
    return 500.0 * width / 640.0 if width != height else 100.0 * width / 128.0


def c3_counts(n_envs: int, seed: int, lo: int = 10_000, hi: int = 200_000) -> np.ndarray:
    """Per-env object Gaussian counts, log-uniform in [lo, hi]."""
    rng = _rng(seed, 9)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), n_envs))).astype(np.int64).clip(lo, hi)


def c3_resolutions(n_envs: int, seed: int) -> np.ndarray:
    rng = _rng(seed, 10)
    return rng.choice(len(C3_RESOLUTIONS), size=n_envs, p=C3_PROBS)


def _c3_object(seed: int, e: int, n: int, sigma: float):
    rng = _rng(seed, 8, e)
    mean = rng.normal(0.0, sigma, size=(n, 3))
    return (mean,) + _attributes(rng, n)


@dataclasses.dataclass
class UnevenWorkload:
    """Envs of different resolutions, each rendering the shared background plus
    its own object (link e of the scene, pose e)."""

    name: str
    background: Gaussians
    link_offsets: np.ndarray  # int64 [E+1]: object of env e = links[off[e]:off[e+1]]
    links: Gaussians
    link_poses: np.ndarray  # f32 [E][7], object pose of env e (link -> world)
    cams: np.ndarray  # CAMERA_DTYPE [E], mixed resolutions

    @property
    def n_envs(self) -> int:
        return int(self.cams.shape[0])

    def env(self, e: int) -> Workload:
        """Env e alone, as a one-link workload (the same bytes)."""
        a, b = int(self.link_offsets[e]), int(self.link_offsets[e + 1])
        return Workload(f"{self.name}[{e}]", self.background, np.array([0, b - a], np.int64), self.links.slice(a, b),
                        self.link_poses[e:e + 1, None, :].copy(), self.cams[e:e + 1].copy())


def make_c3(n_envs: int = 4096, seed: int = 0, n_bg: int = 300_000, count_range=(10_000, 200_000),
            sigma: float = 0.15, threads: int = 16) -> UnevenWorkload:
    """The batched uneven form: a shared room-shell background of n_bg Gaussians;
    env e has its own object of log-uniform size in count_range (means
    N(0, sigma) in the object frame, the c0 attribute distributions) placed in
    front of a jittered head camera, at a resolution drawn from {64x64, 128x128,
    320x240, 640x480} with probabilities {.3, .3, .2, .2}.  Each env's object
    comes from its own seeded stream, so env e can be regenerated alone."""
    from concurrent.futures import ThreadPoolExecutor

    bg = make_room_shell(n_bg, seed)
    counts = c3_counts(n_envs, seed, *count_range)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    N = int(offsets[-1])
    mean = np.empty((N, 3), np.float32)
    quat = np.empty((N, 4), np.float32)
    ls = np.empty((N, 3), np.float32)
    op = np.empty(N, np.float32)
    sh = np.empty((N, SH_COEFFS, 3), np.float32)

    def fill(e):
        a, b = offsets[e], offsets[e + 1]
        m, q, l, o, s = _c3_object(seed, e, int(b - a), sigma)
        mean[a:b], quat[a:b], ls[a:b], op[a:b], sh[a:b] = m, q, l, o, s

    with ThreadPoolExecutor(max(1, threads)) as ex:
        list(ex.map(fill, range(n_envs)))
    links = Gaussians(mean, quat, ls, op, sh)
    rng = _rng(seed, 11)
    pos = np.stack([0.6 + rng.uniform(-0.2, 0.2, n_envs), rng.uniform(-0.3, 0.3, n_envs),
                    0.6 + rng.uniform(0.0, 0.3, n_envs)], 1)
    q = rng.normal(size=(n_envs, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    poses = np.concatenate([q, pos], 1).astype(np.float32)
    res = c3_resolutions(n_envs, seed)
    cams = np.zeros(n_envs, dtype=CAMERA_DTYPE)
    for k, (W, H) in enumerate(C3_RESOLUTIONS):
        idx = np.nonzero(res == k)[0]
        if len(idx):
            c = head_cameras(n_envs, seed, W, H, focal_for(W, H))[idx]
            cams[idx] = c
    return UnevenWorkload("c3", bg, offsets, links, poses, cams)


# ---------------------------------------------------------------- served workload (c4)

@dataclasses.dataclass
class ServedWorkload:
    """Resident scenes and env instances of the request loop: scene k is a
    room-shell background of its own size plus the c1 robot (20 links x 5k
    Gaussians); env i belongs to scene ``env_scene[i]`` and has its own camera
    (c3 resolution mix).  Request poses come from ``request_poses``."""

    name: str
    backgrounds: list          # [n_scenes] Gaussians
    link_offsets: np.ndarray   # int64 [L+1], shared robot
    links: Gaussians
    env_scene: np.ndarray      # int32 [E]
    cams: np.ndarray           # CAMERA_DTYPE [E]
    seed: int

    @property
    def n_envs(self) -> int:
        return int(self.cams.shape[0])

    @property
    def n_links(self) -> int:
        return int(self.link_offsets.shape[0] - 1)

    def request_poses(self, n: int, stream: int = 0) -> np.ndarray:
        """f32 [n][L][7]: link poses of n requests (joint angles U(-1,1) on the
        c1 chain), from stream ``stream`` of this workload's seed."""
        rng = _rng(self.seed, 12, stream)
        return chain_link_poses(rng.uniform(-1.0, 1.0, size=(n, self.n_links)))

    def scene_workload(self, k: int, env_ids, poses: np.ndarray) -> Workload:
        """Envs ``env_ids`` (all of scene k, one resolution) with the given
        poses [len(env_ids)][L][7], as a plain workload."""
        env_ids = np.asarray(env_ids)
        return Workload(f"{self.name}[{k}]", self.backgrounds[k], self.link_offsets, self.links,
                        np.ascontiguousarray(poses, np.float32), self.cams[env_ids].copy())


def c4_background_sizes(n_scenes: int, lo: int = 200_000, hi: int = 1_000_000) -> np.ndarray:
    """Background sizes of the served scenes, evenly spaced from lo to hi."""
    return np.linspace(lo, hi, n_scenes).round().astype(np.int64)


def make_c4(n_scenes: int = 8, n_envs: int = 4096, seed: int = 0, bg_range=(200_000, 1_000_000),
            n_links: int = 20, per_link: int = 5000) -> ServedWorkload:
    """The served form: n_scenes room-shell backgrounds (sizes evenly spaced
    over bg_range, each from its own seed 1000*seed + k + 1, the c0 attribute
    distributions), the c1 robot shared by all, and n_envs env instances
    assigned to scenes round robin, with jittered head cameras at the c3
    resolution mix."""
    sizes = c4_background_sizes(n_scenes, *bg_range)
    bgs = [make_room_shell(int(n), 1000 * seed + k + 1) for k, n in enumerate(sizes)]
    offsets, robot = make_robot(n_links, per_link, seed)
    res = c3_resolutions(n_envs, seed)
    cams = np.zeros(n_envs, dtype=CAMERA_DTYPE)
    for k, (W, H) in enumerate(C3_RESOLUTIONS):
        idx = np.nonzero(res == k)[0]
        if len(idx):
            cams[idx] = head_cameras(n_envs, seed, W, H, focal_for(W, H))[idx]
    env_scene = (np.arange(n_envs) % n_scenes).astype(np.int32)
    return ServedWorkload("c4", bgs, offsets, robot, env_scene, cams, seed)
