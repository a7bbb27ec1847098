"""Batch-LiDAR oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and ``bench.py``'s CPU legs may import this module; it shares
nothing with the CUDA library.

The paper's Batch-LiDAR module ray-casts the same scenes to produce point
clouds for rotating, solid-state and non-repetitive LiDARs, with dynamic
objects and self-occlusion, over the 3DGS representation (Sec. III-E
"Multi-modal Sensor Suite", Table II).  It gives no formulas, so this oracle
states a reading: every ray is composited front to back over the Gaussians
like a camera pixel, with each Gaussian evaluated at its closest approach
along the ray in ray space instead of through a 2D projection:

* a LiDAR of ``rows`` beams x ``cols`` azimuth steps over the azimuth window
  [az_min, az_max) (a rotating LiDAR covers [0, 2 pi); a solid-state one a
  narrower field of view), sensor frame x forward, y left, z up; ray (i, j)
  has azimuth phi = az_min + (az_max - az_min) (i + 1/2) / cols and elevation
  theta = elev_min + (elev_max - elev_min) (j + 1/2) / rows, direction
  d = (cos theta cos phi, cos theta sin phi, sin theta);
* a Gaussian with sensor-frame mean mu and covariance Sigma = R diag(e^2s) R^T
  has q(t) = |G (t d - mu)|^2 with G = diag(e^-s) R^T; with a = G d and
  b = G mu its minimum is at t* = a.b / |a|^2 and equals |a x b|^2 / |a|^2;
* alpha = min(0.99, o exp(-q_min / 2)); Gaussians with alpha < 1/255 or
  t* <= the near range are skipped; order: distance |mu| ascending, ties by
  global index (or a given rank); T' = T (1 - alpha), stop before adding
  when T' < 1e-4;
* outputs: hit = 1 - T and range = sum(alpha T t*) / (1 - T) (0 where
  1 - T = 0).

The non-repetitive patterns of the paper's list have no grid: ``render_rays``
takes the rays as a list of directions and composites each one the same way
(both entry points share ``_composite_rays``).

Computed in FP64 by brute force over every (ray, Gaussian) pair: small inputs
only.  Pinned in ``tests/test_oracle_pins.py`` (closed forms for one and two
Gaussians on grid and off-grid rays, a joint rigid motion of sensor and
scene, a ray list equal to a grid's rays).
"""
from __future__ import annotations

import numpy as np


def quat_to_mat(q) -> np.ndarray:
    """Rotation matrices [..., 3, 3] of (w, x, y, z) quaternions (normalised here)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def ray_directions(rows: int, cols: int, elev_min: float, elev_max: float, az_min: float = 0.0,
                   az_max: float = 2.0 * np.pi) -> np.ndarray:
    """Unit ray directions [rows, cols, 3] in the sensor frame."""
    phi = az_min + (az_max - az_min) * (np.arange(cols) + 0.5) / cols
    theta = elev_min + (elev_max - elev_min) * (np.arange(rows) + 0.5) / rows
    ct, st = np.cos(theta)[:, None], np.sin(theta)[:, None]
    return np.stack([ct * np.cos(phi)[None, :], ct * np.sin(phi)[None, :], np.broadcast_to(st, (rows, cols))], -1)


def _sensor_frame(mean, quat, log_scale, opacity, link_of, link_poses, sensor, rank):
    """Per Gaussian, sensor frame (RLGK then the sensor pose): G = diag(e^-s)
    R^T, b = G mu, opacity; and the compositing order (distance |mu|, ties by
    global index or rank)."""
    mean = np.asarray(mean, np.float64)
    Rg = quat_to_mat(quat)
    s = np.asarray(log_scale, np.float64)
    o = np.asarray(opacity, np.float64)
    link_of = np.asarray(link_of)
    # rigid-link kinematics: link Gaussians move with their link
    mu_w = mean.copy()
    Rw = Rg.copy()
    if link_poses is not None and len(link_poses):
        lp = np.asarray(link_poses, np.float64).reshape(-1, 7)
        RL = quat_to_mat(lp[:, :4])
        m = link_of >= 0
        li = link_of[m]
        mu_w[m] = np.einsum("nij,nj->ni", RL[li], mean[m]) + lp[li, 4:]
        Rw[m] = RL[li] @ Rg[m]
    Rs = quat_to_mat(sensor["q_ws"])
    ts = np.asarray(sensor["t_ws"], np.float64)
    mu = mu_w @ Rs.T + ts
    Rsg = Rs[None] @ Rw                        # sensor <- Gaussian axes
    G = np.exp(-s)[:, :, None] * np.transpose(Rsg, (0, 2, 1))  # rows e^-s_k (R column k)
    b = np.einsum("nij,nj->ni", G, mu)
    dist = np.linalg.norm(mu, axis=1)
    tie = np.arange(len(dist)) if rank is None else np.asarray(rank)
    order = np.lexsort((tie, dist))
    return G[order], b[order], o[order]


def _composite_rays(Go, bo, oo, near, D) -> tuple:
    """Rays D [m, 3] (unit, sensor frame) over Gaussians in compositing order:
    (range [m], hit [m])."""
    m = D.shape[0]
    rng = np.zeros(m)
    hit = np.zeros(m)
    for c0 in range(0, m, 64):
        Dc = D[c0:c0 + 64]
        a = np.einsum("nij,cj->cni", Go, Dc)           # [c, n, 3]
        aa = (a * a).sum(-1)
        ab = (a * bo[None]).sum(-1)
        cr = np.cross(a, np.broadcast_to(bo[None], a.shape))
        qmin = (cr * cr).sum(-1) / aa
        tstar = ab / aa
        alpha = np.minimum(0.99, oo[None] * np.exp(-0.5 * qmin))
        use = (alpha >= 1.0 / 255.0) & (tstar > near)
        for i in range(Dc.shape[0]):
            T, acc = 1.0, 0.0
            for k in np.nonzero(use[i])[0]:
                al = alpha[i, k]
                Tn = T * (1.0 - al)
                if Tn < 1e-4:
                    break
                acc += al * T * tstar[i, k]
                T = Tn
            hit[c0 + i] = 1.0 - T
            rng[c0 + i] = acc / (1.0 - T) if T < 1.0 else 0.0
    return rng, hit


def render_lidar(mean, quat, log_scale, opacity, link_of, link_poses, sensor, rank=None) -> dict:
    """One env.  mean/quat/log_scale/opacity: the scene's Gaussians (background
    then link-major); link_of [n]: -1 for background, else the link index whose
    pose (link_poses [L][7], link -> world) moves it; sensor: dict with q_ws,
    t_ws (world -> sensor), rows, cols, elev_min, elev_max, near and
    optionally az_min, az_max (default: a full revolution); rank [n]
    (optional): the order among Gaussians at equal distance (default: global
    index).  Returns range [rows, cols], hit [rows, cols]."""
    Go, bo, oo = _sensor_frame(mean, quat, log_scale, opacity, link_of, link_poses, sensor, rank)
    D = ray_directions(sensor["rows"], sensor["cols"], sensor["elev_min"], sensor["elev_max"],
                       sensor.get("az_min", 0.0), sensor.get("az_max", 2.0 * np.pi))
    rows, cols = D.shape[:2]
    rng, hit = _composite_rays(Go, bo, oo, sensor["near"], D.reshape(-1, 3))
    return {"range": rng.reshape(rows, cols), "hit": hit.reshape(rows, cols)}


def render_rays(mean, quat, log_scale, opacity, link_of, link_poses, sensor, dirs, rank=None) -> dict:
    """One env along the rays dirs [m, 3] (sensor frame, normalised here);
    sensor: dict with q_ws, t_ws, near.  Returns range [m], hit [m]."""
    Go, bo, oo = _sensor_frame(mean, quat, log_scale, opacity, link_of, link_poses, sensor, rank)
    D = np.asarray(dirs, np.float64).reshape(-1, 3)
    D = D / np.linalg.norm(D, axis=1, keepdims=True)
    rng, hit = _composite_rays(Go, bo, oo, sensor["near"], D)
    return {"range": rng, "hit": hit}
