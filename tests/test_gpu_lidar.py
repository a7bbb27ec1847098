"""Batch-LiDAR scans (ray-space evaluation over the same Gaussians, moving
links included) against the FP64 brute-force LiDAR oracle."""
import numpy as np
import pytest

from gpu_helpers import ensure_built
from oracle import lidar
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


def _sensors(E, rows=16, cols=128, seed=4, az=(0.0, 2.0 * np.pi)):
    rng = np.random.default_rng([seed, 52])
    s = np.zeros(E, dtype=gsbatch.LIDAR_DTYPE)
    s["q_ws"] = [1.0, 0.0, 0.0, 0.0]  # sensor axes = world axes (x forward, z up)
    pos = np.array([-1.0, 0.0, 1.0]) + rng.uniform(-0.2, 0.2, (E, 3))
    s["t_ws"] = -pos
    s["rows"], s["cols"] = rows, cols
    s["elev_min"], s["elev_max"], s["near_range"] = -0.5, 0.35, 0.05
    s["az_min"], s["az_max"] = az
    return s


def _oracle_scan(w, e, sen):
    bg, lk = w.background, w.links
    mean = np.concatenate([bg.mean, lk.mean])
    quat = np.concatenate([bg.quat, lk.quat])
    ls = np.concatenate([bg.log_scale, lk.log_scale])
    op = np.concatenate([bg.opacity, lk.opacity])
    link_of = np.concatenate([np.full(bg.n, -1), np.repeat(np.arange(w.n_links), np.diff(w.link_offsets))])
    return lidar.render_lidar(mean, quat, ls, op, link_of, w.link_poses[e],
                              dict(q_ws=sen["q_ws"].astype(float), t_ws=sen["t_ws"].astype(float),
                                   rows=int(sen["rows"]), cols=int(sen["cols"]), elev_min=float(sen["elev_min"]),
                                   elev_max=float(sen["elev_max"]), near=float(sen["near_range"]),
                                   az_min=float(sen["az_min"]), az_max=float(sen["az_max"])))


@pytest.mark.parametrize("window", ["rotating", "solid_state", "solid_state_across_pi"])
def test_lidar_scan_matches_oracle(window):
    """Rotating scans, and solid-state ones whose azimuth window is narrower
    (one across the direction at +-pi, where the azimuth wraps)."""
    import torch

    ensure_built()
    # the window behind the sensors looks at the far wall: a denser room there
    n_bg = 30_000 if window == "solid_state_across_pi" else 8_000
    w = synth.make_c1(n_envs=2, width=64, height=48, f=50.0, n_bg=n_bg, per_link=200)
    az = {"rotating": (0.0, 2.0 * np.pi), "solid_state": (-0.9, 0.9), "solid_state_across_pi": (2.4, 3.9)}[window]
    sens = _sensors(w.n_envs, cols=64 if window != "rotating" else 128, az=az)
    scene = gsbatch.scene_from_workload(w)
    rng, hit = scene.render_lidar(torch.from_numpy(w.link_poses).cuda(), sens)
    torch.cuda.synchronize()
    scene.sync_status()
    g_r, g_h = rng.cpu().numpy(), hit.cpu().numpy()
    for e in range(w.n_envs):
        ref = _oracle_scan(w, e, sens[e])
        dh = np.abs(g_h[e] - ref["hit"])
        both = (ref["hit"] >= 0.5) & (g_h[e] >= 0.5)
        rel = np.abs(g_r[e] - ref["range"])[both] / ref["range"][both]
        print("lidar env", e, "rays hit >= 0.5:", int(both.sum()), "hit max", dh.max(), "p99",
              np.quantile(dh, 0.99), "range rel max", rel.max() if rel.size else None)
        assert ref["hit"].max() > 0.5 and both.sum() > 20
        # FP32 ray-space arithmetic vs FP64: threshold flips (alpha at 1/255, T at 1e-4) are rare
        assert np.quantile(dh, 0.99) <= 2e-3 and dh.max() <= 0.05
        assert np.quantile(rel, 0.99) <= 1e-4 and rel.max() <= 1e-2
    scene.close()


def _wall_ahead(n=300, seed=23):
    """A patch of wall 3 m straight ahead of a sensor at the origin: y across
    azimuth 0 (where a full turn's columns wrap), z across the beams."""
    rng = np.random.default_rng(seed)
    mean = np.stack([3.0 + rng.normal(0.0, 0.01, n), rng.uniform(-0.25, 0.25, n), rng.uniform(-0.3, 0.3, n)], 1)
    quat = rng.normal(size=(n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)  # uniform random orientations (w, x, y, z)
    ls = np.log(rng.uniform(0.02, 0.05, (n, 3)))
    sh = rng.normal(0, 0.3, size=(n, 16, 3))
    bg = synth.Gaussians(*(np.ascontiguousarray(a, np.float32) for a in
                           (mean, quat, ls, rng.uniform(0.3, 0.95, n), sh)))
    cams = synth.make_cameras(1, 50.0, 50.0, 32.0, 24.0, 64, 48, [[1, 0, 0, 0]], [[0, 0, 0]])
    w = synth.Workload("wall", bg, np.zeros(1, np.int64), bg.slice(0, 0), np.zeros((1, 0, 7), np.float32), cams)
    sens = np.zeros(1, dtype=gsbatch.LIDAR_DTYPE)
    sens["q_ws"] = [1.0, 0.0, 0.0, 0.0]
    sens["rows"], sens["cols"] = 16, 128  # 8 column tiles, one row of tiles
    sens["elev_min"], sens["elev_max"], sens["near_range"] = -0.15, 0.15, 0.05
    sens["az_min"], sens["az_max"] = 0.0, 2.0 * np.pi
    # most of the patch's cones cross azimuth 0 (column width 2 pi / 128)
    az = np.arctan2(mean[:, 1], mean[:, 0])
    assert (np.abs(az) < np.pi / 128).sum() > n // 10
    return w, sens


def test_lidar_cones_across_azimuth_zero():
    """Gaussians straight ahead of a rotating LiDAR, where its columns wrap
    (azimuth 0 is both the first and the last column): their cones reach both
    ends of the grid, so their boxes are stored as two column ranges and each
    Gaussian lands in the tiles of those columns only, not in every tile of
    its rows; the scan there still matches the FP64 oracle."""
    import torch

    ensure_built()
    w, sens = _wall_ahead()
    n = w.background.n
    scene = gsbatch.scene_from_workload(w)
    rg, hit = scene.render_lidar(None, sens)
    torch.cuda.synchronize()
    scene.sync_status()
    keys = scene.stats()["intersections"]
    print("Gaussians", n, "keys", keys)
    assert 0 < keys <= 2 * n  # each in the first and/or last column tile of the one tile row
    g_r, g_h = rg.cpu().numpy()[0], hit.cpu().numpy()[0]
    scene.close()
    ref = _oracle_scan(w, 0, sens[0])
    both = (ref["hit"] >= 0.5) & (g_h >= 0.5)
    print("rays hit >= 0.5 in columns 0 and 127:", int(both[:, [0, 127]].sum()))
    assert both[:, 0].sum() > 3 and both[:, 127].sum() > 3
    _check_scan(g_r, g_h, ref, "wall ahead")


def test_rays_across_azimuth_zero():
    """A ray list straddling azimuth 0, binned on a full turn's grid: the
    Gaussians' wrapped boxes hold every ray of both column ranges (rays just
    left and just right of 0), against the FP64 ray-list oracle."""
    import torch

    ensure_built()
    w, sens = _wall_ahead()
    rng = np.random.default_rng(31)
    R = 4000
    az = rng.uniform(-0.12, 0.12, R)
    el = rng.uniform(-0.14, 0.14, R)
    dirs = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1)[None].astype(np.float32)
    scene = gsbatch.scene_from_workload(w)
    rg, hit = scene.render_rays(None, sens, torch.from_numpy(np.ascontiguousarray(dirs)).cuda())
    torch.cuda.synchronize()
    scene.sync_status()
    g_r, g_h = rg.cpu().numpy()[0], hit.cpu().numpy()[0]
    scene.close()
    ref = _oracle_rays(w, 0, sens[0], dirs[0])
    left, right = az < 0, az >= 0
    print("rays hit >= 0.5 left / right of 0:", int((g_h[left] >= 0.5).sum()), int((g_h[right] >= 0.5).sum()))
    assert (g_h[left] >= 0.5).sum() > 20 and (g_h[right] >= 0.5).sum() > 20
    _check_scan(g_r, g_h, ref, "rays across azimuth 0")


def test_lidar_argument_checks_and_empty_scene():
    import torch

    ensure_built()
    bg = synth.make_gaussians_uniform_cube(0, 0)
    scene = gsbatch.Scene(bg)
    sens = _sensors(2, rows=8, cols=32)
    rng, hit = scene.render_lidar(None, sens)
    torch.cuda.synchronize()
    assert float(rng.abs().max()) == 0.0 and float(hit.abs().max()) == 0.0
    bad = sens.copy()
    bad["elev_max"][1] = -1.0
    with pytest.raises(gsbatch.GsError) as ei:
        scene.render_lidar(None, bad)
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    bad = sens.copy()
    bad["cols"][1] = 64
    with pytest.raises(gsbatch.GsError):
        scene.render_lidar(None, bad)
    for a0, a1 in ((1.0, 1.0), (0.0, 7.0), (np.nan, 1.0)):  # empty, more than a turn, not finite
        bad = sens.copy()
        bad["az_min"][0], bad["az_max"][0] = a0, a1
        with pytest.raises(gsbatch.GsError) as ei:
            scene.render_lidar(None, bad)
        assert ei.value.status == gsbatch.GS_ERR_INVALID
    scene.close()


# ---------------------------------------------------------------- arbitrary rays

def _ray_sensors(E, rows=48, cols=64, seed=4):
    """Sensors whose (azimuth, beam) grid only bins the rays: +-0.65 rad both ways."""
    s = _sensors(E, rows=rows, cols=cols, seed=seed, az=(-0.65, 0.65))
    s["elev_min"], s["elev_max"] = -0.65, 0.65
    return s


def _oracle_rays(w, e, sen, dirs):
    bg, lk = w.background, w.links
    cat = lambda f: np.concatenate([getattr(bg, f), getattr(lk, f)])
    link_of = np.concatenate([np.full(bg.n, -1), np.repeat(np.arange(w.n_links), np.diff(w.link_offsets))])
    return lidar.render_rays(cat("mean"), cat("quat"), cat("log_scale"), cat("opacity"), link_of, w.link_poses[e],
                             dict(q_ws=sen["q_ws"].astype(float), t_ws=sen["t_ws"].astype(float),
                                  near=float(sen["near_range"])), dirs)


def _check_scan(g_r, g_h, ref, label):
    dh = np.abs(g_h - ref["hit"])
    both = (ref["hit"] >= 0.5) & (g_h >= 0.5)
    rel = np.abs(g_r - ref["range"])[both] / ref["range"][both]
    print(label, "rays hit >= 0.5:", int(both.sum()), "of", g_h.size, "hit max", dh.max(), "p99",
          np.quantile(dh, 0.99), "range rel max", rel.max() if rel.size else None)
    assert ref["hit"].max() > 0.5 and both.sum() > 20
    assert np.quantile(dh, 0.99) <= 2e-3 and dh.max() <= 0.05
    assert np.quantile(rel, 0.99) <= 1e-4 and rel.max() <= 1e-2


def test_rays_match_oracle():
    """A non-repetitive (rosette) scan pattern, a different phase per env,
    with the robot's links moving, against the FP64 ray-list oracle."""
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=2, width=64, height=48, f=50.0, n_bg=8_000, per_link=200)
    dirs = synth.rosette_rays(w.n_envs, 3000, seed=3)
    sens = _ray_sensors(w.n_envs)
    scene = gsbatch.scene_from_workload(w)
    rng, hit = scene.render_rays(torch.from_numpy(w.link_poses).cuda(), sens, torch.from_numpy(dirs).cuda())
    torch.cuda.synchronize()
    scene.sync_status()
    g_r, g_h = rng.cpu().numpy(), hit.cpu().numpy()
    scene.close()
    for e in range(w.n_envs):
        _check_scan(g_r[e], g_h[e], _oracle_rays(w, e, sens[e], dirs[e]), f"rays env {e}")


def test_rays_of_a_grid_scan_like_the_grid():
    """The rays of a rotating scan's grid, given as a list (shuffled), scan
    like the grid form within the FP32 rounding of their directions."""
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=2, width=64, height=48, f=50.0, n_bg=8_000, per_link=200)
    sens = _sensors(w.n_envs, rows=16, cols=128)
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    g_rng, g_hit = scene.render_lidar(poses, sens)
    D = lidar.ray_directions(16, 128, -0.5, 0.35).reshape(-1, 3)
    perm = np.random.default_rng(8).permutation(len(D))
    dirs = np.ascontiguousarray(np.broadcast_to(D[perm], (w.n_envs,) + D.shape), np.float32)
    r_rng, r_hit = scene.render_rays(poses, sens, torch.from_numpy(dirs).cuda())
    torch.cuda.synchronize()
    scene.sync_status()
    scene.close()
    g_r = g_rng.cpu().numpy().reshape(w.n_envs, -1)[:, perm]
    g_h = g_hit.cpu().numpy().reshape(w.n_envs, -1)[:, perm]
    for e in range(w.n_envs):
        _check_scan(r_rng.cpu().numpy()[e], r_hit.cpu().numpy()[e], {"range": g_r[e], "hit": g_h[e]},
                    f"grid rays env {e}")


def test_rays_outside_the_grid_and_argument_checks():
    """A zero direction and one outside the binning grid read 0 and set the
    status word; every other ray is bit-identical to the scan without them."""
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=2, width=64, height=48, f=50.0, n_bg=8_000, per_link=200)
    dirs = synth.rosette_rays(w.n_envs, 1000, seed=5)
    sens = _ray_sensors(w.n_envs)
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    r0, h0 = scene.render_rays(poses, sens, torch.from_numpy(dirs).cuda())
    torch.cuda.synchronize()
    scene.sync_status()
    bad = dirs.copy()
    bad[0, 10] = 0.0                  # zero direction
    bad[1, 20] = [-1.0, 0.0, 0.0]     # behind the sensor: outside the +-0.65 rad window
    r1, h1 = scene.render_rays(poses, sens, torch.from_numpy(bad).cuda())
    torch.cuda.synchronize()
    with pytest.raises(gsbatch.GsError) as ei:
        scene.sync_status()
    assert ei.value.status == gsbatch.GS_ERR_DEVICE
    r0, h0, r1, h1 = (t.cpu().numpy() for t in (r0, h0, r1, h1))
    assert r1[0, 10] == 0 and h1[0, 10] == 0 and r1[1, 20] == 0 and h1[1, 20] == 0
    keep = np.ones(r0.shape, bool)
    keep[0, 10] = keep[1, 20] = False
    np.testing.assert_array_equal(r1[keep], r0[keep])
    np.testing.assert_array_equal(h1[keep], h0[keep])
    with pytest.raises(gsbatch.GsError) as ei:  # no rays
        scene.render_rays(poses, sens, torch.zeros((w.n_envs, 0, 3), device="cuda"))
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    scene.close()
