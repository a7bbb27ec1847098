"""Batched uneven form (row A7): environments of different resolutions and
link subsets in one call (gs_render_batch_v), and plans (autotuned tile shape
and claim size, replayed from a captured CUDA graph, capacity regrowth)."""
import numpy as np
import pytest

from gpu_helpers import compare, ensure_built, gpu_render
from oracle import oracle
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


def _small_c3(n_envs=24):
    return synth.make_c3(n_envs=n_envs, n_bg=30_000, count_range=(1_000, 20_000), threads=4)


def _scene(w):
    s = gsbatch.Scene(w.background)
    s.attach_links(w.link_offsets, w.links)
    return s


def _outputs(torch, envs):
    npx = int((envs["cam"]["width"].astype(np.int64) * envs["cam"]["height"]).sum())
    return (torch.full((npx * 3,), -1.0, device="cuda"), torch.full((npx,), -1.0, device="cuda"),
            torch.full((npx,), -1.0, device="cuda"))


def _env_image(out, envs, e):
    c = envs["cam"][e]
    W, H, o = int(c["width"]), int(c["height"]), int(envs["pixel_offset"][e])
    rgb, depth, alpha = (t.cpu().numpy() for t in out)
    return (rgb[3 * o:3 * (o + W * H)].reshape(H, W, 3), depth[o:o + W * H].reshape(H, W),
            alpha[o:o + W * H].reshape(H, W))


def _c3_envs(w):
    E = w.n_envs
    return gsbatch.make_envs(w.cams, link_ranges=np.stack([np.arange(E), np.arange(E) + 1], 1),
                             pose_offsets=np.arange(E))


def test_render_v_equals_each_env_alone_and_oracle():
    import torch

    ensure_built()
    w = _small_c3()
    envs = _c3_envs(w)
    scene = _scene(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    out = _outputs(torch, envs)
    scene.render_v(envs, poses, *out)
    torch.cuda.synchronize()
    scene.sync_status()
    assert set(int(x) for x in w.cams["width"]) >= {64, 128, 320, 640}
    for e in range(w.n_envs):
        alone = gpu_render(w.env(e))
        got = _env_image(out, envs, e)
        for k, g in zip(("rgb", "depth", "alpha"), got):
            np.testing.assert_array_equal(g, alone[k][0], err_msg=f"env {e} {k}")
    for e in (0, 5, 11, 23):
        ref = oracle.render_env(w.env(e), 0)
        rgb, depth, alpha = _env_image(out, envs, e)
        st = compare(rgb, depth, alpha, ref)
        print("c3 env", e, w.cams["width"][e], st)
    scene.close()


def test_render_v_link_subsets_and_scattered_offsets():
    """Envs with no links, a shared link range and reversed output placement."""
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=4, width=96, height=72, f=75.0, n_bg=20_000, per_link=400)
    scene = gsbatch.scene_from_workload(w)
    base = gpu_render(w)
    L = w.n_links
    cams = w.cams
    envs = np.zeros(4, dtype=gsbatch.ENV_DTYPE)
    envs["cam"] = cams
    envs["link_begin"] = [0, 0, 0, 0]
    envs["link_end"] = [L, L, 0, L]
    envs["pose_offset"] = np.arange(4) * L
    px = 96 * 72
    envs["pixel_offset"] = [3 * px, 2 * px, px, 0]  # reversed placement
    out = _outputs(torch, envs)
    poses = torch.from_numpy(w.link_poses).cuda()
    scene.render_v(envs, poses, *out)
    torch.cuda.synchronize()
    for e in (0, 1, 3):
        got = _env_image(out, envs, e)
        for k, g in zip(("rgb", "depth", "alpha"), got):
            np.testing.assert_array_equal(g, base[k][e])
    # env 2 renders the background only
    bg_only = synth.Workload("bg", w.background, np.zeros(1, np.int64), w.links.slice(0, 0),
                             np.zeros((1, 0, 7), np.float32), cams[2:3].copy())
    ref = gpu_render(bg_only)
    got = _env_image(out, envs, 2)
    np.testing.assert_array_equal(got[0], ref["rgb"][0])
    scene.close()


def test_plan_autotune_graph_replay_and_regrow():
    import torch

    ensure_built()
    w = _small_c3(16)
    envs = _c3_envs(w)
    scene = _scene(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    ref = _outputs(torch, envs)
    out = _outputs(torch, envs)
    plan = scene.plan(envs, autotune=True, graph=True)
    for step in range(3):
        if step == 1:  # new poses written in place: the captured graph reads them
            p2 = w.link_poses.copy()
            p2[:, 4] += 0.05
            poses.copy_(torch.from_numpy(p2))
        plan.launch(poses, *out)
        scene.render_v(envs, poses, *ref)
        torch.cuda.synchronize()
        scene.sync_status()
        for a, b in zip(out, ref):
            assert torch.equal(a, b), f"step {step}"
    info = plan.info()
    print("plan", info)
    # 5 tile shapes x 2 claim sizes, plus the quadrant form on 16x16 and 8x8 tiles
    assert info["graph"] == 1 and info["tuned_candidates"] == 14
    assert (info["tile_w"], info["tile_h"]) in ((16, 16), (32, 8), (16, 8), (8, 8), (32, 16))
    assert info["quad"] in (0, 1) and (info["quad"] == 0 or info["tile_w"] == info["tile_h"])
    # objects pulled up to the cameras need far more keys than planned: the
    # replay drops keys and says so, the next launch regrows and is exact again
    p3 = w.link_poses.copy()
    cams = w.cams
    for e in range(w.n_envs):
        q = cams["q_cw"][e].astype(np.float64)
        t = cams["t_cw"][e].astype(np.float64)
        from scipy.spatial.transform import Rotation
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        centre = -R.T @ t
        fwd = R.T @ np.array([0.0, 0.0, 1.0])
        p3[e, 4:7] = centre + 0.35 * fwd
    poses.copy_(torch.from_numpy(p3))
    plan.launch(poses, *out)
    with pytest.raises(gsbatch.GsError) as ei:
        scene.sync_status()
    assert ei.value.status == gsbatch.GS_ERR_DEVICE and "capacity" in str(ei.value)
    plan.launch(poses, *out)
    scene.render_v(envs, poses, *ref)
    torch.cuda.synchronize()
    scene.sync_status()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    assert plan.info()["regrows"] == 1
    plan.close()
    scene.close()
