"""Served form (row A8): the request loop.  Requests of different scenes and
resolutions, submitted with arrival times, are batched continuously on a pool
of CUDA streams under an HBM budget; every result must be bit-identical to
rendering its env alone."""
import numpy as np
import pytest

from gpu_helpers import ensure_built
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu

TILE = (16, 16)


def _setup(n_envs=12, n_scenes=2):
    w = synth.make_c4(n_scenes=n_scenes, n_envs=n_envs, seed=3, bg_range=(20_000, 40_000), per_link=300)
    scenes = []
    for k in range(n_scenes):
        s = gsbatch.Scene(w.backgrounds[k])
        s.attach_links(w.link_offsets, w.links)
        s.set_tile(*TILE)
        scenes.append(s)
    return w, scenes


def _alone(torch, scene, cam, poses, n_links):
    """The env rendered by itself through gs_render_batch_v."""
    envs = gsbatch.make_envs(np.asarray(cam).reshape(1), link_ranges=[[0, n_links]], pose_offsets=[0])
    H, W = int(cam["height"]), int(cam["width"])
    rgb = torch.full((H * W * 3,), -1.0, device="cuda")
    depth = torch.full((H * W,), -1.0, device="cuda")
    scene.render_v(envs, torch.from_numpy(np.ascontiguousarray(poses)).cuda(), rgb, depth)
    torch.cuda.synchronize()
    scene.sync_status()
    return rgb.view(H, W, 3).cpu(), depth.view(H, W).cpu()


def _server(w, scenes, **kw):
    sv = gsbatch.Server(tile=TILE, **kw)
    ids = [sv.add_scene(s) for s in scenes]
    for i in range(w.n_envs):
        assert sv.add_env(ids[int(w.env_scene[i])], w.cams[i], 0, w.n_links) == i
    return sv


def test_served_results_equal_each_env_alone():
    import torch

    ensure_built()
    w, scenes = _setup()
    E, L = w.n_envs, w.n_links
    assert len(set(int(x) for x in w.cams["width"])) >= 3
    pa = w.request_poses(E, stream=0)
    pb = w.request_poses(E, stream=1)
    second = [i for i in range(E) if i % 3 == 0]
    final = {i: (pb[i] if i in second else pa[i]) for i in range(E)}
    ref = {i: _alone(torch, scenes[int(w.env_scene[i])], w.cams[i], final[i][None], L) for i in range(E)}

    sv = _server(w, scenes, budget_bytes=8 << 30, max_inflight=3, max_batch_envs=4)
    first_ids = [sv.submit(i, pa[i], arrival_s=0.0) for i in range(E)]
    second_ids = {i: sv.submit(i, pb[i], arrival_s=0.02 + 0.003 * k) for k, i in enumerate(second)}
    sv.start()
    sv.drain(300.0)
    res = {r["request_id"]: r for r in sv.poll()}
    assert len(res) == E + len(second)
    for r in res.values():
        assert r["status"] == 0
        assert r["admit_s"] >= r["arrival_s"] - 1e-9 and r["done_s"] >= r["admit_s"]
    # an env's requests run one at a time, in submission order
    for i, rid in second_ids.items():
        assert res[rid]["admit_s"] >= res[first_ids[i]]["done_s"]
    st = sv.stats()
    print("serving stats", st)
    assert st["completed"] == E + len(second) and st["cancelled"] == 0
    # 12 requests of two scenes at t = 0, 3 slots, batches of <= 4: the first
    # admission pass fills every slot, so three batches overlap
    assert st["max_concurrent"] == 3 and st["max_batch"] == 4 and st["batches"] >= 4
    for i in range(E):
        rgb, depth = sv.env_output(i)
        assert torch.equal(rgb.cpu(), ref[i][0]), f"env {i} rgb"
        assert torch.equal(depth.cpu(), ref[i][1]), f"env {i} depth"
    sv.close()
    for s in scenes:
        s.close()


def test_budget_admission_serialises_batches():
    """A budget below one request's working set: each request runs alone, one
    batch at a time, and its result is unchanged."""
    import torch

    ensure_built()
    w, scenes = _setup(n_envs=6)
    E, L = w.n_envs, w.n_links
    pa = w.request_poses(E, stream=2)
    sv = _server(w, scenes, budget_bytes=1 << 20, max_inflight=4, max_batch_envs=8)
    for i in range(E):
        sv.submit(i, pa[i], arrival_s=0.0)
    sv.start()
    sv.drain(300.0)
    st = sv.stats()
    assert st["completed"] == E and st["batches"] == E
    assert st["max_concurrent"] == 1 and st["max_batch"] == 1
    for i in range(E):
        ref = _alone(torch, scenes[int(w.env_scene[i])], w.cams[i], pa[i][None], L)
        rgb, depth = sv.env_output(i)
        assert torch.equal(rgb.cpu(), ref[0]) and torch.equal(depth.cpu(), ref[1]), f"env {i}"
    sv.close()
    for s in scenes:
        s.close()


def test_cancel_and_argument_errors():
    ensure_built()
    w, scenes = _setup(n_envs=4)
    pa = w.request_poses(w.n_envs, stream=3)
    sv = _server(w, scenes, budget_bytes=4 << 30, max_inflight=2, max_batch_envs=4)
    late = sv.submit(1, pa[1], arrival_s=1e4)  # arrives long after the test
    sv.submit(0, pa[0], arrival_s=0.0)
    sv.start()
    with pytest.raises(gsbatch.GsError) as ei:
        sv.add_env(0, w.cams[0], 0, w.n_links)
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    with pytest.raises(gsbatch.GsError) as ei:
        sv.submit(99, pa[0])
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    sv.cancel(late)
    with pytest.raises(gsbatch.GsError):
        sv.cancel(late)
    sv.drain(300.0)
    res = {r["request_id"]: r for r in sv.poll()}
    assert res[late]["status"] == 1 and res[late]["admit_s"] < 0
    assert sv.stats()["cancelled"] == 1 and sv.stats()["completed"] == 1
    sv.close()
    for s in scenes:
        s.close()


def _in_front_of_camera(cam, n_links, dist=0.35):
    """Link poses that put every link just in front of the camera (far more
    intersections than the robot at its usual place)."""
    from scipy.spatial.transform import Rotation

    q = cam["q_cw"].astype(np.float64)
    t = cam["t_cw"].astype(np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    centre = -R.T @ t
    fwd = R.T @ np.array([0.0, 0.0, 1.0])
    p = np.zeros((n_links, 7), np.float32)
    p[:, 0] = 1.0
    p[:, 4:7] = centre + dist * fwd
    return p


def test_overflowing_estimate_is_rendered_again_exactly():
    """Once the key estimates are learned, requests that need far more keys
    overflow the planned capacity on the device; the scheduler renders those
    batches again, exactly, before completing them."""
    import torch

    ensure_built()
    w, scenes = _setup(n_envs=8)
    E, L = w.n_envs, w.n_links
    pa = w.request_poses(E, stream=4)
    sv = _server(w, scenes, budget_bytes=8 << 30, max_inflight=2, max_batch_envs=8)
    sv.start()
    for rep in range(2):  # learn the estimates (the first batch of each kind is sized exactly)
        for i in range(E):
            sv.submit(i, pa[i])
        sv.drain(300.0)
    st0 = sv.stats()
    near = {i: _in_front_of_camera(w.cams[i], L) for i in range(E)}
    for i in range(E):
        sv.submit(i, near[i])
    sv.drain(300.0)
    st = sv.stats()
    print("overflow stats", st)
    assert st["retried"] > st0["retried"]
    res = sv.poll(1 << 12)
    assert all(r["status"] == 0 for r in res)
    for i in range(E):
        ref = _alone(torch, scenes[int(w.env_scene[i])], w.cams[i], near[i][None], L)
        rgb, depth = sv.env_output(i)
        assert torch.equal(rgb.cpu(), ref[0]) and torch.equal(depth.cpu(), ref[1]), f"env {i}"
    sv.close()
    for s in scenes:
        s.close()
