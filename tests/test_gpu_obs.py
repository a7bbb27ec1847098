"""Observation form (fused epilogue): 8-bit RGB after per-env appearance
randomisation (exposure, contrast, brightness; Sec. IV-E) and half depth,
written by the compositor."""
import numpy as np
import pytest

from gpu_helpers import ensure_built
from oracle import oracle
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


def _workload():
    return synth.make_c1(n_envs=6, width=96, height=72, f=75.0, n_bg=40_000, per_link=1000)


def _appearance(E, seed=5):
    rng = np.random.default_rng([seed, 77])
    return np.stack([rng.uniform(-0.5, 0.5, E), rng.uniform(0.7, 1.3, E), rng.uniform(-0.1, 0.1, E)],
                    1).astype(np.float32)


def test_identity_observation_equals_quantised_float_render():
    """With no appearance change, rgb8 = round-half-even(255 c) of the float
    render's (clamped) colour in FP32 and depth16 = half(depth), bit for bit."""
    import torch

    ensure_built()
    w = _workload()
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    rgb, depth, _ = scene.render(poses, w.cams, want_alpha=False)
    rgb8, d16 = scene.render_obs(poses, w.cams)
    torch.cuda.synchronize()
    scene.sync_status()
    ref8 = np.rint(rgb.cpu().numpy().astype(np.float32) * np.float32(255.0)).astype(np.uint8)
    np.testing.assert_array_equal(rgb8.cpu().numpy(), ref8)
    np.testing.assert_array_equal(d16.cpu().numpy(), depth.cpu().numpy().astype(np.float16))
    scene.close()


def test_randomised_appearance_against_oracle_and_host_path():
    import torch

    ensure_built()
    w = _workload()
    E = w.n_envs
    ap = _appearance(E)
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    rgb8, d16 = scene.render_obs(poses, w.cams, appearance=torch.from_numpy(ap).cuda())
    torch.cuda.synchronize()
    scene.sync_status()
    g8, gd = rgb8.cpu().numpy(), d16.cpu().numpy()
    # host buffers (pageable: staged; page-locked: written directly): the same bytes
    h8 = np.zeros_like(g8)
    hd = np.zeros_like(gd)
    scene.render_obs_host(w.link_poses, w.cams, ap, h8, hd)
    np.testing.assert_array_equal(h8, g8)
    np.testing.assert_array_equal(hd, gd)
    p8 = torch.zeros(g8.shape, dtype=torch.uint8).pin_memory().numpy()
    pd = torch.zeros(gd.shape, dtype=torch.float16).pin_memory().numpy()
    scene.render_obs_host(w.link_poses, w.cams, ap, p8, pd)
    np.testing.assert_array_equal(p8, g8)
    np.testing.assert_array_equal(pd, gd)
    # against the FP64 oracle: the colour differs by < 2e-3 before quantisation,
    # so the 8-bit value by at most one step (non-ambiguous pixels)
    S = oracle.scene_arrays(w)
    for e in (0, 3, 5):
        ref = oracle.render_env(w, e, S=S)
        o8, od = oracle.observation(ref["rgb"], ref["depth"], ap[e])
        ok = ref["amb"] == 0
        diff = np.abs(g8[e].astype(int) - o8.astype(int))
        assert diff[ok].max() <= 1, (e, diff[ok].max())
        assert (diff[ok] == 0).mean() > 0.97, (e, (diff[ok] == 0).mean())
        both = ok & (ref["alpha"] >= 0.5)
        rel = np.abs(gd[e].astype(np.float64) - od.astype(np.float64)) / np.maximum(od.astype(np.float64), 1e-6)
        assert rel[both].max() <= 2 ** -10, (e, rel[both].max())  # one half-precision step
    scene.close()


def test_empty_scene_and_no_depth():
    """An empty scene gives every pixel the transform of black; depth16 may be
    omitted."""
    import torch

    ensure_built()
    bg = synth.make_gaussians_uniform_cube(0, 0)
    cams = synth.make_cameras(3, 30.0, 30.0, 16.0, 12.0, 32, 24, [[1, 0, 0, 0]] * 3, [[0, 0, 3.0]] * 3)
    scene = gsbatch.Scene(bg)
    ap = np.array([[0.0, 1.0, 0.0], [0.3, 0.5, 0.2], [0.0, 2.0, -0.4]], np.float32)
    rgb8, _ = scene.render_obs(None, cams, appearance=torch.from_numpy(ap).cuda(), want_depth=False)
    torch.cuda.synchronize()
    got = rgb8.cpu().numpy()
    for e in range(3):
        o8, _ = oracle.observation(np.zeros((24, 32, 3)), np.zeros((24, 32)), ap[e])
        np.testing.assert_array_equal(got[e], o8)
    scene.close()
