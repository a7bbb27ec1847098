"""Full-size configurations, in the launch configurations bench.py times, on
sampled envs: the precision form at 2048 envs (both resolutions, BF16 and
FP16 storage) and the batched uneven form at 4096 envs through an autotuned,
graph-replayed plan."""
import numpy as np
import pytest

from gpu_helpers import compare, ensure_built, gpu_render, keyed_check, oracle_env, psnr
from oracle import oracle
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("res", ["128x128", "640x480"])
def test_precision_form_full_batch(res):
    import torch

    ensure_built()
    w = synth.make_c2(n_envs=2048, res=res)
    E = w.n_envs
    H, W = int(w.cams["height"][0]), int(w.cams["width"][0])
    poses = torch.from_numpy(w.link_poses).cuda()
    sampled = [0, 1023, 2047]
    strict = {e: oracle_env(w, e) for e in sampled}
    for dtype in ("f16", "bf16"):
        scene = gsbatch.scene_from_workload(w, dtype)
        rgb, depth, alpha = scene.render(poses, w.cams)
        torch.cuda.synchronize()
        scene.sync_status()
        for e in sampled:
            ref = strict[e]
            got = rgb[e].cpu().numpy()
            ok = ref["amb"] == 0
            err = np.abs(got - ref["rgb"]).max(axis=-1)
            p = psnr(got, ref["rgb"])
            print(f"{dtype} {res} env {e}: PSNR {p:.2f} dB, max abs (non-ambiguous) {err[ok].max():.2e}")
            assert p >= 45.0
            if dtype == "f16":
                assert err[ok].max() <= 8e-3
        assert rgb.shape == (E, H, W, 3)
        scene.close()


def test_batched_uneven_full_plan():
    """c3 at 4096 envs: one autotuned plan replayed from its CUDA graph, as
    bench.py --workload c3 times it; sampled envs of every resolution against
    the oracle."""
    import torch

    ensure_built()
    w = synth.make_c3(n_envs=4096, threads=16)
    E = w.n_envs
    scene = gsbatch.Scene(w.background)
    scene.attach_links(w.link_offsets, w.links)
    envs = gsbatch.make_envs(w.cams, link_ranges=np.stack([np.arange(E), np.arange(E) + 1], 1),
                             pose_offsets=np.arange(E))
    npx = int((w.cams["width"].astype(np.int64) * w.cams["height"]).sum())
    rgb = torch.empty(npx * 3, device="cuda")
    depth = torch.empty(npx, device="cuda")
    alpha = torch.empty(npx, device="cuda")
    poses = torch.from_numpy(w.link_poses).cuda()
    plan = scene.plan(envs, autotune=True, graph=True)
    for _ in range(2):  # tuning launch, then a graph replay
        plan.launch(poses, rgb, depth, alpha)
    torch.cuda.synchronize()
    scene.sync_status()
    assert plan.info()["graph"] == 1
    widths = w.cams["width"]
    sampled = sorted({0, E - 1} | {int(np.nonzero(widths == W)[0][-1]) for W in np.unique(widths)})
    for e in sampled:
        c = w.cams[e]
        Wd, Hd, o = int(c["width"]), int(c["height"]), int(envs["pixel_offset"][e])
        got_rgb = rgb[3 * o:3 * (o + Wd * Hd)].view(Hd, Wd, 3).cpu().numpy()
        got_d = depth[o:o + Wd * Hd].view(Hd, Wd).cpu().numpy()
        got_a = alpha[o:o + Wd * Hd].view(Hd, Wd).cpu().numpy()
        ref = oracle.render_env(w.env(e), 0)
        st = compare(got_rgb, got_d, got_a, ref)
        print("c3 full env", e, Wd, st)
        assert st["amb_frac"] < 0.2
        # keyed: the env alone in debug mode equals its plan output bit for bit,
        # and orders like the oracle fed its float32 depth keys
        one = w.env(e)
        alone = gpu_render(one, debug=True, keep_scene=True)
        for k, g in (("rgb", got_rgb), ("depth", got_d), ("alpha", got_a)):
            np.testing.assert_array_equal(alone[k][0], g, err_msg=f"env {e} {k}: plan vs alone")
        _, st_k, _, _ = keyed_check(one, 0, alone)
        alone["scene"].close()
        print("  keyed", st_k)
        assert st_k["amb_frac"] < 0.2
    plan.close()
    scene.close()
