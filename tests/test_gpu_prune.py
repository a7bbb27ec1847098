"""Contribution pass and pruning (scene transform): per-Gaussian summed
blending weights from the GPU against the oracle's, and the pruned scene."""
import numpy as np
import pytest

from gpu_helpers import ensure_built, gpu_render, psnr
from oracle import oracle
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


def _scores(w):
    import torch

    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda() if w.n_links > 0 else None
    sc = scene.contribution(poses, w.cams)
    torch.cuda.synchronize()
    scene.sync_status()
    scene.close()
    return sc.cpu().numpy().astype(np.float64)


def _oracle_scores(w):
    S = oracle.scene_arrays(w)
    tot = np.zeros(S.n, np.float64)
    alpha = 0.0
    for e in range(w.n_envs):
        ref = oracle.render_env(w, e, S=S, contrib=True)
        tot += ref["contrib"]
        alpha += ref["alpha"].astype(np.float64).sum()
    return tot, alpha


@pytest.mark.parametrize("name", ["c0", "robot"])
def test_contribution_matches_oracle(name):
    ensure_built()
    if name == "c0":
        w = synth.make_c0()
    else:
        w = synth.make_c1(n_envs=3, width=96, height=72, f=75.0, n_bg=20_000, per_link=500)
    got = _scores(w)
    ref, alpha_sum = _oracle_scores(w)
    assert got.shape == ref.shape
    # the weights telescope: their total is the covered area
    assert abs(got.sum() - alpha_sum) <= 1e-4 * alpha_sum
    # per Gaussian: FP32 vs FP64 weights, plus rare threshold flips
    big = ref > 0.05
    rel = np.abs(got[big] - ref[big]) / ref[big]
    print(name, "Gaussians with weight > 0.05:", int(big.sum()), "max rel", rel.max(), "p99", np.quantile(rel, 0.99))
    assert np.quantile(rel, 0.99) < 1e-3 and rel.max() < 0.05
    assert np.abs(got - ref).max() < 0.05
    # ranking: the top 30 % sets agree
    k = int(0.3 * len(ref))
    a = set(np.argsort(-ref)[:k].tolist())
    b = set(np.argsort(-got)[:k].tolist())
    assert len(a & b) >= 0.99 * k


def test_pruned_scene_renders_and_reports_error():
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=4, width=96, height=72, f=75.0, n_bg=40_000, per_link=1000)
    scores = _scores(w)
    p = gsbatch.prune_workload(w, scores, keep_bg=0.3, keep_links=0.1)
    assert p.background.n == int(np.ceil(0.3 * w.background.n))
    assert p.links.n == sum(int(np.ceil(0.1 * 1000)) for _ in range(w.n_links))
    assert (np.diff(p.link_offsets) == 100).all()
    full = gpu_render(w)
    pr = gpu_render(p)
    S = oracle.scene_arrays(w)
    for e in range(w.n_envs):
        ref = oracle.render_env(w, e, S=S)
        print("pruned env", e, "PSNR vs unpruned oracle", psnr(pr["rgb"][e], ref["rgb"]),
              "unpruned", psnr(full["rgb"][e], ref["rgb"]))
    torch.cuda.synchronize()
