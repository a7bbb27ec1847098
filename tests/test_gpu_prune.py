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


def _top(scores, n_bg, offs, keep_bg, keep_links):
    """Reference selection: per group (background, each link) the top
    ceil(f n) by descending score, equal scores by ascending index, returned
    in the original order (background, then link-major)."""
    def top(sc, frac, base):
        k = min(len(sc), int(np.ceil(frac * len(sc))))
        order = np.lexsort((np.arange(len(sc)), -sc.astype(np.float64)))
        return base + np.sort(order[:k])
    parts = [top(scores[:n_bg], keep_bg, 0)]
    for l in range(len(offs) - 1):
        parts.append(top(scores[n_bg + offs[l]:n_bg + offs[l + 1]], keep_links, n_bg + offs[l]))
    return np.concatenate(parts)


@pytest.mark.parametrize("source", ["oracle_c0", "gpu_robot"])
def test_prune_selection_in_the_library(source):
    """gs_scene_prune keeps exactly the top fractions of the given scores
    (here the oracle's contribution ranking on c0, rounded to float32, or the
    GPU's own on a robot scene), per group, in the original order; the new
    scene's link offsets count the kept Gaussians of each link."""
    import torch

    ensure_built()
    if source == "oracle_c0":
        w = synth.make_c0()
        scores = _oracle_scores(w)[0].astype(np.float32)
    else:
        w = synth.make_c1(n_envs=3, width=96, height=72, f=75.0, n_bg=20_000, per_link=500)
        scores = _scores(w).astype(np.float32)
    offs = np.asarray(w.link_offsets, np.int64)
    scene = gsbatch.scene_from_workload(w)
    for kb, kl in ((0.3, 0.1), (0.0, 1.0), (1.0, 0.0), (0.77, 0.5)):
        sub, kept = scene.prune(torch.from_numpy(scores).cuda(), kb, kl)
        np.testing.assert_array_equal(kept, _top(scores, w.background.n, offs, kb, kl))
        assert sub.n_background == min(w.background.n, int(np.ceil(kb * w.background.n)))
        sub.close()
    bad = scores.copy()
    bad[3] = np.nan
    with pytest.raises(gsbatch.GsError) as ei:
        scene.prune(torch.from_numpy(bad).cuda(), 0.3, 0.1)
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    with pytest.raises(gsbatch.GsError) as ei:
        scene.prune(torch.from_numpy(scores).cuda(), 1.5, 0.1)
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    scene.close()


def test_pruned_scene_renders_and_reports_error():
    """The pruned scene renders bit for bit like a scene built from the kept
    Gaussians (its attributes are gathered from the source scene's), and its
    error against the unpruned FP64 oracle is reported."""
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=4, width=96, height=72, f=75.0, n_bg=40_000, per_link=1000)
    scores = _scores(w)
    p, pscene = gsbatch.prune_workload(w, scores, keep_bg=0.3, keep_links=0.1)
    assert p.background.n == int(np.ceil(0.3 * w.background.n))
    assert p.links.n == sum(int(np.ceil(0.1 * 1000)) for _ in range(w.n_links))
    assert (np.diff(p.link_offsets) == 100).all()
    direct = gpu_render(p, scene=pscene)
    pscene.close()
    pr = gpu_render(p)
    for k in ("rgb", "depth", "alpha"):
        np.testing.assert_array_equal(direct[k], pr[k])
    full = gpu_render(w)
    S = oracle.scene_arrays(w)
    for e in range(w.n_envs):
        ref = oracle.render_env(w, e, S=S)
        print("pruned env", e, "PSNR vs unpruned oracle", psnr(pr["rgb"][e], ref["rgb"]),
              "unpruned", psnr(full["rgb"][e], ref["rgb"]))
    torch.cuda.synchronize()
