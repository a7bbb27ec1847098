"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: per-channel max abs <= 2e-3 on [0,1] images and depth relative
error <= 1e-4 where alpha >= 0.5 (FP32 path vs FP64 oracle); binning counts and
per-tile depth-ordered lists bit-exact when the oracle is fed the GPU's keys.
Pixels whose result sits on a threshold within FP32 noise (alpha at 1/255,
T at 1e-4, depth near-ties) are excluded and counted, never hidden.
"""
import numpy as np
import pytest

from gpu_helpers import (compare, ensure_built, gpu_render, keyed_check, oracle_env, render_counted)
from oracle import oracle
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    ensure_built()


def _keyed_check(w, e, out, sh_degree=3):
    return keyed_check(w, e, out, sh_degree)


def test_c0_parity_independent_and_keyed():
    w = synth.make_c0()
    out = gpu_render(w, debug=True, keep_scene=True)
    st_i, st_k, rec, proj = _keyed_check(w, 0, out)
    out["scene"].close()
    print("c0 independent", st_i, "keyed", st_k)
    # the alpha flag window (|alpha - 1/255| <= 1e-3/255) covers ~6e-3 sigma^2 px per splat
    assert st_k["amb_frac"] < 0.1


def test_c0_projection_records():
    """Per-Gaussian records vs the FP64 projection (steps 1-7)."""
    w = synth.make_c0()
    out = gpu_render(w, debug=True, keep_scene=True)
    rec = out["scene"].debug_records(0, w.background.n)
    out["scene"].close()
    S = oracle.scene_arrays(w)
    p = oracle.project(S, w.link_poses[0], w.cams[0])
    vis_g, vis_o = rec["visible"] == 1, p["valid"] == 1
    both = vis_g & vis_o
    # visibility may differ only for supports whose box edge sits on a pixel boundary (rare)
    diff = np.nonzero(vis_g != vis_o)[0]
    assert len(diff) <= max(2, 1e-3 * both.sum())
    np.testing.assert_allclose(rec["u"][both], p["u"][both], atol=2e-3)
    np.testing.assert_allclose(rec["v"][both], p["v"][both], atol=2e-3)
    np.testing.assert_allclose(rec["z"][both], p["z"][both], rtol=2e-6)
    np.testing.assert_allclose(rec["rgb"][both], p["rgb"][both], atol=2e-5)
    np.testing.assert_allclose(rec["conic"][both], p["conic"][both], rtol=2e-3, atol=1e-5)
    np.testing.assert_allclose(rec["hx"][both] / 1.0001, p["hx"][both], rtol=1e-4)
    np.testing.assert_allclose(rec["hy"][both] / 1.0001, p["hy"][both], rtol=1e-4)
    np.testing.assert_allclose(rec["opacity"][both], p["opacity"][both], rtol=1e-7)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8), (16, 8), (32, 16)])
def test_binning_keyed_bit_exact(tile):
    """Counts and depth-ordered per-tile lists equal the binning oracle fed the
    GPU's (u, v, hx, hy, depth bits, index), for a scene whose dense tiles have
    lists longer than the compositor's shared-memory window."""
    w = synth.make_c1(n_envs=2, width=160, height=120, f=125.0, n_bg=60_000, per_link=2000)
    out = gpu_render(w, tile=tile, debug=True, keep_scene=True)
    scene = out["scene"]
    W, H = 160, 120
    ntiles = (-(-W // tile[0])) * (-(-H // tile[1]))
    for e in range(w.n_envs):
        rec = scene.debug_records(e, w.background.n + w.links.n)
        vis = np.nonzero(rec["visible"])[0]
        counts, lists = scene.debug_tiles(e, ntiles)
        oc, ol = oracle.bin_records(rec["u"][vis], rec["v"][vis], rec["hx"][vis], rec["hy"][vis],
                                    rec["z"][vis].view(np.uint32), vis.astype(np.uint32), W, H, *tile)
        np.testing.assert_array_equal(counts.astype(np.int64), oc)
        np.testing.assert_array_equal(lists, ol)
        assert counts.max() > 2048  # the windowed depth selection was exercised
    scene.close()


def test_long_lists_parity():
    """Dense robot tiles (lists far longer than one shared-memory window)."""
    w = synth.make_c1(n_envs=2, width=160, height=120, f=125.0, n_bg=60_000, per_link=2000)
    out = gpu_render(w, debug=True, keep_scene=True)
    for e in range(w.n_envs):
        st_i, st_k, _, _ = _keyed_check(w, e, out)
        print("long lists env", e, st_i, st_k)
    out["scene"].close()


def test_tile_shape_and_batch_invariance_bit_exact():
    """Results do not depend on the tile shape, on the wave size, or on which
    other envs share the batch."""
    w = synth.make_c1(n_envs=6, width=96, height=72, f=75.0, n_bg=40_000, per_link=1000)
    base = gpu_render(w)
    for tile in ((8, 8), (32, 8), (16, 8), (32, 16)):
        o = gpu_render(w, tile=tile)
        for k in ("rgb", "depth", "alpha"):
            np.testing.assert_array_equal(o[k], base[k], err_msg=f"{k} {tile}")
    o = gpu_render(w, wave=2)
    for k in ("rgb", "depth", "alpha"):
        np.testing.assert_array_equal(o[k], base[k])
    alone = gpu_render(w, envs=[3])
    for k in ("rgb", "depth", "alpha"):
        np.testing.assert_array_equal(alone[k][0], base[k][3])


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_match_device(pinned):
    """Host outputs: page-locked buffers are written by the compositor
    directly, pageable ones through device staging and copies; both equal the
    device render."""
    import torch

    w = synth.make_c1(n_envs=5, width=64, height=48, f=50.0, n_bg=20_000, per_link=500)
    base = gpu_render(w)
    scene = gsbatch.scene_from_workload(w)
    scene.set_wave(2)
    E, H, W = 5, 48, 64
    if pinned:
        rgb = torch.empty((E, H, W, 3)).pin_memory().numpy()
        depth = torch.empty((E, H, W)).pin_memory().numpy()
        alpha = torch.empty((E, H, W)).pin_memory().numpy()
    else:
        rgb = np.empty((E, H, W, 3), np.float32)
        depth = np.empty((E, H, W), np.float32)
        alpha = np.empty((E, H, W), np.float32)
    scene.render_host(np.ascontiguousarray(w.link_poses), w.cams, rgb, depth, alpha)
    scene.close()
    np.testing.assert_array_equal(rgb, base["rgb"])
    np.testing.assert_array_equal(depth, base["depth"])
    np.testing.assert_array_equal(alpha, base["alpha"])


def test_c1_full_batch_sampled_envs():
    """The benchmark's workload (2048 envs x 640x480, 600k Gaussians, default
    launch configuration), sampled envs 0, 1023, 2047:
    - each env rendered inside the full batch equals the env rendered alone,
      bit for bit (so the single-env debug and counting renders below speak
      for the batch);
    - against the FP64 oracle, independently and keyed (ordering by the GPU's
      float32 depth keys: no pixel may be excluded for a depth near-tie),
      every pixel within tolerance, ambiguous ones within the bound of their
      flagged decisions; the flagged fraction per decision is printed;
    - the composited-pair count (N_eval, the numerator of the compositor's
      roofline) equals the oracle's count up to flipped decisions."""
    w = synth.make_c1()
    out = gpu_render(w)
    for e in (0, 1023, 2047):
        one = w.env(e)
        alone = gpu_render(one, debug=True, keep_scene=True)
        for k in ("rgb", "depth", "alpha"):
            np.testing.assert_array_equal(alone[k][0], out[k][e], err_msg=f"env {e} {k}: batch vs alone")
        st_i, st_k, _, _ = keyed_check(one, 0, alone)
        alone["scene"].close()
        cnt = render_counted(one)
        n_gpu, n_or = cnt["stats"]["composited"], st_i["neval"]
        print(f"c1 env {e} independent {st_i}\n  keyed {st_k}\n  N_eval gpu {n_gpu} oracle {n_or} "
              f"rel {abs(n_gpu - n_or) / n_or:.2e}")
        assert st_k["amb_frac"] < 0.2
        assert abs(n_gpu - n_or) <= 1e-3 * n_or


def test_fp64_conic_branch_edge_on_discs():
    """Thin discs (scale ratio 1e-4) seen edge-on at depths 0.7 to 8 m
    project to near-degenerate 2D covariances (AC - B^2 far below 2^-10 AC
    before the low-pass), the one case the projection inverts in FP64: the
    counter sees every visible disc take that branch, and records and image
    match the FP64 oracle."""
    import math

    from scipy.spatial.transform import Rotation

    rng = np.random.default_rng(17)
    W, H, f = 96, 80, 70.0
    n = 24
    z = np.concatenate([np.full(8, 0.7), np.full(8, 3.0), np.full(8, 8.0)])
    uv = rng.uniform([10, 10], [W - 10, H - 10], size=(n, 2))
    mean = np.stack([(uv[:, 0] - W / 2) * z / f, (uv[:, 1] - H / 2) * z / f, z], 1)
    quat = np.zeros((n, 4))
    for k in range(n):
        d = mean[k] / np.linalg.norm(mean[k])
        a = rng.normal(size=3)
        nrm = np.cross(d, a)
        nrm /= np.linalg.norm(nrm)  # disc normal perpendicular to the view ray: edge-on
        r, _ = Rotation.align_vectors([nrm], [[0.0, 0.0, 1.0]])
        q = r.as_quat()
        quat[k] = [q[3], q[0], q[1], q[2]]
    thick = np.log(np.where(z < 1, 0.03, 0.15))
    ls = np.stack([thick, thick, thick + math.log(1e-4)], 1)
    sh = rng.normal(0, 0.3, size=(n, 16, 3))
    sh[:, 0, :] += 0.5
    bg = synth.Gaussians(*(np.ascontiguousarray(a, np.float32) for a in
                           (mean, quat, ls, rng.uniform(0.5, 0.95, n), sh)))
    cams = synth.make_cameras(1, f, f, W / 2, H / 2, W, H, [[1, 0, 0, 0]], [[0, 0, 0]])
    w = synth.Workload("discs", bg, np.zeros(1, np.int64), bg.slice(0, 0), np.zeros((1, 0, 7), np.float32), cams)
    cnt = render_counted(w)
    vis = cnt["stats"]["visible"]
    print("edge-on discs: visible", vis, "FP64 conics", cnt["stats"]["fp64_conics"])
    assert vis == n and cnt["stats"]["fp64_conics"] == n
    out = gpu_render(w, debug=True, keep_scene=True)
    np.testing.assert_array_equal(out["rgb"], cnt["rgb"])
    rec = out["scene"].debug_records(0, n)
    st_i, st_k, _, p = keyed_check(w, 0, out)
    out["scene"].close()
    print("edge-on discs independent", st_i, "keyed", st_k)
    both = (rec["visible"] == 1) & (p["valid"] == 1)
    assert both.sum() == n
    # the conic's small eigenvalue comes from the 0.3 px^2 low-pass: relative accuracy on every entry
    np.testing.assert_allclose(rec["conic"][both], p["conic"][both], rtol=2e-3, atol=1e-5)
    A, B, C = p["cov2d"][:, 0], p["cov2d"][:, 1], p["cov2d"][:, 2]
    Ar, Cr = A - 0.3, C - 0.3
    assert np.all(Ar * Cr - B * B < 2.0 ** -10 * Ar * Cr)


# ---------------------------------------------------------------- edge cases

def test_edge_empty_and_degenerate():
    import torch

    ensure_built()
    w = synth.make_tiny(seed=3, n_envs=2)
    scene = gsbatch.scene_from_workload(w)
    # zero envs: no-op
    cams0 = w.cams[:0]
    r = scene.render(None, cams0, want_alpha=True)
    assert r[0].shape[0] == 0
    # camera looking away: nothing visible -> black, alpha 0, depth 0
    cams = w.cams.copy()
    cams["q_cw"] = [[0.0, 0.0, 1.0, 0.0]] * 2  # 180 deg about y, same camera centre
    pos = -w.cams["t_cw"].astype(np.float64)  # centres (the original rotations are identity)
    cams["t_cw"] = np.stack([pos[:, 0], -pos[:, 1], pos[:, 2]], 1)  # t = -R_y(180) pos
    rgb, depth, alpha = scene.render(torch.from_numpy(w.link_poses).cuda(), cams)
    torch.cuda.synchronize()
    assert float(rgb.abs().max()) == 0 and float(alpha.max()) == 0 and float(depth.max()) == 0
    scene.close()
    # no Gaussians at all
    empty = synth.Workload("empty", w.background.slice(0, 0), np.zeros(1, np.int64), w.links.slice(0, 0),
                           np.zeros((2, 0, 7), np.float32), w.cams)
    s2 = gsbatch.scene_from_workload(empty)
    rgb, depth, alpha = s2.render(None, w.cams)
    torch.cuda.synchronize()
    assert float(rgb.abs().max()) == 0
    s2.close()


@pytest.mark.parametrize("wh", [(1, 1), (37, 29), (17, 3)])
def test_edge_ragged_resolutions(wh):
    W, H = wh
    w = synth.make_tiny(seed=6, n_envs=2, width=W, height=H, f=max(W, H) * 0.9)
    out = gpu_render(w)
    for e in range(2):
        compare(out["rgb"][e], out["depth"][e], out["alpha"][e], oracle_env(w, e))


def test_invalid_arguments_rejected_before_launch():
    import torch

    ensure_built()
    w = synth.make_tiny(seed=1, n_envs=2)
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    bad = w.cams.copy()
    bad["fx"][1] = 0.0
    with pytest.raises(gsbatch.GsError) as ei:
        scene.render(poses, bad)
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    bad = w.cams.copy()
    bad["width"][1] = 33
    with pytest.raises(gsbatch.GsError) as ei:
        scene.render(poses, bad)
    assert ei.value.status == gsbatch.GS_ERR_INVALID
    with pytest.raises(gsbatch.GsError):
        scene.set_tile(12, 12)
    # a zero link quaternion is found on the device and reported by the status word
    p2 = w.link_poses.copy()
    p2[0, 0, :4] = 0
    scene.render(torch.from_numpy(p2).cuda(), w.cams)
    with pytest.raises(gsbatch.GsError) as ei:
        scene.sync_status()
    assert ei.value.status == gsbatch.GS_ERR_DEVICE
    scene.sync_status()  # cleared
    scene.close()


def test_scene_with_zero_quaternion_rejected():
    ensure_built()
    w = synth.make_tiny(seed=1)
    bg = w.background
    q = bg.quat.copy()
    q[3] = 0
    bad = synth.Gaussians(bg.mean, q, bg.log_scale, bg.opacity, bg.sh)
    with pytest.raises(gsbatch.GsError) as ei:
        gsbatch.Scene(bad)
    assert ei.value.status == gsbatch.GS_ERR_INVALID


def test_background_storage_order():
    """The scene stores its background in Morton order of the means (a layout
    choice of the library): the order is a permutation whose codes do not
    decrease, and a caller-side shuffle of the background changes neither the
    images (up to pixels where two splats of exactly equal depth swap: ties
    follow the caller's global index) nor the per-Gaussian contribution
    scores, which stay in the caller's order."""
    import torch

    w = synth.make_c1(n_envs=2, width=160, height=120, f=125.0, n_bg=60_000, per_link=2000)
    scene = gsbatch.scene_from_workload(w)
    order = scene.storage_order()
    nb = w.background.n
    assert sorted(order.tolist()) == list(range(nb))
    m = w.background.mean.astype(np.float32)
    lo, hi = m.min(0), m.max(0)
    t = (m - lo).astype(np.float64) / (hi.astype(np.float64) - lo.astype(np.float64)) * 1023.0
    q = np.clip(t, 0.0, 1023.0).astype(np.int64)
    code = np.zeros(nb, np.int64)
    for b in range(10):
        for k in range(3):
            code |= ((q[:, k] >> b) & 1) << (3 * b + k)
    assert np.all(np.diff(code[order]) >= 0)
    poses = torch.from_numpy(w.link_poses).cuda()
    rgb, depth, _ = scene.render(poses, w.cams)
    sc = scene.contribution(poses, w.cams)
    torch.cuda.synchronize()
    scene.sync_status()
    rgb, depth, sc = rgb.cpu().numpy(), depth.cpu().numpy(), sc.cpu().numpy()
    scene.close()

    perm = np.random.default_rng(5).permutation(nb)
    bg = w.background
    shuffled = synth.Gaussians(*[np.ascontiguousarray(getattr(bg, f)[perm])
                                 for f in ("mean", "quat", "log_scale", "opacity", "sh")])
    w2 = synth.Workload(w.name, shuffled, w.link_offsets, w.links, w.link_poses, w.cams)
    scene2 = gsbatch.scene_from_workload(w2)
    rgb2, depth2, _ = scene2.render(poses, w.cams)
    sc2 = scene2.contribution(poses, w.cams)
    torch.cuda.synchronize()
    scene2.sync_status()
    rgb2, depth2, sc2 = rgb2.cpu().numpy(), depth2.cpu().numpy(), sc2.cpu().numpy()
    scene2.close()
    same = np.all(rgb == rgb2, axis=-1) & (depth == depth2)
    print("pixels bit-identical after a caller-side shuffle:", same.mean())
    assert same.mean() >= 0.999
    back = np.empty(nb, sc2.dtype)
    back[perm] = sc2[:nb]
    # (equal scores up to the order of the float atomic adds)
    np.testing.assert_allclose(back, sc[:nb], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(sc2[nb:], sc[nb:], rtol=1e-4, atol=1e-5)


def test_equal_depth_ties_follow_global_index():
    """Two background splats at exactly the same camera depth, overlapping,
    whose Morton storage order (left one first) is the reverse of their global
    order: where both are blended, the lower global index composites first,
    as in the oracle."""
    import math

    import torch

    z, W, H, f = 2.0, 32, 32, 40.0
    mean = np.array([[0.06, 0.0, z], [-0.06, 0.0, z]], np.float32)  # index 0 right, index 1 left
    n = 2
    sh = np.zeros((n, 16, 3), np.float32)
    y0 = 0.5 / math.sqrt(math.pi)
    sh[0, 0, :] = (np.array([1.0, 0.0, 0.0]) - 0.5) / y0  # red
    sh[1, 0, :] = (np.array([0.0, 0.0, 1.0]) - 0.5) / y0  # blue
    bg = synth.Gaussians(mean, np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                         np.full((n, 3), math.log(0.08), np.float32), np.full(n, 0.6, np.float32), sh)
    cams = synth.make_cameras(1, f, f, W / 2, H / 2, W, H, [[1, 0, 0, 0]], [[0, 0, 0]])
    w = synth.Workload("ties", bg, np.zeros(1, np.int64), bg.slice(0, 0), np.zeros((1, 0, 7), np.float32), cams)
    scene = gsbatch.Scene(w.background)
    assert scene.storage_order().tolist() == [1, 0]  # the left splat is stored first
    rgb, depth, alpha = scene.render(None, w.cams)
    torch.cuda.synchronize()
    scene.sync_status()
    rgb = rgb.cpu().numpy()[0]
    scene.close()
    ref = oracle.render_env(w, 0)
    both = ref["alpha"] > 0.6  # pixels where both splats blend
    assert both.sum() > 4
    np.testing.assert_allclose(rgb[both], ref["rgb"][both], atol=2e-3)
    # red (index 0) first: at the centre pixel red carries more weight than blue
    j, i = H // 2, W // 2
    assert rgb[j, i, 0] > rgb[j, i, 2] + 0.1


def test_device_resident_scene_inputs():
    """A scene built from CUDA tensors (the on-device form of gs_gaussians)
    stores the same Gaussians in the same order as one built from host
    arrays, and renders bit-identical images."""
    import types

    import torch

    w = synth.make_c1(n_envs=2, width=96, height=72, f=75.0, n_bg=20_000, per_link=500)

    def on_device(g):
        return types.SimpleNamespace(**{f: torch.from_numpy(np.ascontiguousarray(getattr(g, f))).cuda()
                                        for f in ("mean", "quat", "log_scale", "opacity", "sh")})

    host = gsbatch.scene_from_workload(w)
    dev = gsbatch.Scene(on_device(w.background))
    dev.attach_links(w.link_offsets, on_device(w.links))
    np.testing.assert_array_equal(host.storage_order(), dev.storage_order())
    poses = torch.from_numpy(w.link_poses).cuda()
    outs = []
    for sc in (host, dev):
        rgb, depth, alpha = sc.render(poses, w.cams)
        torch.cuda.synchronize()
        sc.sync_status()
        outs.append((rgb.cpu().numpy(), depth.cpu().numpy(), alpha.cpu().numpy()))
        sc.close()
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_opaque_splats_cap_and_early_stop():
    """c0 with 30 % of its splats near opaque (opacity U(0.9, 0.9999), scales
    e^1.5 larger: alpha meets its 0.99 cap near their centres, and most pixels
    stop, with T just above 1e-4, after a few splats).  The
    compositor walks 32-splat chunks holding a splat of opacity > 0.98 with the
    cap and the others without it, and blends both splats of a step at once
    unless a pixel stops there: against the oracle (independent and keyed), and
    bit for bit between the quadrant form (16x16 tiles at this size) and the
    plain form (16x8 tiles)."""
    w = synth.make_c0()
    bg = w.background
    rng = np.random.default_rng(7)
    op = bg.opacity.copy()
    sel = rng.random(bg.n) < 0.3
    op[sel] = rng.uniform(0.9, 0.9999, int(sel.sum())).astype(op.dtype)
    ls = bg.log_scale.copy()
    ls[sel] += 1.5
    w2 = synth.Workload(w.name, synth.Gaussians(bg.mean, bg.quat, ls, op, bg.sh), w.link_offsets, w.links,
                        w.link_poses, w.cams)
    out = gpu_render(w2, debug=True, keep_scene=True)
    st_i, st_k, rec, proj = _keyed_check(w2, 0, out)
    out["scene"].close()
    print("opaque c0 independent", st_i, "keyed", st_k)
    assert st_k["amb_frac"] < 0.1
    vis = proj["valid"] == 1
    assert int((proj["opacity"][vis] > 0.99).sum()) >= 100  # the cap is reached
    assert float((out["alpha"][0] > 0.999).mean()) > 0.5  # most pixels stop early
    plain = gpu_render(w2, tile=(16, 8))
    for k in ("rgb", "depth", "alpha"):
        assert np.array_equal(plain[k], out[k]), k


def test_crowded_depth_band_partition_and_selection():
    """6,000 splats within 1e-3 m of one depth (3 m) in a few tiles, and a few
    far splats (100 m) that widen the env's depth range.  Long buckets are
    partitioned over the env's range, so the crowd falls into a single
    partition bin, which the compositor cuts by radix selection: per-tile
    depth-ordered lists bit-exact against the binning oracle fed the GPU's
    keys, and the image against the oracle (independent and keyed)."""
    w0 = synth.make_c0()
    rng = np.random.default_rng(11)
    n, nf = 6000, 16
    mean = np.stack([rng.uniform(-0.05, 0.05, n), rng.uniform(-0.05, 0.05, n), rng.uniform(-1e-3, 1e-3, n)], 1)
    q, ls, _, sh = synth._attributes(rng, n)
    crowd = synth._gaussians(mean, q, ls - 0.5, rng.uniform(0.02, 0.2, n), sh)
    fm = np.stack([rng.uniform(-20.0, 20.0, nf), rng.uniform(-15.0, 15.0, nf), np.full(nf, 97.0)], 1)
    q2, ls2, o2, sh2 = synth._attributes(rng, nf)
    far = synth._gaussians(fm, q2, np.zeros_like(ls2), o2, sh2)
    bg = synth.Gaussians.concat([w0.background, crowd, far])
    w = synth.Workload("crowd", bg, w0.link_offsets, w0.links, w0.link_poses, w0.cams)
    W, H = 128, 96
    out = gpu_render(w, debug=True, keep_scene=True)
    scene = out["scene"]
    rec = scene.debug_records(0, bg.n)
    vis = np.nonzero(rec["visible"])[0]
    assert rec["visible"][bg.n - nf:].sum() >= nf // 2  # the far splats widen the range
    counts, lists = scene.debug_tiles(0, (W // 16) * (H // 16))
    zb = rec["z"][vis].view(np.uint32)
    oc, ol = oracle.bin_records(rec["u"][vis], rec["v"][vis], rec["hx"][vis], rec["hy"][vis], zb,
                                vis.astype(np.uint32), W, H, 16, 16)
    np.testing.assert_array_equal(counts.astype(np.int64), oc)
    np.testing.assert_array_equal(lists, ol)
    # the crowd's keys share one bin of the env's range (2048 bins over its depth bits)
    lo, hi = int(zb.min()) << 32, (int(zb.max()) << 32) | 0xFFFFFFFF
    shift = max(0, (hi - lo).bit_length() - 11)
    crowd_keys = (zb[(vis >= w0.background.n) & (vis < bg.n - nf)].astype(np.uint64) << np.uint64(32))
    bins = (crowd_keys - np.uint64(lo)) >> np.uint64(shift)
    assert np.bincount(bins.astype(np.int64)).max() > 384 and counts.max() > 768
    st_i, st_k, _, _ = _keyed_check(w, 0, out)
    scene.close()
    print("crowded band independent", st_i, "keyed", st_k)
