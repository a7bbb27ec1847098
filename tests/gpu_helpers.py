"""Helpers for the GPU parity tests: render through the C ABI, render with the
oracle, compare within the stated tolerances."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle
from paper_2604_25459_gb300 import gsbatch, synth

RGB_TOL = 2e-3      # per-channel max abs on [0,1] images
DEPTH_RTOL = 1e-4   # relative, where the oracle's alpha >= 0.5
AMB_ALPHA, AMB_T, AMB_Z = 1, 2, 4


_built = False


def ensure_built():
    global _built
    if not _built:
        import __graft_entry__

        __graft_entry__.build()
        _built = True


def gpu_render(w, dtype="f32", tile=(16, 16), debug=False, sh_degree=3, scene=None, wave=0, envs=None,
               budget=None, keep_scene=False):
    """Render workload ``w`` (optionally a subset of envs) on cuda:0; numpy outputs."""
    import torch

    ensure_built()
    own = scene is None
    if own:
        scene = gsbatch.scene_from_workload(w, dtype, sh_degree)
    scene.set_tile(*tile)
    scene.set_debug(debug)
    if wave:
        scene.set_wave(wave)
    if budget:
        scene.set_budget(budget)
    lp = w.link_poses if envs is None else w.link_poses[envs]
    cams = w.cams if envs is None else w.cams[envs]
    poses = torch.from_numpy(np.ascontiguousarray(lp)).cuda() if w.n_links > 0 else None
    rgb, depth, alpha = scene.render(poses, cams)
    torch.cuda.synchronize()
    scene.sync_status()
    out = dict(rgb=rgb.cpu().numpy(), depth=depth.cpu().numpy(), alpha=alpha.cpu().numpy())
    if keep_scene:
        out["scene"] = scene
    elif own:
        scene.close()
    return out


def compare(rgb, depth, alpha, ref, amb_bits=AMB_ALPHA | AMB_T | AMB_Z, rgb_tol=RGB_TOL, depth_rtol=DEPTH_RTOL,
            proj=None):
    """Return stats; raise AssertionError when a pixel is out of tolerance.

    Pixels whose flag (ref["amb"]) has none of ``amb_bits`` must meet the
    tolerances.  The others (ambiguous: a threshold decision within FP32 noise)
    must meet them widened by what flipping the flagged decisions can explain:
    the oracle's bound W on the L1 change of the blending weights gives
    rgb <= tol + W max(rgb), alpha <= tol + W and, where both alphas >= 0.5,
    depth (a weighted mean of depths) <= rtol d + 2 W (z_max - z_min)."""
    proj = proj if proj is not None else ref.get("proj")
    if proj is not None and (proj["valid"] == 1).any():
        vis = proj["valid"] == 1
        cmax = float(proj["rgb"][vis].max())
        zspan = float(proj["z"][vis].max() - proj["z"][vis].min())
    else:
        cmax, zspan = 1.0, 0.0
    amb = ref["amb"]
    ok = (amb & amb_bits) == 0
    n_amb = int((~ok).sum())
    err = np.abs(rgb - ref["rgb"]).max(axis=-1)
    aerr = np.abs(alpha - ref["alpha"])
    both = (ref["alpha"] >= 0.5) & (alpha >= 0.5)
    dmask = ok & both
    derr = np.abs(depth - ref["depth"]) / np.maximum(ref["depth"], 1e-30)
    wb = ref["wbound"].astype(np.float64)
    rgb_lim = np.where(ok, rgb_tol, rgb_tol + wb * cmax)
    a_lim = np.where(ok, rgb_tol, rgb_tol + wb)
    d_lim = depth_rtol * np.abs(ref["depth"]) + np.where(ok, 0.0, 2.0 * wb * zspan)
    dcheck = both
    px = ok.size
    st = dict(pixels=int(px), ambiguous=n_amb, amb_frac=n_amb / px,
              flag_floor=float(((amb & AMB_ALPHA) != 0).mean()), flag_stop=float(((amb & AMB_T) != 0).mean()),
              flag_tie=float(((amb & AMB_Z) != 0).mean()),
              amb_beyond_tol=int(((~ok) & ((err > rgb_tol) | (aerr > rgb_tol))).sum()),
              amb_rgb_max=float(err[~ok].max()) if (~ok).any() else 0.0,
              amb_bound_use=float((err / rgb_lim)[~ok].max()) if (~ok).any() else 0.0,
              rgb_max=float(err[ok].max()) if ok.any() else 0.0,
              alpha_max=float(aerr[ok].max()) if ok.any() else 0.0,
              depth_rel_max=float(derr[dmask].max()) if dmask.any() else 0.0)
    bad = (err > rgb_lim) | (aerr > a_lim)
    if bad.any():
        j, i = np.argwhere(bad)[0]
        raise AssertionError(f"{int(bad.sum())} pixels out of tolerance, first ({i},{j}) flag {int(amb[j, i])} "
                             f"bound {wb[j, i]:.3g}: gpu rgb {rgb[j, i]} oracle {ref['rgb'][j, i]} alpha "
                             f"{alpha[j, i]} vs {ref['alpha'][j, i]}; {st}")
    dbad = dcheck & (np.abs(depth - ref["depth"]) > d_lim)
    if dbad.any():
        j, i = np.argwhere(dbad)[0]
        raise AssertionError(f"{int(dbad.sum())} depth pixels out of tolerance, first ({i},{j}) flag "
                             f"{int(amb[j, i])}: {depth[j, i]} vs {ref['depth'][j, i]}; {st}")
    return st


def psnr(a, b) -> float:
    mse = float(np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


def keyed_zkey(proj, rec):
    """Depth keys for the keyed comparison: the GPU's float32 depth where it
    projected the Gaussian, the oracle's depth rounded to float32 elsewhere."""
    zk = proj["z"].astype(np.float32)
    vis = rec["visible"] == 1
    zk[vis] = rec["z"][vis]
    return zk


def oracle_env(w, e, sh_degree=3, zkey=None, widened=None):
    """Oracle render of env e (optionally with quantised attributes ``widened``)."""
    if widened is not None:
        bg, links = widened
        w = synth.Workload(w.name, bg, w.link_offsets, links, w.link_poses, w.cams)
    S = oracle.scene_arrays(w, sh_degree)
    cam = w.cams[e]
    proj = oracle.project(S, w.link_poses[e], cam)
    img = oracle.render_projected(proj, int(cam["width"]), int(cam["height"]), zkey=None)
    img["proj"] = proj
    if zkey is not None:
        img2 = oracle.render_projected(proj, int(cam["width"]), int(cam["height"]), zkey=zkey)
        img2["proj"] = proj
        return img, img2
    return img


def keyed_check(w, e, out, sh_degree=3):
    """Independent and keyed comparisons of env e of a debug-mode render
    (``out`` from gpu_render(..., debug=True, keep_scene=True)).  Keyed: the
    oracle orders by the GPU's float32 depth keys (FP64 elsewhere), so the
    depth near-tie flag may not exclude a pixel; only alpha-floor and
    transmittance-stop decisions may."""
    scene = out["scene"]
    rec = scene.debug_records(e, w.background.n + w.links.n)
    S = oracle.scene_arrays(w, sh_degree)
    proj = oracle.project(S, w.link_poses[e], w.cams[e])
    zk = keyed_zkey(proj, rec)
    W, H = int(w.cams[e]["width"]), int(w.cams[e]["height"])
    ind = oracle.render_projected(proj, W, H)
    key = oracle.render_projected(proj, W, H, zkey=zk)
    st_i = compare(out["rgb"][e], out["depth"][e], out["alpha"][e], ind, proj=proj)
    st_k = compare(out["rgb"][e], out["depth"][e], out["alpha"][e], key, amb_bits=AMB_ALPHA | AMB_T, proj=proj)
    st_i["neval"] = int(ind["neval"].sum())
    return st_i, st_k, rec, proj


def render_counted(w, tile=(16, 16)):
    """Render every env of w with the library's counters on; returns the
    images and the counters (composited pairs, visible records, FP64 conics)."""
    import torch

    ensure_built()
    scene = gsbatch.scene_from_workload(w)
    scene.set_tile(*tile)
    scene.set_counters(True)
    poses = torch.from_numpy(np.ascontiguousarray(w.link_poses)).cuda() if w.n_links > 0 else None
    rgb, depth, alpha = scene.render(poses, w.cams)
    torch.cuda.synchronize()
    scene.sync_status()
    st = scene.stats()
    out = dict(rgb=rgb.cpu().numpy(), depth=depth.cpu().numpy(), alpha=alpha.cpu().numpy(), stats=st)
    scene.close()
    return out
