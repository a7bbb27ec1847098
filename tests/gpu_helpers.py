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


def compare(rgb, depth, alpha, ref, amb_bits=AMB_ALPHA | AMB_T | AMB_Z, rgb_tol=RGB_TOL, depth_rtol=DEPTH_RTOL):
    """Return stats; raise AssertionError when a non-ambiguous pixel is out of tolerance."""
    ok = (ref["amb"] & amb_bits) == 0
    n_amb = int((~ok).sum())
    err = np.abs(rgb - ref["rgb"]).max(axis=-1)
    aerr = np.abs(alpha - ref["alpha"])
    dmask = ok & (ref["alpha"] >= 0.5) & (alpha >= 0.5)
    derr = np.abs(depth - ref["depth"]) / np.maximum(ref["depth"], 1e-30)
    st = dict(pixels=int(ok.size), ambiguous=n_amb, amb_frac=n_amb / ok.size,
              amb_rgb_max=float(err[~ok].max()) if (~ok).any() else 0.0,
              rgb_max=float(err[ok].max()) if ok.any() else 0.0,
              alpha_max=float(aerr[ok].max()) if ok.any() else 0.0,
              depth_rel_max=float(derr[dmask].max()) if dmask.any() else 0.0)
    bad = ok & ((err > rgb_tol) | (aerr > rgb_tol))
    if bad.any():
        j, i = np.argwhere(bad)[0]
        raise AssertionError(f"{int(bad.sum())} pixels out of tolerance, first ({i},{j}): gpu rgb {rgb[j, i]} "
                             f"oracle {ref['rgb'][j, i]} alpha {alpha[j, i]} vs {ref['alpha'][j, i]}; {st}")
    dbad = dmask & (derr > depth_rtol)
    if dbad.any():
        j, i = np.argwhere(dbad)[0]
        raise AssertionError(f"{int(dbad.sum())} depth pixels out of tolerance, first ({i},{j}): "
                             f"{depth[j, i]} vs {ref['depth'][j, i]}; {st}")
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
