"""gs_render_batch_noalloc, the entry point that allocates nothing.

It serves callers that may not allocate device memory while they render (GPU
memory already reserved by another allocator, places where an allocation
would stall the device or is not allowed).  Its working memory is a fixed
32 MiB device array shared by all calls, so these tests call it twice in a
row and compare each result with gs_render_batch, which allocates its own
scratch.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import ensure_built
from paper_2604_25459_gb300 import gsbatch, synth

pytestmark = pytest.mark.gpu


def _outputs(torch, E, H, W):
    return (torch.full((E, H, W, 3), -1.0, device="cuda"), torch.full((E, H, W), -1.0, device="cuda"),
            torch.full((E, H, W), -1.0, device="cuda"))


@pytest.mark.parametrize("make", [lambda: synth.make_c0(),
                                  lambda: synth.make_tiny(seed=7, n_envs=3),
                                  lambda: synth.make_c1(n_envs=3, width=96, height=72, f=75.0, n_bg=20_000,
                                                        per_link=500)])
def test_noalloc_matches_allocating_path_twice(make):
    import torch

    ensure_built()
    w = make()
    E, H, W = w.n_envs, int(w.cams["height"][0]), int(w.cams["width"][0])
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(np.ascontiguousarray(w.link_poses)).cuda() if w.n_links else None
    ref = scene.render(poses, w.cams)
    torch.cuda.synchronize()
    L = gsbatch.lib()
    for _ in range(2):  # the second call starts from the first call's leftovers in the shared array
        rgb, depth, alpha = _outputs(torch, E, H, W)
        st = L.gs_render_batch_noalloc(scene._h, E, gsbatch._ptr(poses), gsbatch._ptr(np.ascontiguousarray(w.cams)),
                                       C.c_void_p(rgb.data_ptr()), C.c_void_p(depth.data_ptr()),
                                       C.c_void_p(alpha.data_ptr()), None)
        assert st == gsbatch.GS_OK, L.gs_last_error()
        torch.cuda.synchronize()
        scene.sync_status()
        for got, exp in zip((rgb, depth, alpha), ref):
            assert float((got - exp).abs().max()) <= 2e-3
            assert torch.equal(got, exp)  # same kernels, same inputs: identical bits
    scene.close()


def _c0_batch(E):
    """E envs of the c0 scene (16,384 Gaussians, 128x96), each camera shifted
    by its own offset."""
    w = synth.make_c0()
    rng = np.random.default_rng(3)
    t = np.zeros((E, 3))
    t[:, :2] = rng.uniform(-0.2, 0.2, (E, 2))
    t[:, 2] = 3.0
    cams = synth.make_cameras(E, 110.0, 110.0, 64.0, 48.0, 128, 96, [[1.0, 0.0, 0.0, 0.0]] * E, t)
    return synth.Workload("c0 batch", w.background, w.link_offsets, w.links, np.zeros((E, 0, 7), np.float32), cams)


def _near_far_batch(E, near_from):
    """E envs of a 1,024-Gaussian cube of large splats (scale ~0.15 m), 128x96:
    envs before near_from view it from 8 m (~3.4k intersection keys each),
    envs from near_from on from 1.5 m (~16k keys each)."""
    rng = np.random.default_rng(5)
    n = 1024
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh = rng.normal(0, 0.3, (n, 16, 3))
    sh[:, 0, :] += 0.5
    bg = synth.Gaussians(*(np.ascontiguousarray(a, np.float32) for a in
                           (rng.uniform(-1, 1, (n, 3)), q, np.log(0.15) + rng.normal(0, 0.2, (n, 3)),
                            rng.uniform(0.5, 0.9, n), sh)))
    t = np.zeros((E, 3))
    t[:, :2] = rng.uniform(-0.1, 0.1, (E, 2))
    t[:, 2] = np.where(np.arange(E) < near_from, 8.0, 1.5)
    cams = synth.make_cameras(E, 110.0, 110.0, 64.0, 48.0, 128, 96, [[1.0, 0.0, 0.0, 0.0]] * E, t)
    return synth.Workload("near/far", bg, np.zeros(1, np.int64), bg.slice(0, 0), np.zeros((E, 0, 7), np.float32), cams)


def _noalloc(L, scene, w, outs):
    rgb, depth, alpha = outs
    return L.gs_render_batch_noalloc(scene._h, w.n_envs, None, gsbatch._ptr(np.ascontiguousarray(w.cams)),
                                     C.c_void_p(rgb.data_ptr()), C.c_void_p(depth.data_ptr()),
                                     C.c_void_p(alpha.data_ptr()), None)


def test_noalloc_several_waves():
    """60 envs of 16,384 Gaussians do not fit one pass of the 32 MiB array
    (about 1 MiB of projected records per env), so the call renders them in
    waves: every wave's images land at their own offsets, from the array's
    leftovers of the wave before, equal to gs_render_batch bit for bit."""
    import torch

    ensure_built()
    w = _c0_batch(60)
    scene = gsbatch.scene_from_workload(w)
    ref = scene.render(None, w.cams)
    torch.cuda.synchronize()
    L = gsbatch.lib()
    for _ in range(2):
        outs = _outputs(torch, 60, 96, 128)
        st = _noalloc(L, scene, w, outs)
        assert st == gsbatch.GS_OK, L.gs_last_error()
        torch.cuda.synchronize()
        scene.sync_status()
        for got, exp in zip(outs, ref):
            assert float((got - exp).abs().max()) <= 2e-3
            assert torch.equal(got, exp)
    scene.close()


def test_noalloc_later_wave_overflow():
    """512 envs in waves of 256 (about 65 KiB of records per env): the first
    wave's 256 distant views fit the array's room for intersection keys
    (~7 MB of ~16 MB), the second wave's 212 close views do not (~28 MB).
    The call fails with GS_ERR_UNSUPPORTED when that wave is binned; the
    first wave's images are complete (equal to gs_render_batch) and every
    later env still holds the -1 fill."""
    import torch

    ensure_built()
    E = 512
    w = _near_far_batch(E, near_from=300)
    scene = gsbatch.scene_from_workload(w)
    ref = scene.render(None, w.cams)
    torch.cuda.synchronize()
    L = gsbatch.lib()
    outs = _outputs(torch, E, 96, 128)
    st = _noalloc(L, scene, w, outs)
    assert st == gsbatch.GS_ERR_UNSUPPORTED
    assert b"intersection keys" in L.gs_last_error()
    torch.cuda.synchronize()
    scene.sync_status()
    rgb = outs[0]
    unwritten = [bool((rgb[e] == -1.0).all()) for e in range(E)]
    k = unwritten.index(True)
    assert 1 <= k <= 300 and all(unwritten[k:])  # a later wave failed; nothing after it was written
    print("first unwritten env", k)
    for got, exp in zip(outs, ref):
        assert torch.equal(got[:k], exp[:k])
        assert bool((got[k:] == -1.0).all())
    scene.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    ensure_built()
    w = synth.make_c1(n_envs=1, width=64, height=48, f=50.0)  # 600k Gaussians: 38 MB of records per env
    scene = gsbatch.scene_from_workload(w)
    poses = torch.from_numpy(w.link_poses).cuda()
    rgb, depth, alpha = _outputs(torch, 1, 48, 64)
    with pytest.raises(gsbatch.GsError) as ei:
        scene.render_noalloc(poses, w.cams, rgb, depth, alpha)
    assert ei.value.status == gsbatch.GS_ERR_UNSUPPORTED
    assert "no-allocation" in str(ei.value)
    assert float(rgb.min()) == -1.0  # nothing was written
    scene.close()
