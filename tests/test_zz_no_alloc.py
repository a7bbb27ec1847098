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
