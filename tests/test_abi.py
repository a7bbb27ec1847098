"""The C-ABI library loads and exports every entry point declared in
include/gsbatch.h; argument checks that need no GPU return GS_ERR_INVALID."""
import ctypes as C
import os
import re

import pytest

from paper_2604_25459_gb300 import build as cuda_build
from paper_2604_25459_gb300 import gsbatch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gsbatch.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return gsbatch.lib()


def test_every_declared_symbol_exported(lib):
    names = _declared()
    assert "gs_render_batch" in names and "gs_scene_create" in names and "gs_scene_attach_links" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(gsbatch._SIGS), set(names) - set(gsbatch._SIGS)


def test_argument_checks_without_gpu(lib):
    assert lib.gs_scene_create(None, None) == gsbatch.GS_ERR_INVALID
    h = C.c_void_p()
    v = gsbatch.GsGaussians(-1, None, None, None, None, None, 3, 0, 0)
    assert lib.gs_scene_create(C.byref(v), C.byref(h)) == gsbatch.GS_ERR_INVALID
    assert b"negative" in lib.gs_last_error()
    v = gsbatch.GsGaussians(10, None, None, None, None, None, 3, 0, 0)
    assert lib.gs_scene_create(C.byref(v), C.byref(h)) == gsbatch.GS_ERR_INVALID
    v = gsbatch.GsGaussians(0, None, None, None, None, None, 5, 0, 0)
    assert lib.gs_scene_create(C.byref(v), C.byref(h)) == gsbatch.GS_ERR_INVALID
    assert lib.gs_scene_set_tile(None, 16, 16) == gsbatch.GS_ERR_INVALID
    assert lib.gs_render_batch(None, 1, None, None, None, None, None, None) == gsbatch.GS_ERR_INVALID
    assert lib.gs_version().startswith(b"gsbatch")


def test_server_config_checks_without_gpu(lib):
    h = C.c_void_p()
    assert lib.gs_server_create(None, C.byref(h)) == gsbatch.GS_ERR_INVALID
    for cfg in [(0, 2, 8, 16, 16), (1 << 30, 0, 8, 16, 16), (1 << 30, 65, 8, 16, 16), (1 << 30, 2, 0, 16, 16),
                (1 << 30, 2, 8, 12, 16)]:
        c = gsbatch.GsServerConfig(*cfg)
        assert lib.gs_server_create(C.byref(c), C.byref(h)) == gsbatch.GS_ERR_INVALID, cfg
        assert not h.value
    assert lib.gs_server_submit(None, 0, None, 0.0, None) == gsbatch.GS_ERR_INVALID
    assert lib.gs_server_poll(None, None, 0, None) == gsbatch.GS_ERR_INVALID
    lib.gs_server_destroy(None)
