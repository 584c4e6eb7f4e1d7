"""The C ABI library builds, loads and exports every declared entry point;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2606_21381_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(name="osog.h"):
    text = open(os.path.join(ROOT, "include", name)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(osog_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("osog_plan_create", "osog_plan_destroy", "osog_workspace_size",
                     "osog_render", "osog_batch_submit", "osog_sync_status",
                     "osog_last_error"):
        assert required in names
    assert sorted(_lib.EXPORTS) == names


def test_library_exports_every_declared_symbol(L):
    raw = ctypes.CDLL(build.LIB)
    for name in header_functions() + header_functions("osog_cnn.h"):
        assert hasattr(raw, name), name
    assert sorted(_lib.CNN_EXPORTS) == header_functions("osog_cnn.h")


def test_conv_shape_checks_on_the_host(L):
    s = _lib.ConvShape(2, 20, 20, 8, 16, 3, 3, 2, 1)
    assert L.osog_conv_out_h(ctypes.byref(s)) == 10
    bad = _lib.ConvShape(2, 20, 20, 6, 16, 3, 3, 1, 1)  # C not a multiple of 8
    assert L.osog_conv_out_h(ctypes.byref(bad)) == 0
    assert L.osog_conv2d_forward(ctypes.byref(bad), None, None, None, 1, None, None, None) == 1


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_plan_create_rejects_bad_sizes_on_the_host(L):
    plan = ctypes.c_void_p()
    for H, W in [(100, 256), (256, 16), (4096, 256), (256, 0)]:
        rc = L.osog_plan_create(ctypes.byref(plan), H, W)
        assert rc == 2, (H, W)
        assert not plan
        assert b"power" in L.osog_last_error()


def test_null_plan_arguments_are_reported(L):
    o = _lib.Optics()
    assert L.osog_workspace_size(None, 10, 1, 1) == 0
    assert L.osog_render(None, None, 0, 0, ctypes.byref(o), None, None, 0, None) == 1
    assert L.osog_sync_status(None, None) == 1
    assert L.osog_plan_launch_count(None) == 0
    assert L.osog_profile_begin(None) == 1


def test_optics_struct_mirrors_header_layout():
    # 2 int32 + 5 doubles + uint32 + 6 doubles with natural alignment
    assert ctypes.sizeof(_lib.Optics) == 8 + 5 * 8 + 8 + 6 * 8
    assert _lib.Optics.modes.offset == 48
    assert _lib.Optics.oblique_frac.offset == 56
