"""CPU checks of the C ABI library: it builds for sm_103a, loads without a GPU, exports every
function include/gs.h declares with the prototypes the binding uses, and its host-side argument
checks answer without touching a device."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2408_07967_gb300 import _native, build as gsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gslib():
    gsbuild.build()
    return _native.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gs_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_parses():
    names = header_functions()
    assert "gs_render" in names and "gs_sort_pairs" in names and len(names) >= 20


def test_library_exports_every_header_symbol(gslib):
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(gs_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing
    assert set(header_functions()) <= set(_native.PROTOTYPES), set(header_functions()) - set(_native.PROTOTYPES)


def test_build_targets_sm103a_only():
    flags = " ".join(gsbuild.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags and flags.count("-gencode") == 1


def test_host_side_argument_checks(gslib):
    o = _native.gs_render_opts()
    assert gslib.gs_default_opts(C.byref(o)) == 0
    assert abs(o.tau - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7 and o.clamp_fov == 1
    assert gslib.gs_default_opts(None) == -1
    assert b"NULL" in gslib.gs_last_error()
    assert gslib.gs_version() >= 100
    h = C.c_void_p()
    assert gslib.gs_frame_create(None, 10, 10, 16, 16, C.byref(h)) == -1
    assert gslib.gs_sort(None, None) == -1
    assert gslib.gs_render(None, None, None, None, None, None, None, None) == -1
    assert gslib.gs_frame_destroy(None) == 0 and gslib.gs_scene_destroy(None) == 0


def test_no_device_is_an_error_not_a_crash(gslib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = C.c_void_p()
    st = gslib.gs_context_create(0, C.byref(h))
    assert st in (-8, -4), st
