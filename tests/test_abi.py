"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/kbe.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2505_19467_gb300 as kbe
from paper_2505_19467_gb300 import builder

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "kbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kbe_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    builder.build()
    return kbe.load()


def test_library_exports_every_declared_function(lib):
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", kbe.LIB_PATH], capture_output=True, text=True).stdout
    for name in names:
        assert re.search(rf"\bT {name}\b", out), name


def test_binding_export_list_matches_header():
    assert sorted(kbe.EXPORTS) == header_functions()


@pytest.mark.gpu
def test_library_kernels_are_built_for_sm103(lib):
    """the loaded kernels report compute capability 10.3 (cudaFuncGetAttributes)
    and grids are sized against the device's own SM count"""
    import torch
    torch.cuda.init()
    bv, sms = kbe.device_info()
    assert bv == 103, bv
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count


def test_create_rejects_bad_config_without_gpu(lib):
    cfg = kbe._binding.kbe_config()
    cfg.nb, cfg.dim = 5, 1          # N_b = 5 is not compiled in
    cfg.L[0], cfg.L[1] = 8, 1
    cfg.nt_max, cfg.dt = 4, 0.1
    h = ctypes.c_void_p()
    rc = lib.kbe_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -7 and not h.value
    assert b"nb" in lib.kbe_last_error(None)
    cfg.nb, cfg.dt = 2, -1.0
    assert lib.kbe_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
