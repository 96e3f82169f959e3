"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, and exports every entry point include/hfx.h declares."""
import ctypes
import os
import re

import pytest

import paper_2009_12505_gb300 as hfx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hfx_[a-z_A-Z0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_boundary():
    names = declared()
    for n in ("hfx_create", "hfx_set_C", "hfx_set_V", "hfx_set_D", "hfx_set_many", "hfx_build",
              "hfx_H_count", "hfx_H_keys", "hfx_get_H", "hfx_get_H_all", "hfx_grad",
              "hfx_stats", "hfx_last_error", "hfx_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = hfx.build_library()
    lib = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(lib, n), n


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hfx.HfxError):
        hfx.Context([13], [60])
