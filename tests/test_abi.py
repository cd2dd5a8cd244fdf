"""The C-ABI library builds, loads without a GPU, and exports every declared entry point."""
import ctypes
import os
import re

import pytest

from paper_2108_05021_gb300 import build as libbuild
from paper_2108_05021_gb300 import osbf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(osbf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("osbf_create", "osbf_destroy", "osbf_filter", "osbf_filter_ex", "osbf_filter_backward",
              "osbf_filter_batched", "osbf_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string(lib):
    lib.osbf_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.osbf_version()


def test_null_context_is_rejected(lib):
    lib.osbf_filter.restype = ctypes.c_int
    assert lib.osbf_filter(None, None, None, 1, 1, 1, 1, 1, 1, 0, None) == 1  # OSBF_EINVAL
    lib.osbf_last_error.restype = ctypes.c_char_p
    assert lib.osbf_last_error(None) == b"null context"


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(osbf, "LIB_PATH", "/nonexistent/libosbf.so")
    monkeypatch.setattr(osbf, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        osbf.lib()


def test_maps_pitch_rounds_frame_width_to_16_bytes(lib):
    for W in (1, 7, 16, 100, 4096):
        for r in (0, 1, 3, 8, 16):
            assert lib.osbf_maps_pitch(W, r) == -(-(W + 2 * r) // 16) * 16


def test_binding_has_no_cpu_path():
    """Every device entry of the binding refuses host tensors (there is no CPU fallback;
    host buffers go through filter_host, which copies to the device)."""
    import torch

    from paper_2108_05021_gb300 import osbf

    x = torch.zeros(1, 1, 8, 8)
    maps = torch.zeros(osbf.maps_shape(x, 1, 1), dtype=torch.uint8)
    calls = [
        lambda: osbf.filter(x, 1, 1),
        lambda: osbf.filter_fast(x, 1, 1),
        lambda: osbf.filter_gauss(x, 1, 1.0, 1),
        lambda: osbf.filter3d(torch.zeros(1, 1, 4, 8, 8), 1, 1),
        lambda: osbf.backward(x, maps, 1, 1),
    ]
    for call in calls:
        with pytest.raises(ValueError):
            call()
