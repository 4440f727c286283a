"""The C ABI library without a GPU: it builds, loads, and exports every entry point that
include/*.h declares; calls fail cleanly (a status, not a crash) when no device exists."""

import ctypes
import glob
import os
import re

import pytest
import torch

from paper_1811_10074_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:sws_status|const char\s*\*|int|void)\s+\**\s*(sws_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("sws_sliding_sum", "sws_kmers", "sws_minimizers", "sws_minimizers_batch", "sws_create", "sws_sync"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} is declared in include/ but not exported"


def test_binding_signatures_cover_header():
    assert set(declared_functions()) <= set(binding.SIGNATURES)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_create_without_device_fails_cleanly(lib):
    h = ctypes.c_void_p()
    st = lib.sws_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value
    assert len(lib.sws_last_error()) > 0


def test_null_context_is_rejected(lib):
    st = lib.sws_sliding_sum(None, 0, 4, None, None, 100, 0, None)
    assert st == 1  # SWS_ERR_INVALID
    assert b"context" in lib.sws_last_error()
