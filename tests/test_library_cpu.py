"""CPU-side checks of the CUDA library: it builds, loads, exports every symbol
include/szx.h declares, and its host-only geometry agrees with the oracle's.
No kernel runs here (no GPU)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2201_13020_b300 import _lib
from paper_2201_13020_b300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "szx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(szx_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    libbuild.build()
    L = _lib.lib()
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(_lib.EXPORTED)


def test_no_cpu_fallback_when_library_missing(monkeypatch):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libszx.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()


def test_status_strings_and_version():
    L = _lib.lib()
    for code in range(7):
        assert L.szx_status_string(code)
    assert b"sm_103a" in L.szx_version()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("block", [32, 64, 128, 256, 512, 1024])
def test_stream_max_matches_oracle_bound(dtype, block):
    # two independent statements of the worst-case stream size (all raw blocks)
    L = _lib.lib()
    for n in (1, 7, 31, block, block + 1, 8191, 8192 * 3 + 5, 1 << 20, 10**6 + 3):
        assert L.szx_stream_max_bytes(n, dtype, block) == oracle.compress_bound(n, dtype, block)
        assert L.szx_compress_bound(n, dtype, block) > L.szx_stream_max_bytes(n, dtype, block)


def test_invalid_geometry_returns_zero():
    L = _lib.lib()
    assert L.szx_compress_bound(0, 0, 128) == 0
    assert L.szx_compress_bound(10, 0, 100) == 0
    assert L.szx_compress_bound(10, 2, 128) == 0
    assert L.szx_compress_bound(10, 0, 2048) == 0


def test_compiled_for_sm103a():
    log = open(os.path.join(ROOT, "paper_2201_13020_b300", "lib", "ptxas.log")).read()
    assert "sm_103a" in log
    assert "compress_kernel" in log and "decompress_kernel" in log
