"""The C ABI library builds for sm_103a, loads, and exports every function include/im.h declares (no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions() -> list[str]:
    text = open(os.path.join(ROOT, "include", "im.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:im_status|const char \*)\s*(im_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libim():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2105_04023_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_api():
    names = declared_functions()
    for required in ["im_ctx_create", "im_ctx_destroy", "im_build_sketches", "im_estimate", "im_select_seeds",
                     "im_select_seeds_batch", "im_sketch_registers", "im_sketch_destroy", "im_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libim):
    missing = [n for n in declared_functions() if not hasattr(libim, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2105_04023_gb300 import _lib

    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_structs_match_header_layout():
    # field order and types of the ctypes mirrors follow the header
    from paper_2105_04023_gb300 import _lib

    text = open(os.path.join(ROOT, "include", "im.h")).read()
    for cname, py in [("im_graph", _lib.im_graph), ("im_params", _lib.im_params), ("im_trace", _lib.im_trace),
                      ("im_stats", _lib.im_stats), ("im_tuning", _lib.im_tuning)]:
        plain = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", plain).group(1)
        fields = re.findall(r"(\w+)\s*;", body)
        assert fields == [f for f, _ in py._fields_], (cname, fields)


def test_context_creation_without_a_gpu_fails_cleanly(libim):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    from paper_2105_04023_gb300 import _lib

    L = _lib.load()
    h = ctypes.c_void_p()
    assert L.im_ctx_create(0, None, ctypes.byref(h)) == _lib.IM_ECUDA
    assert not h.value


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2105_04023_gb300 import _lib

    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
