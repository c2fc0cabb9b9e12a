"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/npm.h declares, and rejects bad arguments on the
host before any device work."""
import ctypes as C
import os
import re

import pytest

import paper_2504_04315_gb300 as npm
from paper_2504_04315_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    npm.build()
    return _lib.load()


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if not name.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        syms |= set(re.findall(r"\b(npm_[a-z0-9_]+)\s*\(", text))
    return syms


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for core in ["npm_create", "npm_query_sample", "npm_eval_pdf", "npm_train_step", "npm_destroy"]:
        assert core in syms


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    # The Python binding types every one of them.
    assert syms <= set(_lib.SIGNATURES), syms - set(_lib.SIGNATURES)


def test_config_struct_layout_matches_header():
    # int fields, 32 level resolutions, 9 widths, 4 floats, int64, uint64
    assert C.sizeof(_lib.NpmConfig) == 232
    assert _lib.NpmConfig.max_batch.offset == 216


@pytest.mark.parametrize("field,value", [
    ("mode", 7), ("n_levels", 0), ("feat_per_level", 9), ("K", 0), ("kappa_act", 5),
    ("precision", 5), ("log2_table", 30), ("max_batch", -1)])
def test_invalid_config_rejected_on_host(lib, field, value):
    cfg = npm.make_config(npm.RADIANCE, [16], 4, 19, [4, 32, 32, 16], 4)
    setattr(cfg, field, value)
    h = C.c_void_p()
    st = lib.npm_create(C.byref(cfg), C.byref(h))
    assert st == _lib.ERR_INVALID_ARG
    assert h.value is None
    assert lib.npm_last_error()


def test_width_rules_rejected_on_host(lib):
    bad = [
        ([4, 30, 16], 4),       # width not a multiple of 4
        ([4, 32, 32, 12], 4),   # last width != 4K
        ([2, 32, 16], 4),       # input narrower than the encoding (1 level x 4)
        ([4, 256, 16], 4),      # width above the maximum
    ]
    for widths, K in bad:
        cfg = npm.make_config(npm.RADIANCE, [16], 4, 19, widths, K)
        h = C.c_void_p()
        assert lib.npm_create(C.byref(cfg), C.byref(h)) == _lib.ERR_INVALID_ARG


def test_null_handle_calls_are_errors(lib):
    assert lib.npm_query_sample(None, 1, None, None, None, 1, 0.0, None, None, None, None) \
        == _lib.ERR_INVALID_ARG
    assert lib.npm_destroy(None) == _lib.OK
    assert lib.npm_num_params(None) == -1


def test_normal_build_compiles_bounds_checks_out(lib):
    # The bounds-checking kernels exist only in the debug build
    # (_build.build_debug, NPM_DEBUG_BOUNDS); the normal build reports -1.
    assert lib.npm_debug_bounds_violations() == -1
