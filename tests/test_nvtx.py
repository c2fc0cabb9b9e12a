"""Every entry point opens an NVTX range named after itself. Checked on the
CPU with a minimal NVTX tool library (tests/nvtx_probe.c) that the NVTX
headers inside libnpm_gb300 load through NVTX_INJECTION64_PATH: calls that
return on their argument checks already open and close their range, so no
GPU is needed."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import ctypes as C, sys
sys.path.insert(0, {root!r})
import paper_2504_04315_gb300 as npm
from paper_2504_04315_gb300 import _lib
lib = _lib.load()
cfg = npm.make_config(npm.RADIANCE, [16], 4, 19, [4, 32, 32, 16], 4)
cfg.K = 0                                    # invalid: rejected on the host
h = C.c_void_p()
assert lib.npm_create(C.byref(cfg), C.byref(h)) == _lib.ERR_INVALID_ARG
assert lib.npm_query_sample(None, 1, None, None, None, 1, 0.0, None, None, None, None) == _lib.ERR_INVALID_ARG
assert lib.npm_eval_pdf(None, 1, None, None, None, 1, None, None) == _lib.ERR_INVALID_ARG
assert lib.npm_train_step(None, 1, None, None, None, None, None, 1, None, None) == _lib.ERR_INVALID_ARG
"""


def test_entry_points_open_named_ranges(tmp_path):
    npm_build = pytest.importorskip("paper_2504_04315_gb300._build")
    npm_build.build()
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    probe = str(tmp_path / "libnvtx_probe.so")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", cuda_inc, os.path.join(HERE, "nvtx_probe.c"),
                    "-o", probe], check=True)
    out = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=probe, NPM_NVTX_PROBE_OUT=str(out))
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    names = out.read_text().split()
    assert names == ["npm_create", "npm_query_sample", "npm_eval_pdf", "npm_train_step"], names
