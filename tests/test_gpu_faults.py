"""Failure handling without a GPU fault: host-side injection of a failed
device allocation (every earlier allocation of npm_create freed again) and
of a failed launch (the next call succeeds on the same context), and the
bounds-checking debug build of the library (every grid-entry index and
queue slot checked before its access) on ordinary workloads."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from gpu_helpers import cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3])
def test_failed_allocation_frees_everything(precision):
    import paper_2504_04315_gb300 as npm
    from paper_2504_04315_gb300 import _lib
    w = synth.PAPER_HASH.with_(precision=precision)
    cfg = npm.config_from(w, max_batch=1 << 16)
    m = npm.NPM(cfg)  # warm the context and the allocator's pools
    m.close()
    free0 = _free_bytes()
    failures = 0
    try:
        for k in range(1, 40):
            os.environ["NPM_TEST_FAIL_ALLOC"] = str(k)
            try:
                npm.NPM(cfg).close()
                break  # k is beyond the number of allocations: created
            except _lib.NpmError as e:
                assert e.status == _lib.ERR_OOM, e
                failures += 1
            assert _free_bytes() >= free0 - (4 << 20), k
    finally:
        os.environ.pop("NPM_TEST_FAIL_ALLOC", None)
    assert failures >= 8, failures
    # Nothing left behind, and the next create works.
    m = make_model(w, synth.random_params(w, 3), 1 << 10, precision=precision)
    m.close()
    assert _free_bytes() >= free0 - (4 << 20)


CHILD_LAUNCH = r"""
import sys
sys.path[:0] = [{here!r}, {root!r}]
import numpy as np, torch, synth
from gpu_helpers import cuda, host, make_model
from paper_2504_04315_gb300 import _lib
w = synth.TINY_BF16
n = 4096
m = make_model(w, synth.random_params(w, 3), n)
pos, u = cuda(synth.positions(4, n)), cuda(synth.sample_uniforms(4, n))
d1, p1, _ = m.query_sample(pos, u)
first = host(p1).copy()
try:
    m.query_sample(pos, u)
    raise SystemExit("the second call should have failed")
except _lib.NpmError as e:
    assert e.status == _lib.ERR_CUDA and "injected" in str(e), e
d3, p3, _ = m.query_sample(pos, u)
assert np.array_equal(host(p3), first)
m.check_device_status()
print("launch injection ok")
"""


def test_failed_launch_is_reported_and_the_next_call_works():
    env = dict(os.environ, NPM_TEST_FAIL_LAUNCH="2")
    r = subprocess.run([sys.executable, "-c", CHILD_LAUNCH.format(here=HERE, root=ROOT)], env=env,
                       capture_output=True, text=True, timeout=600)
    print(r.stdout[-1000:], r.stderr[-3000:])
    assert r.returncode == 0


CHILD_DEBUG = r"""
import sys
sys.path[:0] = [{here!r}, {root!r}]
import numpy as np, torch, oracle, synth
from gpu_helpers import PRODUCT_SMALL, cuda, host, make_model
import paper_2504_04315_gb300 as npm
from paper_2504_04315_gb300 import _lib
lib = _lib.load()
assert lib.npm_debug_bounds_violations() == 0
n = 1 << 14
for w in (synth.TINY, synth.TINY_BF16, synth.PAPER_HASH, synth.PAPER_HASH.with_(precision=synth.BF16X3),
          PRODUCT_SMALL, PRODUCT_SMALL.with_(precision=synth.BF16X3)):
    params = synth.random_params(w, 9)
    pos, u = synth.positions(9, n), synth.sample_uniforms(9, n)
    aux = synth.aux_inputs(9, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n, precision=w.precision)
    d, p, _ = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux))
    ref = oracle.eval_pdf64(w, params, pos, host(d).astype(np.float64), aux)
    err = np.abs(host(p) - ref) / np.maximum(ref, 1e-2 / (4 * np.pi))
    assert np.quantile(err, 0.999) <= 2e-2, (w.name, np.quantile(err, 0.999))
    b = synth.train_batch_uniform(w, n, seed=9)
    m.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf), None if b.aux is None else cuda(b.aux))
    m.check_device_status()
    m.close()
w = synth.TINY_BF16
m = make_model(w, synth.random_params(w, 3), 1 << 16)
with npm.Wavefront(m, 1 << 16, bounces=4, survival=0.7, train_batch=1 << 12, seed=3, use_graph=True,
                   max_frames=8) as wf:
    wf.run(2)
m.close()
v = lib.npm_debug_bounds_violations()
assert v == 0, v
print("debug build ok: no index out of bounds")
"""


def test_debug_bounds_build_finds_no_violation():
    from paper_2504_04315_gb300 import _build
    lib = _build.build_debug()
    env = dict(os.environ, NPM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD_DEBUG.format(here=HERE, root=ROOT)], env=env,
                       capture_output=True, text=True, timeout=900)
    print(r.stdout[-1000:], r.stderr[-3000:])
    assert r.returncode == 0
