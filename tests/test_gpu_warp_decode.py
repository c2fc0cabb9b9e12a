"""The warp-per-query decode of the general tensor-core kernel (one lane per
lobe; selected by the tuning override NPM_TC_DECODE=1, read once per
process, so each case runs in a child process): the same sampler-stage
check, directions against the oracle and densities as the thread-per-query
decode."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def _child(name):
    import oracle
    import synth
    from gpu_helpers import compare_rp_directions, cuda, host, make_model
    from test_gpu_rp_sampler import _stage_check
    w = {"tiny": synth.TINY_BF16, "paper_hash": synth.PAPER_HASH.with_(precision=synth.BF16X3)}[name]
    n = 1 << 14
    params = synth.random_params(w, 71)
    pos = synth.positions(71, n)
    u = synth.sample_uniforms(71, n, rows=4)
    m = make_model(w, params, n, precision=synth.BF16X3)
    d, p, mix = m.query_sample(cuda(pos), cuda(u), want_mix=True)
    gd = host(d).astype(np.float64)
    _stage_check(host(mix), u, gd, w.K)
    compare_rp_directions(w, params, pos, u[:3], None, gd)
    ref = oracle.eval_pdf64(w, params, pos, gd)
    err = np.abs(host(p) - ref) / np.maximum(ref, 1e-2 / (4 * np.pi))
    assert np.quantile(err, 0.999) <= 2e-2, np.quantile(err, 0.999)
    # uniform-sphere mixture and density / log-density evaluation
    d2, p2, mix2 = m.query_sample(cuda(pos), cuda(u), uniform_frac=0.3, want_mix=True)
    _stage_check(host(mix2), u, host(d2).astype(np.float64), w.K, ufrac=0.3)
    uu = synth.uniform_rows(72, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    ref = oracle.eval_pdf(w, params, pos, dirs)
    ev = host(m.eval_pdf(cuda(pos), cuda(dirs)))
    lv = host(m.eval_log_pdf(cuda(pos), cuda(dirs)))
    assert np.quantile(np.abs(ev - ref) / np.maximum(ref, 1e-2 / (4 * np.pi)), 0.999) <= 2e-2
    assert np.quantile(np.abs(lv - np.log(ref)), 0.999) <= 2e-2
    m.check_device_status()
    print(f"warp decode {name}: ok")


@pytest.mark.parametrize("name", ["tiny", "paper_hash"])
def test_warp_decode_matches_oracle(name):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    env = dict(os.environ, NPM_TC_DECODE="1", NPM_TC_TINY="0")
    r = subprocess.run([sys.executable, "-c",
                        f"import sys; sys.path[:0] = [{HERE!r}, {os.path.dirname(HERE)!r}]; "
                        f"import test_gpu_warp_decode as t; t._child({name!r})"],
                       env=env, capture_output=True, text=True, timeout=600)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0
