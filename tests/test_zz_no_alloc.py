"""npm_eval_pdf_noalloc: the allocation-free density evaluation for callers
that cannot allocate device memory (a renderer with its own allocator, a
plug-in that may not call cudaMalloc during a frame). It must give the same
densities as npm_eval_pdf on a handle with the same parameters and as the
FP64 oracle, call after call, although every call shares one static scratch
array.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import PDF_RTOL_FP32, PRODUCT_SMALL, cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(cfg, params_dev, pos, dirs, aux, out):
    from paper_2504_04315_gb300 import _lib
    lib = _lib.load()
    ld = pos.shape[1]
    st = lib.npm_eval_pdf_noalloc(C.byref(cfg), params_dev.data_ptr(), ld, pos.data_ptr(),
                                  None if aux is None else aux.data_ptr(), dirs.data_ptr(), ld,
                                  out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    _lib.check(st, "npm_eval_pdf_noalloc")


def _case(w, n, seed):
    import paper_2504_04315_gb300 as npm
    params = synth.random_params(w, seed)
    pos = synth.positions(seed, n)
    uu = synth.uniform_rows(seed, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    aux = synth.aux_inputs(seed, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n, precision=synth.FP32)
    ref = host(m.eval_pdf(cuda(pos), cuda(dirs), None if aux is None else cuda(aux)))
    m.close()
    orc = oracle.eval_pdf(w, params, pos, dirs, aux)
    cfg = npm.config_from(w, max_batch=n, precision=synth.FP32)
    return cfg, cuda(params), cuda(pos), cuda(dirs), None if aux is None else cuda(aux), ref, orc


def test_noalloc_matches_eval_pdf_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    # The tiny model, a product-mode model and the paper-shaped hash grid
    # (16 levels, 32-64-64-64-32, K = 8: 12,288 padded weight floats, the
    # network on which npm_eval_pdf runs the warp-specialised kernel).
    cases = [_case(synth.TINY, 4096 + 37, 31), _case(PRODUCT_SMALL, 3000, 32),
             _case(synth.PAPER_HASH, 5000, 33)]
    # Calls in a row on different models: each overwrites the shared
    # scratch left by the one before. Then the first model again.
    for cfg, p, pos, dirs, aux, ref, orc in cases + cases[:1]:
        out = torch.full((pos.shape[1],), -1.0, device="cuda")
        _noalloc(cfg, p, pos, dirs, aux, out)
        got = host(out)
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)
        assert err.max() <= PDF_RTOL_FP32, err.max()
        err_o = np.abs(got - orc) / np.maximum(np.abs(orc), 1e-30)
        assert err_o.max() <= PDF_RTOL_FP32, err_o.max()


def test_noalloc_rejects_weights_beyond_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2504_04315_gb300 as npm
    from paper_2504_04315_gb300 import _lib
    w = synth.Workload(name="too wide for the static scratch", mode=synth.RADIANCE,
                       level_res=[16], feat=4, log2_table=19, widths=[64, 128, 128, 64, 32], K=8)
    cfg = npm.config_from(w, max_batch=16)
    p = torch.zeros(synth.n_params(w), device="cuda")
    pos = torch.zeros((3, 16), device="cuda")
    out = torch.zeros(16, device="cuda")
    lib = _lib.load()
    st = lib.npm_eval_pdf_noalloc(C.byref(cfg), p.data_ptr(), 16, pos.data_ptr(), None,
                                  pos.data_ptr(), 16, out.data_ptr(), None)
    assert st == _lib.ERR_CAPACITY
    assert b"NPM_NOALLOC_MAX_WEIGHT_FLOATS" in lib.npm_last_error()
