"""GPU parity of the FP32-accuracy tensor-core mode (NPM_FP32_TC) against the
FP64 oracle, through the C ABI, at the FP32 path's bars.

The mode gathers the FP32 grid table and multiplies every activation and
weight as an FP16 high part plus an FP16 residual (three MMAs per K step,
FP32 accumulation); its decode, sampler and density are the FP32 path's. A
numpy model of that operand format puts the density within 5e-6 of FP64 on
these networks, so the FP32 bars (relative density 1e-4, directions 1e-4
rad, decoded lobes 1e-4) apply unchanged. Training in this mode runs the
FP32 kernels, held to the FP32 gradient bar.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import (DIR_TOL_FP32, MARGIN_FP32, PDF_RTOL_FP32, PRODUCT_SMALL, compare_samples,
                         cuda, host, make_model, rel_err)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _tc(w):
    return w.with_(precision=synth.FP32_TC)


@pytest.mark.parametrize("w,n", [(synth.TINY, 4096 + 37), (PRODUCT_SMALL, 3000),
                                 (synth.TINY.with_(kappa_act=synth.EXP), 2048),
                                 (synth.PAPER_OWN, 3000), (synth.PAPER_HASH, 4096)])
def test_query_sample_parity(w, n):
    w = _tc(w)
    params = synth.random_params(w, 3, kappa_boost=6.0 if w.kappa_act == synth.SOFTPLUS else 1.0)
    pos = synth.positions(7, n)
    u = synth.sample_uniforms(7, n)
    aux = synth.aux_inputs(7, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n)
    d, p, mix = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux), want_mix=True)
    gd, gp, gm = host(d), host(p), host(mix)
    stats = compare_samples(w, params, pos, u, aux, 0.0, gd, gp, PDF_RTOL_FP32, DIR_TOL_FP32,
                            MARGIN_FP32)
    assert np.abs(np.linalg.norm(gd, axis=0) - 1).max() < 1e-5
    om = oracle.decode_batch(w, params, pos, aux)
    # lambda, theta, phi absolute; kappa relative.
    for r in range(4):
        g, o = gm[r::4], om[r::4]
        err = rel_err(g, o, 1.0) if r == 1 else np.abs(g - o)
        assert err.max() < 1e-4, (r, err.max())
    print(stats)


def test_query_sample_with_uniform_branch():
    w = _tc(synth.PAPER_HASH)
    n = 4096
    params = synth.random_params(w, 4)
    pos = synth.positions(8, n)
    u = synth.sample_uniforms(8, n, rows=4)
    m = make_model(w, params, n)
    d, p, _ = m.query_sample(cuda(pos), cuda(u), uniform_frac=0.5)
    compare_samples(w, params, pos, u, None, 0.5, host(d), host(p), PDF_RTOL_FP32, DIR_TOL_FP32,
                    MARGIN_FP32)


def test_paper_hash_full_size_sampled():
    # The benchmark's launch: 2^20 queries in one call; the oracle checks a
    # seeded subset of 2^14 queries one by one.
    w = _tc(synth.PAPER_HASH)
    n = w.n_query
    params = synth.random_params(w, 3)
    pos = synth.positions(0, n)
    u = synth.sample_uniforms(0, n)
    m = make_model(w, params, n)
    d, p, _ = m.query_sample(cuda(pos), cuda(u))
    gd, gp = host(d), host(p)
    assert np.all(np.isfinite(gp)) and np.all(gp > 0)
    pick = np.sort(np.random.default_rng(0).choice(n, 1 << 14, replace=False))
    compare_samples(w, params, pos[:, pick], u[:, pick], None, 0.0, gd[:, pick], gp[pick],
                    PDF_RTOL_FP32, DIR_TOL_FP32, MARGIN_FP32)


@pytest.mark.parametrize("w,n", [(synth.TINY, 4096), (synth.PAPER_HASH, 8192), (PRODUCT_SMALL, 4096)])
def test_eval_pdf_and_log_pdf_parity(w, n):
    w = _tc(w)
    params = synth.random_params(w, 5)
    pos = synth.positions(9, n)
    uu = synth.uniform_rows(9, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    aux = synth.aux_inputs(9, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n)
    a = None if aux is None else cuda(aux)
    got = host(m.eval_pdf(cuda(pos), cuda(dirs), a))
    ref = oracle.eval_pdf(w, params, pos, dirs, aux)
    err = rel_err(got, ref, 1e-30)
    assert err.max() < PDF_RTOL_FP32, err.max()
    lg = host(m.eval_log_pdf(cuda(pos), cuda(dirs), a)).astype(np.float64)
    assert np.abs(lg - np.log(ref)).max() < PDF_RTOL_FP32


def test_ragged_ld_and_untouched_tail():
    w = _tc(synth.PAPER_HASH)
    n, ld = 1000, 1100
    params = synth.random_params(w, 6)
    pos = np.full((3, ld), np.nan, dtype=np.float32)
    pos[:, :n] = synth.positions(10, n)
    u = np.full((3, ld), np.nan, dtype=np.float32)
    u[:, :n] = synth.sample_uniforms(10, n)
    m = make_model(w, params, ld)
    d = torch.full((3, ld), -7.0, device="cuda")
    p = torch.full((ld,), -7.0, device="cuda")
    m.query_sample(cuda(pos), cuda(u), n=n, out=(d, p))
    gd, gp = host(d), host(p)
    assert np.all(gd[:, n:] == -7.0) and np.all(gp[n:] == -7.0)
    compare_samples(w, params, pos[:, :n], u[:, :n], None, 0.0, gd[:, :n], gp[:n], PDF_RTOL_FP32,
                    DIR_TOL_FP32, MARGIN_FP32)


def test_sizes_zero_and_one():
    w = _tc(synth.PAPER_HASH)
    params = synth.random_params(w, 6)
    m = make_model(w, params, 16)
    pos = synth.positions(11, 16)
    u = synth.sample_uniforms(11, 16)
    m.query_sample(cuda(pos), cuda(u), n=0)
    d, p, _ = m.query_sample(cuda(pos[:, :1]), cuda(u[:, :1]))
    compare_samples(w, params, pos[:, :1], u[:, :1], None, 0.0, host(d), host(p), PDF_RTOL_FP32,
                    DIR_TOL_FP32, MARGIN_FP32)


def _grad_blocks(w, g):
    ng = sum(synth.grid_sizes(w)) * w.feat
    out = [("grid", g[:ng])]
    o = ng
    for i in range(len(w.widths) - 1):
        k = w.widths[i] * w.widths[i + 1]
        out.append((f"W{i + 1}", g[o:o + k]))
        o += k
    return out


@pytest.mark.parametrize("w,n", [(synth.TINY, 4096), (synth.PAPER_HASH, 4096)])
def test_gradient_parity(w, n):
    w = _tc(w)
    params = synth.random_params(w, 12, kappa_boost=6.0)
    b = synth.train_batch_uniform(w, n, seed=12)
    m = make_model(w, params, n)
    dlogv = -(b.radiance.astype(np.float64) / b.pdf) / n
    m.backward(cuda(b.pos), cuda(b.dir), cuda(dlogv), None if b.aux is None else cuda(b.aux))
    g = m.get_grads()
    _, ref = oracle.train_grad(w, params, b.pos, b.dir, b.radiance, b.pdf, b.aux)
    for (name, gb), (_, rb) in zip(_grad_blocks(w, g), _grad_blocks(w, ref)):
        e = np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-30)
        assert e < 1e-4, (name, e)


def test_trained_model_serves_updated_weights():
    # After training steps, the tensor-core weights and the FP32 table the
    # queries read are the updated parameters: the same densities as a fresh
    # model built from them.
    w = _tc(synth.PAPER_HASH)
    n = 4096
    params = synth.random_params(w, 14)
    m = make_model(w, params, n)
    b = synth.train_batch_uniform(w, n, seed=14)
    for _ in range(3):
        m.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf))
    cur = m.get_params()
    assert np.abs(cur - params).max() > 0
    pos = synth.positions(15, n)
    uu = synth.uniform_rows(15, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    got = host(m.eval_pdf(cuda(pos), cuda(dirs)))
    ref = oracle.eval_pdf(w, cur, pos, dirs)
    assert rel_err(got, ref, 1e-30).max() < PDF_RTOL_FP32
