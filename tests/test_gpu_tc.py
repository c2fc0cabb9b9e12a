"""GPU parity of the tensor-core path (tcgen05 MLP, FP16 grid, FP32 vMF)
against the FP64 oracle run with the FP32 master parameters.

Bar for the reduced-precision path: relative density error at the
GPU-sampled direction, denominator floored at 1e-2/(4 pi), at most 2e-2 at
the 99.9th percentile. Split BF16 (NPM_BF16X3) meets it on every workload.

Single-pass BF16 inference (NPM_BF16) does not meet it on these sharp-lobe
parameters (kappa up to ~35): its 8-bit significands put the density 1.5e-2
to 6e-2 off at the 99.9th percentile. Its kernels are checked instead
against a model of exactly that quantisation (tests/bf16_model.py: FP16
table, BF16 operands rounded to nearest, FP32 sums), within 2e-3 at the
99.9th percentile, and its distance from the oracle is printed. Training
takes split operands in both reduced-precision modes and is held to the
2e-2 gradient bar.
"""
import math

import numpy as np
import pytest

import bf16_model
import oracle
import synth
from gpu_helpers import PRODUCT_SMALL, compare_rp_directions, cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PDF_P999_BF16 = 2e-2
# Single-pass BF16 against the model of its own operand rounding.
PDF_P999_BF16_MODEL = 2e-3
FLOOR = 1e-2 / (4 * math.pi)


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _bf16_stats(w, n, seed, params=None, precision=synth.BF16X3):
    params = synth.random_params(w, seed) if params is None else params
    pos = synth.positions(seed, n)
    u = synth.sample_uniforms(seed, n)
    aux = synth.aux_inputs(seed, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n, precision=precision)
    d, p, mix = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux),
                               want_mix=True)
    gd, gp, gm = host(d), host(p), host(mix)
    assert np.all(np.isfinite(gp)) and np.all(gp > 0)
    assert np.abs(np.linalg.norm(gd, axis=0) - 1).max() < 1e-5
    ref = oracle.eval_pdf64(w, params, pos, gd.astype(np.float64), aux)
    err = np.abs(gp - ref) / np.maximum(ref, FLOOR)
    om = oracle.decode_batch(w, params, pos, aux)
    m.check_device_status()
    return err, gm, om, m, params, pos, aux


def _bf16_single_vs_model(n, seed, dirs=None):
    """Single-pass BF16: density at the sampled (or given) directions
    against the BF16 quantisation model; returns (error vs model, error vs
    oracle)."""
    w = synth.TINY_BF16.with_(precision=synth.BF16)
    params = synth.random_params(w, seed)
    pos = synth.positions(seed, n)
    m = make_model(w, params, n, precision=synth.BF16)
    if dirs is None:
        d, p, _ = m.query_sample(cuda(pos), cuda(synth.sample_uniforms(seed, n)))
        gd = host(d).astype(np.float64)
    else:
        gd = dirs.astype(np.float64)
        p = m.eval_pdf(cuda(pos), cuda(dirs))
    gp = host(p).astype(np.float64)
    m.check_device_status()
    model = bf16_model.density(w, bf16_model.raw_outputs(w, params, pos), gd)
    ref = oracle.eval_pdf64(w, params, pos, gd)
    e_model = np.abs(gp - model) / np.maximum(model, FLOOR)
    e_oracle = np.abs(gp - ref) / np.maximum(ref, FLOOR)
    print(f"bf16 n={n}: vs quantisation model p99.9 {np.quantile(e_model, 0.999):.2e} max {e_model.max():.2e}; "
          f"vs oracle p99.9 {np.quantile(e_oracle, 0.999):.2e} (outside the 2e-2 bar is expected)")
    return e_model, e_oracle


@pytest.mark.parametrize("n", [1, 128, 1000, 1 << 16])
def test_tc_bf16_single_matches_quantisation_model(n):
    e_model, _ = _bf16_single_vs_model(n, 21 if n < 4096 else 22)
    assert np.quantile(e_model, 0.999) <= PDF_P999_BF16_MODEL


@pytest.mark.parametrize("precision", [synth.BF16X3, synth.FP16], ids=["split-bf16", "fp16"])
@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 1 << 16),
                                 (synth.PAPER_HASH, 1 << 14),
                                 (synth.PAPER_OWN, 1 << 14),
                                 (PRODUCT_SMALL, 4096),
                                 (synth.PRODUCT_BF16, 1 << 14)])
def test_tc_reduced_precision_parity(w, n, precision):
    # Split BF16 (hi + residual operands, three MMAs per K step): the error
    # left is the FP16 rounding of the grid features. FP16 operands (weights
    # with an FP16 residual, two MMAs per K step): the FP16 rounding of the
    # activations as well.
    w = w.with_(precision=precision)
    err, gm, om, _, _, _, _ = _bf16_stats(w, n, 22, precision=precision)
    print(f"precision {precision} {w.name[:30]} n={n} pdf err p50 {np.median(err):.2e} p99.9 "
          f"{np.quantile(err, 0.999):.2e} max {err.max():.2e}")
    assert np.quantile(err, 0.999) <= (1e-2 if precision == synth.BF16X3 else PDF_P999_BF16)
    assert np.median(err) <= 1e-3


@pytest.mark.parametrize("dirs_from", ["mixture", "uniform"])
def test_tc_bf16_single_eval_pdf_matches_quantisation_model(dirs_from):
    n = 4096
    if dirs_from == "uniform":
        uu = synth.uniform_rows(23, synth.S_DIR, 2, n)
        dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    else:
        w = synth.TINY_BF16
        dirs = oracle.query_sample(w, synth.random_params(w, 23), synth.positions(23, n),
                                   synth.sample_uniforms(23, n))[0].astype(np.float32)
    e_model, _ = _bf16_single_vs_model(n, 23, dirs=dirs)
    assert np.quantile(e_model, 0.999) <= PDF_P999_BF16_MODEL


@pytest.mark.parametrize("precision", [synth.BF16X3, synth.FP16], ids=["split-bf16", "fp16"])
@pytest.mark.parametrize("dirs_from", ["mixture", "uniform"])
def test_tc_eval_pdf_matches_oracle(dirs_from, precision):
    # Split BF16 and FP16 densities at directions drawn from the mixture
    # (where the guide is used) and uniformly.
    w = synth.TINY_BF16
    n = 4096
    params = synth.random_params(w, 23)
    pos = synth.positions(23, n)
    if dirs_from == "uniform":
        uu = synth.uniform_rows(23, synth.S_DIR, 2, n)
        dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    else:
        dirs = oracle.query_sample(w, params, pos, synth.sample_uniforms(23, n))[0].astype(np.float32)
    m = make_model(w, params, n, precision=precision)
    got = host(m.eval_pdf(cuda(pos), cuda(dirs)))
    ref = oracle.eval_pdf(w, params, pos, dirs)
    err = np.abs(got - ref) / np.maximum(ref, FLOOR)
    print(f"eval precision {precision} dirs={dirs_from}: p99.9 {np.quantile(err, 0.999):.2e}")
    assert np.quantile(err, 0.999) <= PDF_P999_BF16


@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 4096), (PRODUCT_SMALL.with_(precision=synth.BF16X3), 4096),
                                 (synth.PAPER_HASH.with_(precision=synth.BF16X3), 4096),
                                 (synth.PAPER_OWN.with_(precision=synth.BF16X3), 4096),
                                 (synth.PRODUCT_BF16, 3000),
                                 (synth.TINY_BF16.with_(precision=synth.BF16), 4096),
                                 (synth.TINY_BF16.with_(precision=synth.FP16), 4096),
                                 (synth.PAPER_HASH.with_(precision=synth.FP16), 4096)])
def test_tc_gradient_parity(w, n):
    # Training on tensor cores (FP32 TMEM accumulation, split BF16
    # operands in both reduced-precision modes) against the FP64 oracle
    # with the FP32 master parameters: per-tensor relative L2 <= 2e-2.
    params = synth.random_params(w, 12)
    b = synth.train_batch_uniform(w, n, seed=12)
    m = make_model(w, params, n, precision=w.precision)
    dlogv = -(b.radiance.astype(np.float64) / b.pdf) / n
    m.backward(cuda(b.pos), cuda(b.dir), cuda(dlogv), None if b.aux is None else cuda(b.aux))
    g = m.get_grads()
    m.check_device_status()
    loss, ref = oracle.train_grad(w, params, b.pos, b.dir, b.radiance, b.pdf, b.aux)
    ng = sum(synth.grid_sizes(w)) * w.feat
    blocks = [("grid", slice(0, ng))]
    o = ng
    for i in range(len(w.widths) - 1):
        k = w.widths[i] * w.widths[i + 1]
        blocks.append((f"W{i + 1}", slice(o, o + k)))
        o += k
    errs = {}
    for name, sl in blocks:
        errs[name] = np.linalg.norm(g[sl] - ref[sl]) / max(np.linalg.norm(ref[sl]), 1e-30)
    print(f"tc grad rel L2 {w.name[:30]} precision {w.precision}: "
          + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    bar = 2e-2
    assert max(errs.values()) <= bar, errs
    # The training loss of the same batch through train_step.
    m2 = make_model(w, params, n, precision=w.precision)
    l2 = m2.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf),
                       None if b.aux is None else cuda(b.aux))
    assert abs(float(host(l2)[0]) - loss) <= bar * abs(loss)


@pytest.mark.parametrize("w", [synth.TINY_BF16, synth.PAPER_HASH.with_(precision=synth.BF16X3),
                               synth.TINY_BF16.with_(precision=synth.FP16)],
                         ids=["tiny-split-bf16", "paper-hash-split-bf16", "tiny-fp16"])
def test_tc_kl_estimate_matches_oracle(w):
    # KL estimate of the guide against the noise-free target on a seeded
    # 2^16 subset: (1/N) sum_j (D_j / p_j) (log D_j - log V_j), directions
    # uniform on the sphere (p_j = 1/(4 pi)) and D the analytic radiance
    # field, itself a normalised density in w (amplitudes summing to 1 times
    # normalised lobes). The reduced-precision path's estimate stays within
    # 1e-3 absolute of the same estimate with the FP64 oracle's density.
    n = 1 << 16
    params = synth.random_params(w, 17)
    pos = synth.positions(17, n)
    uu = synth.uniform_rows(17, synth.S_DIR, 2, n)
    d32 = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    m = make_model(w, params, n, precision=w.precision)
    vg = host(m.eval_pdf(cuda(pos), cuda(d32))).astype(np.float64)
    m.check_device_status()
    assert np.all(np.isfinite(vg)) and np.all(vg > 0)
    dirs = d32.astype(np.float64)
    vo = oracle.eval_pdf64(w, params, pos, dirs)
    target = synth.radiance(pos.astype(np.float64), dirs)
    wgt = target * (4 * math.pi)
    kl_g = float(np.mean(wgt * (np.log(target) - np.log(vg))))
    kl_o = float(np.mean(wgt * (np.log(target) - np.log(vo))))
    print(f"KL {w.name[:30]}: gpu {kl_g:.6f} oracle {kl_o:.6f} diff {abs(kl_g - kl_o):.2e}")
    assert abs(kl_g - kl_o) <= 1e-3


@pytest.mark.parametrize("precision", [synth.BF16X3, synth.FP16], ids=["split-bf16", "fp16"])
def test_tc_tiny_full_size_launch_sampled(precision):
    # The reduced-precision workload as the benchmark launches it: 2^22
    # queries in one call; the oracle checks a seeded 2^16 subset: the
    # density at the GPU-sampled directions and the directions themselves
    # (oracle.query_sample on the same uniforms).
    w = synth.TINY_BF16.with_(precision=precision)
    n = w.n_query
    params = synth.random_params(w, 3)
    pos = synth.positions(0, n)
    u = synth.sample_uniforms(0, n)
    m = make_model(w, params, n, precision=w.precision)
    d, p, _ = m.query_sample(cuda(pos), cuda(u))
    m.check_device_status()
    gd, gp = host(d), host(p)
    assert np.all(np.isfinite(gp)) and np.all(gp > 0)
    pick = np.sort(np.random.default_rng(1).choice(n, 1 << 16, replace=False))
    assert np.abs(np.linalg.norm(gd[:, pick], axis=0) - 1).max() < 1e-5
    ref = oracle.eval_pdf64(w, params, pos[:, pick], gd[:, pick].astype(np.float64))
    err = np.abs(gp[pick] - ref) / np.maximum(ref, FLOOR)
    print(f"tiny 2^22 launch, 2^16 subset: p99.9 {np.quantile(err, 0.999):.2e} max {err.max():.2e}")
    assert np.quantile(err, 0.999) <= PDF_P999_BF16
    compare_rp_directions(w, params, pos[:, pick], u[:, pick], None, gd[:, pick].astype(np.float64),
                          median_bar=3e-4 if precision == synth.BF16X3 else 1e-3)
