"""GPU parity of the tensor-core path (tcgen05 MLP, FP16 grid, FP32 vMF)
against the FP64 oracle run with the FP32 master parameters.

Bar for the reduced-precision path: relative density error at the
GPU-sampled direction, denominator floored at 1e-2/(4 pi), at most 2e-2 at
the 99.9th percentile. Split BF16 (NPM_BF16X3) meets it on every workload.
Single-pass BF16 (NPM_BF16) is held to a looser 5e-2: on these sharp-lobe
parameters (kappa up to ~35) the BF16 rounding of the lobe means alone is
amplified to 1.5e-2 .. 4e-2.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import PRODUCT_SMALL, cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PDF_P999_BF16 = 2e-2
PDF_P999_BF16_SINGLE = 5e-2
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


@pytest.mark.parametrize("n", [1, 128, 1000])
def test_tc_small_tiny(n):
    err, gm, om, _, _, _, _ = _bf16_stats(synth.TINY_BF16, n, 21, precision=synth.BF16)
    print(f"n={n} pdf err p50 {np.median(err):.2e} p99.9 {np.quantile(err, 0.999):.2e} max {err.max():.2e}")
    assert np.quantile(err, 0.999) <= PDF_P999_BF16_SINGLE
    # decoded weights match to BF16 accuracy
    assert np.abs(gm[0::4] - om[0::4]).max() < 3e-2


@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 1 << 16)])
def test_tc_pdf_parity(w, n):
    err, gm, om, _, _, _, _ = _bf16_stats(w, n, 22, precision=synth.BF16)
    print(f"{w.name[:30]} n={n} pdf err p50 {np.median(err):.2e} p99.9 "
          f"{np.quantile(err, 0.999):.2e} max {err.max():.2e}")
    assert np.quantile(err, 0.999) <= PDF_P999_BF16_SINGLE


@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 1 << 16),
                                 (synth.PAPER_HASH.with_(precision=synth.BF16X3), 1 << 14),
                                 (synth.PAPER_OWN.with_(precision=synth.BF16X3), 1 << 14),
                                 (PRODUCT_SMALL.with_(precision=synth.BF16X3), 4096),
                                 (synth.PRODUCT_BF16.with_(precision=synth.BF16X3), 1 << 14)])
def test_tc_split_bf16_parity(w, n):
    # Split BF16 (hi + residual operands, three MMAs per K step): the error
    # left is the FP16 rounding of the grid features.
    err, gm, om, _, _, _, _ = _bf16_stats(w, n, 22, precision=synth.BF16X3)
    print(f"bf16x3 {w.name[:30]} n={n} pdf err p50 {np.median(err):.2e} p99.9 "
          f"{np.quantile(err, 0.999):.2e} max {err.max():.2e}")
    assert np.quantile(err, 0.999) <= 1e-2
    assert np.median(err) <= 1e-3


@pytest.mark.parametrize("precision,dirs_from", [(synth.BF16, "mixture"), (synth.BF16X3, "mixture"),
                                                 (synth.BF16X3, "uniform")])
def test_tc_eval_pdf_matches_oracle(precision, dirs_from):
    # Plain BF16 is held to the bar at directions drawn from the mixture
    # (where the guide is used); split BF16 also at uniform directions.
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
    print(f"eval precision={precision} dirs={dirs_from}: p99.9 {np.quantile(err, 0.999):.2e}")
    bar = PDF_P999_BF16 if precision == synth.BF16X3 else PDF_P999_BF16_SINGLE
    assert np.quantile(err, 0.999) <= bar


def test_tc_matches_fp32_path_on_lobe_choice():
    # The BF16 path picks the same lobe as the FP32 path except near CDF
    # boundaries: compare directions from both GPU paths.
    w = synth.TINY_BF16
    n = 1 << 14
    params = synth.random_params(w, 24)
    pos = synth.positions(24, n)
    u = synth.sample_uniforms(24, n)
    mb = make_model(w, params, n, precision=synth.BF16X3)
    mf = make_model(w, params, n, precision=synth.FP32)
    db, _, _ = mb.query_sample(cuda(pos), cuda(u))
    df, _, _ = mf.query_sample(cuda(pos), cuda(u))
    ang = np.linalg.norm(host(db) - host(df), axis=0)
    assert np.median(ang) < 2e-2
    assert (ang > 0.5).mean() < 2e-2


@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 4096), (PRODUCT_SMALL.with_(precision=synth.BF16X3), 4096),
                                 (synth.PAPER_HASH.with_(precision=synth.BF16X3), 4096),
                                 (synth.PAPER_OWN.with_(precision=synth.BF16X3), 4096),
                                 (synth.PRODUCT_BF16, 3000),
                                 (synth.TINY_BF16.with_(precision=synth.BF16), 4096)])
def test_tc_gradient_parity(w, n):
    # Training on tensor cores (FP32 TMEM accumulation, FP16 grid features)
    # against the FP64 oracle with the FP32 master parameters. Split BF16:
    # per-tensor relative L2 <= 2e-2. Single-pass BF16 compounds its rounding
    # down the layers and the grid sums cancel heavily: held to 0.3.
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
    bar = 2e-2 if w.precision == synth.BF16X3 else 0.3
    assert max(errs.values()) <= bar, errs
    # The training loss of the same batch through train_step.
    m2 = make_model(w, params, n, precision=w.precision)
    l2 = m2.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf),
                       None if b.aux is None else cuda(b.aux))
    assert abs(float(host(l2)[0]) - loss) <= bar * abs(loss)


@pytest.mark.parametrize("w", [synth.TINY_BF16, synth.PAPER_HASH.with_(precision=synth.BF16X3)],
                         ids=["tiny-split-bf16", "paper-hash-split-bf16"])
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


def test_tc_tiny_full_size_launch_sampled():
    # The reduced-precision workload as the benchmark launches it: 2^22
    # queries in one call, split BF16; the oracle checks a seeded 2^16 subset
    # at the GPU-sampled directions.
    w = synth.TINY_BF16
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
