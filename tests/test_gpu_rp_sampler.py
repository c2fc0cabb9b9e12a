"""Directions drawn by the reduced-precision (tensor-core) path against the
FP64 oracle.

The tensor-core kernels sample with their own FP32 routine (Sec. 5.3, the
inversion of Jakob 2012 on hardware exponential, logarithm and divide, with
series for 1 - e^{-2 kappa} below 2 kappa = 0.1 and for log(1 + y) below
|y| = 1/16) and their own lobe pick. Three checks:

1. The sampling stage alone: every direction against the FP64 inversion of
   the same lobe, evaluated by the oracle's vMF sampler from the mixture the
   kernel decoded (mix_out) and the same uniforms. The lobe pick is the
   smallest i with u0 below the running FP32 sum of the decoded weights,
   reproduced exactly. Tolerance: 2e-5 rad plus the propagated error of the
   inversion's FP32 inputs and hardware logarithm. With y = u1 (e^{-2 kappa}
   - 1) and t = 1 - W = -log(1 + y) / kappa, an error e in log(1 + y) moves
   the angle by e / (kappa sin(angle)); e is at most 2^-19 |y| / (1 + y)
   from the rounding of y and e^{-2 kappa} (a few units), plus, where the
   kernel takes the hardware logarithm (|y| >= 1/16), its absolute error
   2^-21.4 on [1/2, 2] or 3 units of log(1 + y) below 1/2.
   Each series branch and the largest kappa must be exercised.
2. End to end (split BF16): directions against oracle.query_sample on the
   master parameters, within the direction error that the 2e-2 density bar
   allows at that direction (2e-2 over the tangential gradient of log V,
   capped at 2e-2 rad), with a median bar; where the oracle's u0 sits within
   1e-3 of a lobe boundary the kernel may pick the neighbouring lobe, and
   where the chosen lobe's mean lies within 1e-3 of the equator the two
   branches of the Duff et al. 2017 frame meet and only the angle to the
   mean is unique.
3. A chi-square test of 10^6 tensor-core samples at one position against the
   oracle's density integrated over 8192 bins.
"""
import math

import numpy as np
import pytest

import mixtures
import oracle
import synth
from gpu_helpers import PRODUCT_SMALL, compare_rp_directions, cuda, host, lobe_means, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# A mixture that reaches every branch of the sampler at one position: a
# nearly flat lobe (2 kappa < 0.1: the series of 1 - e^{-2 kappa}), the
# sharpest lobe of the workloads (kappa 50), and moderate ones.
RP_MIX = dict(lams=[0.3, 0.3, 0.25, 0.15], kaps=[0.02, 50.0, 5.0, 0.3],
              thetas=[0.7, 1.9, 2.6, 1.2], phis=[5.5, 2.2, 0.9, 3.7])


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _lobes(mix, K):
    m = np.asarray(mix, dtype=np.float32)
    return m[0::4].T, m[1::4].T, m[2::4].T, m[3::4].T  # [n][K] each


def _stage_check(mix, u, gd, K, ufrac=0.0, min_branch=0):
    """Check 1 of the module docstring; returns branch counts."""
    lam, kap, th, ph = _lobes(mix, K)
    n = lam.shape[0]
    u = np.asarray(u, dtype=np.float32)
    # The kernel's pick: running FP32 sum of the decoded weights.
    cum = np.zeros(n, dtype=np.float32)
    sel = np.full(n, K - 1)
    found = np.zeros(n, dtype=bool)
    for i in range(K):
        cum = (cum + lam[:, i]).astype(np.float32)
        hit = ~found & (u[0] < cum)
        sel[hit] = i
        found |= hit
    uni = (u[3] < ufrac) if ufrac > 0 else np.zeros(n, dtype=bool)
    rows = np.arange(n)
    ks = kap[rows, sel].astype(np.float64)
    mus = lobe_means(th[rows, sel], ph[rows, sel])
    u1 = u[1].astype(np.float64)
    u2 = u[2].astype(np.float64)
    exp_d = np.zeros((3, n))
    for j in range(n):
        if uni[j]:
            z = 1.0 - 2.0 * u1[j]
            r = math.sqrt(max(0.0, 1.0 - z * z))
            exp_d[:, j] = (r * math.cos(2 * math.pi * u2[j]), r * math.sin(2 * math.pi * u2[j]), z)
        else:
            exp_d[:, j] = oracle.vmf_sample(mus[j], ks[j], u1[j], u2[j])
    y = u1 * np.expm1(-2.0 * ks)
    lg = np.log1p(y)
    t = -lg / np.maximum(ks, 1e-30)
    sin_a = np.sqrt(np.clip(t * (2.0 - t), 0.0, None))
    e_log = np.where(np.abs(y) < 0.0625, 0.0,
                     np.where(1.0 + y >= 0.5, 2.0 ** -21.41, 3 * 2.0 ** -23 * np.abs(lg)))
    e_in = 2.0 ** -19 * np.abs(y) / np.maximum(1.0 + y, 1e-300)
    tol = 2e-5 + (e_log + e_in) / (np.maximum(ks, 1e-30) * np.maximum(sin_a, 1e-7))
    tol[uni] = 2e-5
    ang = np.linalg.norm(gd - exp_d, axis=0)
    # Mean on the equator: both frame branches are valid; the angle to the
    # mean is what is unique.
    eq = ~uni & (np.abs(mus[:, 2]) < 1e-5)
    w_gpu = np.einsum("jc,cj->j", mus, gd)
    w_exp = np.einsum("jc,cj->j", mus, exp_d)
    ok = np.where(eq, np.abs(w_gpu - w_exp) <= tol, ang <= tol)
    bad = np.where(~ok)[0]
    assert bad.size == 0, (
        f"{bad.size} directions off; worst {ang[bad].max():.3e} rad at {bad[:8]}, "
        f"kappa {ks[bad[:8]]}, u {u[:3, bad[:8]].T.tolist()}")
    counts = {
        "series_1_minus_exp": int(np.sum(~uni & (2.0 * ks < 0.1))),
        "series_log1p": int(np.sum(~uni & (np.abs(y) < 0.0625))),
        "kappa_ge_30": int(np.sum(~uni & (ks >= 30.0))),
        "uniform": int(uni.sum()),
        "equator": int(eq.sum()),
    }
    print("sampler stage:", counts, f"max angle {ang[~eq].max(initial=0.0):.2e}")
    if min_branch:
        for k in ("series_1_minus_exp", "series_log1p", "kappa_ge_30"):
            assert counts[k] >= min_branch, counts
    return counts


def _designed(w, n, seed):
    params = mixtures.diverse_params(w, mixtures.raw_for(**RP_MIX), mixtures.X0).astype(np.float32)
    pos = np.repeat(np.array(mixtures.X0, np.float32)[:, None], n, axis=1)
    return params, pos, synth.sample_uniforms(seed, n, rows=4)


@pytest.mark.parametrize("precision", [synth.BF16X3, synth.BF16, synth.FP16], ids=["split-bf16", "bf16", "fp16"])
@pytest.mark.parametrize("ufrac", [0.0, 0.3])
def test_rp_sampler_stage_designed_mixture(precision, ufrac):
    w = synth.TINY_BF16.with_(precision=precision)
    n = 1 << 16
    params, pos, u = _designed(w, n, 41)
    m = make_model(w, params, n, precision=precision)
    d, p, mix = m.query_sample(cuda(pos), cuda(u), uniform_frac=ufrac, want_mix=True)
    m.check_device_status()
    gd = host(d).astype(np.float64)
    assert np.abs(np.linalg.norm(gd, axis=0) - 1).max() < 1e-5
    _stage_check(host(mix), u, gd, w.K, ufrac=ufrac, min_branch=0 if ufrac else 200)


@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 1 << 16),
                                 (synth.TINY_BF16.with_(precision=synth.BF16), 1 << 16),
                                 (synth.TINY_BF16.with_(precision=synth.FP16), 1 << 16),
                                 (synth.PAPER_HASH.with_(precision=synth.BF16X3), 1 << 14),
                                 (synth.PAPER_HASH.with_(precision=synth.FP16), 1 << 14),
                                 (synth.PAPER_OWN.with_(precision=synth.BF16X3), 1 << 14),
                                 (PRODUCT_SMALL.with_(precision=synth.BF16X3), 4096),
                                 (synth.PRODUCT_BF16, 1 << 14)])
def test_rp_sampler_stage_random_models(w, n):
    params = synth.random_params(w, 42)
    pos = synth.positions(42, n)
    u = synth.sample_uniforms(42, n)
    aux = synth.aux_inputs(42, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n, precision=w.precision)
    d, _, mix = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux), want_mix=True)
    m.check_device_status()
    _stage_check(host(mix), u, host(d).astype(np.float64), w.K)


@pytest.mark.parametrize("precision", [synth.BF16X3, synth.FP16], ids=["split-bf16", "fp16"])
@pytest.mark.parametrize("w,n", [(synth.TINY_BF16, 1 << 16),
                                 (synth.PAPER_HASH, 1 << 14),
                                 (synth.PAPER_OWN, 1 << 14),
                                 (PRODUCT_SMALL, 4096),
                                 (synth.PRODUCT_BF16, 1 << 14)])
def test_rp_directions_match_oracle(w, n, precision):
    params = synth.random_params(w, 43)
    pos = synth.positions(43, n)
    u = synth.sample_uniforms(43, n)
    aux = synth.aux_inputs(43, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n, precision=precision)
    d, _, _ = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux))
    m.check_device_status()
    compare_rp_directions(w, params, pos, u, aux, host(d).astype(np.float64),
                          median_bar=3e-4 if precision == synth.BF16X3 else 1e-3)


def test_rp_directions_designed_mixture_match_oracle():
    w = synth.TINY_BF16
    n = 1 << 16
    params, pos, u = _designed(w, n, 44)
    m = make_model(w, params, n, precision=synth.BF16X3)
    d, _, _ = m.query_sample(cuda(pos), cuda(u[:3].copy()))
    m.check_device_status()
    compare_rp_directions(w, params, pos, u[:3], None, host(d).astype(np.float64))


@pytest.mark.parametrize("precision", [synth.BF16X3, synth.FP16], ids=["split-bf16", "fp16"])
def test_rp_chi_square_against_oracle_density(precision):
    # 10^6 tensor-core samples at X0 against the oracle's V integrated over
    # 64 x 128 equal-area bins.
    w = synth.TINY_BF16
    n = 1_000_000
    params, pos, u = _designed(w, n, 45)
    m = make_model(w, params, n, precision=precision)
    d, _, _ = m.query_sample(cuda(pos), cuda(u[:3].copy()))
    m.check_device_status()
    gd = host(d).astype(np.float64)

    def density(dirs):
        posq = np.repeat(np.array(mixtures.X0, np.float32)[:, None], dirs.shape[1], axis=1)
        return oracle.eval_pdf64(w, params, posq, dirs)

    p, chi2 = mixtures.chi2_directions(gd, density)
    print(f"chi-square {chi2:.1f}, p = {p:.3f}")
    assert p > 0.01, p
