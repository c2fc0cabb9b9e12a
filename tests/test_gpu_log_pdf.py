"""npm_eval_log_pdf: log V from the kernels in log-sum-exp form, against the
log of the FP64 oracle's density -- at ordinary directions (FP32 and split
BF16 paths) and at directions where V itself underflows FP32 (far from every
lobe of a sharp mixture), where only the log-domain form stays finite."""
import math

import numpy as np
import pytest

import mixtures
import oracle
import synth
from gpu_helpers import PRODUCT_SMALL, cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Four sharp lobes around the north pole: at the south pole every term is
# about e^{-2 kappa} <= e^{-120} (underflows FP32) while log V ~ -120.
SHARP = dict(lams=[0.4, 0.3, 0.2, 0.1], kaps=[60.0, 80.0, 70.0, 90.0],
             thetas=[0.2, 0.3, 0.25, 0.35], phis=[0.5, 2.0, 3.5, 5.0])


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@pytest.mark.parametrize("w,precision,tol", [(synth.TINY, synth.FP32, 1e-4),
                                             (synth.PAPER_HASH, synth.FP32, 1e-4),
                                             (PRODUCT_SMALL, synth.FP32, 1e-4),
                                             (synth.TINY_BF16, synth.BF16X3, 2e-2),
                                             (synth.TINY_BF16, synth.FP16, 2e-2),
                                             (synth.PAPER_HASH, synth.BF16X3, 2e-2)])
def test_log_pdf_matches_oracle(w, precision, tol):
    n = 4096
    params = synth.random_params(w, 51)
    pos = synth.positions(51, n)
    uu = synth.uniform_rows(51, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    aux = synth.aux_inputs(51, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n, precision=precision)
    lv = host(m.eval_log_pdf(cuda(pos), cuda(dirs), None if aux is None else cuda(aux))).astype(np.float64)
    v = host(m.eval_pdf(cuda(pos), cuda(dirs), None if aux is None else cuda(aux))).astype(np.float64)
    m.check_device_status()
    ref = np.log(oracle.eval_pdf(w, params, pos, dirs, aux))
    err = np.abs(lv - ref)
    print(f"{w.name[:30]} precision {precision}: |log V err| max {err.max():.2e} p99.9 {np.quantile(err, 0.999):.2e}")
    # An absolute error eps in log V is a relative density error of about eps.
    assert np.quantile(err, 0.999) <= tol
    if precision == synth.FP32:
        assert err.max() <= tol
    # Where V is representable, log V agrees with the log of npm_eval_pdf.
    ok = v > 1e-30
    assert np.abs(lv[ok] - np.log(v[ok])).max() <= 1e-5 * np.maximum(1.0, np.abs(lv[ok])).max()


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3])
def test_log_pdf_finite_where_density_underflows(precision):
    w = synth.TINY.with_(precision=precision)
    params = mixtures.diverse_params(w, mixtures.raw_for(**SHARP), mixtures.X0).astype(np.float32)
    n = 256
    pos = np.repeat(np.array(mixtures.X0, np.float32)[:, None], n, axis=1)
    # Directions in a cap around the south pole.
    th = math.pi - 0.3 * np.linspace(0, 1, n)
    ph = np.linspace(0, 2 * math.pi, n)
    dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]).astype(np.float32)
    m = make_model(w, params, n, precision=precision)
    lv = host(m.eval_log_pdf(cuda(pos), cuda(dirs))).astype(np.float64)
    v = host(m.eval_pdf(cuda(pos), cuda(dirs)))
    m.check_device_status()
    ref = np.log(oracle.eval_pdf64(w, params, pos, dirs.astype(np.float64)))
    assert ref.max() < -100, ref.max()        # the density is far below FP32's range
    assert np.all(v < 1e-37)                    # the linear form underflows
    assert np.all(np.isfinite(lv))
    err = np.abs(lv - ref) / np.abs(ref)
    print(f"precision {precision}: log V {ref.min():.1f} .. {ref.max():.1f}, max rel err {err.max():.2e}")
    assert err.max() <= (1e-5 if precision == synth.FP32 else 2e-3)
