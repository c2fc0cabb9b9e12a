"""FP64 validation reduction on the GPU: the mixture density integrates to 1.

V(w | x) is a density on the sphere (Eq. 3-4), so its integral is 1 for any
network outputs. npm_pdf_integral evaluates V through the same kernels as
every query (FP32 CUDA cores or tensor cores) on a Gauss-Legendre (cos theta)
x uniform (phi) grid of 320,000 directions and reduces the weighted sum in
FP64 on the GPU; the FP64 oracle reaches 1e-10 on the same grid.
"""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import PRODUCT_SMALL, cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def sphere_quadrature(nz, nphi):
    z, wz = np.polynomial.legendre.leggauss(nz)
    ph = (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
    Z, P = np.meshgrid(z, ph, indexing="ij")
    r = np.sqrt(1 - Z * Z)
    dirs = np.stack([r * np.cos(P), r * np.sin(P), Z]).reshape(3, -1)
    wts = (wz[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).ravel()
    return dirs, wts


@pytest.mark.parametrize("w", [synth.TINY, synth.PAPER_HASH, PRODUCT_SMALL, synth.TINY_BF16],
                         ids=["tiny-fp32", "paper-hash-fp32", "product-fp32", "tiny-split-bf16"])
def test_pdf_integrates_to_one_fp64_reduction_on_gpu(w):
    dirs, wts = sphere_quadrature(400, 800)
    n_dir = dirs.shape[1]
    n_pos = 12
    params = synth.random_params(w, 13)  # sharp lobes: kappa up to ~35
    pos = synth.positions(13, n_pos)
    aux = synth.aux_inputs(13, n_pos) if w.mode == synth.PRODUCT else None
    # max_batch of two positions' grids: the call works in six chunks.
    m = make_model(w, params, 2 * n_dir, precision=w.precision)
    out = m.pdf_integral(cuda(pos), cuda(dirs), torch.from_numpy(wts).cuda(),
                         None if aux is None else cuda(aux))
    assert out.dtype == torch.float64
    integ = host(out)
    m.check_device_status()
    print(f"{w.name[:40]}: max |I - 1| = {np.abs(integ - 1).max():.2e}")
    assert np.abs(integ - 1).max() < 1e-5
