"""The hand-written backward behind a torch.autograd.Function (log_density):
its gradient matches the FP64 oracle's and central finite differences of the
GPU forward, for the FP32 path."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import PRODUCT_SMALL, cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _batch(w, n, seed):
    b = synth.train_batch_uniform(w, n, seed=seed)
    wts = (b.radiance.astype(np.float64) / b.pdf) / n  # loss = -sum wts log V
    return b, wts


@pytest.mark.parametrize("w", [synth.TINY, PRODUCT_SMALL], ids=["tiny", "product"])
def test_log_density_gradient_matches_oracle(w):
    import paper_2504_04315_gb300 as npm
    n = 4096
    params = synth.random_params(w, 21)
    b, wts = _batch(w, n, 21)
    m = make_model(w, synth.init_params(w), n)  # theta, not the handle, holds the parameters
    theta = torch.from_numpy(params.astype(np.float32)).cuda().requires_grad_(True)
    aux = None if b.aux is None else cuda(b.aux)
    logv = npm.log_density(theta, m, cuda(b.pos), cuda(b.dir), aux)
    loss = -(torch.from_numpy(wts.astype(np.float32)).cuda() * logv).sum()
    loss.backward()
    m.check_device_status()
    ref_loss, ref = oracle.train_grad(w, params, b.pos, b.dir, b.radiance, b.pdf, b.aux)
    # log V itself, and the loss
    ov = oracle.eval_pdf(w, params, b.pos, b.dir, b.aux)
    assert np.abs(host(logv) - np.log(ov)).max() < 1e-4
    assert abs(float(loss.detach()) - ref_loss) <= 1e-4 * abs(ref_loss)
    g = host(theta.grad).astype(np.float64)
    ng = sum(synth.grid_sizes(w)) * w.feat
    blocks = [slice(0, ng)]
    o = ng
    for i in range(len(w.widths) - 1):
        k = w.widths[i] * w.widths[i + 1]
        blocks.append(slice(o, o + k))
        o += k
    for sl in blocks:
        err = np.linalg.norm(g[sl] - ref[sl]) / max(np.linalg.norm(ref[sl]), 1e-30)
        assert err <= 1e-4, (sl, err)


def test_log_density_gradient_matches_finite_differences():
    # Central differences of the GPU forward along random directions of the
    # whole parameter vector against the autograd directional derivative.
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    n = 4096
    params = synth.random_params(w, 22).astype(np.float64)
    b, wts = _batch(w, n, 22)
    m = make_model(w, synth.init_params(w), n)
    pos, dirs = cuda(b.pos), cuda(b.dir)
    wt = torch.from_numpy(wts).cuda()

    def f(p):
        with torch.no_grad():
            lv = npm.log_density(torch.from_numpy(p.astype(np.float32)).cuda(), m, pos, dirs)
            return float(-(wt * lv.double()).sum())

    theta = torch.from_numpy(params.astype(np.float32)).cuda().requires_grad_(True)
    loss = -(wt * npm.log_density(theta, m, pos, dirs).double()).sum()
    loss.backward()
    g = host(theta.grad).astype(np.float64)
    rng = np.random.default_rng(22)
    h = 1e-2
    for _ in range(3):
        v = rng.standard_normal(params.size)
        v /= np.linalg.norm(v)
        fd = (f(params + h * v) - f(params - h * v)) / (2 * h)
        an = float(g @ v)
        assert abs(fd - an) <= 1e-2 * max(abs(an), 1e-3), (fd, an)
