"""Training on the GPU: the device input generator matches the host one, the
multi-step loss curve tracks the FP64 oracle, and online training (Sec. 5.2)
gains over sampling without the guide."""
import math

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


@pytest.mark.parametrize("product", [False, True])
def test_device_generator_matches_host(product):
    from paper_2504_04315_gb300 import scene
    n, seed = 5000, 17
    pos, aux, u = scene.generate(seed, n, product, urows=4)
    assert np.array_equal(host(pos), synth.positions(seed, n))
    assert np.array_equal(host(u), synth.sample_uniforms(seed, n, rows=4))
    ref_aux = synth.aux_inputs(seed, n) if product else None
    if product:
        a = host(aux)
        # The hemisphere flip may differ only where wo is nearly tangent.
        ok = np.abs(np.sum(ref_aux[0:3] * ref_aux[3:6], axis=0)) > 1e-4
        assert np.abs(a[:, ok] - ref_aux[:, ok]).max() < 2e-6
    uu = synth.uniform_rows(seed, synth.S_DIR, 2, n)
    d = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    clean, noisy = scene.radiance(product, pos, None if aux is None else cuda(ref_aux), cuda(d),
                                  noise_seed=seed)
    ref = synth.target(synth.positions(seed, n), d, ref_aux)
    assert np.abs(host(clean) - ref).max() <= 2e-5 * ref.max()
    assert np.allclose(host(noisy), ref * synth.exp_noise(seed, n), rtol=2e-5, atol=2e-5 * ref.max())


def test_multistep_loss_curve_tracks_oracle():
    # 30 Adam steps on fixed samples (directions uniform, so the data do not
    # depend on the model): GPU FP32 and the FP64 oracle give the same loss
    # at every step within 1e-3 relative.
    w = synth.TINY
    n = 4096
    params = synth.random_params(w, 51)
    b = synth.train_batch_uniform(w, n, seed=51)
    m = make_model(w, params, n)
    tb = [cuda(a) for a in (b.pos, b.dir, b.radiance, b.pdf)]
    p = params.astype(np.float64)
    mm, vv = np.zeros_like(p), np.zeros_like(p)
    gl, ol = [], []
    for t in range(1, 31):
        loss = m.train_step(*tb)
        gl.append(float(host(loss)[0]))
        lo, g = oracle.train_grad(w, p, b.pos, b.dir, b.radiance, b.pdf)
        ol.append(lo)
        oracle.adam(p, g, mm, vv, t, w.lr, w.beta1, w.beta2, w.eps)
    gl, ol = np.array(gl), np.array(ol)
    assert ol[-1] < ol[0]
    assert np.abs(gl - ol).max() <= 1e-3 * np.abs(ol).max(), np.abs(gl - ol).max()


def _online(m, steps, n, seed0, fixed_position=None):
    from paper_2504_04315_gb300 import scene
    losses = []
    for s in range(steps):
        losses.append(scene.online_step(m, seed0 + s, n, fixed_position=fixed_position))
    return [float(x) for x in torch.stack(losses).cpu().numpy().ravel()]


def test_online_training_gains_over_uniform_radiance():
    from paper_2504_04315_gb300 import scene
    w = synth.TINY.with_(lr=1e-2)
    m = make_model(w, synth.init_params(w), 1 << 16)
    m0 = make_model(w, synth.init_params(w), 1 << 16)  # stays untrained
    rv_untrained, _ = scene.relative_variance(m, False, 999, 1 << 16)
    rv_uniform, mean_u = scene.relative_variance(m, False, 999, 1 << 16, uniform=True)
    # About the paper's budget (~1000 steps); batches of 2^16.
    losses, curve = [], []
    for chunk in range(5):
        losses += _online(m, 200, 1 << 16, 1000 + 200 * chunk)
        curve.append(scene.relative_variance(m, False, 999, 1 << 16)[0])
    rv_trained, mean_t = scene.relative_variance(m, False, 999, 1 << 16)
    # The guide alone (alpha = 0) has a heavy-tailed estimator: a rare
    # direction where the guide is far below the target can dominate one
    # measurement (one run read 6.2 after 2.4 at the previous checkpoint).
    # The assertions use the defensive mixture the method samples with
    # (alpha = 0.5), whose estimator is bounded.
    mix_untrained = scene.relative_variance(m0, False, 999, 1 << 16, alpha=0.5)[0]
    mix_trained, _ = scene.relative_variance(m, False, 999, 1 << 16, alpha=0.5)
    print(f"radiance: rel. variance uniform {rv_uniform:.3f} untrained {rv_untrained:.3f} "
          f"trained every 200 steps {[round(c, 3) for c in curve]}; "
          f"loss {losses[0]:.3f} -> {losses[-1]:.3f}; with the 50 % uniform mixture: "
          f"untrained {mix_untrained:.3f} trained {mix_trained:.3f}")
    assert abs(mean_u - 1.0) < 0.05 and abs(mean_t - 1.0) < 0.05  # the target integrates to 1
    assert mix_trained < 0.5 * rv_uniform
    assert mix_trained < 0.5 * mix_untrained
    assert np.mean(losses[-20:]) < np.mean(losses[:20])
    # Position-independent guide: the same network and training, but every
    # vertex is presented at one point, so it can only learn a single mixture
    # for the whole scene. The spatially varying guide must beat it.
    g = make_model(w, synth.init_params(w), 1 << 16)
    _online(g, 1000, 1 << 16, 1000, fixed_position=0.5)
    rv_global, _ = scene.relative_variance(g, False, 999, 1 << 16, fixed_position=0.5)
    mix_global, _ = scene.relative_variance(g, False, 999, 1 << 16, fixed_position=0.5, alpha=0.5)
    print(f"radiance: position-independent single mixture {rv_global:.3f} "
          f"(50 % uniform mixture {mix_global:.3f})")
    assert mix_global < rv_uniform
    assert mix_trained < 0.7 * mix_global


def test_product_workload_200_steps():
    # Product-mode workload: hash grid + SH(wo) + SH(n) + roughness, MLP
    # 64-64-64-64-32, K = 8, batch 2^19, Adam lr 1e-2 / betas 0.9, 0.99,
    # 200 online steps; split-BF16 forward for sampling.
    from paper_2504_04315_gb300 import scene
    w = synth.PRODUCT_BF16
    m = make_model(w, synth.init_params(w), w.n_train)
    rv_uniform, _ = scene.relative_variance(m, True, 4242, 1 << 16, uniform=True)
    rv_untrained, _ = scene.relative_variance(m, True, 4242, 1 << 16)
    losses = _online(m, 200, w.n_train, 2000)
    rv_trained, _ = scene.relative_variance(m, True, 4242, 1 << 16)
    mix_trained, _ = scene.relative_variance(m, True, 4242, 1 << 16, alpha=0.5)
    m.check_device_status()
    print(f"product: rel. variance uniform {rv_uniform:.3f} untrained {rv_untrained:.3f} "
          f"trained {rv_trained:.3f} (50 % uniform mixture {mix_trained:.3f}); "
          f"loss {losses[0]:.3f} -> {losses[-1]:.3f}")
    assert all(math.isfinite(x) for x in losses)
    assert np.mean(losses[-20:]) < np.mean(losses[:20])
    assert mix_trained < 0.5 * rv_uniform


_FULL_BATCH_REF = {}


def _full_batch_ref(w, params, b):
    key = id(params)
    if key not in _FULL_BATCH_REF:
        _FULL_BATCH_REF.clear()
        _FULL_BATCH_REF[key] = oracle.train_grad(w, params, b.pos, b.dir, b.radiance, b.pdf, b.aux)[1]
    return _FULL_BATCH_REF[key]


_FULL_BATCH = {}


@pytest.mark.parametrize("precision,bar", [(synth.BF16X3, 2e-2), (synth.FP32, 1e-4)],
                         ids=["split-bf16", "fp32"])
def test_product_full_batch_gradient_matches_oracle(precision, bar):
    # The product workload's full training batch (2^19 samples, the batch
    # the benchmark times) against the FP64 oracle with the FP32 master
    # parameters, per-tensor relative L2 of the gradient: <= 2e-2 through the
    # tensor-core training path (encode kernel, training kernel with each
    # tile's grid scatter issued during the next tile's MMAs, many tiles per
    # CTA) and <= 1e-4 through the FP32 training kernel (many 64-sample
    # tiles per CTA, grid atomics from every tile).
    w = synth.PRODUCT_BF16
    n = w.n_train
    if not _FULL_BATCH:
        _FULL_BATCH["params"] = synth.random_params(w, 12)
        _FULL_BATCH["batch"] = synth.train_batch_uniform(w, n, seed=12)
    params, b = _FULL_BATCH["params"], _FULL_BATCH["batch"]
    m = make_model(w, params, n, precision=precision)
    dlogv = -(b.radiance.astype(np.float64) / b.pdf) / n
    m.backward(cuda(b.pos), cuda(b.dir), cuda(dlogv), cuda(b.aux))
    g = m.get_grads().astype(np.float64)
    m.check_device_status()
    ref = _full_batch_ref(w, params, b)
    ng = sum(synth.grid_sizes(w)) * w.feat
    blocks = [("grid", slice(0, ng))]
    o = ng
    for i in range(len(w.widths) - 1):
        k = w.widths[i] * w.widths[i + 1]
        blocks.append((f"W{i + 1}", slice(o, o + k)))
        o += k
    errs = {name: np.linalg.norm(g[sl] - ref[sl]) / max(np.linalg.norm(ref[sl]), 1e-30) for name, sl in blocks}
    print(f"full-batch product gradient rel L2 (precision {precision}): "
          + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= bar, errs
