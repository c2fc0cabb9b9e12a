"""GPU parity of the FP32 path against the FP64 oracle, through the C ABI.

Bars: bit-exact grid indices; relative density error <= 1e-4 and direction
error <= 1e-4 rad for sampling; per-tensor relative L2 <= 1e-4 for gradients.
"""
import math

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


def edge_positions():
    pts = [[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [1.2, -0.3, 0.7], [0.99999994, 0.0, 1e-8],
           [-0.0, 2.0, -5.0], [0.25, 0.75, 0.125]]
    for d in [16, 20, 25, 101, 512]:
        for i in [0, 1, d // 3, d - 2, d - 1]:
            pts.append([i / (d - 1), (d - 1 - i) / (d - 1), 0.5])
    return np.array(pts, dtype=np.float32).T


@pytest.mark.parametrize("w", [synth.TINY, synth.PAPER_HASH, PRODUCT_SMALL, synth.PAPER_OWN])
def test_grid_indices_bit_exact(w):
    n = 50_000
    pos = np.concatenate([synth.positions(5, n), edge_positions()], axis=1)
    nan_col = np.array([[np.nan], [0.3], [np.nan]], dtype=np.float32)
    pos = np.concatenate([pos, nan_col], axis=1)
    m = make_model(w, synth.init_params(w), pos.shape[1])
    got = host(m.grid_indices(cuda(pos)))
    ref = oracle.grid_indices(w, pos)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("w,n", [(synth.TINY, 4096 + 37), (PRODUCT_SMALL, 3000),
                                 (synth.TINY.with_(kappa_act=synth.EXP), 2048),
                                 (synth.PAPER_OWN, 3000)])
def test_query_sample_parity(w, n):
    params = synth.random_params(w, 3, kappa_boost=6.0 if w.kappa_act == synth.SOFTPLUS else 1.0)
    pos = synth.positions(7, n)
    u = synth.sample_uniforms(7, n)
    aux = synth.aux_inputs(7, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n)
    d, p, mix = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux),
                               want_mix=True)
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
    w = synth.TINY
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
    w = synth.PAPER_HASH
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


@pytest.mark.parametrize("w,n", [(synth.TINY, 4096), (synth.PAPER_HASH, 8192),
                                 (PRODUCT_SMALL, 4096)])
def test_eval_pdf_parity(w, n):
    params = synth.random_params(w, 5)
    pos = synth.positions(9, n)
    uu = synth.uniform_rows(9, synth.S_DIR, 2, n)
    dirs = synth.sphere_dirs(uu[0], uu[1]).astype(np.float32)
    aux = synth.aux_inputs(9, n) if w.mode == synth.PRODUCT else None
    m = make_model(w, params, n)
    got = host(m.eval_pdf(cuda(pos), cuda(dirs), None if aux is None else cuda(aux)))
    ref = oracle.eval_pdf(w, params, pos, dirs, aux)
    err = rel_err(got, ref, 1e-30)
    assert err.max() < PDF_RTOL_FP32, err.max()


def test_ragged_ld_and_untouched_tail():
    w = synth.TINY
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


def test_sizes_zero_one_and_capacity():
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    params = synth.random_params(w, 6)
    m = make_model(w, params, 16)
    pos = synth.positions(11, 16)
    u = synth.sample_uniforms(11, 16)
    m.query_sample(cuda(pos), cuda(u), n=0)
    d, p, _ = m.query_sample(cuda(pos[:, :1]), cuda(u[:, :1]))
    compare_samples(w, params, pos[:, :1], u[:, :1], None, 0.0, host(d), host(p), PDF_RTOL_FP32,
                    DIR_TOL_FP32, MARGIN_FP32)
    big = cuda(synth.positions(11, 17))
    with pytest.raises(npm.NpmError) as e:
        m.query_sample(big, cuda(synth.sample_uniforms(11, 17)))
    assert e.value.status == 4  # NPM_ERR_CAPACITY


# ------------------------------------------------------------- training

def _grad_blocks(w, g):
    ng = sum(synth.grid_sizes(w)) * w.feat
    out = [("grid", g[:ng])]
    o = ng
    for i in range(len(w.widths) - 1):
        k = w.widths[i] * w.widths[i + 1]
        out.append((f"W{i + 1}", g[o:o + k]))
        o += k
    return out


@pytest.mark.parametrize("w,n", [(synth.TINY, 4096), (PRODUCT_SMALL, 4096),
                                 (synth.TINY.with_(kappa_act=synth.EXP), 2048),
                                 (synth.PAPER_HASH, 4096), (synth.PAPER_OWN, 4096)])
def test_gradient_parity(w, n):
    # Table 1's exp mapping of kappa needs milder raw outputs than softplus.
    params = synth.random_params(w, 12, kappa_boost=6.0 if w.kappa_act == synth.SOFTPLUS else 1.0)
    b = synth.train_batch_uniform(w, n, seed=12)
    m = make_model(w, params, n)
    dlogv = -(b.radiance.astype(np.float64) / b.pdf) / n
    m.backward(cuda(b.pos), cuda(b.dir), cuda(dlogv), None if b.aux is None else cuda(b.aux))
    g = m.get_grads()
    loss, ref = oracle.train_grad(w, params, b.pos, b.dir, b.radiance, b.pdf, b.aux)
    for (name, gb), (_, rb) in zip(_grad_blocks(w, g), _grad_blocks(w, ref)):
        e = np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-30)
        assert e < 1e-4, (name, e)


def test_train_step_loss_and_adam_parity():
    w = synth.TINY
    n = 4096
    params = synth.random_params(w, 13)
    b = synth.train_batch_uniform(w, n, seed=13)
    m = make_model(w, params, n)
    # Gradient from the GPU, then one Adam step on each side from it.
    dlogv = -(b.radiance.astype(np.float64) / b.pdf) / n
    m.backward(cuda(b.pos), cuda(b.dir), cuda(dlogv))
    g = m.get_grads().astype(np.float64)
    m.adam_step()
    got = m.get_params().astype(np.float64)
    p = params.astype(np.float64)
    mm, vv = np.zeros_like(p), np.zeros_like(p)
    oracle.adam(p, g, mm, vv, 1, w.lr, w.beta1, w.beta2, w.eps)
    assert np.abs(got - p).max() < 1e-6 * max(1.0, np.abs(p).max())
    # train_step: same loss as the oracle, and the same update as
    # backward + adam_step on a fresh model.
    m2 = make_model(w, params, n)
    loss = m2.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf))
    ref_loss = oracle.train_loss(w, params, b.pos, b.dir, b.radiance, b.pdf)
    assert abs(float(host(loss)[0]) - ref_loss) < 1e-5 * abs(ref_loss)
    p2 = m2.get_params().astype(np.float64)
    same = np.abs(p2 - got) < 1e-6
    # Entries whose gradient is within rounding of zero may flip the sign of
    # the unit Adam step; they must be a tiny minority.
    assert same.mean() > 0.999
    step, mom, _ = m2.get_adam()
    assert step == 1


def test_non_finite_loss_skips_update():
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    n = 256
    params = synth.random_params(w, 14)
    b = synth.train_batch_uniform(w, n, seed=14)
    rad = b.radiance.copy()
    rad[3] = np.inf
    m = make_model(w, params, n)
    m.train_step(cuda(b.pos), cuda(b.dir), cuda(rad), cuda(b.pdf))
    with pytest.raises(npm.NpmError) as e:
        m.check_device_status()
    assert e.value.status == 6  # NPM_ERR_NUMERIC
    assert np.array_equal(m.get_params(), params)
    m.check_device_status()  # cleared


def test_checkpoint_round_trip(tmp_path):
    w = synth.TINY
    n = 1024
    params = synth.random_params(w, 15)
    b = synth.train_batch_uniform(w, n, seed=15)
    m = make_model(w, params, n)
    for _ in range(3):
        m.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf))
    path = str(tmp_path / "ck.bin")
    m.save(path)
    m2 = make_model(w, synth.init_params(w), n)
    m2.load(path)
    assert np.array_equal(m.get_params(), m2.get_params())
    s1, m1, v1 = m.get_adam()
    s2, mb, vb = m2.get_adam()
    assert s1 == s2 == 3 and np.array_equal(m1, mb) and np.array_equal(v1, vb)
    m.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf))
    m2.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf))
    # Identical up to the summation order of the gradient atomics.
    assert (np.abs(m.get_params() - m2.get_params()) < 1e-6).mean() > 0.999


def test_bounded_wait_timeout_is_reported_and_context_survives():
    # The paper-shaped FP32 forward hands each tile from its encoder thread
    # group to an MLP group through shared-memory mailboxes guarded by
    # mbarriers whose waits are bounded. With a zero wait budget every wait
    # is one non-blocking test, and the MLP groups' first wait (before the
    # encoder has finished a tile) gives up: the kernel ends early and
    # reports NPM_ERR_TIMEOUT; nothing hangs. With the default budget the
    # next call on the same handle and context is correct again.
    from paper_2504_04315_gb300 import _lib
    w = synth.PAPER_HASH
    n = 1 << 16
    params = synth.random_params(w, 3)
    pos = synth.positions(11, n)
    u = synth.sample_uniforms(11, n)
    m = make_model(w, params, n)
    m.set_wait_limit(0)
    m.query_sample(cuda(pos), cuda(u))
    with pytest.raises(_lib.NpmError) as exc:
        m.check_device_status()
    assert exc.value.status == _lib.ERR_TIMEOUT
    m.set_wait_limit(1 << 31)
    d, p, _ = m.query_sample(cuda(pos), cuda(u))
    m.check_device_status()
    pick = np.arange(0, n, 16)
    compare_samples(w, params, pos[:, pick], u[:, pick], None, 0.0, host(d)[:, pick], host(p)[pick],
                    PDF_RTOL_FP32, DIR_TOL_FP32, MARGIN_FP32)


@pytest.mark.parametrize("w,n,ld,alpha", [(synth.PAPER_HASH, 200_003, 200_064, 0.0),
                                          (PRODUCT_SMALL, 70_001, 70_001, 0.5)],
                         ids=["paper-hash", "product-uniform-branch"])
def test_query_sample_host_buffers_match_device(w, n, ld, alpha):
    # The end-to-end entry point (pinned host buffers, strided chunk copies
    # on two internal streams) returns exactly what the device entry point
    # returns for the same inputs: per-query results do not depend on the
    # chunking. Several chunks, a ragged tail and ld > n; columns beyond n
    # of the host outputs stay untouched.
    params = synth.random_params(w, 31)
    pos = np.zeros((3, ld), np.float32)
    pos[:, :n] = synth.positions(31, n)
    u = np.zeros((4, ld), np.float32)
    u[:, :n] = synth.sample_uniforms(31, n, rows=4)
    aux = None
    if w.mode == synth.PRODUCT:
        aux = np.zeros((7, ld), np.float32)
        aux[:, :n] = synth.aux_inputs(31, n)
    m = make_model(w, params, ld)
    d_dev, p_dev, _ = m.query_sample(cuda(pos), cuda(u), None if aux is None else cuda(aux),
                                     uniform_frac=alpha, n=n)
    hpos = torch.from_numpy(pos).pin_memory()
    hu = torch.from_numpy(u).pin_memory()
    haux = None if aux is None else torch.from_numpy(aux).pin_memory()
    hd = torch.full((3, ld), -7.0).pin_memory()
    hp = torch.full((ld,), -7.0).pin_memory()
    m.query_sample_host(hpos, hu, hd, hp, haux, uniform_frac=alpha, n=n)
    m.check_device_status()
    assert np.array_equal(hd.numpy()[:, :n], host(d_dev)[:, :n])
    assert np.array_equal(hp.numpy()[:n], host(p_dev)[:n])
    assert np.all(hd.numpy()[:, n:] == -7.0) and np.all(hp.numpy()[n:] == -7.0)


def test_readme_session():
    # The usage shown in the README, at 2^16 vertices: densities of the
    # library's own seeded initialisation match the oracle, and one training
    # step on the sampled directions runs and moves the parameters.
    import paper_2504_04315_gb300 as npm
    w = synth.PAPER_HASH
    n = 1 << 16
    cfg = npm.make_config(npm.RADIANCE, level_res=w.level_res, feat=2, log2_table=19,
                          widths=[32, 64, 64, 64, 32], K=8, precision=npm.FP32, max_batch=n)
    m = npm.NPM(cfg)
    p_init = m.get_params()
    g = torch.Generator(device="cuda").manual_seed(0)
    pos = torch.rand(3, n, device="cuda", generator=g)
    u = torch.rand(3, n, device="cuda", generator=g)
    d, pdf, _ = m.query_sample(pos, u)
    k = 4096
    ref = oracle.eval_pdf(w, p_init, host(pos)[:, :k], host(d)[:, :k], None)
    assert rel_err(host(pdf)[:k], ref, 1e-30).max() < PDF_RTOL_FP32
    radiance = torch.rand(n, device="cuda", generator=g)
    loss = m.train_step(pos, d, radiance, pdf)
    m.check_device_status()
    assert math.isfinite(float(loss.item()))
    assert not np.array_equal(m.get_params(), p_init)
    m.close()
