"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each checks a closed form, an
invariant, a special case that reduces to a textbook result, quadrature, a
chi-square test, or central finite differences.
"""
import math
import os

import mpmath
import numpy as np
import pytest
from scipy import optimize, special

import mixtures
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hash_and_levels.txt")


def _golden():
    hashes, levels, total = [], None, None
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "hash":
            hashes.append(tuple(int(v) for v in line[1:]))
        elif line[0] == "levels":
            levels = [int(v) for v in line[1:]]
        elif line[0] == "total_entries":
            total = int(line[1])
    return hashes, levels, total


# ------------------------------------------------------------ a2: index

def test_hash_worked_values():
    hashes, _, _ = _golden()
    w = synth.PAPER_HASH
    level = 8  # D = 101: 101^3 > 2^19, hashed
    for i, j, k, v in hashes:
        assert oracle.lattice_index(w, level, i, j, k) == v


def test_level_table_and_sizes():
    _, levels, total = _golden()
    assert synth.PAPER_HASH.level_res == levels
    off = oracle.grid_offsets(synth.PAPER_HASH)
    assert off[0] == 0
    assert oracle.n_params(synth.PAPER_HASH) == total * 2 + (32 * 64 + 64 * 64 * 2 + 64 * 32)
    # Levels 0-7 are dense (D^3 <= 2^19), 8-15 hashed (2^19 entries each).
    sizes = np.diff(np.append(off, total))
    assert list(sizes[:8]) == [d ** 3 for d in levels[:8]]
    assert list(sizes[8:]) == [1 << 19] * 8


def test_dense_index_is_row_major():
    w = synth.PAPER_HASH
    for level, d in enumerate(w.level_res[:8]):
        for (i, j, k) in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (d - 1, d - 1, d - 1), (3, 5, 7)]:
            assert oracle.lattice_index(w, level, i, j, k) == i + d * (j + d * k)


def test_cell_and_fraction_edges():
    w = synth.TINY  # D = 16
    idx, wt = oracle.grid_corners(w, 0, [0.0, 0.0, 0.0])
    assert idx[0] == 0 and wt[0] == 1.0 and wt[1:].sum() == 0.0
    # x = 1 lands in the last cell with fraction 1: all weight on corner 7.
    idx, wt = oracle.grid_corners(w, 0, [1.0, 1.0, 1.0])
    assert idx[7] == 15 + 16 * (15 + 16 * 15) and wt[7] == 1.0
    # Out-of-range inputs clamp to the box.
    idx2, wt2 = oracle.grid_corners(w, 0, [1.5, 2.0, 7.0])
    assert np.array_equal(idx, idx2) and np.array_equal(wt, wt2)
    idx3, wt3 = oracle.grid_corners(w, 0, [-0.5, -1.0, -3.0])
    assert idx3[0] == 0 and wt3[0] == 1.0


# --------------------------------------------------------- a3: trilinear

def test_trilinear_weights_partition_of_unity():
    w = synth.PAPER_HASH
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = rng.random(3).astype(np.float32)
        for level in range(16):
            _, wt = oracle.grid_corners(w, level, x)
            assert np.all(wt >= 0.0) and np.all(wt <= 1.0)
            assert abs(wt.sum() - 1.0) < 1e-14


def test_trilinear_reproduces_affine_field():
    # Trilinear blending is exact on affine functions of the lattice
    # coordinate: store V[i,j,k] = a + b i + c j + d k and read back a + b p.
    w = synth.Workload(name="affine", mode=0, level_res=[7, 12], feat=2, log2_table=19,
                       widths=[4, 4], K=1)
    n_entries = 7 ** 3 + 12 ** 3
    params = np.zeros(oracle.n_params(w))
    coef = [(0.5, 1.0, -2.0, 0.25), (-1.0, 0.125, 0.5, 3.0)]
    base = 0
    for level, d in enumerate(w.level_res):
        ii, jj, kk = np.meshgrid(np.arange(d), np.arange(d), np.arange(d), indexing="ij")
        lin = (ii + d * (jj + d * kk)).ravel()
        for q in range(2):
            a, b, c, e = coef[q]
            params[(base + lin) * 2 + q] = (a + b * ii + c * jj + e * kk).ravel()
        base += d ** 3
    assert base == n_entries
    rng = np.random.default_rng(2)
    for _ in range(100):
        x = rng.random(3).astype(np.float32)
        g = oracle.grid_encode(w, params, x)
        for level, d in enumerate(w.level_res):
            p = (x * np.float32(d - 1)).astype(np.float64)  # lattice coordinate
            for q in range(2):
                a, b, c, e = coef[q]
                assert abs(g[level * 2 + q] - (a + b * p[0] + c * p[1] + e * p[2])) < 1e-12


def test_trilinear_hits_lattice_values():
    w = synth.TINY
    rng = np.random.default_rng(3)
    params = rng.standard_normal(oracle.n_params(w))
    for (i, j, k) in [(0, 0, 0), (3, 7, 11), (15, 15, 15), (15, 0, 8)]:
        x = np.array([i, j, k], dtype=np.float32) / np.float32(15)
        g = oracle.grid_encode(w, params, x)
        e = (i + 16 * (j + 16 * k)) * 4
        assert np.allclose(g, params[e:e + 4], rtol=0, atol=1e-6)


# ------------------------------------------------------- a4: SH encoding

def _sphere_quadrature(nz, nphi):
    z, wz = np.polynomial.legendre.leggauss(nz)
    ph = (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
    Z, P = np.meshgrid(z, ph, indexing="ij")
    r = np.sqrt(1 - Z * Z)
    dirs = np.stack([r * np.cos(P), r * np.sin(P), Z]).reshape(3, -1)
    wts = (wz[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).ravel()
    return dirs, wts


def test_sh_orthonormal_by_quadrature():
    dirs, wts = _sphere_quadrature(24, 48)
    Y = np.stack([oracle.sh(4, dirs[:, i]) for i in range(dirs.shape[1])])
    gram = (Y * wts[:, None]).T @ Y
    assert np.abs(gram - np.eye(16)).max() < 1e-12
    assert abs(oracle.sh(1, [0, 0, 1])[0] - 1 / (2 * math.sqrt(math.pi))) < 1e-16


def test_sh_addition_theorem():
    # sum_m Y_lm(a) Y_lm(b) = (2l + 1) / (4 pi) P_l(a . b) for every band l.
    rng = np.random.default_rng(4)
    for _ in range(20):
        a = rng.standard_normal(3)
        b = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        ya, yb = oracle.sh(4, a), oracle.sh(4, b)
        for l in range(4):
            s = np.dot(ya[l * l:(l + 1) ** 2], yb[l * l:(l + 1) ** 2])
            ref = (2 * l + 1) / (4 * math.pi) * special.eval_legendre(l, np.dot(a, b))
            assert abs(s - ref) < 1e-13


def test_product_encoding_layout():
    w = synth.FD_TINY_PRODUCT
    rng = np.random.default_rng(5)
    params = rng.standard_normal(oracle.n_params(w))
    x = np.array([0.3, 0.6, 0.9], dtype=np.float32)
    aux = synth.aux_inputs(0, 1)[:, 0]
    enc = oracle.encode(w, params, x, aux)
    assert np.allclose(enc[:4], oracle.grid_encode(w, params, x))
    assert np.allclose(enc[4:20], oracle.sh(4, aux[0:3].astype(np.float64)))
    assert np.allclose(enc[20:24], oracle.sh(2, aux[3:6].astype(np.float64)))
    assert enc[24] == np.float64(aux[6])
    assert np.all(enc[25:] == 0.0)


# ---------------------------------------------------------- a5: the MLP

def test_mlp_matches_matmul():
    w = synth.PAPER_HASH
    rng = np.random.default_rng(6)
    params = rng.standard_normal(oracle.n_params(w)) * 0.3
    ng = oracle.n_params(w) - sum(a * b for a, b in zip(w.widths[:-1], w.widths[1:]))
    mats, o = [], ng
    for a, b in zip(w.widths[:-1], w.widths[1:]):
        mats.append(params[o:o + a * b].reshape(b, a))
        o += a * b
    for _ in range(10):
        h = rng.standard_normal(w.widths[0])
        raw = oracle.mlp(w, params, h)
        ref = h
        for i, M in enumerate(mats):
            ref = M @ ref
            if i < len(mats) - 1:
                ref = np.maximum(ref, 0.0)
        assert np.allclose(raw, ref, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------- a6: the mapping

def _zero_mlp(w, params):
    ng = oracle.n_params(w) - sum(a * b for a, b in zip(w.widths[:-1], w.widths[1:]))
    params = params.copy()
    params[ng:] = 0.0
    return params


@pytest.mark.parametrize("act", [synth.SOFTPLUS, synth.EXP])
def test_mapping_at_zero_raw(act):
    w = synth.TINY.with_(kappa_act=act)
    params = _zero_mlp(w, synth.init_params(w).astype(np.float64))
    out = oracle.decode_batch(w, params, synth.positions(0, 8))
    lam, kap, th, ph = out[0::4], out[1::4], out[2::4], out[3::4]
    assert np.allclose(lam, 1.0 / w.K, atol=1e-15)
    assert np.allclose(kap, math.log(2.0) if act == synth.SOFTPLUS else 1.0, atol=1e-15)
    assert np.allclose(th, math.pi / 2, atol=1e-15)
    assert np.allclose(ph, math.pi, atol=1e-15)


def test_mapping_invariants():
    w = synth.PAPER_HASH
    rng = np.random.default_rng(7)
    params = rng.standard_normal(oracle.n_params(w)) * 0.2
    out = oracle.decode_batch(w, params, synth.positions(1, 512))
    lam, kap, th, ph = out[0::4], out[1::4], out[2::4], out[3::4]
    assert np.abs(lam.sum(axis=0) - 1.0).max() < 1e-14
    assert np.all(lam > 0) and np.all(kap > 0)
    assert np.all((th > 0) & (th < math.pi)) and np.all((ph > 0) & (ph < 2 * math.pi))


# --------------------------------------------- a7: vMF and mixture pdf

@pytest.mark.parametrize("k", [1e-9, 1e-6, 1e-3, 0.5, 1.0, 5.0, 50.0, 300.0, 700.0])
def test_vmf_normaliser_closed_form(k):
    # c(k) e^{-k} must equal k / (4 pi sinh k) (Eq. 3); checked at 40 digits.
    mpmath.mp.dps = 40
    K = mpmath.mpf(k)
    ref = K / (4 * mpmath.pi * mpmath.sinh(K)) * mpmath.exp(K)
    got = oracle.vmf_scaled_norm(k)
    assert abs(mpmath.mpf(got) / ref - 1) < 1e-13


_diverse_params = mixtures.diverse_params
_raw_for = mixtures.raw_for
MIX = mixtures.MIX
X0 = mixtures.X0


def test_mixture_decodes_to_target():
    w = synth.TINY
    params = _diverse_params(w, _raw_for(**MIX), X0)
    out = oracle.decode_batch(w, params, np.array(X0, np.float32)[:, None])[:, 0]
    assert np.allclose(out[0::4], MIX["lams"], atol=1e-12)
    assert np.allclose(out[1::4], MIX["kaps"], atol=1e-10)
    assert np.allclose(out[2::4], MIX["thetas"], atol=1e-12)
    assert np.allclose(out[3::4], MIX["phis"], atol=1e-12)


@pytest.mark.parametrize("w", [synth.TINY, synth.PAPER_HASH, synth.FD_TINY_PRODUCT])
def test_mixture_integrates_to_one(w):
    # Quadrature of V over the sphere: Gauss-Legendre in cos(theta) times
    # the periodic trapezoid rule in phi, converging exponentially.
    if w is synth.TINY:
        params = _diverse_params(w, _raw_for(**MIX), X0)
        xs = [X0]
    else:
        params = np.random.default_rng(9).standard_normal(oracle.n_params(w)) * 0.3
        xs = [X0, [0.9, 0.05, 0.5]]
    dirs, wts = _sphere_quadrature(400, 800)
    n = dirs.shape[1]
    for x in xs:
        pos = np.repeat(np.array(x, np.float32)[:, None], n, axis=1)
        aux = None
        if w.mode == synth.PRODUCT:
            aux = np.repeat(synth.aux_inputs(3, 1), n, axis=1)
        v = oracle.eval_pdf64(w, params, pos, dirs, aux)
        assert abs(np.dot(v, wts) - 1.0) < 1e-10


# ------------------------------------------------------- a8: the sampler

@pytest.mark.parametrize("k", [1e-4, 0.5, 5.0, 50.0, 500.0])
def test_sampler_inverts_closed_form_cdf(k):
    # P(W <= w) = (e^{k w} - e^{-k}) / (2 sinh k); the sampler maps u1 to the
    # w with P(W <= w) = 1 - u1 (it is decreasing in u1).
    mpmath.mp.dps = 40
    K = mpmath.mpf(k)
    for u1 in [0.0, 1e-6, 0.1, 0.37, 0.5, 0.9, 0.999999]:
        W = oracle.vmf_sample_w(k, u1)
        cdf = (mpmath.exp(K * W) - mpmath.exp(-K)) / (2 * mpmath.sinh(K))
        assert abs(float(cdf) - (1.0 - u1)) < 1e-9 + 1e-9 * k


def test_frame_is_orthonormal_right_handed():
    rng = np.random.default_rng(10)
    ns = list(rng.standard_normal((200, 3))) + [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 0, -1 + 1e-12]]
    for n in ns:
        n = np.asarray(n, float)
        n /= np.linalg.norm(n)
        t, b = oracle.frame(n)
        M = np.stack([t, b, n])
        assert np.abs(M @ M.T - np.eye(3)).max() < 1e-12
        assert np.allclose(np.cross(t, b), n, atol=1e-12)


def _chi2_sampling(w, params, alpha, n=1_000_000, seed=11, sample_params=None):
    """p-value of a chi-square test of sampled directions (drawn with
    sample_params, default params) against the density of params."""
    pos = np.repeat(np.array(X0, np.float32)[:, None], n, axis=1)
    u = synth.sample_uniforms(seed, n, rows=4 if alpha > 0 else 3)
    sp = params if sample_params is None else sample_params
    d, pdf, _, _ = oracle.query_sample(w, sp, pos, u, alpha=alpha)
    assert np.abs(np.linalg.norm(d, axis=0) - 1.0).max() < 1e-12

    def density(dirs):
        posq = np.repeat(np.array(X0, np.float32)[:, None], dirs.shape[1], axis=1)
        return alpha / (4 * math.pi) + (1 - alpha) * oracle.eval_pdf64(w, params, posq, dirs)

    p, _ = mixtures.chi2_directions(d, density)
    return p, pdf, d


@pytest.mark.parametrize("alpha", [0.0, 0.5])
def test_sampling_chi_square(alpha):
    w = synth.TINY
    params = _diverse_params(w, _raw_for(**MIX), X0)
    p, pdf, d = _chi2_sampling(w, params, alpha)
    assert p > 0.01, p
    # Returned density equals the strategy's density at the sample.
    n = 4096
    pos = np.repeat(np.array(X0, np.float32)[:, None], n, axis=1)
    v = oracle.eval_pdf64(w, params, pos, d[:, :n])
    assert np.allclose(pdf[:n], alpha / (4 * math.pi) + (1 - alpha) * v, rtol=1e-12)


def test_chi_square_detects_wrong_density():
    # The statistic must reject when sampler and density disagree slightly:
    # sample a mixture whose second lobe has kappa 22 instead of 20.
    w = synth.TINY
    params = _diverse_params(w, _raw_for(**MIX), X0)
    mix2 = dict(MIX)
    mix2["kaps"] = [2.0, 22.0, 50.0, 0.5]
    params2 = _diverse_params(w, _raw_for(**mix2), X0)
    p, _, _ = _chi2_sampling(w, params, 0.0, sample_params=params2)
    assert p < 1e-6, p


# --------------------------------------------- a9-a10: loss and gradient

def _fd_setup(w, seed=13, n=16):
    rng = np.random.default_rng(seed)
    npar = oracle.n_params(w)
    params = rng.uniform(-1, 1, npar)
    ng = npar - sum(a * b for a, b in zip(w.widths[:-1], w.widths[1:]))
    params[ng:] *= 0.8
    pos = synth.positions(seed, n)
    aux = synth.aux_inputs(seed, n) if w.mode == synth.PRODUCT else None
    u = synth.uniform_rows(seed, synth.S_DIR, 2, n)
    d = synth.sphere_dirs(u[0], u[1]).astype(np.float32)
    L = (synth.target(pos, d, aux) + 0.05).astype(np.float32)
    pt = np.full(n, 1 / (4 * math.pi), np.float32)
    # Keep clear of cell faces (C14): the gradient is not smooth there.
    return params, pos, aux, d, L, pt


@pytest.mark.parametrize("w", [synth.FD_TINY, synth.FD_TINY.with_(kappa_act=synth.EXP),
                               synth.FD_TINY_PRODUCT])
def test_gradient_matches_central_differences(w):
    params, pos, aux, d, L, pt = _fd_setup(w)
    loss, g = oracle.train_grad(w, params, pos, d, L, pt, aux)
    assert abs(loss - oracle.train_loss(w, params, pos, d, L, pt, aux)) < 1e-12 * abs(loss)
    h = 1e-6
    fd = np.zeros_like(g)
    for i in range(params.size):
        p1 = params.copy()
        p1[i] += h
        p2 = params.copy()
        p2[i] -= h
        fd[i] = (oracle.train_loss(w, p1, pos, d, L, pt, aux)
                 - oracle.train_loss(w, p2, pos, d, L, pt, aux)) / (2 * h)
    scale = np.abs(g).max()
    assert scale > 1e-3
    err = np.abs(fd - g)
    assert err.max() < 1e-6 * scale, (err.max(), scale)
    touched = np.abs(g) > 1e-3 * scale
    assert np.all(err[touched] < 1e-5 * np.abs(g[touched]) + 1e-8 * scale)


def test_gradient_detects_planted_sign_error():
    # A plausible slip (dropping the sign of one lobe's kappa term) changes the
    # gradient well beyond the finite-difference tolerance used above.
    w = synth.FD_TINY
    params, pos, aux, d, L, pt = _fd_setup(w)
    _, g = oracle.train_grad(w, params, pos, d, L, pt, aux)
    last = oracle.n_params(w) - w.widths[-1] * w.widths[-2]
    row = 1  # kappa' of lobe 0
    h = 1e-6
    i = last + row * w.widths[-2] + 2
    p1, p2 = params.copy(), params.copy()
    p1[i] += h
    p2[i] -= h
    fd = (oracle.train_loss(w, p1, pos, d, L, pt) - oracle.train_loss(w, p2, pos, d, L, pt)) / (2 * h)
    assert abs(fd - g[i]) < 1e-6 * abs(g).max()
    assert abs(fd + g[i]) > 1e-3 * abs(g).max()


def test_single_lobe_fit_is_weighted_vmf_mle():
    # K = 1 at a single position with a constant sampling density: the loss
    # is the weighted vMF negative log-likelihood, whose minimiser is the
    # textbook MLE (mean = normalised weighted resultant, coth k - 1/k = Rbar).
    w = synth.Workload(name="mle", mode=0, level_res=[2], feat=4, log2_table=19,
                       widths=[4, 4], K=1)
    n = 4000
    u = synth.uniform_rows(21, synth.S_DIR, 2, n)
    d = synth.sphere_dirs(u[0], u[1]).astype(np.float32)
    dd = d.astype(np.float64)
    mu0 = np.array([0.2, -0.5, 0.84])
    mu0 /= np.linalg.norm(mu0)
    L = (np.exp(6.0 * (mu0 @ dd - 1.0)) + 0.05).astype(np.float32)
    pt = np.full(n, 1 / (4 * math.pi), np.float32)
    wts = L.astype(np.float64) / pt.astype(np.float64)
    R = dd @ wts
    mu = R / np.linalg.norm(R)
    rbar = np.linalg.norm(R) / wts.sum()
    kap = optimize.brentq(lambda k: 1 / math.tanh(k) - 1 / k - rbar, 1e-6, 1e4, xtol=1e-15)
    th = math.acos(mu[2])
    ph = math.atan2(mu[1], mu[0]) % (2 * math.pi)
    raw = np.array([0.0, math.log(math.expm1(kap)), special.logit(th / math.pi),
                    special.logit(ph / (2 * math.pi))])
    npar = oracle.n_params(w)
    params = np.zeros(npar)
    params[: 8 * 4] = 1.0  # constant features -> encoding (1, 1, 1, 1)
    params[32:] = np.repeat(raw / 4.0, 4)
    pos = np.repeat(np.array(X0, np.float32)[:, None], n, axis=1)
    _, g_opt = oracle.train_grad(w, params, pos, d, L, pt)
    off = params.copy()
    off[32:] = np.repeat((raw + np.array([0.0, 0.3, 0.05, -0.05])) / 4.0, 4)
    _, g_off = oracle.train_grad(w, off, pos, d, L, pt)
    assert np.abs(g_off[32:]).max() > 1e-2
    assert np.abs(g_opt[32:]).max() < 1e-9 * np.abs(g_off[32:]).max() + 1e-12


# -------------------------------------------------------------- a11: Adam

def test_ema_closed_form():
    """Sec. 5.3 weight averaging: with the parameters held at p, t updates of
    e <- d e + (1 - d) p leave e_t = p + d^t (e_0 - p); d = 0 copies p; the
    average of a parameter path stays inside its range."""
    rng = np.random.default_rng(21)
    n, d = 257, 0.9
    e0, p = rng.standard_normal(n), rng.standard_normal(n)
    e = e0.copy()
    for _ in range(7):
        oracle.ema(e, p, d)
    assert np.allclose(e, p + d ** 7 * (e0 - p), rtol=0, atol=1e-14)
    e = e0.copy()
    oracle.ema(e, p, 0.0)
    assert np.array_equal(e, p)
    path = rng.uniform(-1.0, 2.0, size=(20, n))
    e = path[0].copy()
    for q in path[1:]:
        oracle.ema(e, q, 0.7)
    assert np.all(e >= path.min(axis=0) - 1e-15) and np.all(e <= path.max(axis=0) + 1e-15)


def test_adam_closed_form_two_steps():
    rng = np.random.default_rng(14)
    n = 1000
    p0 = rng.standard_normal(n)
    g1, g2 = rng.standard_normal(n) * 1e-2, rng.standard_normal(n) * 3e-2
    lr, b1, b2, eps = 1e-2, 0.9, 0.99, 1e-8
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    oracle.adam(p, g1, m, v, 1, lr, b1, b2, eps)
    assert np.allclose(p, p0 - lr * g1 / (np.abs(g1) + eps), rtol=0, atol=1e-15)
    p1 = p.copy()
    oracle.adam(p, g2, m, v, 2, lr, b1, b2, eps)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    assert np.allclose(p, p1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-14)
