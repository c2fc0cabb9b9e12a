"""Test helpers shared by the oracle pins and the GPU sampler tests: models
whose network decodes to a chosen vMF mixture at one position, and a
chi-square test of sampled directions against a density integrated over
equal-area bins of the sphere.

Nothing here computes a step of the method: the designed parameters solve one
linear system for the last layer through the oracle's own forward pass, and
the chi-square statistic takes the density as a callable."""
import math

import numpy as np
from scipy import special, stats

import oracle

X0 = [0.31, 0.62, 0.17]

# A four-lobe mixture with uneven weights, kappa from smooth to sharp and
# means spread over the sphere.
MIX = dict(lams=[0.4, 0.3, 0.2, 0.1], kaps=[2.0, 20.0, 50.0, 0.5],
           thetas=[0.4, 2.0, 1.2, 2.9], phis=[0.3, 4.0, 2.5, 5.9])


def diverse_params(w, raw_target, x):
    """Parameters whose network outputs exactly raw_target at position x:
    constant grid features, random hidden layers, and a last layer solved so
    that its outputs equal the target."""
    rng = np.random.default_rng(8)
    npar = oracle.n_params(w)
    params = rng.standard_normal(npar) * 0.5
    ng = npar - sum(a * b for a, b in zip(w.widths[:-1], w.widths[1:]))
    params[:ng] = np.tile([1.0, 0.5, -0.3, 0.8][: w.feat], ng // w.feat)
    enc = oracle.encode(w, params, np.asarray(x, np.float32))
    _, acts = oracle.mlp(w, params, enc, want_acts=True)
    h = np.maximum(acts[-(w.widths[-1] + w.widths[-2]):-w.widths[-1]], 0.0)
    last = npar - w.widths[-1] * w.widths[-2]
    W = np.outer(raw_target, h) / np.dot(h, h)
    params[last:] = W.ravel()
    return params


def raw_for(lams, kaps, thetas, phis):
    """Raw network outputs that Table 1 maps to the given lobes (softplus
    kappa): weight logit, kappa', theta', phi' per lobe."""
    raw = []
    for l, k, t, p in zip(lams, kaps, thetas, phis):
        raw += [math.log(l), math.log(math.expm1(k)), special.logit(t / math.pi),
                special.logit(p / (2 * math.pi))]
    return np.array(raw)


def chi2_directions(d, density, nz=64, nph=128):
    """p-value and statistic of a chi-square test of the directions d [3][n]
    against density(dirs [3][m]) -> [m] over nz x nph equal-area bins in
    (cos theta, phi); expected counts by 6 x 6 Gauss-Legendre per bin, bins
    expecting fewer than 5 pooled."""
    n = d.shape[1]
    z = np.clip(d[2], -1, 1)
    ph = np.mod(np.arctan2(d[1], d[0]), 2 * math.pi)
    bz = np.minimum(((z + 1) / 2 * nz).astype(int), nz - 1)
    bp = np.minimum((ph / (2 * math.pi) * nph).astype(int), nph - 1)
    obs = np.bincount(bz * nph + bp, minlength=nz * nph).astype(float)
    g, gw = np.polynomial.legendre.leggauss(6)
    zc = (np.arange(nz) + 0.5) / nz * 2 - 1
    pc = (np.arange(nph) + 0.5) / nph * 2 * math.pi
    hz, hp = 1.0 / nz, math.pi / nph
    Z = (zc[:, None] + hz * g[None, :]).ravel()
    P = (pc[:, None] + hp * g[None, :]).ravel()
    ZZ, PP = np.meshgrid(Z, P, indexing="ij")
    r = np.sqrt(np.clip(1 - ZZ ** 2, 0, None))
    dirs = np.stack([r * np.cos(PP), r * np.sin(PP), ZZ]).reshape(3, -1)
    dens = np.asarray(density(dirs), dtype=np.float64).reshape(nz, 6, nph, 6)
    wgt = (gw[:, None] * gw[None, :]) * hz * hp
    exp_c = np.einsum("aibj,ij->ab", dens, wgt).ravel() * n
    assert abs(exp_c.sum() / n - 1.0) < 1e-6
    keep = exp_c >= 5
    pooled_o, pooled_e = obs[~keep].sum(), exp_c[~keep].sum()
    o = np.append(obs[keep], pooled_o)
    e = np.append(exp_c[keep], pooled_e)
    if pooled_e < 5:
        o, e = obs[keep], exp_c[keep]
    chi2 = ((o - e) ** 2 / e).sum()
    dof = len(o) - 1
    return stats.chi2.sf(chi2, dof), chi2
