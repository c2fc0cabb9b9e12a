"""A numpy model of the operand rounding of single-pass BF16 inference
(NPM_BF16) on the tiny workloads (one dense grid level, radiance mode).

Used to show that the BF16 path's distance from the FP64 oracle is the
declared quantisation and nothing else: FP16 grid table, FP32 trilinear
blend, every MMA operand (encoding, hidden activations, weights) rounded to
nearest BF16, exact products summed in FP32, then the Table 1 mapping and the
mixture density in FP64 (Eq. 3-4). It is a model of a number format, not of
the method: the mapping and density it needs come from the oracle's own
definitions restated in closed form below, and the tests compare it only
with the GPU."""
import math

import numpy as np

import synth


def bf16_rn(x):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _encode_dense_level(w, params, pos, fp16_grid):
    D, F = w.level_res[0], w.feat
    g = params[: D ** 3 * F]
    g = (g.astype(np.float16) if fp16_grid else g).astype(np.float32).reshape(-1, F)
    p = np.clip(pos, 0, 1).astype(np.float32) * np.float32(D - 1)
    c = np.minimum(np.floor(p).astype(np.int64), D - 2)
    f = (p - c).astype(np.float32)
    acc = np.zeros((pos.shape[1], F), np.float32)
    for k in range(8):
        d = [(k >> a) & 1 for a in range(3)]
        wt = np.ones(pos.shape[1], np.float32)
        for a in range(3):
            wt = (wt * (f[a] if d[a] else np.float32(1) - f[a])).astype(np.float32)
        idx = (c[0] + d[0]) + D * ((c[1] + d[1]) + D * (c[2] + d[2]))
        acc = (acc + wt[:, None] * g[idx]).astype(np.float32)
    return acc


def raw_outputs(w, params, pos, rounding=bf16_rn, fp16_grid=True):
    """[n][4K] network outputs with BF16 operands and FP32 sums (rounding
    and the FP16 table can be switched off to check the model itself)."""
    assert w.mode == synth.RADIANCE and len(w.level_res) == 1
    assert w.level_res[0] ** 3 <= (1 << w.log2_table)
    params = np.asarray(params, np.float32)
    h = _encode_dense_level(w, params, pos, fp16_grid)
    h = np.concatenate([h, np.zeros((h.shape[0], w.widths[0] - h.shape[1]), np.float32)], 1)
    o = sum(synth.grid_sizes(w)) * w.feat
    L = len(w.widths) - 1
    for l in range(L):
        k = w.widths[l] * w.widths[l + 1]
        W = rounding(params[o:o + k]).reshape(w.widths[l + 1], w.widths[l])
        o += k
        z = (rounding(h).astype(np.float64) @ W.astype(np.float64).T).astype(np.float32)
        h = np.maximum(z, 0) if l < L - 1 else z
    return h.astype(np.float64)


def density(w, raw, dirs):
    """V(dirs [3][n]) of the mixtures that Table 1 maps raw [n][4K] to."""
    lam = raw[:, 0::4]
    lam = np.exp(lam - lam.max(1, keepdims=True))
    lam /= lam.sum(1, keepdims=True)
    rk = raw[:, 1::4]
    kap = np.where(rk > 0, rk + np.log1p(np.exp(-rk)), np.log1p(np.exp(rk))) if w.kappa_act == synth.SOFTPLUS \
        else np.exp(rk)
    th = math.pi / (1 + np.exp(-raw[:, 2::4]))
    ph = 2 * math.pi / (1 + np.exp(-raw[:, 3::4]))
    mu = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    c = kap / (2 * math.pi * -np.expm1(-2 * kap))
    dot = np.einsum("nkc,cn->nk", mu, dirs)
    return (lam * c * np.exp(kap * (dot - 1))).sum(1)
