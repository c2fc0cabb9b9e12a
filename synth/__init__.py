"""Seeded synthetic inputs for the NPM hot path.

This module is shared by the tests, the benchmark and the smoke check. It
produces inputs only: random numbers, positions, directions, initial
parameters and the analytic stand-in scenes. It holds none of the method's own
arithmetic (no grid index, no network, no mixture pdf, no sampler, no
gradient). Neither the oracle nor the CUDA path is imported here.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
evaluated at state ``s0 + (i + 1) * gamma`` with a keyed start state
``s0 = mix(mix(seed) ^ stream)``. A uniform float is ``(bits >> 40) * 2**-24``,
which is an exact float32 in [0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Named random streams. Each input kind has its own stream so that changing
# one workload size never shifts the numbers of another input.
S_POS = 1
S_U = 2
S_DIR = 3
S_NOISE = 4
S_GRID_INIT = 5
S_MLP_INIT = 6
S_AUX = 7
S_BRANCH = 8
S_SURVIVE = 9


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (xor-shift-multiply finaliser)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def counter_bits(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """64 random bits for counters start .. start+n-1 of (seed, stream)."""
    s0 = mix64(mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF)) ^ np.uint64(stream))
    i = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = s0 + (i + np.uint64(1)) * GAMMA
    return mix64(state)


def uniform(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """Exact float32 uniforms in [0, 1)."""
    b = counter_bits(seed, stream, start, n) >> np.uint64(40)
    return (b.astype(np.float64) * 2.0 ** -24).astype(np.float32)


def uniform_rows(seed: int, stream: int, rows: int, n: int) -> np.ndarray:
    """[rows][n] float32 uniforms; row r uses counters r*n .. r*n+n-1."""
    return uniform(seed, stream, rows * n).reshape(rows, n)


def sphere_dirs(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """Area-uniform unit vectors from two uniforms, float64 [3][n]."""
    z = 1.0 - 2.0 * u1.astype(np.float64)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = 2.0 * math.pi * u2.astype(np.float64)
    return np.stack([r * np.cos(ph), r * np.sin(ph), z])


# --------------------------------------------------------------------------
# Workload definitions: sizes and shapes of the five stand-in workloads.
# --------------------------------------------------------------------------

RES16 = [16, 20, 25, 32, 40, 50, 64, 80, 101, 128, 161, 203, 256, 322, 406, 512]

RADIANCE, PRODUCT = 0, 1
SOFTPLUS, EXP = 0, 1
FP32, BF16, BF16X3, FP16, FP32_TC = 0, 1, 2, 3, 4


@dataclass
class Workload:
    name: str
    mode: int
    level_res: List[int]
    feat: int
    log2_table: int
    widths: List[int]
    K: int
    kappa_act: int = SOFTPLUS
    precision: int = FP32
    n_query: int = 4096
    n_train: int = 0
    lr: float = 5e-3
    beta1: float = 0.9
    beta2: float = 0.99
    eps: float = 1e-8
    seed: int = 0

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


TINY = Workload(
    name="tiny dense 16^3x4, MLP 4-32-32-16, K=4, fp32",
    mode=RADIANCE, level_res=[16], feat=4, log2_table=19,
    widths=[4, 32, 32, 16], K=4, n_query=4096, n_train=4096)

PAPER_HASH = Workload(
    name="hash grid 16 levels x 2 feats, T=2^19, MLP 32-64-64-64-32, K=8, fp32",
    mode=RADIANCE, level_res=list(RES16), feat=2, log2_table=19,
    widths=[32, 64, 64, 64, 32], K=8, n_query=1 << 20)

TINY_BF16 = TINY.with_(
    name="tiny dense 16^3x4, MLP 4-32-32-16, K=4, split-bf16 tensor-core MLP / fp16 grid",
    precision=BF16X3, n_query=1 << 22)

PRODUCT_BF16 = Workload(
    name="product mode, hash grid + SH4(wo) + SH2(n) + roughness, MLP 64-64-64-64-32, K=8, split-bf16",
    mode=PRODUCT, level_res=list(RES16), feat=2, log2_table=19,
    widths=[64, 64, 64, 64, 32], K=8, precision=BF16X3,
    n_query=1 << 19, n_train=1 << 19, lr=1e-2, beta1=0.9, beta2=0.99)

# The paper's own shape (Sec. 5.3): L = 8 dense levels whose resolution grows
# geometrically from D = 8 to D = 86 (D_l = floor(8 (86/8)^(l/7))), F = 4
# features (3.95 M grid parameters), three hidden layers of width 64, K = 8.
RES8_PAPER = [8, 11, 15, 22, 31, 43, 61, 86]
PAPER_OWN = Workload(
    name="paper's own shape: 8 dense levels D 8..86 x 4 feats, MLP 32-64-64-64-32, K=8, fp32",
    mode=RADIANCE, level_res=list(RES8_PAPER), feat=4, log2_table=20,
    widths=[32, 64, 64, 64, 32], K=8, n_query=1 << 20, n_train=1 << 18)

# Finite-difference net: 2 dense levels, hidden width 8, K=2.
FD_TINY = Workload(
    name="finite-difference net: 2 dense levels (4, 8), hidden 8, K=2",
    mode=RADIANCE, level_res=[4, 8], feat=2, log2_table=19,
    widths=[4, 8, 8, 8], K=2, n_query=64, n_train=64)

FD_TINY_PRODUCT = FD_TINY.with_(
    name="finite-difference net, product mode: 2 dense levels, hidden 8, K=2",
    mode=PRODUCT, widths=[32, 8, 8, 8])

WORKLOADS = {
    "tiny": TINY,
    "paper_hash": PAPER_HASH,
    "tiny_bf16": TINY_BF16,
    "tiny_fp16": TINY_BF16.with_(
        name="tiny dense 16^3x4, MLP 4-32-32-16, K=4, fp16 tensor-core MLP / fp16 grid", precision=FP16),
    # The serving loop's per-frame training batch on the tiny network.
    "tiny_bf16_train": TINY_BF16.with_(
        name="tiny dense 16^3x4, MLP 4-32-32-16, K=4, split-bf16, training batch 2^18", n_train=1 << 18),
    "product_bf16": PRODUCT_BF16,
    "paper_own": PAPER_OWN,
    "paper_hash_fp32tc": PAPER_HASH.with_(
        name="hash grid 16 levels x 2 feats, T=2^19, MLP 32-64-64-64-32, K=8, FP32 accuracy on tensor cores "
             "(split FP16 operands, FP32 grid)", precision=FP32_TC),
    "paper_hash_bf16": PAPER_HASH.with_(
        name="hash grid 16 levels x 2 feats, T=2^19, MLP 32-64-64-64-32, K=8, split-bf16",
        precision=BF16X3),
    "paper_own_bf16": PAPER_OWN.with_(
        name="paper's own shape: 8 dense levels D 8..86 x 4 feats, MLP 32-64-64-64-32, K=8, split-bf16",
        precision=BF16X3),
}


def encoding_width(w: Workload) -> int:
    """Number of meaningful MLP inputs (grid features, plus SH and roughness)."""
    g = len(w.level_res) * w.feat
    return g + (16 + 4 + 1 if w.mode == PRODUCT else 0)


def grid_sizes(w: Workload) -> List[int]:
    """Entries per level as the configuration defines them: min(T, D^3)."""
    T = 1 << w.log2_table
    return [min(T, d ** 3) for d in w.level_res]


def n_params(w: Workload) -> int:
    g = sum(grid_sizes(w)) * w.feat
    m = sum(w.widths[i] * w.widths[i + 1] for i in range(len(w.widths) - 1))
    return g + m


# --------------------------------------------------------------------------
# Initial parameters (grid U[-1e-4, 1e-4]; MLP Glorot-uniform, no biases).
# --------------------------------------------------------------------------

def init_params(w: Workload, seed: Optional[int] = None) -> np.ndarray:
    """Flat float32 parameter blob: grid (level, entry, feature), then each
    weight matrix row-major [out][in]."""
    seed = w.seed if seed is None else seed
    ng = sum(grid_sizes(w)) * w.feat
    grid = (uniform(seed, S_GRID_INIT, ng).astype(np.float64) * 2.0 - 1.0) * 1e-4
    mats = []
    off = 0
    for i in range(len(w.widths) - 1):
        fi, fo = w.widths[i], w.widths[i + 1]
        a = math.sqrt(6.0 / (fi + fo))
        u = uniform(seed, S_MLP_INIT, fi * fo, start=off).astype(np.float64)
        off += fi * fo
        mats.append((u * 2.0 - 1.0) * a)
    # Zero the weight columns that read the zero padding of the input.
    ew = encoding_width(w)
    if ew < w.widths[0]:
        mats[0].reshape(w.widths[1], w.widths[0])[:, ew:] = 0.0
    return np.concatenate([grid] + mats).astype(np.float32)


def random_params(w: Workload, seed: int = 1, grid_scale: float = 1.0,
                  gain: float = 2.0, kappa_boost: float = 6.0) -> np.ndarray:
    """Parameters that decode to varied mixtures (uneven weights, lobes spread
    over the sphere, kappa up to tens), standing in for a trained model:
    grid features U[-grid_scale, grid_scale], Glorot-uniform layers times
    gain, and the kappa' rows of the last layer scaled by kappa_boost."""
    ng = sum(grid_sizes(w)) * w.feat
    grid = (uniform(seed, S_GRID_INIT, ng).astype(np.float64) * 2.0 - 1.0) * grid_scale
    mats = []
    off = 0
    ew = encoding_width(w)
    for i in range(len(w.widths) - 1):
        fi, fo = w.widths[i], w.widths[i + 1]
        # Fan-in of the first layer counts only the meaningful inputs.
        fan_in = min(fi, ew) if i == 0 else fi
        a = gain * math.sqrt(6.0 / (fan_in + fo))
        u = uniform(seed, S_MLP_INIT, fi * fo, start=off).astype(np.float64)
        off += fi * fo
        m = ((u * 2.0 - 1.0) * a).reshape(fo, fi)
        if i == 0 and ew < fi:
            m[:, ew:] = 0.0
        mats.append(m)
    last = mats[-1]
    for k in range(w.K):
        last[4 * k + 1] *= kappa_boost
    return np.concatenate([grid] + [m.ravel() for m in mats]).astype(np.float32)


# --------------------------------------------------------------------------
# Query inputs.
# --------------------------------------------------------------------------

def positions(seed: int, n: int) -> np.ndarray:
    return uniform_rows(seed, S_POS, 3, n)


def sample_uniforms(seed: int, n: int, rows: int = 3) -> np.ndarray:
    return uniform_rows(seed, S_U, rows, n)


def aux_inputs(seed: int, n: int) -> np.ndarray:
    """Product-mode auxiliary inputs [7][n]: wo (3), normal (3), roughness.
    The normal is uniform on the sphere, wo uniform on its hemisphere, and the
    roughness uniform in [0.05, 1]."""
    u = uniform_rows(seed, S_AUX, 5, n)
    nrm = sphere_dirs(u[0], u[1])
    wo = sphere_dirs(u[2], u[3])
    flip = np.sum(wo * nrm, axis=0) < 0.0
    wo[:, flip] *= -1.0
    r = 0.05 + 0.95 * u[4].astype(np.float64)
    return np.concatenate([wo, nrm, r[None]]).astype(np.float32)


# --------------------------------------------------------------------------
# Analytic stand-in scene: a radiance field that is a sum of three lobes whose
# means and sharpness vary smoothly with position.
# --------------------------------------------------------------------------

_AMP = (0.5, 0.3, 0.2)
_E = (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]),
      np.array([-1.0, -1.0, 1.0]) / math.sqrt(3.0))


def field_lobes(x: np.ndarray):
    """Means [3 lobes][3][n] and sharpness [3][n] of the stand-in field."""
    x = np.asarray(x, dtype=np.float64)
    mus, kaps = [], []
    for m in range(3):
        p = 0.5 * np.stack([np.sin(2 * math.pi * x[1] + m),
                            np.sin(2 * math.pi * x[2] + 2 * m),
                            np.sin(2 * math.pi * x[0] + 3 * m)])
        v = _E[m][:, None] + p
        v = v / np.linalg.norm(v, axis=0, keepdims=True)
        k = 1.0 + 49.0 * (0.5 + 0.5 * np.sin(2 * math.pi * (m + 1) * (x[0] + x[1] + x[2]) / 3.0 + m))
        mus.append(v)
        kaps.append(k)
    return np.stack(mus), np.stack(kaps)


def _lobe(w: np.ndarray, mu: np.ndarray, k: np.ndarray) -> np.ndarray:
    # Normalised spherical lobe written from its textbook definition
    # k exp(k mu.w) / (4 pi sinh k), in a form safe for k up to 50.
    d = np.sum(mu * w, axis=0)
    return k * np.exp(k * (d - 1.0)) / (2.0 * math.pi * (1.0 - np.exp(-2.0 * k)))


def radiance(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Noise-free stand-in radiance L(x, w), float64 [n]."""
    mus, kaps = field_lobes(x)
    w = np.asarray(w, dtype=np.float64)
    return sum(_AMP[m] * _lobe(w, mus[m], kaps[m]) for m in range(3))


def glossy_factor(w: np.ndarray, aux: np.ndarray) -> np.ndarray:
    """Product-mode BSDF-and-cosine stand-in:
    max(0, n.w) * (0.3 + 0.7 * D(n.h) / D(1)) with a GGX-like normal
    distribution D of alpha = roughness^2 and h = normalize(w + wo)."""
    w = np.asarray(w, dtype=np.float64)
    aux = np.asarray(aux, dtype=np.float64)
    wo, nrm, r = aux[0:3], aux[3:6], aux[6]
    cos_i = np.maximum(0.0, np.sum(nrm * w, axis=0))
    h = w + wo
    hl = np.linalg.norm(h, axis=0)
    ok = hl > 1e-9
    h = h / np.where(ok, hl, 1.0)
    ch = np.clip(np.sum(nrm * h, axis=0), -1.0, 1.0)
    a2 = (r * r) ** 2
    ratio = a2 * a2 / (ch * ch * (a2 - 1.0) + 1.0) ** 2
    ratio = np.where(ok & (ch > 0), ratio, 0.0)
    return cos_i * (0.3 + 0.7 * ratio)


def target(x: np.ndarray, w: np.ndarray, aux: Optional[np.ndarray]) -> np.ndarray:
    L = radiance(x, w)
    if aux is not None:
        L = L * glossy_factor(w, aux)
    return L


def exp_noise(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Exponential(1) multiplicative noise, -log(1 - u)."""
    u = uniform(seed, S_NOISE, n, start=start).astype(np.float64)
    return -np.log1p(-u)


@dataclass
class TrainBatch:
    pos: np.ndarray      # [3][n] float32
    aux: Optional[np.ndarray]  # [7][n] float32 or None
    dir: np.ndarray      # [3][n] float32
    radiance: np.ndarray  # [n] float32, noisy estimate
    pdf: np.ndarray      # [n] float32, density the directions were drawn from
    clean: np.ndarray    # [n] float64, noise-free target at the samples


def train_batch_uniform(w: Workload, n: int, seed: Optional[int] = None) -> TrainBatch:
    """Training samples with directions drawn uniformly on the sphere, so the
    sampling density is the constant 1/(4 pi)."""
    seed = w.seed if seed is None else seed
    pos = positions(seed + 1000, n)
    aux = aux_inputs(seed + 1000, n) if w.mode == PRODUCT else None
    u = uniform_rows(seed, S_DIR, 2, n)
    d = sphere_dirs(u[0], u[1]).astype(np.float32)
    clean = target(pos, d, aux)
    noisy = clean * exp_noise(seed, n)
    pdf = np.full(n, 1.0 / (4.0 * math.pi), dtype=np.float32)
    return TrainBatch(pos, aux, d, noisy.astype(np.float32), pdf, clean)
