"""Synthetic stand-in scene on the device (npm_scene_* C ABI) and the online
training loop of Sec. 5.2 driven by it: each step draws path vertices,
samples directions from the current guide mixed with uniform-sphere
sampling (the BSDF stand-in, 50 % selection as in Sec. 6.1), evaluates the
noisy target there and takes one training step."""
from __future__ import annotations

from typing import Optional

from . import NPM, PRODUCT, _lib, _ptr, _stream_ptr


def _torch():
    import torch
    return torch


def generate(seed: int, n: int, product: bool, urows: int = 3, stream=None):
    """Device tensors pos [3][n], aux [7][n] or None, u [urows][n]."""
    torch = _torch()
    pos = torch.empty((3, n), device="cuda")
    aux = torch.empty((7, n), device="cuda") if product else None
    u = torch.empty((max(urows, 1), n), device="cuda")
    _lib.check(_lib.load().npm_scene_generate(int(seed), n, 1 if product else 0, _ptr(pos), _ptr(aux),
                                              _ptr(u), urows, n, _stream_ptr(stream)),
               "npm_scene_generate")
    return pos, aux, u


def radiance(product: bool, pos, aux, dirs, noise_seed: int = 0, clean: bool = True,
             noisy: bool = True, stream=None):
    """(clean [n] or None, noisy [n] or None) device tensors."""
    torch = _torch()
    n = pos.shape[1]
    c = torch.empty((n,), device="cuda") if clean else None
    z = torch.empty((n,), device="cuda") if noisy else None
    _lib.check(_lib.load().npm_scene_radiance(1 if product else 0, int(noise_seed), n, _ptr(pos),
                                              _ptr(aux), _ptr(dirs), n, _ptr(c), _ptr(z),
                                              _stream_ptr(stream)), "npm_scene_radiance")
    return c, z


def _guide_input(pos, fixed_position: Optional[float]):
    """The positions the guide sees: the vertices', or one constant point for
    every vertex (a position-independent guide: a single mixture for the
    whole scene)."""
    return pos if fixed_position is None else _torch().full_like(pos, float(fixed_position))


def online_step(model: NPM, seed: int, n: int, uniform_frac: float = 0.5,
                fixed_position: Optional[float] = None, stream=None):
    """One online training step on n fresh samples; returns the loss tensor.
    With fixed_position the guide is queried and trained at that constant
    point, while the target is evaluated at the real vertices."""
    product = model.mode == PRODUCT
    pos, aux, u = generate(seed, n, product, urows=4, stream=stream)
    gpos = _guide_input(pos, fixed_position)
    d, p, _ = model.query_sample(gpos, u, aux, uniform_frac=uniform_frac, stream=stream)
    _, noisy = radiance(product, pos, aux, d, noise_seed=seed, clean=False, stream=stream)
    return model.train_step(gpos, d, noisy, p, aux, stream=stream)


def relative_variance(model: NPM, product: bool, seed: int, n: int, uniform: bool = False,
                      fixed_position: Optional[float] = None, alpha: float = 0.0, stream=None):
    """Relative variance var(I) / mean(I)^2 of the one-sample estimator
    I = target(x, w) / pdf(w | x) over n vertices, with w drawn from the
    model's guide, or uniformly on the sphere (uniform=True, the "no guide"
    baseline: the same kernel with uniform_frac = 1). alpha > 0 draws from
    the defensive one-sample mixture alpha uniform + (1 - alpha) guide (the
    strategy the method samples with, Sec. 6.1), whose estimator is bounded
    by target 4 pi / alpha. fixed_position: the guide sees that constant
    point (see online_step)."""
    pos, aux, u = generate(seed, n, product, urows=4, stream=stream)
    d, p, _ = model.query_sample(_guide_input(pos, fixed_position), u, aux,
                                 uniform_frac=1.0 if uniform else alpha, stream=stream)
    clean, _ = radiance(product, pos, aux, d, noisy=False, stream=stream)
    est = clean.double() / p.double()
    return float(est.var() / est.mean() ** 2), float(est.mean())
