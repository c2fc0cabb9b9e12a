"""GB300-native hot path of Neural Parametric Mixtures (NPM) for path guiding.

The compute runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/npm.h``; this module only marshals torch tensors (device memory and
streams) into those calls. See ``NPM`` for the entry points.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._build import build  # noqa: F401
from ._lib import NpmError  # noqa: F401

RADIANCE, PRODUCT = 0, 1
SOFTPLUS, EXP = 0, 1
FP32, BF16, BF16X3, FP16, FP32_TC = 0, 1, 2, 3, 4


def _torch():
    import torch
    return torch


def make_config(mode: int, level_res: Sequence[int], feat: int, log2_table: int,
                widths: Sequence[int], K: int, kappa_act: int = SOFTPLUS,
                precision: int = FP32, lr: float = 5e-3, beta1: float = 0.9,
                beta2: float = 0.99, eps: float = 1e-8, max_batch: int = 1 << 20,
                seed: int = 0) -> _lib.NpmConfig:
    c = _lib.NpmConfig()
    c.mode = mode
    c.n_levels = len(level_res)
    c.feat_per_level = feat
    c.log2_table = log2_table
    for i, r in enumerate(level_res):
        c.level_res[i] = int(r)
    c.n_layers = len(widths) - 1
    for i, w in enumerate(widths):
        c.widths[i] = int(w)
    c.K = K
    c.kappa_act = kappa_act
    c.precision = precision
    c.lr, c.beta1, c.beta2, c.eps = lr, beta1, beta2, eps
    c.max_batch = int(max_batch)
    c.seed = int(seed)
    return c


def config_from(w, max_batch: Optional[int] = None, precision: Optional[int] = None,
                seed: int = 0) -> _lib.NpmConfig:
    """Config from any object with the fields of a workload description
    (mode, level_res, feat, log2_table, widths, K, kappa_act, precision, lr,
    beta1, beta2, eps, n_query, n_train)."""
    mb = max_batch if max_batch is not None else max(w.n_query, w.n_train, 1)
    return make_config(w.mode, w.level_res, w.feat, w.log2_table, w.widths, w.K, w.kappa_act,
                       w.precision if precision is None else precision, w.lr, w.beta1, w.beta2,
                       w.eps, mb, seed)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        torch = _torch()
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream


def _soa(t, rows: int, name: str):
    """Validate a [rows][ld] float32 CUDA tensor; returns ld."""
    torch = _torch()
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if t.dim() != 2 or t.shape[0] < rows or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous [{rows}][ld] tensor")
    return t.shape[1]


class NPM:
    """One NPM model on the current CUDA device (library-owned parameters,
    gradient and Adam state)."""

    def __init__(self, config: _lib.NpmConfig):
        self._L = _lib.load()
        self.config = config
        h = C.c_void_p()
        _lib.check(self._L.npm_create(C.byref(config), C.byref(h)), "npm_create")
        self._h = h
        self.K = config.K
        self.mode = config.mode

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._L.npm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- hot path
    def query_sample(self, pos, u, aux=None, uniform_frac: float = 0.0, n: Optional[int] = None,
                     want_mix: bool = False, out=None, stream=None):
        """Guided directions and densities. pos [3][ld], u [3 or 4][ld],
        aux [7][ld] (product mode). Returns (dir [3][ld], pdf [ld], mix)."""
        torch = _torch()
        ld = _soa(pos, 3, "pos")
        n = ld if n is None else n
        _soa(u, 4 if uniform_frac > 0 else 3, "u")
        if aux is not None:
            _soa(aux, 7, "aux")
        if out is None:
            d = torch.empty((3, ld), device=pos.device, dtype=torch.float32)
            p = torch.empty((ld,), device=pos.device, dtype=torch.float32)
        else:
            d, p = out
        m = torch.empty((4 * self.K, ld), device=pos.device, dtype=torch.float32) if want_mix else None
        _lib.check(self._L.npm_query_sample(self._h, n, _ptr(pos), _ptr(aux), _ptr(u), ld,
                                            float(uniform_frac), _ptr(d), _ptr(p), _ptr(m),
                                            _stream_ptr(stream)), "npm_query_sample")
        return d, p, m

    def query_sample_host(self, pos, u, dir_out, pdf_out, aux=None, uniform_frac: float = 0.0,
                          n: Optional[int] = None, stream=None):
        """Same as query_sample with all arrays in (preferably pinned) HOST
        memory -- torch CPU tensors; copies run inside the library."""
        ld = pos.shape[1]
        n = ld if n is None else n
        for t in (pos, u, dir_out, pdf_out) + ((aux,) if aux is not None else ()):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host tensors must be contiguous CPU tensors")
        _lib.check(self._L.npm_query_sample_host(self._h, n, _ptr(pos), _ptr(aux), _ptr(u), ld,
                                                 float(uniform_frac), _ptr(dir_out),
                                                 _ptr(pdf_out), _stream_ptr(stream)),
                   "npm_query_sample_host")

    def eval_pdf(self, pos, dirs, aux=None, n: Optional[int] = None, out=None, stream=None):
        torch = _torch()
        ld = _soa(pos, 3, "pos")
        n = ld if n is None else n
        _soa(dirs, 3, "dir")
        p = torch.empty((ld,), device=pos.device, dtype=torch.float32) if out is None else out
        _lib.check(self._L.npm_eval_pdf(self._h, n, _ptr(pos), _ptr(aux), _ptr(dirs), ld, _ptr(p),
                                        _stream_ptr(stream)), "npm_eval_pdf")
        return p

    def eval_log_pdf(self, pos, dirs, aux=None, n: Optional[int] = None, out=None, stream=None):
        """log V at the given directions, computed in the kernel in
        log-sum-exp form (npm_eval_log_pdf)."""
        torch = _torch()
        ld = _soa(pos, 3, "pos")
        n = ld if n is None else n
        _soa(dirs, 3, "dir")
        p = torch.empty((ld,), device=pos.device, dtype=torch.float32) if out is None else out
        _lib.check(self._L.npm_eval_log_pdf(self._h, n, _ptr(pos), _ptr(aux), _ptr(dirs), ld, _ptr(p),
                                            _stream_ptr(stream)), "npm_eval_log_pdf")
        return p

    def train_step(self, pos, dirs, radiance, sample_pdf, aux=None, n: Optional[int] = None,
                   loss_out=None, stream=None):
        torch = _torch()
        ld = _soa(pos, 3, "pos")
        n = ld if n is None else n
        loss = torch.zeros((1,), device=pos.device, dtype=torch.float32) if loss_out is None else loss_out
        _lib.check(self._L.npm_train_step(self._h, n, _ptr(pos), _ptr(aux), _ptr(dirs),
                                          _ptr(radiance), _ptr(sample_pdf), ld, _ptr(loss),
                                          _stream_ptr(stream)), "npm_train_step")
        return loss

    def backward(self, pos, dirs, dlogv, aux=None, n: Optional[int] = None, stream=None):
        ld = _soa(pos, 3, "pos")
        n = ld if n is None else n
        _lib.check(self._L.npm_backward(self._h, n, _ptr(pos), _ptr(aux), _ptr(dirs), _ptr(dlogv),
                                        ld, _stream_ptr(stream)), "npm_backward")

    def adam_step(self, stream=None):
        _lib.check(self._L.npm_adam_step(self._h, _stream_ptr(stream)), "npm_adam_step")

    # -- support
    def num_params(self) -> int:
        return int(self._L.npm_num_params(self._h))

    def set_params(self, params: np.ndarray):
        a = np.ascontiguousarray(params, dtype=np.float32)
        _lib.check(self._L.npm_set_params(self._h, a.ctypes.data_as(C.c_void_p), a.size),
                   "npm_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(self.num_params(), dtype=np.float32)
        _lib.check(self._L.npm_get_params(self._h, a.ctypes.data_as(C.c_void_p), a.size),
                   "npm_get_params")
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(self.num_params(), dtype=np.float32)
        _lib.check(self._L.npm_get_grads(self._h, a.ctypes.data_as(C.c_void_p), a.size),
                   "npm_get_grads")
        return a

    def set_params_device(self, theta, stream=None):
        """Parameters from a float32 CUDA tensor [npm_num_params] in the
        public layout (npm_set_params_device; stream-ordered)."""
        torch = _torch()
        if theta.dtype != torch.float32 or not theta.is_cuda or not theta.is_contiguous():
            raise TypeError("theta must be a contiguous float32 CUDA tensor")
        _lib.check(self._L.npm_set_params_device(self._h, _ptr(theta), theta.numel(), _stream_ptr(stream)),
                   "npm_set_params_device")

    def grads_device(self, out=None, stream=None):
        """The gradient buffer as a float32 CUDA tensor in the public layout
        (npm_get_grads_device; stream-ordered)."""
        torch = _torch()
        g = torch.empty((self.num_params(),), dtype=torch.float32, device="cuda") if out is None else out
        _lib.check(self._L.npm_get_grads_device(self._h, _ptr(g), g.numel(), _stream_ptr(stream)),
                   "npm_get_grads_device")
        return g

    def set_ema(self, decay: float, stream=None):
        """Inference evaluates the moving average of the weights (npm_set_ema);
        decay 0 turns it off."""
        _lib.check(self._L.npm_set_ema(self._h, float(decay), _stream_ptr(stream)), "npm_set_ema")

    def get_ema_params(self) -> np.ndarray:
        a = np.empty(self.num_params(), dtype=np.float32)
        _lib.check(self._L.npm_get_ema_params(self._h, a.ctypes.data_as(C.c_void_p), a.size),
                   "npm_get_ema_params")
        return a

    def get_adam(self):
        n = self.num_params()
        m = np.empty(n, dtype=np.float32)
        v = np.empty(n, dtype=np.float32)
        step = C.c_int()
        _lib.check(self._L.npm_get_adam(self._h, C.byref(step), m.ctypes.data_as(C.c_void_p),
                                        v.ctypes.data_as(C.c_void_p)), "npm_get_adam")
        return step.value, m, v

    def set_adam(self, step: int, m: np.ndarray, v: np.ndarray):
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        _lib.check(self._L.npm_set_adam(self._h, int(step), m.ctypes.data_as(C.c_void_p),
                                        v.ctypes.data_as(C.c_void_p)), "npm_set_adam")

    def grid_indices(self, pos, n: Optional[int] = None, stream=None):
        torch = _torch()
        ld = _soa(pos, 3, "pos")
        n = ld if n is None else n
        out = torch.empty((self.config.n_levels, 8, n), device=pos.device, dtype=torch.int32)
        _lib.check(self._L.npm_grid_indices(self._h, n, _ptr(pos), ld, _ptr(out),
                                            _stream_ptr(stream)), "npm_grid_indices")
        return out

    def save(self, path: str):
        _lib.check(self._L.npm_save(self._h, path.encode()), "npm_save")

    def load(self, path: str):
        _lib.check(self._L.npm_load(self._h, path.encode()), "npm_load")

    def check_device_status(self, stream=None):
        _lib.check(self._L.npm_check_device_status(self._h, _stream_ptr(stream)),
                   "npm_check_device_status")

    def pdf_integral(self, pos, dirs, weights, aux=None, stream=None):
        """Integral over the sphere of the mixture density at each position
        (npm_pdf_integral): sum_k weights[k] V(dirs[:, k] | pos[:, p]),
        reduced in FP64 on the GPU. pos [3][n] (and aux [7][n]) float32,
        dirs [3][n_dir] float32, weights [n_dir] float64, device tensors;
        returns a float64 device tensor [n]."""
        import torch
        n, n_dir = pos.shape[1], dirs.shape[1]
        out = torch.empty((n,), dtype=torch.float64, device=pos.device)
        _lib.check(self._L.npm_pdf_integral(
            self._h, n, _ptr(pos), _ptr(aux) if aux is not None else None, pos.stride(0), n_dir,
            _ptr(dirs), _ptr(weights), _ptr(out), _stream_ptr(stream)), "npm_pdf_integral")
        return out

    def set_wait_limit(self, cycles: int):
        """Bound (SM clock cycles) of the FP32 forward kernel's internal
        waits (npm_set_wait_limit); <= 0 makes each wait one test."""
        _lib.check(self._L.npm_set_wait_limit(self._h, int(cycles)), "npm_set_wait_limit")


def _make_log_density():
    torch = _torch()

    class LogDensity(torch.autograd.Function):
        """log V(dir_j | Theta(x_j); theta) for a batch, differentiable in the
        parameters theta (float32 CUDA tensor [npm_num_params], public layout).

        Forward loads theta into the model (npm_set_params_device) and
        evaluates log V with the library's kernels (npm_eval_log_pdf, in
        log-sum-exp form); backward reloads theta and runs the hand-written
        backward (npm_backward: decode, MLP and grid, activations recomputed,
        with the incoming gradient as the per-query weight of d log V),
        returning the parameter gradient (npm_get_grads_device)."""

        @staticmethod
        def forward(ctx, theta, model, pos, dirs, aux=None):
            model.set_params_device(theta)
            lv = model.eval_log_pdf(pos, dirs, aux)
            n = pos.shape[1]
            ctx.model = model
            ctx.save_for_backward(theta, pos, dirs, aux if aux is not None else theta.new_empty(0))
            ctx.has_aux = aux is not None
            return lv[:n]

        @staticmethod
        def backward(ctx, grad_out):
            theta, pos, dirs, aux = ctx.saved_tensors
            model = ctx.model
            model.set_params_device(theta)
            model.backward(pos, dirs, grad_out.contiguous().to(torch.float32), aux if ctx.has_aux else None)
            return model.grads_device(), None, None, None, None

    return LogDensity


_LOG_DENSITY = None


def log_density(theta, model, pos, dirs, aux=None):
    """Differentiable log V (LogDensity.apply): see _make_log_density."""
    global _LOG_DENSITY
    if _LOG_DENSITY is None:
        _LOG_DENSITY = _make_log_density()
    return _LOG_DENSITY.apply(theta, model, pos, dirs, aux)


class Server:
    """Continuous-batching request loop over one NPM model (npm_server_* C
    ABI). Requests carry host (CPU) tensors in the [c][ld] layout; pinned
    memory lets the copies overlap. The model must not be used directly while
    the server is open."""

    def __init__(self, model: NPM, pool_queries: int):
        self._L = _lib.load()
        self.model = model
        h = C.c_void_p()
        _lib.check(self._L.npm_server_create(model.handle, int(pool_queries), C.byref(h)),
                   "npm_server_create")
        self._s = h
        self._keep = {}

    @staticmethod
    def _host(*ts):
        for t in ts:
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("server requests take contiguous host tensors")

    def submit_query(self, pos, u, dir_out, pdf_out, aux=None, uniform_frac: float = 0.0,
                     n: Optional[int] = None) -> int:
        self._host(pos, u, dir_out, pdf_out, aux)
        ld = pos.shape[1]
        n = ld if n is None else n
        t = C.c_uint64()
        _lib.check(self._L.npm_server_submit_query(self._s, n, _ptr(pos), _ptr(aux), _ptr(u), ld,
                                                   float(uniform_frac), _ptr(dir_out),
                                                   _ptr(pdf_out), C.byref(t)),
                   "npm_server_submit_query")
        self._keep[t.value] = (pos, u, dir_out, pdf_out, aux)
        return t.value

    def submit_train(self, pos, dirs, radiance, sample_pdf, aux=None, n: Optional[int] = None) -> int:
        self._host(pos, dirs, radiance, sample_pdf, aux)
        ld = pos.shape[1]
        n = ld if n is None else n
        t = C.c_uint64()
        _lib.check(self._L.npm_server_submit_train(self._s, n, _ptr(pos), _ptr(aux), _ptr(dirs),
                                                   _ptr(radiance), _ptr(sample_pdf), ld,
                                                   C.byref(t)), "npm_server_submit_train")
        self._keep[t.value] = (pos, dirs, radiance, sample_pdf, aux)
        return t.value

    def hold(self, on: bool = True):
        """Pause (True) or resume (False) admission; requests submitted while
        held are admitted together on resume."""
        _lib.check(self._L.npm_server_hold(self._s, 1 if on else 0), "npm_server_hold")

    def wait(self, ticket: int) -> float:
        lat = C.c_double()
        try:
            _lib.check(self._L.npm_server_wait(self._s, int(ticket), C.byref(lat)), "npm_server_wait")
        finally:
            self._keep.pop(ticket, None)
        return lat.value

    def stats(self) -> dict:
        s = _lib.NpmServerStats()
        _lib.check(self._L.npm_server_get_stats(self._s, C.byref(s)), "npm_server_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_s", None):
            self._L.npm_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Wavefront:
    """Synthetic wavefront frame driver around a radiance-mode model
    (npm_wavefront_* C ABI)."""

    def __init__(self, model: NPM, paths: int, bounces: int = 8, survival: float = 0.7,
                 train_batch: int = 1 << 18, uniform_frac: float = 0.5, seed: int = 0,
                 use_graph: bool = True, max_frames: int = 1024):
        self._L = _lib.load()
        self.model = model
        c = _lib.NpmFrameConfig()
        self.bounces = int(bounces)
        c.paths, c.bounces, c.survival = int(paths), int(bounces), float(survival)
        c.train_batch, c.uniform_frac, c.seed = int(train_batch), float(uniform_frac), int(seed)
        c.use_graph, c.max_frames = 1 if use_graph else 0, int(max_frames)
        h = C.c_void_p()
        _lib.check(self._L.npm_wavefront_create(model.handle, C.byref(c), C.byref(h)),
                   "npm_wavefront_create")
        self._w = h

    def run(self, frames: int, stream=None) -> dict:
        s = _lib.NpmFrameStats()
        _lib.check(self._L.npm_wavefront_run(self._w, int(frames), _stream_ptr(stream), C.byref(s)),
                   "npm_wavefront_run")
        out = {k: getattr(s, k) for k, _ in s._fields_}
        nb = min(self.bounces, _lib.FRAME_BOUNCE_STATS)
        out["bounce_queries"] = list(s.bounce_queries)[:nb]
        out["bounce_query_ms"] = list(s.bounce_query_ms)[:nb]
        return out

    def close(self):
        if getattr(self, "_w", None):
            self._L.npm_wavefront_destroy(self._w)
            self._w = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def measure_unit_peaks(stream=None) -> dict:
    """Measured FP32 FMA, MUFU, L2 sector-read and L2 atomic throughput of
    the current device (npm_measure_unit_peaks)."""
    L = _lib.load()
    p = _lib.NpmUnitPeaks()
    _lib.check(L.npm_measure_unit_peaks(C.byref(p), _stream_ptr(stream)), "npm_measure_unit_peaks")
    return {k: getattr(p, k) for k, _ in p._fields_}
