"""FP64 CPU oracle of the NPM hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product path never does. The C source
(``npm_oracle.c``) shares no code with the CUDA library.

``build()`` compiles the C file with gcc (OpenMP when available) into
``oracle/_build/libnpm_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libnpm_oracle.so")
_lib = None


class OrcCfg(C.Structure):
    _fields_ = [
        ("mode", C.c_int), ("n_levels", C.c_int), ("feat", C.c_int),
        ("log2_table", C.c_int), ("level_res", C.c_int * 32),
        ("n_layers", C.c_int), ("widths", C.c_int * 17), ("K", C.c_int),
        ("kappa_act", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle; returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        d, f, i32, i64 = C.c_double, C.c_float, C.c_int32, C.c_int64
        vp = C.c_void_p
        sig = {
            "orc_grid_offsets": (i64, [P(OrcCfg), vp]),
            "orc_n_params": (i64, [P(OrcCfg)]),
            "orc_lattice_index": (C.c_uint32, [P(OrcCfg), C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]),
            "orc_grid_corners": (None, [P(OrcCfg), C.c_int, vp, vp, vp]),
            "orc_grid_encode": (None, [P(OrcCfg), vp, vp, vp]),
            "orc_sh": (None, [C.c_int, vp, vp]),
            "orc_encode": (None, [P(OrcCfg), vp, vp, vp, vp]),
            "orc_mlp": (None, [P(OrcCfg), vp, vp, vp, vp]),
            "orc_vmf_scaled_norm": (d, [d]),
            "orc_vmf_sample_w": (d, [d, d]),
            "orc_vmf_sample": (None, [vp, d, d, d, vp]),
            "orc_frame": (None, [vp, vp, vp]),
            "orc_decode_batch": (None, [P(OrcCfg), vp, i64, vp, vp, i64, vp]),
            "orc_query_sample": (None, [P(OrcCfg), vp, i64, vp, vp, vp, i64, d, vp, vp, vp, vp, vp]),
            "orc_eval_pdf": (None, [P(OrcCfg), vp, i64, vp, vp, vp, i64, vp]),
            "orc_eval_pdf64": (None, [P(OrcCfg), vp, i64, vp, vp, vp, i64, vp]),
            "orc_grid_indices": (None, [P(OrcCfg), i64, vp, i64, vp]),
            "orc_train_grad": (d, [P(OrcCfg), vp, i64, vp, vp, vp, vp, vp, i64, vp]),
            "orc_train_loss": (d, [P(OrcCfg), vp, i64, vp, vp, vp, vp, vp, i64]),
            "orc_adam": (None, [i64, vp, vp, vp, vp, C.c_int, d, d, d, d]),
            "orc_ema": (None, [i64, vp, vp, d]),
            "orc_num_threads": (C.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def cfg_of(w) -> OrcCfg:
    """Oracle configuration from a synth.Workload (plain field copy)."""
    c = OrcCfg()
    c.mode = w.mode
    c.n_levels = len(w.level_res)
    c.feat = w.feat
    c.log2_table = w.log2_table
    for i, r in enumerate(w.level_res):
        c.level_res[i] = r
    c.n_layers = len(w.widths) - 1
    for i, x in enumerate(w.widths):
        c.widths[i] = x
    c.K = w.K
    c.kappa_act = w.kappa_act
    return c


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def n_params(w) -> int:
    c = cfg_of(w)
    return int(lib().orc_n_params(C.byref(c)))


def grid_offsets(w) -> np.ndarray:
    c = cfg_of(w)
    off = np.zeros(32, dtype=np.int64)
    lib().orc_grid_offsets(C.byref(c), _p(off))
    return off[: len(w.level_res)]


def lattice_index(w, level: int, i: int, j: int, k: int) -> int:
    c = cfg_of(w)
    return int(lib().orc_lattice_index(C.byref(c), level, i, j, k))


def grid_corners(w, level: int, x):
    c = cfg_of(w)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    idx = np.zeros(8, dtype=np.uint32)
    wt = np.zeros(8, dtype=np.float64)
    lib().orc_grid_corners(C.byref(c), level, _p(xx), _p(idx), _p(wt))
    return idx, wt


def grid_encode(w, params, x) -> np.ndarray:
    c = cfg_of(w)
    out = np.zeros(len(w.level_res) * w.feat, dtype=np.float64)
    lib().orc_grid_encode(C.byref(c), _p(_f64(params)), _p(_f32(x)), _p(out))
    return out


def sh(bands: int, d) -> np.ndarray:
    dd = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(bands * bands, dtype=np.float64)
    lib().orc_sh(bands, _p(dd), _p(out))
    return out


def encode(w, params, x, aux7=None) -> np.ndarray:
    c = cfg_of(w)
    out = np.zeros(w.widths[0], dtype=np.float64)
    a = _f32(aux7 if aux7 is not None else np.zeros(7))
    lib().orc_encode(C.byref(c), _p(_f64(params)), _p(_f32(x)), _p(a), _p(out))
    return out


def mlp(w, params, inp, want_acts: bool = False):
    c = cfg_of(w)
    inp = np.ascontiguousarray(inp, dtype=np.float64)
    raw = np.zeros(w.widths[-1], dtype=np.float64)
    acts = np.zeros(sum(w.widths[1:]), dtype=np.float64) if want_acts else None
    lib().orc_mlp(C.byref(c), _p(_f64(params)), _p(inp), _p(raw), _p(acts))
    return (raw, acts) if want_acts else raw


def vmf_scaled_norm(k: float) -> float:
    return float(lib().orc_vmf_scaled_norm(k))


def vmf_sample_w(k: float, u1: float) -> float:
    return float(lib().orc_vmf_sample_w(k, u1))


def vmf_sample(mu, k: float, u1: float, u2: float) -> np.ndarray:
    m = np.ascontiguousarray(mu, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_vmf_sample(_p(m), k, u1, u2, _p(out))
    return out


def frame(n):
    nn = np.ascontiguousarray(n, dtype=np.float64)
    t = np.zeros(3)
    b = np.zeros(3)
    lib().orc_frame(_p(nn), _p(t), _p(b))
    return t, b


def decode_batch(w, params, pos, aux=None) -> np.ndarray:
    """[4K][n] rows of (lambda, kappa, theta, phi) per lobe."""
    c = cfg_of(w)
    pos = _f32(pos)
    n = pos.shape[1]
    out = np.zeros((4 * w.K, n), dtype=np.float64)
    lib().orc_decode_batch(C.byref(c), _p(_f64(params)), n, _p(pos), _p(_f32(aux)), n, _p(out))
    return out


def query_sample(w, params, pos, u, aux=None, alpha: float = 0.0, forced=None):
    """Returns dir [3][n], pdf [n], lobe [n], margin [n] (all float64/int)."""
    c = cfg_of(w)
    pos = _f32(pos)
    u = _f32(u)
    n = pos.shape[1]
    assert u.shape[1] == n
    d = np.zeros((3, n), dtype=np.float64)
    pdf = np.zeros(n, dtype=np.float64)
    lobe = np.zeros(n, dtype=np.int32)
    margin = np.zeros(n, dtype=np.float64)
    fo = None if forced is None else np.ascontiguousarray(forced, dtype=np.int32)
    lib().orc_query_sample(C.byref(c), _p(_f64(params)), n, _p(pos), _p(_f32(aux)), _p(u), n,
                           float(alpha), _p(fo), _p(d), _p(pdf), _p(lobe), _p(margin))
    return d, pdf, lobe, margin


def eval_pdf(w, params, pos, dirs, aux=None) -> np.ndarray:
    c = cfg_of(w)
    pos = _f32(pos)
    n = pos.shape[1]
    out = np.zeros(n, dtype=np.float64)
    lib().orc_eval_pdf(C.byref(c), _p(_f64(params)), n, _p(pos), _p(_f32(aux)), _p(_f32(dirs)),
                       n, _p(out))
    return out


def eval_pdf64(w, params, pos, dirs, aux=None) -> np.ndarray:
    """Mixture density at FP64 directions."""
    c = cfg_of(w)
    pos = _f32(pos)
    n = pos.shape[1]
    out = np.zeros(n, dtype=np.float64)
    lib().orc_eval_pdf64(C.byref(c), _p(_f64(params)), n, _p(pos), _p(_f32(aux)), _p(_f64(dirs)),
                         n, _p(out))
    return out


def grid_indices(w, pos) -> np.ndarray:
    c = cfg_of(w)
    pos = _f32(pos)
    n = pos.shape[1]
    out = np.zeros((len(w.level_res), 8, n), dtype=np.int32)
    lib().orc_grid_indices(C.byref(c), n, _p(pos), n, _p(out))
    return out


def train_grad(w, params, pos, dirs, radiance, pdf, aux=None):
    """(loss, grad[n_params] float64)."""
    c = cfg_of(w)
    pos = _f32(pos)
    n = pos.shape[1]
    g = np.zeros(n_params(w), dtype=np.float64)
    loss = lib().orc_train_grad(C.byref(c), _p(_f64(params)), n, _p(pos), _p(_f32(aux)),
                                _p(_f32(dirs)), _p(_f32(radiance)), _p(_f32(pdf)), n, _p(g))
    return float(loss), g


def train_loss(w, params, pos, dirs, radiance, pdf, aux=None) -> float:
    c = cfg_of(w)
    pos = _f32(pos)
    n = pos.shape[1]
    return float(lib().orc_train_loss(C.byref(c), _p(_f64(params)), n, _p(pos), _p(_f32(aux)),
                                      _p(_f32(dirs)), _p(_f32(radiance)), _p(_f32(pdf)), n))


def adam(p, g, m, v, t: int, lr: float, b1: float, b2: float, eps: float):
    """In place on float64 arrays p, m, v."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(p.size, _p(p), _p(g), _p(m), _p(v), int(t), lr, b1, b2, eps)


def ema(e, p, decay: float):
    """In place on float64 array e: e <- decay e + (1 - decay) p (Sec. 5.3)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert e.dtype == np.float64 and e.flags.c_contiguous and e.size == p.size
    lib().orc_ema(e.size, _p(e), _p(p), float(decay))


def num_threads() -> int:
    return int(lib().orc_num_threads())
