"""Shared helpers of the GPU parity tests: device upload, model creation and
comparison of sampled directions / densities against the oracle."""
import numpy as np

import oracle
import synth

# FP32 path tolerances: relative density and direction error (radians).
PDF_RTOL_FP32 = 1e-4
DIR_TOL_FP32 = 1e-4
# Lobe-choice boundary margin: when u0 is this close to a cumulative weight,
# FP32 and FP64 may legitimately pick neighbouring lobes.
MARGIN_FP32 = 1e-5


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def make_model(w, params, max_batch, precision=None):
    import paper_2504_04315_gb300 as npm
    m = npm.NPM(npm.config_from(w, max_batch=max_batch, precision=precision))
    m.set_params(params)
    return m


def rel_err(got, ref, floor=1e-30):
    return np.abs(got - ref) / np.maximum(np.abs(ref), floor)


def compare_samples(w, params, pos, u, aux, alpha, gd, gp, pdf_rtol, dir_tol, margin,
                    pdf_floor=1e-30, max_near_frac=1e-3):
    """Compare GPU samples (gd [3][n], gp [n]) with the oracle on the same
    inputs. Where u0 sits within `margin` of a lobe boundary, the GPU result
    may match the oracle conditioned on another lobe; such cases are
    counted, must be rare, and must match the oracle for some lobe."""
    od, op, _, omargin = oracle.query_sample(w, params, pos, u, aux, alpha)
    dir_err = np.linalg.norm(gd - od, axis=0)
    pdf_err = np.abs(gp - op) / np.maximum(op, pdf_floor)
    bad = (dir_err > dir_tol) | (pdf_err > pdf_rtol) | ~np.isfinite(gp)
    near = omargin < margin
    idx = np.where(bad & near)[0]
    if idx.size:
        ok = np.zeros(idx.size, dtype=bool)
        sub_aux = None if aux is None else aux[:, idx]
        for k in range(w.K):
            fd, fp, _, _ = oracle.query_sample(w, params, pos[:, idx], u[:, idx], sub_aux, alpha,
                                               forced=np.full(idx.size, k, dtype=np.int32))
            ok |= ((np.linalg.norm(gd[:, idx] - fd, axis=0) <= dir_tol)
                   & (np.abs(gp[idx] - fp) / np.maximum(fp, pdf_floor) <= pdf_rtol))
        bad[idx[ok]] = False
    n_bad = int(bad.sum())
    assert near.mean() <= max_near_frac, f"near-boundary fraction {near.mean():.2e}"
    assert n_bad == 0, (
        f"{n_bad} mismatches; worst dir {dir_err[bad].max() if n_bad else 0:.3e} "
        f"worst pdf {pdf_err[bad].max() if n_bad else 0:.3e} at {np.where(bad)[0][:10]}")
    return dict(max_dir=float(dir_err[~near].max(initial=0.0)),
                max_pdf=float(pdf_err[~near].max(initial=0.0)),
                near=int(near.sum()))


PRODUCT_SMALL = synth.Workload(
    name="product mode, 4 levels (2 dense, 2 hashed in 2^12), MLP 32-32-32-32, K=8",
    mode=synth.PRODUCT, level_res=[8, 12, 20, 32], feat=2, log2_table=12,
    widths=[32, 32, 32, 32], K=8, n_query=4096, n_train=4096)
