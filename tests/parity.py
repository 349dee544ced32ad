"""Shared helpers of the GPU parity tests: seeded inputs, oracle references and
the scale-aware tolerances.

Tolerances (FP32 evaluation and accumulation against the FP64 oracle):
  value:                 |gpu - oracle| <= 1e-5 * max(|oracle|, S)
  spatial gradient:      |gpu - oracle| <= 1e-5 * max(|oracle|, G)
  coefficient gradient:  |gpu - oracle| <= 1e-4 * max(|oracle|, A)
where S = sum_i w_i sum_k |theta_k phi_k| (the magnitude of the terms the
FP32 sum cancels), G is the same magnitude for d f / d x_a,
sum_i |d w_i / d x_a| sum_k |theta_k phi_k| + w_i sum_k |theta_k d phi_k / d x_a|,
and A = the sum of |contribution| into that coefficient.
"""
import numpy as np
import torch

import oracle
import workloads as W

VAL_RTOL = 1e-5
GRAD_RTOL = 1e-4


def edge_points(dim: int, res: int) -> np.ndarray:
    """Domain corners, vertex and face coordinates, out-of-domain and NaN coordinates."""
    h = 1.0 / (res - 1)
    r = np.random.default_rng(123)
    pts = [np.zeros(dim), np.ones(dim), np.full(dim, 0.5), np.full(dim, -0.25), np.full(dim, 1.75)]
    for j in [0, 1, res // 2, res - 2, res - 1]:
        p = r.random(dim)
        p[0] = j * h
        pts.append(p)
        q = r.random(dim)
        q[:] = j * h
        pts.append(q)
    nanp = r.random(dim); nanp[dim - 1] = np.nan
    pts.append(nanp)
    return np.asarray(pts, np.float32)


def points(dim: int, res: int, n: int, seed: int = 1) -> np.ndarray:
    p = W.uniform_points(seed, n, dim)
    return np.concatenate([edge_points(dim, res), p]).astype(np.float32)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def check_forward(gpu_out, gpu_gx, dim, res, order, C, coefs64, pts):
    ref, ref_gx, _, _ = oracle.query(dim, res, order, C, coefs64, pts)
    S = oracle.query_absscale(dim, res, order, C, coefs64, pts)
    tol = VAL_RTOL * np.maximum(np.abs(ref), S)
    err = np.abs(gpu_out.reshape(ref.shape) - ref)
    bad = err > tol
    assert not bad.any(), f"value mismatch at {np.argwhere(bad)[:5].tolist()}: max err {err.max()}"
    if gpu_gx is not None:
        G = oracle.query_gradscale(dim, res, order, C, coefs64, pts)
        tolg = VAL_RTOL * np.maximum(np.abs(ref_gx), G)
        errg = np.abs(gpu_gx.reshape(ref_gx.shape) - ref_gx)
        badg = errg > tolg
        assert not badg.any(), f"grad_x mismatch at {np.argwhere(badg)[:5].tolist()}: max err {errg.max()}"
    return ref


def check_coef_grad(gpu_grad, dim, res, order, C, pts, dLdf, dLdg=None):
    ref, A = oracle.query_backward(dim, res, order, C, pts, dLdf.astype(np.float64),
                                   None if dLdg is None else dLdg.astype(np.float64), want_abs=True)
    tol = GRAD_RTOL * np.maximum(np.abs(ref), A) + 1e-30
    err = np.abs(gpu_grad - ref)
    bad = err > tol
    assert not bad.any(), f"coef grad mismatch at {np.argwhere(bad)[:5].ravel().tolist()}: max err {err.max()}"
    return ref
