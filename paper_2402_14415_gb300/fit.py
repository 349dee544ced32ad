"""SDF fitting driver (Sec. 3.2) over the C ABI: sample -> step -> Adam.

Orchestration only: every step of the fit (sampling, binning, forward, loss,
backward, Adam) runs in the library's kernels on one CUDA stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import binding as tg


@dataclass
class FitResult:
    steps: int
    final_error: float                 # mean |f - d| on the evaluation points
    losses: list = field(default_factory=list)   # (step, mean L1, mean eikonal) every `log_every` steps
    errors: list = field(default_factory=list)   # (step, mean |SDF error|) at every evaluation


def fit_sdf(grid: tg.Grid, shape: tg.DeviceShape, steps: int, n_points: int, lr: float, lambda_eik: float = 0.0,
            seed: int = 1, eval_pts: torch.Tensor | None = None, eval_every: int = 0, tol: float = 0.0,
            points_fn=None, log_every: int = 0, k_weight: float = 0.0, lambda_tv: float = 0.0,
            stream=None) -> FitResult:
    """Runs up to `steps` Adam steps of the SDF loss (Eq. 8 of Sec. 3.2: the reconstruction term of Eq. 6 with
    Eq. 7's weight when k_weight > 0, lambda_eik times the eikonal term, lambda_tv times the TV term).

    points_fn(step) -> (n, 3) device tensor overrides the device sampler (used
    to feed both the library and the oracle the same batches). With tol > 0
    the fit stops at the first evaluation whose mean |SDF error| is below tol.
    """
    batch = tg.Batch(3, grid.res, n_points)
    grad = torch.zeros(grid.n_coefs, device="cuda", dtype=torch.float32)
    loss = torch.zeros(2, device="cuda", dtype=torch.float32)
    err = torch.zeros(1, device="cuda", dtype=torch.float32)
    res = FitResult(steps=0, final_error=float("nan"))
    for k in range(steps):
        pts = points_fn(k) if points_fn is not None else None
        if log_every and k % log_every == 0:
            loss.zero_()
        tg.tg_sdf_step(grid, batch, shape, grad, loss, pts=pts, n=n_points, seed=seed, step=k,
                       lambda_eik=lambda_eik, k_weight=k_weight, stream=stream)
        if lambda_tv > 0:
            tg.tg_tv_step(grid, lambda_tv, grad, stream=stream)
        tg.tg_adam_step(grid, grad, lr=lr, step=k + 1, stream=stream)
        res.steps = k + 1
        if log_every and k % log_every == 0:
            l = loss.tolist()
            res.losses.append((k, l[0] / n_points, l[1] / n_points))
        if eval_pts is not None and eval_every and (k + 1) % eval_every == 0:
            err.zero_()
            tg.tg_sdf_error(grid, shape, eval_pts, err, stream=stream)
            e = err.item() / eval_pts.shape[0]
            res.errors.append((k + 1, e))
            if tol > 0 and e < tol:
                break
    if eval_pts is not None:
        err.zero_()
        tg.tg_sdf_error(grid, shape, eval_pts, err, stream=stream)
        res.final_error = err.item() / eval_pts.shape[0]
    batch.close()
    return res
