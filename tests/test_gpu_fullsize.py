"""Parity at the full size of the benchmark: a 256^3 order-2 grid (N(0,1)
coefficients, seed 0) and 2^24 uniform points, run exactly as the benchmark
step runs them (tg_batch_bin -> tg_query_binned -> tg_query_backward_binned,
outputs and upstream in input order, and again in binned order).

At 256^3 the batch has exactly 32768 bricks, the largest count the
shared-memory histogram binning takes, and the grid and the point records
are both larger than L2. The oracle checks sampled outputs one by one, and
the coefficient gradient of every vertex of a z-slab of the grid against
the oracle's backward over all points whose cells touch that slab.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from parity import GRAD_RTOL, check_forward, to_dev

pytestmark = pytest.mark.gpu

RES, ORDER, K = 256, 2, 10
N = 1 << 24


@pytest.fixture(scope="module")
def inputs():
    pts = W.uniform_points(1, N)
    up = W.normal(4, W.STREAM_UPSTREAM, np.arange(N, dtype=np.uint64)).astype(np.float32).reshape(-1, 1)
    return pts, up


def cells_z(pts):
    """Cell z index by the FP32 index rule of Eq. 2 (clamp, one FP32 multiply, floor, clamp to res - 2)."""
    u = np.clip(pts[:, 2], np.float32(0), np.float32(1)) * np.float32(RES - 1)
    return np.minimum(np.floor(u).astype(np.int64), RES - 2)


def check_slab_gradient(grad_gpu, pts, up, z0, z1):
    """Gradient of the vertices with z in [z0 + 1, z1 - 1]: every contribution comes from a point in a cell with
    z in [z0, z1 - 1], so the oracle's backward over those points alone gives their exact value."""
    cz = cells_z(pts)
    sel = (cz >= z0) & (cz < z1)
    ref, A = oracle.query_backward(3, RES, ORDER, 1, pts[sel], up[sel].astype(np.float64), want_abs=True)
    lo, hi = (z0 + 1) * RES * RES * K, z1 * RES * RES * K
    ref, A, gpu = ref[lo:hi], A[lo:hi], grad_gpu[lo:hi].astype(np.float64)
    tol = GRAD_RTOL * np.maximum(np.abs(ref), A) + 1e-30
    err = np.abs(gpu - ref)
    bad = err > tol
    assert not bad.any(), f"{bad.sum()} gradient entries off, first {np.argwhere(bad)[:5].ravel().tolist()}"
    assert (A > 0).mean() > 0.99          # the slab's vertices all received contributions


@pytest.mark.parametrize("binned_order", [False, True])
def test_benchmark_step_matches_oracle_at_full_size(tg, inputs, binned_order):
    pts, up = inputs
    g = tg.tg_create(3, RES, ORDER, 1, "f32", seed=0, init_std=1.0)
    P, U = to_dev(pts), to_dev(up)
    batch = tg.tg_batch_create(3, RES, N)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_batch_bin(batch, P)
    idx = tg.tg_batch_order(batch).long()
    if binned_order:
        out = tg.tg_query_binned(g, batch, binned_order=True)
        tg.tg_query_backward_binned(g, batch, U[idx].contiguous(), grad, binned_order=True)
        out = torch.empty_like(out).index_copy_(0, idx, out)      # back to input order
    else:
        out = tg.tg_query_binned(g, batch)
        tg.tg_query_backward_binned(g, batch, U, grad)
    torch.cuda.synchronize()
    assert tg.tg_batch_timeouts(batch) == 0
    # the binning is a permutation, every brick's records are its own points
    assert torch.equal(torch.sort(idx).values, torch.arange(N, device="cuda"))
    coefs = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)
    sample = np.random.default_rng(0).choice(N, 1 << 20, replace=False)
    check_forward(out.cpu().numpy()[sample], None, 3, RES, ORDER, 1, coefs, pts[sample])
    check_slab_gradient(grad.cpu().numpy(), pts, up, 120, 136)


def test_spatial_gradient_and_bf16_storage_at_full_size(tg, inputs):
    """The forward with spatial gradients (what the SDF step asks for), FP32 and BF16 storage, on the same points."""
    pts, _ = inputs
    P = to_dev(pts)
    batch = tg.tg_batch_create(3, RES, N)
    tg.tg_batch_bin(batch, P)
    sample = np.random.default_rng(1).choice(N, 1 << 18, replace=False)
    for dtype in ("f32", "bf16"):
        g = tg.tg_create(3, RES, ORDER, 1, dtype, seed=0, init_std=1.0)
        out, gx = tg.tg_query_binned(g, batch, want_grad=True)
        torch.cuda.synchronize()
        assert tg.tg_batch_timeouts(batch) == 0
        stored = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)    # dequantised for BF16
        check_forward(out.cpu().numpy()[sample], gx.cpu().numpy()[sample], 3, RES, ORDER, 1, stored, pts[sample])
        del g


def test_fit_sized_batch_on_the_record_path(tg):
    """The SDF fit's batch on the full grid: 2^20 points (half uniform, half on the union's surface), 32 points
    per brick, so the binned forward with spatial gradients and the backward with value and spatial-gradient
    upstreams take one thread per record. Sampled outputs and a z-slab of the gradient against the oracle."""
    shape = W.union_shape(0)
    n = 1 << 20
    pts = W.sdf_points(shape, seed=1, step=0, n=n)
    r = np.random.default_rng(6)
    up = r.normal(size=(n, 1)).astype(np.float32)
    ug = r.normal(size=(n, 1, 3)).astype(np.float32)
    g = tg.tg_create(3, RES, ORDER, 1, "f32", seed=0, init_std=1.0)
    batch = tg.tg_batch_create(3, RES, n)
    tg.tg_batch_bin(batch, to_dev(pts))
    out, gx = tg.tg_query_binned(g, batch, want_grad=True)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward_binned(g, batch, to_dev(up), grad, dL_dgradx=to_dev(ug))
    torch.cuda.synchronize()
    coefs = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)
    sample = np.random.default_rng(2).choice(n, 1 << 16, replace=False)
    check_forward(out.cpu().numpy()[sample], gx.cpu().numpy()[sample], 3, RES, ORDER, 1, coefs, pts[sample])
    cz = cells_z(pts)
    z0, z1 = 120, 136
    sel = (cz >= z0) & (cz < z1)
    ref, A = oracle.query_backward(3, RES, ORDER, 1, pts[sel], up[sel].astype(np.float64),
                                   ug[sel].astype(np.float64), want_abs=True)
    lo, hi = (z0 + 1) * RES * RES * K, z1 * RES * RES * K
    err = np.abs(grad.cpu().numpy()[lo:hi].astype(np.float64) - ref[lo:hi])
    tol = GRAD_RTOL * np.maximum(np.abs(ref[lo:hi]), A[lo:hi]) + 1e-30
    assert (err <= tol).all(), f"{(err > tol).sum()} gradient entries off"
    assert (A[lo:hi] > 0).mean() > 0.1           # a few hundred thousand slab entries were reached
