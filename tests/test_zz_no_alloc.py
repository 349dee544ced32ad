"""tg_query_noalloc against the allocating entry points and the oracle.

Some callers cannot call cudaMalloc: code embedded in a host framework that
owns every device allocation, or a latency-critical serving path that must
never reach the allocator. tg_query_noalloc serves them from one fixed
scratch array compiled into the library. This file runs last so that a
failure here does not hide the rest of the suite; it must also pass alone.
"""
import numpy as np
import pytest
import torch

import workloads as W
from parity import VAL_RTOL, check_forward, edge_points, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_binned_query_on_two_calls(tg):
    res = 34
    g = tg.tg_create(3, res, 2, 1, "f32", seed=5, init_std=0.5)
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)
    # two calls in a row: the second runs on the scratch the first one left behind
    for seed, n in [(11, 200000), (12, 3001)]:
        pts = np.concatenate([edge_points(3, res), W.uniform_points(seed, n)]).astype(np.float32)
        P = to_dev(pts)
        out, gx = tg.tg_query_noalloc(g, P, want_grad=True)
        batch = tg.tg_batch_create(3, res, pts.shape[0])
        tg.tg_batch_bin(batch, P)
        ref, ref_gx = tg.tg_query_binned(g, batch, want_grad=True)
        torch.cuda.synchronize()
        assert tg.tg_noalloc_timeouts() == 0
        torch.testing.assert_close(out, ref, rtol=VAL_RTOL, atol=1e-6)
        torch.testing.assert_close(gx, ref_gx, rtol=VAL_RTOL, atol=1e-5)
        check_forward(out.cpu().numpy(), gx.cpu().numpy(), 3, res, 2, 1, stored, pts)


def test_noalloc_rejects_sizes_over_its_limit(tg):
    g = tg.tg_create(3, 10, 2, 1, "f32")
    with pytest.raises(tg.TGError, match="fixed scratch limit"):
        tg.tg_query_noalloc(g, torch.rand(((1 << 18) + 1, 3), device="cuda"))
    big = tg.tg_create(3, 300, 0, 1, "f32")
    with pytest.raises(tg.TGError, match="bricks"):
        tg.tg_query_noalloc(big, torch.rand((16, 3), device="cuda"))


def test_noalloc_at_its_maximum_sizes(tg):
    """res 257 (32768 bricks: the brick counters and offsets are full, the scan writes offsets[32768]) and
    exactly 2^18 points (the record and permutation arrays are full), against tg_query_binned and the oracle."""
    res, n = 257, 1 << 18
    g = tg.tg_create(3, res, 1, 1, "f32", seed=7, init_std=0.5)      # 257 * 4 coefficients * 4 B: TMA rows align
    pts = W.uniform_points(14, n)
    e = edge_points(3, res)
    pts[:e.shape[0]] = e
    P = to_dev(pts)
    for _ in range(2):
        out, gx = tg.tg_query_noalloc(g, P, want_grad=True)
    batch = tg.tg_batch_create(3, res, n)
    tg.tg_batch_bin(batch, P)
    ref, ref_gx = tg.tg_query_binned(g, batch, want_grad=True)
    torch.cuda.synchronize()
    assert tg.tg_noalloc_timeouts() == 0
    torch.testing.assert_close(out, ref, rtol=VAL_RTOL, atol=1e-6)
    torch.testing.assert_close(gx, ref_gx, rtol=VAL_RTOL, atol=1e-5)
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)
    sub = np.r_[0:e.shape[0], np.random.default_rng(3).choice(n, 20000, replace=False)]
    check_forward(out.cpu().numpy()[sub], gx.cpu().numpy()[sub], 3, res, 1, 1, stored, pts[sub])


def test_noalloc_bf16_storage(tg):
    res = 36                                # 36 * 10 coefficients * 2 B: TMA rows align
    g = tg.tg_create(3, res, 2, 1, "bf16", seed=8, init_std=0.5)
    pts = np.concatenate([edge_points(3, res), W.uniform_points(15, 100000)]).astype(np.float32)
    P = to_dev(pts)
    out, gx = tg.tg_query_noalloc(g, P, want_grad=True)
    batch = tg.tg_batch_create(3, res, pts.shape[0])
    tg.tg_batch_bin(batch, P)
    ref, ref_gx = tg.tg_query_binned(g, batch, want_grad=True)
    torch.cuda.synchronize()
    assert tg.tg_noalloc_timeouts() == 0
    torch.testing.assert_close(out, ref, rtol=VAL_RTOL, atol=1e-6)
    torch.testing.assert_close(gx, ref_gx, rtol=VAL_RTOL, atol=1e-5)
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)     # the dequantised BF16 values
    check_forward(out.cpu().numpy(), gx.cpu().numpy(), 3, res, 2, 1, stored, pts)


def test_noalloc_spatial_gradient_with_several_channels(tg):
    res = 20
    g = tg.tg_create(3, res, 1, 3, "f32", seed=6, init_std=0.5)
    P = to_dev(W.uniform_points(13, 50000))
    out, gx = tg.tg_query_noalloc(g, P, want_grad=True)
    ref, ref_gx = tg.tg_query(g, P, want_grad=True)
    torch.cuda.synchronize()
    assert tg.tg_noalloc_timeouts() == 0
    torch.testing.assert_close(out, ref, rtol=VAL_RTOL, atol=1e-6)
    torch.testing.assert_close(gx, ref_gx, rtol=VAL_RTOL, atol=1e-5)
