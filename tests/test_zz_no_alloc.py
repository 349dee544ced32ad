"""tg_query_noalloc against the allocating entry points.

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
from parity import VAL_RTOL, edge_points, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_binned_query_on_two_calls(tg):
    res = 34
    g = tg.tg_create(3, res, 2, 1, "f32", seed=5, init_std=0.5)
    # two calls in a row: the second runs on the scratch the first one left behind
    for seed, n in [(11, 200000), (12, 3001)]:
        pts = np.concatenate([edge_points(3, res), W.uniform_points(seed, n)]).astype(np.float32)
        P = to_dev(pts)
        out, gx = tg.tg_query_noalloc(g, P, want_grad=True)
        batch = tg.tg_batch_create(3, res, pts.shape[0])
        tg.tg_batch_bin(batch, P)
        ref, ref_gx = tg.tg_query_binned(g, batch, want_grad=True)
        torch.cuda.synchronize()
        torch.testing.assert_close(out, ref, rtol=VAL_RTOL, atol=1e-6)
        torch.testing.assert_close(gx, ref_gx, rtol=VAL_RTOL, atol=1e-5)


def test_noalloc_rejects_sizes_over_its_limit(tg):
    g = tg.tg_create(3, 10, 2, 1, "f32")
    with pytest.raises(tg.TGError, match="fixed scratch limit"):
        tg.tg_query_noalloc(g, torch.rand(((1 << 18) + 1, 3), device="cuda"))
    big = tg.tg_create(3, 300, 0, 1, "f32")
    with pytest.raises(tg.TGError, match="bricks"):
        tg.tg_query_noalloc(big, torch.rand((16, 3), device="cuda"))


def test_noalloc_spatial_gradient_with_several_channels(tg):
    res = 20
    g = tg.tg_create(3, res, 1, 3, "f32", seed=6, init_std=0.5)
    P = to_dev(W.uniform_points(13, 50000))
    out, gx = tg.tg_query_noalloc(g, P, want_grad=True)
    ref, ref_gx = tg.tg_query(g, P, want_grad=True)
    torch.cuda.synchronize()
    torch.testing.assert_close(out, ref, rtol=VAL_RTOL, atol=1e-6)
    torch.testing.assert_close(gx, ref_gx, rtol=VAL_RTOL, atol=1e-5)
