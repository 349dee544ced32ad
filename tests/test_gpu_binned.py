"""GPU parity of the brick-binned path (TMA-staged forward, TMA reduce-add
backward) against the FP64 oracle and against the point-parallel path."""
import numpy as np
import pytest
import torch

import workloads as W
from parity import check_coef_grad, check_forward, points, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [  # res, order, C, dtype  (res - 1 not a multiple of 8: ragged last brick)
    (34, 2, 1, "f32"), (20, 1, 3, "f32"), (24, 0, 1, "f32"), (18, 2, 2, "f32"), (36, 2, 1, "bf16"),
    (28, 1, 1, "f16"), (10, 2, 1, "f32"),
    (300, 0, 1, "f32"),      # more than 32768 bricks: the global-atomic binning path
]


def clustered(n, seed=3):
    """Dense clusters: several hundred points inside single bricks."""
    r = np.random.default_rng(seed)
    c = r.random((4, 3)) * 0.8 + 0.1
    return np.concatenate([c[k] + 0.01 * r.standard_normal((n // 4, 3)) for k in range(4)]).astype(np.float32)


@pytest.fixture(params=["auto", "brick", "records"])
def binned_path(request, monkeypatch):
    """The binned passes take the brick kernels or, for batches with few points per brick, one thread per record;
    TG_BINNED_PATH forces either (read by the library at every call)."""
    if request.param != "auto":
        monkeypatch.setenv("TG_BINNED_PATH", request.param)
    return request.param


@pytest.mark.parametrize("res,order,C,dtype", SHAPES)
def test_binned_forward_backward_parity(tg, res, order, C, dtype, binned_path):
    coefs = W.init_coefs(3, res, order, C, seed=1, std=0.5)
    g = tg.tg_create(3, res, order, C, dtype)
    tg.tg_set_coefs(g, to_dev(coefs))
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)
    pts = np.concatenate([points(3, res, 20000, seed=2), clustered(2000)])
    N = pts.shape[0]
    P = to_dev(pts)
    batch = tg.tg_batch_create(3, res, N)
    tg.tg_batch_bin(batch, P)
    out, gx = tg.tg_query_binned(g, batch, want_grad=True)
    out_p, gx_p = tg.tg_query(g, P, want_grad=True)
    r = np.random.default_rng(4)
    dLdf = r.normal(size=(N, C)).astype(np.float32)
    dLdg = r.normal(size=(N, C, 3)).astype(np.float32)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward_binned(g, batch, to_dev(dLdf), grad, dL_dgradx=to_dev(dLdg))
    torch.cuda.synchronize()
    assert tg.tg_batch_timeouts(batch) == 0
    check_forward(out.cpu().numpy(), gx.cpu().numpy(), 3, res, order, C, stored, pts)
    torch.testing.assert_close(out, out_p, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(gx, gx_p, rtol=1e-5, atol=1e-5)
    check_coef_grad(grad.cpu().numpy(), 3, res, order, C, pts, dLdf, dLdg)


@pytest.mark.parametrize("C,order", [(1, 2), (3, 1)])
def test_binned_order_io(tg, C, order, binned_path):
    """TG_ORDER_BINNED outputs/upstreams equal the input-order ones through the batch permutation."""
    res = 26
    coefs = W.init_coefs(3, res, order, C, seed=2, std=0.4)
    g = tg.tg_create(3, res, order, C, "f32")
    tg.tg_set_coefs(g, to_dev(coefs))
    pts = np.concatenate([points(3, res, 30000, seed=9), clustered(1000)])
    N = pts.shape[0]
    batch = tg.tg_batch_create(3, res, N)
    tg.tg_batch_bin(batch, to_dev(pts))
    idx = tg.tg_batch_order(batch).long()
    assert torch.equal(torch.sort(idx).values, torch.arange(N, device="cuda"))
    torch.testing.assert_close(tg.tg_batch_points(batch), to_dev(pts)[idx], rtol=0, atol=0, equal_nan=True)
    out_i, gx_i = tg.tg_query_binned(g, batch, want_grad=True)
    out_b, gx_b = tg.tg_query_binned(g, batch, want_grad=True, binned_order=True)
    assert torch.equal(out_b, out_i[idx]) and torch.equal(gx_b, gx_i[idx])
    r = np.random.default_rng(5)
    uf = to_dev(r.normal(size=(N, C)).astype(np.float32))
    ug = to_dev(r.normal(size=(N, C, 3)).astype(np.float32))
    g_i = torch.zeros(g.n_coefs, device="cuda")
    g_b = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward_binned(g, batch, uf, g_i, dL_dgradx=ug)
    tg.tg_query_backward_binned(g, batch, uf[idx].contiguous(), g_b, dL_dgradx=ug[idx].contiguous(), binned_order=True)
    torch.cuda.synchronize()
    check_coef_grad(g_b.cpu().numpy(), 3, res, order, C, pts, uf.cpu().numpy(), ug.cpu().numpy())
    # bricks sharing a face add into the gradient in either order (L2 reduce-add): FP32 rounding only
    torch.testing.assert_close(g_b, g_i, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("width", [1, 3, 10])
def test_batch_gather_scatter(tg, width):
    """tg_batch_gather / tg_batch_scatter are the permutation of tg_batch_order, row by row, bit for bit."""
    res = 26
    pts = np.concatenate([points(3, res, 20001, seed=4), clustered(777)])
    N = pts.shape[0]
    batch = tg.tg_batch_create(3, res, N)
    tg.tg_batch_bin(batch, to_dev(pts))
    idx = tg.tg_batch_order(batch).long()
    src = torch.randn((N, width), device="cuda")
    binned = tg.tg_batch_gather(batch, src)
    assert torch.equal(binned, src[idx])
    back = tg.tg_batch_scatter(batch, binned)
    assert torch.equal(back, src)
    # the public permutation + TG_ORDER_BINNED reproduce TG_ORDER_INPUT
    g = tg.tg_create(3, res, 2, 1, "f32", seed=1, init_std=0.5)
    out_i = tg.tg_query_binned(g, batch)
    out_b = tg.tg_query_binned(g, batch, binned_order=True)
    assert torch.equal(tg.tg_batch_scatter(batch, out_b), out_i)
    with pytest.raises(tg.TGError):
        tg.tg_batch_gather(batch, src, dst=src)


def test_binned_value_only_backward_and_rebin(tg):
    res, order, C = 26, 2, 1
    g = tg.tg_create(3, res, order, C, "f32", seed=3, init_std=0.3)
    coefs = tg.tg_get_coefs(g, which=1).cpu().numpy()
    batch = tg.tg_batch_create(3, res, 50000)
    for seed, n in [(5, 50000), (6, 777), (7, 1)]:
        pts = W.uniform_points(seed, n)
        tg.tg_batch_bin(batch, to_dev(pts))
        out = tg.tg_query_binned(g, batch)
        dLdf = np.random.default_rng(seed).normal(size=(n, 1)).astype(np.float32)
        grad = torch.zeros(g.n_coefs, device="cuda")
        tg.tg_query_backward_binned(g, batch, to_dev(dLdf), grad)
        torch.cuda.synchronize()
        check_forward(out.cpu().numpy(), None, 3, res, order, C, coefs.astype(np.float64), pts)
        check_coef_grad(grad.cpu().numpy(), 3, res, order, C, pts, dLdf)


def test_binned_empty_batch(tg):
    g = tg.tg_create(3, 10, 2, 1, "f32", init_std=0.1)
    batch = tg.tg_batch_create(3, 10, 16)
    tg.tg_batch_bin(batch, torch.empty((0, 3), device="cuda"))
    out = tg.tg_query_binned(g, batch)
    assert out.shape == (0, 1)


def test_binned_rows_tma_cannot_move(tg):
    """11 x 40-byte rows are not whole 16-byte units, so no brick tile can be moved by TMA: the binned passes take
    the per-record path (equal to the point-parallel query), and the deterministic backward, which needs the
    brick kernels, is refused."""
    g = tg.tg_create(3, 11, 2, 1, "f32", seed=3, init_std=0.5)
    P = torch.rand((5000, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
    batch = tg.tg_batch_create(3, 11, 5000)
    tg.tg_batch_bin(batch, P)
    out, gx = tg.tg_query_binned(g, batch, want_grad=True)
    out_p, gx_p = tg.tg_query(g, P, want_grad=True)
    assert torch.equal(out, out_p) and torch.equal(gx, gx_p)
    U = torch.randn((5000, 1), device="cuda")
    grad_b = torch.zeros(g.n_coefs, device="cuda")
    grad_p = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward_binned(g, batch, U, grad_b)
    tg.tg_query_backward(g, P, U, grad_p)
    torch.testing.assert_close(grad_b, grad_p, rtol=1e-4, atol=1e-5)
    with pytest.raises(tg.TGError):
        tg.tg_query_backward_binned(g, batch, U, grad_b, deterministic=True)


def test_binned_rejects_unsupported(tg):
    batch = tg.tg_batch_create(3, 11, 16)
    tg.tg_batch_bin(batch, torch.rand((16, 3), device="cuda"))
    with pytest.raises(tg.TGError):
        tg.tg_batch_create(2, 10, 16)
    with pytest.raises(tg.TGError):
        tg.tg_batch_bin(batch, torch.rand((17, 3), device="cuda"))


@pytest.mark.parametrize("with_g,res,N,clustered", [
    (False, 40, 60000, False),                # about 480 points per brick: every brick fits one round
    (True, 40, 60000, False),
    (False, 10, 60000, False),                # 8 bricks of about 7500 points: rounds taken by input index
    (True, 26, 50000, True),                  # half the points in one corner: single- and multi-round bricks
])
def test_deterministic_backward_is_bitwise_reproducible(tg, with_g, res, N, clustered):
    """TG_DETERMINISTIC: the same gradient bit for bit from three independent binnings (whose binned order
    differs from run to run), and the oracle's within tolerance."""
    g = tg.tg_create(3, res, 2, 1, "f32", seed=2, init_std=0.5)
    pts = W.uniform_points(51, N)
    if clustered:
        pts[: N // 2] *= 0.15
    P = to_dev(pts)
    r = np.random.default_rng(52)
    up = r.normal(size=(N, 1)).astype(np.float32)
    ug = r.normal(size=(N, 1, 3)).astype(np.float32) if with_g else None
    grads = []
    for _ in range(3):
        batch = tg.tg_batch_create(3, res, N)
        tg.tg_batch_bin(batch, P)
        grad = torch.zeros(g.n_coefs, device="cuda")
        tg.tg_query_backward_binned(g, batch, to_dev(up), grad, dL_dgradx=None if ug is None else to_dev(ug),
                                    deterministic=True)
        grads.append(grad)
    torch.cuda.synchronize()
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])
    check_coef_grad(grads[0].cpu().numpy(), 3, res, 2, 1, pts, up, ug)
