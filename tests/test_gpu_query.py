"""GPU parity of the query path (Eq. 2 - Eq. 4), its coefficient gradient and
Adam against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from parity import check_coef_grad, check_forward, points, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [  # dim, res, order, C
    (3, 5, 0, 1), (3, 9, 1, 1), (3, 12, 2, 1), (3, 7, 2, 3), (3, 6, 1, 3), (3, 6, 2, 2), (3, 5, 0, 4),
    (2, 11, 2, 1), (2, 9, 1, 2), (2, 6, 0, 3),
]


def make_grid(tg, dim, res, order, C, dtype="f32", std=0.5, seed=0):
    coefs = W.init_coefs(dim, res, order, C, seed=seed, std=std)
    g = tg.tg_create(dim, res, order, C, dtype)
    tg.tg_set_coefs(g, to_dev(coefs))
    return g, coefs


@pytest.mark.parametrize("dim,res", [(3, 7), (3, 256), (2, 33), (3, 2)])
def test_locate_bit_exact(tg, dim, res):
    pts = points(dim, res, 20000, seed=5)
    cells, t = tg.tg_locate(dim, res, to_dev(pts))
    rc, rt = oracle.locate(dim, res, pts)
    assert np.array_equal(cells.cpu().numpy(), rc)
    assert np.array_equal(t.cpu().numpy().astype(np.float64), rt)


@pytest.mark.parametrize("dim,res,order,C", SHAPES)
def test_forward_parity(tg, dim, res, order, C):
    g, coefs = make_grid(tg, dim, res, order, C)
    pts = points(dim, res, 3000)
    out, gx = tg.tg_query(g, to_dev(pts), want_grad=True)
    torch.cuda.synchronize()
    check_forward(out.cpu().numpy(), gx.cpu().numpy(), dim, res, order, C, coefs.astype(np.float64), pts)


@pytest.mark.parametrize("dim,res,order,C", SHAPES)
def test_backward_parity(tg, dim, res, order, C):
    g, coefs = make_grid(tg, dim, res, order, C)
    pts = points(dim, res, 3000)
    N = pts.shape[0]
    r = np.random.default_rng(7)
    dLdf = r.normal(size=(N, C)).astype(np.float32)
    dLdg = r.normal(size=(N, C, dim)).astype(np.float32)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, to_dev(pts), to_dev(dLdf), grad)
    torch.cuda.synchronize()
    check_coef_grad(grad.cpu().numpy(), dim, res, order, C, pts, dLdf)
    grad.zero_()
    tg.tg_query_backward(g, to_dev(pts), to_dev(dLdf), grad, dL_dgradx=to_dev(dLdg))
    torch.cuda.synchronize()
    check_coef_grad(grad.cpu().numpy(), dim, res, order, C, pts, dLdf, dLdg)


def test_backward_sorted_points_warp_aggregation(tg):
    """Many points per cell in warp order exercises the match/shuffle combine."""
    dim, res, order, C = 3, 6, 2, 1
    g, _ = make_grid(tg, dim, res, order, C)
    pts = W.uniform_points(9, 8192)
    cells, _ = oracle.locate(dim, res, pts)
    key = cells[:, 0] + res * (cells[:, 1] + res * cells[:, 2])
    pts = pts[np.argsort(key, kind="stable")]
    r = np.random.default_rng(8)
    dLdf = r.normal(size=(pts.shape[0], 1)).astype(np.float32)
    dLdg = r.normal(size=(pts.shape[0], 1, 3)).astype(np.float32)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, to_dev(pts), to_dev(dLdf), grad, dL_dgradx=to_dev(dLdg))
    torch.cuda.synchronize()
    check_coef_grad(grad.cpu().numpy(), dim, res, order, C, pts, dLdf, dLdg)


def test_backward_accumulates(tg):
    dim, res, order, C = 3, 5, 2, 1
    g, _ = make_grid(tg, dim, res, order, C)
    pts = points(dim, res, 500)
    dLdf = np.ones((pts.shape[0], 1), np.float32)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, to_dev(pts), to_dev(dLdf), grad)
    once = grad.clone()
    tg.tg_query_backward(g, to_dev(pts), to_dev(dLdf), grad)
    torch.testing.assert_close(grad, 2 * once, rtol=1e-5, atol=1e-6)


def test_empty_and_single_point(tg):
    g, coefs = make_grid(tg, 3, 4, 2, 1)
    empty = torch.empty((0, 3), device="cuda")
    out = tg.tg_query(g, empty)
    assert out.shape == (0, 1)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, empty, torch.empty((0, 1), device="cuda"), grad)
    assert not grad.any()
    p = np.array([[0.3, 0.6, 0.9]], np.float32)
    out = tg.tg_query(g, to_dev(p))
    torch.cuda.synchronize()
    check_forward(out.cpu().numpy(), None, 3, 4, 2, 1, coefs.astype(np.float64), p)


def test_invalid_arguments_raise(tg):
    with pytest.raises(tg.TGError):
        tg.tg_create(3, 1, 2, 1)
    with pytest.raises(tg.TGError):
        tg.tg_create(3, 8, 5, 1)
    g, _ = make_grid(tg, 3, 4, 1, 1)
    with pytest.raises(ValueError):
        tg.tg_query(g, torch.zeros((4, 3)))            # host tensor: no CPU path


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_low_precision_storage(tg, dtype, order):
    """(i) against the oracle on the dequantised coefficients: FP32-level error;
    (ii) against the oracle on the FP32 master: within 1e-2 relative."""
    dim, res, C = 3, 10, 1
    g, coefs = make_grid(tg, dim, res, order, C, dtype=dtype)
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy().astype(np.float64)
    master = tg.tg_get_coefs(g, which=1).cpu().numpy()
    assert np.array_equal(master, coefs)
    pts = points(dim, res, 3000)
    out, gx = tg.tg_query(g, to_dev(pts), want_grad=True)
    torch.cuda.synchronize()
    check_forward(out.cpu().numpy(), gx.cpu().numpy(), dim, res, order, C, stored, pts)
    ref, _, _, _ = oracle.query(dim, res, order, C, coefs.astype(np.float64), pts, want_grad=False)
    S = oracle.query_absscale(dim, res, order, C, coefs.astype(np.float64), pts)
    assert (np.abs(out.cpu().numpy() - ref) <= 1e-2 * np.maximum(np.abs(ref), S)).all()


# the hyper-parameters as the kernel receives them (tg_adam holds FP32 lr, betas and eps)
F32_ADAM = tuple(float(np.float32(x)) for x in (1e-2, 0.9, 0.999, 1e-8))


def moments_close(tg, g, m, v, scale_m, scale_v, dtype, where):
    """GPU moments against the oracle's. FP32: within a few rounding units of the magnitude of all the terms the
    moment has summed so far (S_t = beta1 S_{t-1} + (1 - beta1) |g_t|; the terms of v are non-negative), since
    beta1 m and (1 - beta1) g may cancel and the error of a step is carried into the next. BF16 (BF16 / FP16 storage): equal but for the rare entries where FP32 arithmetic and the oracle's
    exact arithmetic fall on two sides of a rounding boundary, which differ by one BF16 unit. Returns the
    entries that differed."""
    gm = tg.tg_get_coefs(g, which=2).cpu().numpy().astype(np.float64)
    gv = tg.tg_get_coefs(g, which=3).cpu().numpy().astype(np.float64)
    if dtype == "f32":
        assert (np.abs(gm - m) <= 1e-6 * scale_m + 1e-38).all(), where
        assert (np.abs(gv - v) <= 1e-6 * scale_v + 1e-38).all(), where
        return np.zeros(m.shape, bool)
    off = (gm != m) | (gv != v)
    assert off.mean() < 0.01, (where, off.mean())
    assert (np.abs(gm - m) <= 2.0 ** -7 * np.abs(m) + 1e-38).all(), where
    assert (np.abs(gv - v) <= 2.0 ** -7 * np.abs(v) + 1e-38).all(), where
    return off


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_adam_parity(tg, dtype):
    """Five fused Adam steps against the oracle's (moments rounded to BF16 for BF16 / FP16 storage)."""
    dim, res, order, C = 3, 8, 2, 1
    g, coefs = make_grid(tg, dim, res, order, C, dtype=dtype)
    n = g.n_coefs
    lp = dtype != "f32"
    p = coefs.astype(np.float64).copy(); m = np.zeros(n); v = np.zeros(n)
    r = np.random.default_rng(11)
    grad = torch.zeros(n, device="cuda")
    drift = np.zeros(n, bool)
    sm, sv = np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        gnp = r.normal(size=n).astype(np.float32) * (10.0 ** r.uniform(-3, 1, size=n)).astype(np.float32)
        grad.copy_(to_dev(gnp))
        tg.tg_adam_step(g, grad, lr=1e-2, step=step)
        gg = gnp.astype(np.float64)
        sm = F32_ADAM[1] * sm + (1 - F32_ADAM[1]) * np.abs(gg)
        sv = F32_ADAM[2] * sv + (1 - F32_ADAM[2]) * gg ** 2
        oracle.adam(p, gg, m, v, *F32_ADAM, step, bf16_moments=lp)
        torch.cuda.synchronize()
        assert not grad.any()
        drift |= moments_close(tg, g, m, v, sm, sv, dtype, f"step {step}")
        got = tg.tg_get_coefs(g, which=1).cpu().numpy()
        tol = 2e-6 * step * 1e-2 * 10 + 1e-6 * np.abs(p).max()
        np.testing.assert_allclose(got[~drift], p[~drift], rtol=0, atol=tol)
        # a moment one BF16 unit off moves that step by at most 2^-7 of the learning rate
        np.testing.assert_allclose(got[drift], p[drift], rtol=0, atol=tol + step * 1e-2 * 2.0 ** -6)
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy()
    master = tg.tg_get_coefs(g, which=1).cpu()
    want = master.to(torch.bfloat16 if dtype == "bf16" else torch.float16 if dtype == "f16" else torch.float32)
    assert np.array_equal(stored, want.float().numpy())


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_lazy_adam_parity(tg, dtype):
    """tg_adam_step_lazy against the oracle's lazy Adam on gradients that leave whole vertices (groups of 4
    coefficients and more) and single coefficients at 0; untouched entries keep their bits."""
    dim, res, order, C = 3, 7, 2, 1                    # 3430 coefficients: a scalar tail after the float4 groups
    g, coefs = make_grid(tg, dim, res, order, C, dtype=dtype)
    n = g.n_coefs
    p = coefs.astype(np.float64).copy(); m = np.zeros(n); v = np.zeros(n)
    r = np.random.default_rng(12)
    grad = torch.zeros(n, device="cuda")
    drift = np.zeros(n, bool)
    sm, sv = np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        gnp = r.normal(size=n).astype(np.float32)
        gnp *= np.repeat(r.random(n // 10 + 1) < 0.5, 10)[:n]          # whole vertices untouched
        gnp[r.random(n) < 0.05] = 0.0                                   # and single coefficients
        before = tg.tg_get_coefs(g, which=1).cpu().numpy()
        grad.copy_(to_dev(gnp))
        tg.tg_adam_step_lazy(g, grad, lr=1e-2, step=step)
        gg = gnp.astype(np.float64)
        t = gg != 0                                    # lazy: untouched entries keep their moments
        sm = np.where(t, F32_ADAM[1] * sm + (1 - F32_ADAM[1]) * np.abs(gg), sm)
        sv = np.where(t, F32_ADAM[2] * sv + (1 - F32_ADAM[2]) * gg ** 2, sv)
        oracle.adam_lazy(p, gg, m, v, *F32_ADAM, step, bf16_moments=dtype != "f32")
        torch.cuda.synchronize()
        assert not grad.any()
        drift |= moments_close(tg, g, m, v, sm, sv, dtype, f"step {step}")
        got = tg.tg_get_coefs(g, which=1).cpu().numpy()
        z = gnp == 0
        assert np.array_equal(got[z], before[z])
        tol = 2e-6 * step * 1e-2 * 10 + 1e-6 * np.abs(p).max()
        np.testing.assert_allclose(got[~drift], p[~drift], rtol=0, atol=tol)
        np.testing.assert_allclose(got[drift], p[drift], rtol=0, atol=tol + step * 1e-2 * 2.0 ** -6)
    stored = tg.tg_get_coefs(g, which=0).cpu().numpy()
    master = tg.tg_get_coefs(g, which=1).cpu()
    want = master.to(torch.bfloat16 if dtype == "bf16" else torch.float32)
    assert np.array_equal(stored, want.float().numpy())


def test_init_matches_generator(tg):
    g = tg.tg_create(3, 6, 2, 1, "f32", seed=42, init_std=0.01)
    got = tg.tg_get_coefs(g, which=1).cpu().numpy()
    want = W.init_coefs(3, 6, 2, 1, seed=42, std=0.01)
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-9)


@pytest.mark.parametrize("order,C", [(2, 1), (1, 3)])
def test_large_batches_take_the_binned_path(tg, order, C):
    """N >= 2^18 on a 3-D grid: tg_query / tg_query_backward bin into the grid's own batch; the
    results match the oracle and the point-parallel kernels (the same points in chunks below 2^18)."""
    res, N = 34, 300000
    coefs = W.init_coefs(3, res, order, C, seed=8, std=0.5)
    g = tg.tg_create(3, res, order, C, "f32")
    tg.tg_set_coefs(g, to_dev(coefs))
    pts = np.concatenate([points(3, res, N - 1000, seed=31), W.uniform_points(32, 1000)])
    N = pts.shape[0]                       # the helper adds the edge cases
    P = to_dev(pts)
    out, gx = tg.tg_query(g, P, want_grad=True)
    chunks = [tg.tg_query(g, P[i:i + 100000], want_grad=True) for i in range(0, N, 100000)]
    torch.cuda.synchronize()
    check_forward(out.cpu().numpy(), gx.cpu().numpy(), 3, res, order, C, coefs.astype(np.float64), pts)
    torch.testing.assert_close(out, torch.cat([c[0] for c in chunks]), rtol=1e-5, atol=1e-5)
    up = np.random.default_rng(3).normal(size=(N, C)).astype(np.float32)
    grad = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, P, to_dev(up), grad)
    ref = torch.zeros(g.n_coefs, device="cuda")
    for i in range(0, N, 100000):
        tg.tg_query_backward(g, P[i:i + 100000], to_dev(up[i:i + 100000]), ref)
    torch.cuda.synchronize()
    check_coef_grad(grad.cpu().numpy(), 3, res, order, C, pts, up)
    torch.testing.assert_close(grad, ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))


def test_large_batches_on_two_streams_share_the_grid_batch(tg):
    res, N = 34, 1 << 18
    g = tg.tg_create(3, res, 2, 1, "f32", seed=4, init_std=0.5)
    Ps = [to_dev(W.uniform_points(40 + k, N)) for k in range(2)]
    refs = [torch.cat([tg.tg_query(g, P[i:i + 65536]) for i in range(0, N, 65536)]) for P in Ps]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    outs = []
    for rep in range(3):
        for P, s in zip(Ps, streams):
            outs.append(tg.tg_query(g, P, stream=s))
    torch.cuda.synchronize()
    for k, o in enumerate(outs):
        torch.testing.assert_close(o, refs[k % 2], rtol=1e-5, atol=1e-5)


def test_large_batches_under_cuda_graph_capture(tg):
    """Calls captured into a CUDA graph take the point-parallel kernels (binning allocates and reads back
    sizes, so it stays out of graphs); the replayed graph matches the oracle and the binned calls."""
    res, order, C, N = 34, 2, 1, 1 << 18
    coefs = W.init_coefs(3, res, order, C, seed=9, std=0.5)
    g = tg.tg_create(3, res, order, C, "f32")
    tg.tg_set_coefs(g, to_dev(coefs))
    pts = W.uniform_points(44, N)
    P = to_dev(pts)
    up = np.random.default_rng(6).normal(size=(N, C)).astype(np.float32)
    U = to_dev(up)
    out_binned = tg.tg_query(g, P)
    grad_binned = torch.zeros(g.n_coefs, device="cuda")
    tg.tg_query_backward(g, P, U, grad_binned)
    out = torch.empty((N, C), device="cuda")
    grad = torch.zeros(g.n_coefs, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        tg.tg_query(g, P, out=out)
        tg.tg_query_backward(g, P, U, grad)
    for rep in range(2):                   # the capture itself runs nothing; each replay adds one backward
        grad.zero_()
        graph.replay()
        torch.cuda.synchronize()
        check_forward(out.cpu().numpy(), None, 3, res, order, C, coefs.astype(np.float64), pts)
        check_coef_grad(grad.cpu().numpy(), 3, res, order, C, pts, up)
        torch.testing.assert_close(out, out_binned, rtol=1e-5, atol=1e-5)
        torch.testing.assert_close(grad, grad_binned, rtol=1e-4, atol=1e-4 * float(grad_binned.abs().max()))
