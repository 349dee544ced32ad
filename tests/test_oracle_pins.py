"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own formulas: a library
routine (torch grid_sample, torch.optim.Adam), a closed form (polynomial
reproduction, homogeneous-medium transmittance, analytic SDFs), an invariant
(face continuity, linearity) or finite differences. Each is chosen so that a
plausible slip in the oracle (dropped 1/2, wrong corner bit, swapped Hessian
entry, wrong sign in the compositing derivative) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# Generator
# --------------------------------------------------------------------------
def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    st = np.uint64(1234567)
    got = []
    for _ in range(5):
        got.append(int(W.splitmix64(np.asarray([st]))[0]))
        with np.errstate(over="ignore"):
            st = np.uint64(st + np.uint64(0x9E3779B97F4A7C15))
    assert got == vals


def test_oracle_uniform_matches_input_generator():
    idx = np.arange(64, dtype=np.uint64)
    a = W.uniform(7, 11, idx).astype(np.float64)
    b = np.array([oracle.uniform(7, 11, int(i)) for i in idx])
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# Eq. 2: the index rule
# --------------------------------------------------------------------------
def test_locate_rule_edges():
    res = 5
    pts = np.array([[0.0], [1.0], [0.25], [0.2499999], [-0.5], [1.5], [np.nan], [0.999]], np.float32)
    cells, ts = oracle.locate(1, res, pts)
    assert cells[:, 0].tolist() == [0, 3, 1, 0, 0, 3, 0, 3]
    assert ts[0, 0] == 0.0 and ts[1, 0] == 1.0 and ts[2, 0] == 0.0
    assert ts[4, 0] == 0.0 and ts[5, 0] == 1.0 and ts[6, 0] == 0.0
    # t is the FP32 difference of the FP32 product
    u = np.float32(np.float32(0.999) * np.float32(4.0))
    assert ts[7, 0] == float(np.float32(u - np.float32(3.0)))


# --------------------------------------------------------------------------
# Order 0 is the linear grid (Sec. 4.1 "Linear only considers the zero-order
# Taylor series"): the field must equal trilinear / bilinear interpolation.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,res,C", [(3, 5, 1), (3, 4, 3), (2, 6, 2)])
def test_order0_equals_grid_sample(dim, res, C):
    r = rng(1)
    coefs = r.normal(size=res ** dim * C)
    pts = r.random((300, dim)).astype(np.float32)
    out, _, _, _ = oracle.query(dim, res, 0, C, coefs, pts, want_grad=False)
    vol = torch.tensor(coefs.reshape((res,) * dim + (C,))).movedim(-1, 0)[None]   # (1, C, [D,] H, W)
    g = torch.tensor(pts.astype(np.float64) * 2.0 - 1.0)
    g = g.reshape((1,) + (1,) * (dim - 1) + (pts.shape[0], dim))
    ref = torch.nn.functional.grid_sample(vol, g, mode="bilinear", align_corners=True)
    ref = ref.reshape(C, -1).T.numpy()
    np.testing.assert_allclose(out, ref, rtol=0, atol=2e-6 * np.abs(coefs).max())


# --------------------------------------------------------------------------
# Polynomial reproduction (Eq. 1 + the partition of unity of Eq. 4)
# --------------------------------------------------------------------------
def taylor_data_of_poly(dim, res, order, p, grad, hess):
    """Exact Taylor data (derivatives in x, Eq. 1) of a polynomial at every vertex, exchange layout."""
    h = 1.0 / (res - 1)
    K = W.n_coefs(dim, order)
    axes = np.meshgrid(*[np.arange(res) * h] * dim, indexing="ij")
    X = np.stack([a.reshape(-1) for a in axes[::-1]], 1) if dim == 3 else None
    # vertex v = x + res*(y + res*z): enumerate in that order
    idx = np.arange(res ** dim)
    coords = np.stack([(idx // res ** d) % res for d in range(dim)], 1) * h
    out = np.zeros((res ** dim, K))
    out[:, 0] = [p(c) for c in coords]
    if order >= 1:
        out[:, 1:1 + dim] = np.array([grad(c) for c in coords])
    if order >= 2:
        Hs = np.array([hess(c) for c in coords])
        diag = [Hs[:, a, a] for a in range(dim)]
        off = [Hs[:, 0, 1], Hs[:, 0, 2], Hs[:, 1, 2]] if dim == 3 else [Hs[:, 0, 1]]
        out[:, 1 + dim:] = np.stack(diag + off, 1)
    return out.reshape(-1)


def quadratic(dim, seed):
    r = rng(seed)
    a = r.normal(); b = r.normal(size=dim); A = r.normal(size=(dim, dim)); A = A + A.T
    p = lambda x: a + b @ x + 0.5 * x @ A @ x
    return p, (lambda x: b + A @ x), (lambda x: A)


@pytest.mark.parametrize("dim,res", [(3, 4), (3, 7), (2, 5)])
def test_order2_reproduces_quadratics(dim, res):
    p, gp, hp = quadratic(dim, 3 + dim)
    coefs = taylor_data_of_poly(dim, res, 2, p, gp, hp)
    pts = rng(4).random((500, dim)).astype(np.float32)
    out, gx, _, _ = oracle.query(dim, res, 2, 1, coefs, pts)
    x = pts.astype(np.float64)
    np.testing.assert_allclose(out[:, 0], [p(v) for v in x], atol=5e-6)
    np.testing.assert_allclose(gx[:, 0, :], [gp(v) for v in x], atol=5e-5)


@pytest.mark.parametrize("dim,res", [(3, 5), (2, 4)])
def test_order1_reproduces_affine(dim, res):
    r = rng(5)
    a, b = r.normal(), r.normal(size=dim)
    coefs = taylor_data_of_poly(dim, res, 1, lambda x: a + b @ x, lambda x: b, None)
    pts = r.random((400, dim)).astype(np.float32)
    out, gx, _, _ = oracle.query(dim, res, 1, 1, coefs, pts)
    np.testing.assert_allclose(out[:, 0], a + pts.astype(np.float64) @ b, atol=5e-6)
    np.testing.assert_allclose(gx[:, 0, :], np.broadcast_to(b, (400, dim)), atol=5e-6)


def test_order1_does_not_reproduce_quadratics():
    p, gp, hp = quadratic(3, 9)
    coefs = taylor_data_of_poly(3, 4, 1, p, gp, None)
    pts = rng(6).random((200, 3)).astype(np.float32)
    out, _, _, _ = oracle.query(3, 4, 1, 1, coefs, pts, want_grad=False)
    assert np.abs(out[:, 0] - [p(v) for v in pts.astype(np.float64)]).max() > 1e-3


def test_order2_does_not_reproduce_cubics():
    res = 4
    p = lambda x: x[0] ** 3
    coefs = taylor_data_of_poly(3, res, 2, p, lambda x: np.array([3 * x[0] ** 2, 0, 0]),
                                lambda x: np.diag([6 * x[0], 0, 0]))
    pts = rng(7).random((200, 3)).astype(np.float32)
    out, _, _, _ = oracle.query(3, res, 2, 1, coefs, pts, want_grad=False)
    assert np.abs(out[:, 0] - pts[:, 0].astype(np.float64) ** 3).max() > 1e-5


def test_order0_reproduces_multilinear():
    r = rng(8)
    c = r.normal(size=8)
    p = lambda x: (c[0] + c[1] * x[0] + c[2] * x[1] + c[3] * x[2] + c[4] * x[0] * x[1]
                   + c[5] * x[0] * x[2] + c[6] * x[1] * x[2] + c[7] * x[0] * x[1] * x[2])
    coefs = taylor_data_of_poly(3, 2, 0, p, None, None)       # one cell: exact
    pts = r.random((300, 3)).astype(np.float32)
    out, _, _, _ = oracle.query(3, 2, 0, 1, coefs, pts, want_grad=False)
    np.testing.assert_allclose(out[:, 0], [p(v) for v in pts.astype(np.float64)], atol=5e-6)


def test_zero_derivatives_reduce_to_order0():
    r = rng(9)
    res, C = 4, 2
    f0 = r.normal(size=(res ** 3, C))
    c2 = np.zeros((res ** 3, C, 10)); c2[:, :, 0] = f0
    pts = r.random((300, 3)).astype(np.float32)
    a, ga, _, _ = oracle.query(3, res, 2, C, c2.reshape(-1), pts)
    b, gb, _, _ = oracle.query(3, res, 0, C, f0.reshape(-1), pts)
    np.testing.assert_allclose(a, b, atol=1e-12)
    np.testing.assert_allclose(ga, gb, atol=1e-11)


def test_hessian_offdiagonal_order():
    """The field x z stores its second derivative in the H_xz slot only (value 1 at every vertex)."""
    res = 3
    p = lambda x: x[0] * x[2]
    coefs = taylor_data_of_poly(3, res, 2, p, lambda x: np.array([x[2], 0.0, x[0]]),
                                lambda x: np.array([[0, 0, 1.0], [0, 0, 0], [1.0, 0, 0]]))
    c = coefs.reshape(-1, 10)
    assert np.allclose(c[:, 8], 1.0) and np.allclose(c[:, 7], 0) and np.allclose(c[:, 9], 0)
    pts = rng(10).random((100, 3)).astype(np.float32)
    out, _, _, _ = oracle.query(3, res, 2, 1, coefs, pts, want_grad=False)
    np.testing.assert_allclose(out[:, 0], pts[:, 0].astype(np.float64) * pts[:, 2], atol=5e-6)


# --------------------------------------------------------------------------
# Continuity across cell faces (Eq. 4 weights vanish off the face)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [0, 1, 2])
def test_face_continuity(order):
    r = rng(11 + order)
    res, C = 4, 2
    K = W.n_coefs(3, order)
    coefs = r.normal(size=res ** 3 * C * K)
    for axis in range(3):
        for _ in range(10):
            cell = r.integers(0, res - 2, size=3)          # both cell and cell+e_axis valid
            t = r.random(3)
            t_lo = t.copy(); t_lo[axis] = 1.0
            t_hi = t.copy(); t_hi[axis] = 0.0
            up = cell.copy(); up[axis] += 1
            fa, _ = oracle.eval_cell(3, res, order, C, coefs, cell, t_lo)
            fb, _ = oracle.eval_cell(3, res, order, C, coefs, up, t_hi)
            np.testing.assert_allclose(fa, fb, atol=1e-12)


# --------------------------------------------------------------------------
# Spatial gradient: central finite differences inside a cell
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,order", [(3, 2), (3, 1), (2, 2), (3, 0)])
def test_spatial_gradient_finite_differences(dim, order):
    r = rng(20 + order + dim)
    res, C = 4, 2
    coefs = r.normal(size=res ** dim * C * W.n_coefs(dim, order))
    eps = 1e-5
    for _ in range(20):
        cell = r.integers(0, res - 1, size=dim)
        t = 0.1 + 0.8 * r.random(dim)
        _, gx = oracle.eval_cell(dim, res, order, C, coefs, cell, t)
        for a in range(dim):
            tp = t.copy(); tp[a] += eps
            tm = t.copy(); tm[a] -= eps
            fp, _ = oracle.eval_cell(dim, res, order, C, coefs, cell, tp)
            fm, _ = oracle.eval_cell(dim, res, order, C, coefs, cell, tm)
            # x = (cell + t) h: d/dx = (res - 1) d/dt
            np.testing.assert_allclose(gx[:, a], (fp - fm) / (2 * eps) * (res - 1), atol=1e-7)


def test_query_gradient_is_world_units():
    r = rng(30)
    res = 6
    coefs = r.normal(size=res ** 3 * 10)
    pts = r.random((50, 3)).astype(np.float32)
    _, gx, cells, ts = oracle.query(3, res, 2, 1, coefs, pts, want_cells=True)
    for n in range(50):
        _, gc = oracle.eval_cell(3, res, 2, 1, coefs, cells[n], ts[n])
        np.testing.assert_allclose(gx[n, 0], gc[0], rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# Coefficient gradient: central finite differences (exact by linearity)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,res,order,C", [(3, 2, 2, 1), (3, 3, 1, 2), (3, 4, 2, 1), (2, 3, 2, 2), (3, 3, 0, 3)])
def test_coef_gradient_finite_differences(dim, res, order, C):
    r = rng(40 + res + order)
    K = W.n_coefs(dim, order)
    coefs = r.normal(size=res ** dim * C * K)
    N = 40
    pts = r.random((N, dim)).astype(np.float32)
    pts[0] = 0.0; pts[1] = 1.0                          # domain corners
    dLdf = r.normal(size=(N, C)); dLdg = r.normal(size=(N, C, dim))

    def L(c):
        f, g, _, _ = oracle.query(dim, res, order, C, c, pts)
        return float((f * dLdf).sum() + (g * dLdg).sum())

    grad = oracle.query_backward(dim, res, order, C, pts, dLdf, dLdg)
    eps = 1e-3
    fd = np.zeros_like(coefs)
    for j in range(coefs.size):
        e = np.zeros_like(coefs); e[j] = eps
        fd[j] = (L(coefs + e) - L(coefs - e)) / (2 * eps)
    np.testing.assert_allclose(grad, fd, atol=1e-8 * max(1.0, np.abs(fd).max()))


def test_adjoint_identity():
    r = rng(50)
    res, order, C, dim = 6, 2, 2, 3
    K = W.n_coefs(dim, order)
    theta = r.normal(size=res ** 3 * C * K)
    pts = r.random((2000, 3)).astype(np.float32)
    g = r.normal(size=(2000, C))
    f, _, _, _ = oracle.query(dim, res, order, C, theta, pts, want_grad=False)
    At_g = oracle.query_backward(dim, res, order, C, pts, g)
    assert abs((f * g).sum() - theta @ At_g) < 1e-9 * abs(theta @ At_g) + 1e-9


# --------------------------------------------------------------------------
# Adam: torch.optim.Adam in float64
# --------------------------------------------------------------------------
def test_adam_matches_torch():
    r = rng(60)
    n = 1000
    p0 = r.normal(size=n)
    p = p0.copy(); m = np.zeros(n); v = np.zeros(n)
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = r.normal(size=n)
        gg = g.copy()
        oracle.adam(p, gg, m, v, 3e-3, 0.9, 0.999, 1e-8, step)
        assert not gg.any()
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)

def test_lazy_adam_matches_torch_sparse_adam():
    """Lazy Adam against torch.optim.SparseAdam (float64) fed the nonzero entries as a sparse gradient; entries
    with a zero gradient keep p, m and v; with no zero entries it is plain Adam. SparseAdam adds eps to sqrt(v)
    before the bias correction, Adam (and the oracle) to sqrt(v_hat): the two agree to rounding at eps = 1e-30
    (SparseAdam refuses 0), and the dense case pins the eps placement to the Adam oracle, itself pinned to
    torch.optim.Adam."""
    r = rng(61)
    n = 1000
    p0 = r.normal(size=n)
    p = p0.copy(); m = np.zeros(n); v = np.zeros(n)
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.SparseAdam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-30)
    for step in range(1, 7):
        g = r.normal(size=n) * (r.random(n) < 0.4)          # about 60 % untouched entries per step
        before = (p.copy(), m.copy(), v.copy())
        gg = g.copy()
        oracle.adam_lazy(p, gg, m, v, 3e-3, 0.9, 0.999, 1e-30, step)
        assert not gg.any()
        idx = np.nonzero(g)[0]
        tp.grad = torch.sparse_coo_tensor(torch.tensor(idx)[None], torch.tensor(g[idx]), (n,),
                                          check_invariants=True)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)
        z = g == 0
        for a, b in zip((p, m, v), before):
            assert np.array_equal(a[z], b[z])
    # dense gradient: the lazy rule is plain Adam
    q = p0.copy(); mq = np.zeros(n); vq = np.zeros(n)
    p = p0.copy(); m = np.zeros(n); v = np.zeros(n)
    for step in range(1, 4):
        g = r.normal(size=n)
        g[g == 0] = 1.0
        oracle.adam(q, g.copy(), mq, vq, 1e-2, 0.9, 0.999, 1e-8, step)
        oracle.adam_lazy(p, g.copy(), m, v, 1e-2, 0.9, 0.999, 1e-8, step)
    assert np.array_equal(p, q) and np.array_equal(m, mq) and np.array_equal(v, vq)


# --------------------------------------------------------------------------
# SDF targets and the SDF step (Sec. 3.2)
# --------------------------------------------------------------------------
def test_sdf_closed_forms():
    sph = np.array([[0.5, 0.5, 0.5, 0.3]], np.float32)
    box = np.array([[0.2, 0.3, 0.4, 0.1, 0.05, 0.2]], np.float32)
    none_s = np.zeros((0, 4), np.float32); none_b = np.zeros((0, 6), np.float32)
    f32 = lambda v: float(np.float32(v))
    # sphere: centre, surface, outside
    d = oracle.sdf_union(sph, none_b, np.array([[0.5, 0.5, 0.5], [0.8, 0.5, 0.5], [0.5, 0.5, 1.0]]))
    np.testing.assert_allclose(d, [-f32(0.3), 0.8 - 0.5 - f32(0.3), 1.0 - 0.5 - f32(0.3)], atol=1e-12)
    c = np.array([f32(0.2), f32(0.3), f32(0.4)]); h = np.array([f32(0.1), f32(0.05), f32(0.2)])
    pts = np.array([c,                                  # centre: -min half extent
                    c + [h[0] + 0.1, 0, 0],             # outside a face
                    c + [h[0] + 0.03, h[1] + 0.04, 0],  # outside an edge
                    c + h + [0.01, 0.02, 0.02],         # outside a corner
                    c + [0, h[1] - 0.01, 0]])           # inside near a face
    want = [-h.min(), 0.1, 0.05, 0.03, -0.01]
    np.testing.assert_allclose(oracle.sdf_union(none_s, box, pts), want, atol=1e-12)
    # union = min
    both = oracle.sdf_union(sph, box, pts)
    np.testing.assert_allclose(both, np.minimum(oracle.sdf_union(sph, none_b, pts), want), atol=1e-12)


def test_box_sdf_brute_force():
    box = np.array([[0.5, 0.45, 0.55, 0.2, 0.1, 0.15]], np.float32)
    c = box[0, :3].astype(np.float64); h = box[0, 3:].astype(np.float64)
    g = np.linspace(-1, 1, 121)
    A, B = np.meshgrid(g, g, indexing="ij")
    surf = []
    for ax in range(3):
        a1, a2 = (ax + 1) % 3, (ax + 2) % 3
        for s in (-1, 1):
            P = np.zeros((A.size, 3))
            P[:, ax] = c[ax] + s * h[ax]; P[:, a1] = c[a1] + A.ravel() * h[a1]; P[:, a2] = c[a2] + B.ravel() * h[a2]
            surf.append(P)
    surf = np.concatenate(surf)
    x = rng(70).random((60, 3))
    inside = np.all(np.abs(x - c) < h, axis=1)
    brute = np.array([np.linalg.norm(surf - p, axis=1).min() for p in x]) * np.where(inside, -1, 1)
    got = oracle.sdf_union(np.zeros((0, 4), np.float32), box, x)
    np.testing.assert_allclose(got, brute, atol=2.5e-3)


def test_sdf_step_loss_gradient_finite_differences():
    r = rng(80)
    res, order = 3, 2
    coefs = r.normal(size=res ** 3 * 10) * 0.2
    shape = W.sphere_shape((0.45, 0.5, 0.55), 0.3)
    pts = r.random((64, 3)).astype(np.float32)
    lam = 0.1
    g, _ = oracle.sdf_step(res, order, coefs, pts, shape.spheres, shape.boxes, lam)

    def L(c):
        _, (l1, eik) = oracle.sdf_step(res, order, c, pts, shape.spheres, shape.boxes, lam)
        return l1 + lam * eik

    eps = 1e-6
    for j in r.choice(coefs.size, 40, replace=False):
        e = np.zeros_like(coefs); e[j] = eps
        fd = (L(coefs + e) - L(coefs - e)) / (2 * eps)
        assert abs(fd - g[j]) < 1e-6 + 1e-5 * abs(fd), (j, fd, g[j])


def test_sdf_step_loss_values():
    """With the exact Taylor data of an affine SDF-like field the residual and the eikonal term are known."""
    res = 5
    b = np.array([0.6, 0.0, 0.8])                         # |b| = 1: eikonal term zero
    coefs = taylor_data_of_poly(3, res, 2, lambda x: -0.2 + b @ x, lambda x: b, lambda x: np.zeros((3, 3)))
    sph = np.array([[0.5, 0.5, 0.5, 0.25]], np.float32)
    pts = rng(81).random((100, 3)).astype(np.float32)
    _, (l1, eik) = oracle.sdf_step(res, 2, coefs, pts, sph, np.zeros((0, 6), np.float32), 0.1)
    x = pts.astype(np.float64)
    d = np.linalg.norm(x - 0.5, axis=1) - np.float32(0.25)
    np.testing.assert_allclose(l1, np.abs(-0.2 + x @ b - d).mean(), atol=1e-6)
    assert eik < 1e-10


def test_adaptive_weight_closed_form():
    """Eq. 7: w'(z) = 1 - |2 sigmoid(k z) - 1| = 1 - tanh(|k z| / 2); 1 on the surface, even in z, towards 0 away."""
    for k in (10.0, 100.0):
        for z in (-0.3, -0.01, 0.0, 0.004, 0.2):
            assert abs(oracle.adaptive_weight1(k, z) - (1 - math.tanh(abs(k * z) / 2))) < 1e-14
    assert oracle.adaptive_weight1(100.0, 0.0) == 1.0
    assert oracle.adaptive_weight1(100.0, 1.0) < 1e-40
    assert oracle.adaptive_weight1(0.0, 0.7) == 1.0 and oracle.adaptive_weight1(-3.0, 0.7) == 1.0


def test_adaptive_weight_k0_is_plain_l1_and_weighted_step_matches_fixed_weight_fd():
    r = rng(82)
    res, order = 3, 2
    coefs = r.normal(size=res ** 3 * 10) * 0.2
    shape = W.sphere_shape((0.45, 0.5, 0.55), 0.3)
    pts = r.random((64, 3)).astype(np.float32)
    g0, (l0, _) = oracle.sdf_step(res, order, coefs, pts, shape.spheres, shape.boxes, 0.0)
    gk0, (lk0, _) = oracle.sdf_step(res, order, coefs, pts, shape.spheres, shape.boxes, 0.0, k_weight=0.0)
    assert l0 == lk0
    np.testing.assert_allclose(g0, gk0, rtol=1e-12, atol=1e-18)     # the oracle's OpenMP sums vary in the last bits
    k = 20.0
    g, (lw, _) = oracle.sdf_step(res, order, coefs, pts, shape.spheres, shape.boxes, 0.0, k_weight=k)
    # the weight is held at its value for the current coefficients
    f0, _, _, _ = oracle.query(3, res, order, 1, coefs, pts, want_grad=False)
    d = oracle.sdf_union(shape.spheres, shape.boxes, np.clip(pts.astype(np.float64), 0, 1))
    w = np.maximum([oracle.adaptive_weight1(k, v) for v in f0[:, 0]], [oracle.adaptive_weight1(k, v) for v in d])
    assert w.min() < 0.9 and abs(lw - np.mean(w * np.abs(f0[:, 0] - d))) < 1e-12

    def L(c):
        f, _, _, _ = oracle.query(3, res, order, 1, c, pts, want_grad=False)
        return np.mean(w * np.abs(f[:, 0] - d))

    eps = 1e-6
    for j in r.choice(coefs.size, 40, replace=False):
        e = np.zeros_like(coefs); e[j] = eps
        fd = (L(coefs + e) - L(coefs - e)) / (2 * eps)
        assert abs(fd - g[j]) < 1e-7 + 1e-5 * abs(fd), (j, fd, g[j])


def test_tv_constant_and_ramp_closed_forms():
    res, nv = 6, 3
    const = np.tile(np.array([0.3, -1.0, 2.0]), res ** 3)
    L, g = oracle.tv(res, nv, const)
    assert L == 0.0 and not g.any()
    # theta(v, 0) = a i along x, other channels zero: n = |a| except on the last x plane
    a = -0.7
    i = np.arange(res ** 3) % res
    ramp = np.zeros((res ** 3, nv)); ramp[:, 0] = a * i
    L, g = oracle.tv(res, nv, ramp.ravel(), lam=2.0)
    np.testing.assert_allclose(L, (res - 1) * res * res * abs(a) / res ** 3, rtol=1e-14)
    g = g.reshape(-1, nv)
    want = np.zeros(res ** 3)
    want[i == 0] = -np.sign(a) * 2.0 / res ** 3        # only the first and last planes keep a gradient
    want[i == res - 1] = np.sign(a) * 2.0 / res ** 3
    np.testing.assert_allclose(g[:, 0], want, atol=1e-15)
    assert not g[:, 1:].any()


def test_tv_gradient_finite_differences_and_channel_separability():
    r = rng(83)
    res, nv = 4, 2
    c = r.normal(size=res ** 3 * nv)
    L, g = oracle.tv(res, nv, c, lam=0.5)
    L0, _ = oracle.tv(res, 1, c.reshape(-1, nv)[:, 0].copy(), want_grad=False)
    L1, _ = oracle.tv(res, 1, c.reshape(-1, nv)[:, 1].copy(), want_grad=False)
    np.testing.assert_allclose(L, L0 + L1, rtol=1e-13)
    eps = 1e-6
    for j in r.choice(c.size, 40, replace=False):
        e = np.zeros_like(c); e[j] = eps
        fd = 0.5 * (oracle.tv(res, nv, c + e, want_grad=False)[0] - oracle.tv(res, nv, c - e, want_grad=False)[0]) / (2 * eps)
        assert abs(fd - g[j]) < 1e-8 + 1e-6 * abs(fd), (j, fd, g[j])


def fp32_vertex_coords(res):
    """The dst vertex coordinates of the resampling rule: fl32(j / (res - 1)) in x-fastest vertex order."""
    v = (np.arange(res, dtype=np.float32) / np.float32(res - 1)).astype(np.float64)
    idx = np.arange(res ** 3)
    return np.stack([v[idx % res], v[(idx // res) % res], v[idx // res ** 2]], 1)


def taylor_at(points, order, p, grad, hess):
    out = [np.array([p(x) for x in points])[:, None]]
    if order >= 1:
        out.append(np.array([grad(x) for x in points]))
    if order >= 2:
        Hs = np.array([hess(x) for x in points])
        out.append(np.stack([Hs[:, 0, 0], Hs[:, 1, 1], Hs[:, 2, 2], Hs[:, 0, 1], Hs[:, 0, 2], Hs[:, 1, 2]], 1))
    return np.concatenate(out, 1).reshape(-1)


@pytest.mark.parametrize("res_dst", [9, 4, 7])
def test_resample_reproduces_quadratics_and_affine_fields(res_dst):
    p, gp, hp = quadratic(3, 90)
    src = taylor_data_of_poly(3, 5, 2, p, gp, hp)
    dst = oracle.resample(5, 2, 1, src, res_dst, 2)
    np.testing.assert_allclose(dst, taylor_at(fp32_vertex_coords(res_dst), 2, p, gp, hp), atol=1e-10)
    b = rng(91).normal(size=3)
    aff = taylor_data_of_poly(3, 5, 1, lambda x: 0.3 + b @ x, lambda x: b, None)
    dst = oracle.resample(5, 1, 1, aff, res_dst, 2)
    np.testing.assert_allclose(dst, taylor_at(fp32_vertex_coords(res_dst), 2, lambda x: 0.3 + b @ x,
                                              lambda x: b, lambda x: np.zeros((3, 3))), atol=1e-12)


def test_resample_keeps_the_value_at_coincident_vertices():
    src = rng(92).normal(size=5 ** 3 * 2 * 10)
    dst = oracle.resample(5, 2, 2, src, 9, 2).reshape(9, 9, 9, 2, 10)      # [z][y][x][channel][k]
    np.testing.assert_array_equal(dst[::2, ::2, ::2, :, 0], src.reshape(5, 5, 5, 2, 10)[..., 0])


def test_resample_derivatives_match_finite_differences():
    res_src, res_dst = 5, 7                 # dst coordinates j / 6 meet src faces k / 4 only at j = 0, 3, 6
    src = rng(93).normal(size=res_src ** 3 * 10)
    dst = oracle.resample(res_src, 2, 1, src, res_dst, 2).reshape(-1, 10)
    X = fp32_vertex_coords(res_dst)
    on_face = np.any(np.isin(np.round(X * 6).astype(int), [0, 3, 6]), axis=1)
    sel = np.flatnonzero(~on_face)
    eps = 1e-4
    for a in range(3):
        e = np.zeros(3); e[a] = eps
        fp, gp, _, _ = oracle.query(3, res_src, 2, 1, src, (X[sel] + e).astype(np.float32))
        fm, gm, _, _ = oracle.query(3, res_src, 2, 1, src, (X[sel] - e).astype(np.float32))
        # the points are rounded to FP32 by the query: difference over the rounded step
        step = ((X[sel] + e).astype(np.float32).astype(np.float64) - (X[sel] - e).astype(np.float32).astype(np.float64))[:, a]
        np.testing.assert_allclose(dst[sel, 1 + a], (fp[:, 0] - fm[:, 0]) / step, rtol=1e-4, atol=1e-4)
        Hrow = (gp[:, 0, :] - gm[:, 0, :]) / step[:, None]
        H = np.zeros((sel.size, 3, 3))
        H[:, 0, 0], H[:, 1, 1], H[:, 2, 2] = dst[sel, 4], dst[sel, 5], dst[sel, 6]
        H[:, 0, 1] = H[:, 1, 0] = dst[sel, 7]
        H[:, 0, 2] = H[:, 2, 0] = dst[sel, 8]
        H[:, 1, 2] = H[:, 2, 1] = dst[sel, 9]
        np.testing.assert_allclose(H[:, a, :], Hrow, rtol=1e-3, atol=1e-3 * np.abs(Hrow).max())


# --------------------------------------------------------------------------
# Volume rendering (Sec. 3.3, Eq. 10 / Eq. 11)
# --------------------------------------------------------------------------
def sp(x):
    return math.log1p(math.exp(x))


def sg(x):
    return 1.0 / (1.0 + math.exp(-x))


def test_render_homogeneous_closed_form():
    res = 4
    f0, g0 = 0.7, -0.3
    dco = np.full(res ** 3, f0)                           # order 0 density
    cco = np.tile([g0, 0.1, 0.9], res ** 3)               # order 0 colour, 3 channels
    o = np.array([[-0.5, 0.5, 0.5], [0.3, -1.0, 0.4], [2.0, 2.0, 2.0], [0.5, 0.5, 0.5]], np.float32)
    d = np.array([[1, 0, 0], [0.1, 1, 0.05], [1, 0, 0], [0, 0, 1]], np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    rgb = oracle.render(res, 0, dco, 0, cco, o, d, S=64, seed=3, bg=1.0)
    sigma = sp(f0)
    for r in range(4):
        hit, n, f = oracle.ray_box(o[r].astype(np.float64), d[r].astype(np.float64))
        if not hit:
            np.testing.assert_allclose(rgb[r], [1, 1, 1]); continue
        # stratified samples: delta_i = t_{i+1} - t_i with t_S = far, so the
        # optical depth covers [t_0, far], t_0 = near + xi_0 (far - near) / S
        # (the oracle places samples by the FP32 rule, so t_0 and far carry FP32 rounding: rtol 1e-6)
        t0 = n + float(W.uniform(3, r, 0)) * (f - n) / 64
        T = math.exp(-sigma * (f - t0))
        want = [sg(c) * (1 - T) + T for c in (g0, 0.1, 0.9)]
        np.testing.assert_allclose(rgb[r], want, rtol=1e-6)
    assert not oracle.ray_box(o[2].astype(np.float64), d[2].astype(np.float64))[0]


def test_render_black_background_is_eq10():
    """bg = 0 leaves exactly the sum of Eq. 10; a dense medium saturates to the colour."""
    res = 3
    dco = np.full(res ** 3, 40.0); cco = np.tile([0.0, 2.0, -2.0], res ** 3)
    o = np.array([[-1.0, 0.5, 0.5]], np.float32); d = np.array([[1.0, 0.0, 0.0]], np.float32)
    rgb = oracle.render(res, 0, dco, 0, cco, o, d, S=16, seed=1, bg=0.0)
    np.testing.assert_allclose(rgb[0], [sg(0.0), sg(2.0), sg(-2.0)], rtol=1e-12)


def test_render_gradient_finite_differences():
    r = rng(90)
    res, od, oc = 3, 2, 1
    dco = r.normal(size=res ** 3 * 10) * 0.5
    cco = r.normal(size=res ** 3 * 3 * 4) * 0.5
    o, d = W.random_rays(5, 3, radius=1.2, spread=0.3)
    tgt = r.random((3, 3)).astype(np.float32)
    S = 12
    _, loss, dg, cg = oracle.render(res, od, dco, oc, cco, o, d, S, seed=9, target=tgt)

    def L(a, b):
        return oracle.render(res, od, a, oc, b, o, d, S, seed=9, target=tgt)[1]

    eps = 1e-6
    for j in r.choice(dco.size, 25, replace=False):
        e = np.zeros_like(dco); e[j] = eps
        fd = (L(dco + e, cco) - L(dco - e, cco)) / (2 * eps)
        assert abs(fd - dg[j]) < 1e-7 + 1e-5 * abs(fd), ("density", j, fd, dg[j])
    for j in r.choice(cco.size, 25, replace=False):
        e = np.zeros_like(cco); e[j] = eps
        fd = (L(dco, cco + e) - L(dco, cco - e)) / (2 * eps)
        assert abs(fd - cg[j]) < 1e-7 + 1e-5 * abs(fd), ("colour", j, fd, cg[j])


def test_render_term_magnitudes_bound_the_gradient():
    """The per-coefficient sums of term magnitudes (want_abs) bound the gradients, vanish where a coefficient
    receives nothing, and equal |gradient| where every term is positive: an order-0 colour grid against a zero
    target (C - 0 > 0, T alpha > 0, sigmoid' > 0, corner weights >= 0)."""
    r = rng(91)
    res = 3
    o, d = W.random_rays(6, 4, radius=1.2, spread=0.3)
    for od, oc, tgt in ((2, 1, r.random((4, 3)).astype(np.float32)), (1, 0, np.zeros((4, 3), np.float32))):
        dco = r.normal(size=res ** 3 * oracle.num_coefs(3, od)) * 0.5
        cco = r.normal(size=res ** 3 * 3 * oracle.num_coefs(3, oc)) * 0.5
        _, _, dg, cg, da, ca = oracle.render(res, od, dco, oc, cco, o, d, 10, seed=4, target=tgt, want_abs=True)
        assert (da >= np.abs(dg) * (1 - 1e-12)).all() and (ca >= np.abs(cg) * (1 - 1e-12)).all()
        assert (dg[da == 0] == 0).all() and (cg[ca == 0] == 0).all()
        assert (ca > 0).any() and (da > 0).any()
        if oc == 0:
            np.testing.assert_allclose(ca, np.abs(cg), rtol=1e-12, atol=0)


def test_blob_scene_renderer_limits():
    """A dense blob saturates to its colour; a ray that misses the cube renders bg; an empty scene is bg."""
    mu = np.array([[0.5, 0.5, 0.5]]); icov = np.eye(3)[None] / 0.05 ** 2
    amp = np.array([5000.0]); rgb = np.array([[0.2, 0.4, 0.8]])
    o = np.array([[-1.0, 0.5, 0.5], [2.0, 2.0, 2.0]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]], np.float32)
    c = oracle.render_blobs((mu, icov, amp, rgb), o, d, n_samples=4096, bg=1.0)
    np.testing.assert_allclose(c[0], rgb[0], atol=1e-3)
    np.testing.assert_allclose(c[1], [1, 1, 1])
    c0 = oracle.render_blobs((mu, icov, np.array([0.0]), rgb), o, d, n_samples=64, bg=0.25)
    np.testing.assert_allclose(c0, 0.25)


# --------------------------------------------------------------------------
# Mesh extraction (marching tetrahedra), mesh sampling and the Chamfer distance
# --------------------------------------------------------------------------
def _lattice(M, fn):
    a = np.arange(M, dtype=np.float64) / (M - 1)
    z, y, x = np.meshgrid(a, a, a, indexing="ij")
    return fn(x, y, z).ravel()


@pytest.mark.parametrize("M", [9, 17])
def test_marching_tets_plane(M):
    """f = z - 0.37: every vertex lies on the plane, the triangles tile the unit square (area 1) and face +z."""
    T = oracle.marching_tets(M, _lattice(M, lambda x, y, z: z - 0.37))
    np.testing.assert_allclose(T[..., 2], 0.37, atol=1e-12)
    n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
    assert abs(0.5 * np.linalg.norm(n, axis=1).sum() - 1.0) < 1e-12
    assert (n[:, 2] > 0).all()


def _edges(T):
    key = lambda v: tuple(np.round(v, 12))
    directed = {}
    for tri in T:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            e = (key(tri[a]), key(tri[b]))
            directed[e] = directed.get(e, 0) + 1
    return directed


def test_marching_tets_sphere_closed_oriented_and_accurate():
    """|x - c| - r: a closed, consistently oriented surface (every directed edge once, its reverse once, Euler
    characteristic 2) whose area and enclosed volume approach 4 pi r^2 and 4/3 pi r^3 as the lattice refines."""
    c, r = np.array([0.5, 0.52, 0.48]), 0.3
    errs = []
    for M in (17, 33):
        T = oracle.marching_tets(M, _lattice(M, lambda x, y, z: np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2
                                                                        + (z - c[2]) ** 2) - r))
        d = _edges(T)
        assert all(v == 1 for v in d.values())
        assert all((b, a) in d for (a, b) in d)
        V = len({v for e in d for v in e}); E = len(d) // 2; F = T.shape[0]
        assert V - E + F == 2
        area = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1).sum()
        vol = (T[:, 0] * np.cross(T[:, 1], T[:, 2])).sum() / 6.0
        errs.append((abs(area / (4 * np.pi * r * r) - 1), abs(vol / (4 / 3 * np.pi * r ** 3) - 1)))
    assert errs[1][0] < 0.01 and errs[1][1] < 0.01
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]


def test_marching_tets_empty_and_full():
    assert oracle.marching_tets(5, np.ones(125)).shape[0] == 0
    assert oracle.marching_tets(5, -np.ones(125)).shape[0] == 0


def test_lattice_values_of_quadratic_grids():
    """Two order-2 channels holding the Taylor data of two different quadratics (exchange layout
    [vertex][channel][k]) reproduce them on a lattice that does not coincide with the grid's vertices: the
    lattice is i (x) fastest and the channel argument selects the channel. A transposed lattice or the wrong
    channel misses by O(1), since the quadratics differ along every axis."""
    res, M = 6, 9
    quads = [quadratic(3, 21), quadratic(3, 22)]
    per = [taylor_data_of_poly(3, res, 2, *q).reshape(res ** 3, 1, -1) for q in quads]
    coefs = np.concatenate(per, axis=1).reshape(-1)
    a = np.arange(M, dtype=np.float64) / (M - 1)
    lat = np.stack(np.meshgrid(a, a, a, indexing="ij")[::-1], -1).reshape(-1, 3)     # (x, y, z), x fastest
    lat = lat.astype(np.float32).astype(np.float64)                                 # the FP32 query points
    for ch, (p, _, _) in enumerate(quads):
        vals = oracle.lattice_values(res, 2, 2, coefs, M, channel=ch)
        np.testing.assert_allclose(vals, [p(v) for v in lat], atol=5e-6)
    assert np.abs(oracle.lattice_values(res, 2, 2, coefs, M, channel=0)
                  - np.array([quads[1][0](v) for v in lat])).max() > 0.1


def test_sample_mesh_area_weighting_and_support():
    """Two triangles with areas 1 : 3: the samples split 1 : 3 and lie on their triangles; the mean of the
    samples on one triangle is its centroid."""
    T = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]],
                  [[0, 0, 1], [3, 0, 1], [0, 1, 1]]], np.float32)
    n = 40000
    P = oracle.sample_mesh(T, n, seed=7)
    on0 = np.abs(P[:, 2]) < 1e-12
    on1 = np.abs(P[:, 2] - 1) < 1e-12
    assert (on0 | on1).all()
    frac = on0.mean()
    assert abs(frac - 0.25) < 4 * np.sqrt(0.25 * 0.75 / n)
    for tri, m in ((T[0], on0), (T[1], on1)):
        Q = P[m]
        ux, uy = tri[1, 0], tri[2, 1]
        assert (Q[:, 0] >= -1e-12).all() and (Q[:, 1] >= -1e-12).all()
        assert (Q[:, 0] / ux + Q[:, 1] / uy <= 1 + 1e-9).all()
        cen = tri.astype(np.float64).mean(0)
        sd = max(ux, uy) / np.sqrt(18)                  # the largest coordinate deviation on the triangle
        np.testing.assert_allclose(Q.mean(0)[:2], cen[:2], atol=5 * sd / np.sqrt(m.sum()))


def test_chamfer_closed_forms():
    """A set against itself is 0; against a copy translated by s (much shorter than the spacing) each direction
    sums N |s|^2; small sets match the double loop."""
    r = rng(70)
    g = np.stack(np.meshgrid(*[np.arange(6) / 5.0] * 3, indexing="ij"), -1).reshape(-1, 3)
    assert oracle.chamfer(g, g) == (0.0, 0.0)
    s = np.array([0.01, -0.02, 0.015])
    a, b = oracle.chamfer(g, g + s)
    np.testing.assert_allclose([a, b], [g.shape[0] * (s @ s)] * 2, rtol=1e-12)
    A = r.random((40, 3)); B = r.random((55, 3))
    ab = sum(min(((p - q) ** 2).sum() for q in B) for p in A)
    ba = sum(min(((p - q) ** 2).sum() for p in A) for q in B)
    np.testing.assert_allclose(oracle.chamfer(A, B), [ab, ba], rtol=1e-12)


# --------------------------------------------------------------------------
# The tolerance scale of the parity tests: sum_i w_i sum_k |theta_ik phi_k|
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,order,C", [(3, 2, 1), (3, 1, 3), (2, 2, 2)])
def test_absscale_bounds_the_value_and_is_exact_for_nonnegative_terms(dim, order, C):
    """It is never below |f| (triangle inequality), equals f when every term is non-negative (order 0 with
    non-negative coefficients, and order 2 with only non-negative value and diagonal-Hessian coefficients),
    and scales linearly with the coefficients."""
    res = 6
    r = rng(80 + dim + order)
    K = W.n_coefs(dim, order)
    coefs = r.normal(size=res ** dim * C * K)
    pts = r.random((300, dim)).astype(np.float32)
    f, _, _, _ = oracle.query(dim, res, order, C, coefs, pts, want_grad=False)
    S = oracle.query_absscale(dim, res, order, C, coefs, pts)
    assert (S >= np.abs(f).reshape(S.shape) - 1e-12).all()
    np.testing.assert_allclose(oracle.query_absscale(dim, res, order, C, 3.0 * coefs, pts), 3.0 * S, rtol=1e-12)
    pos = np.abs(r.normal(size=res ** dim * C))
    f0, _, _, _ = oracle.query(dim, res, 0, C, pos, pts, want_grad=False)
    np.testing.assert_allclose(oracle.query_absscale(dim, res, 0, C, pos, pts), f0.reshape(-1, C), rtol=1e-12)
    if order == 2:                              # value and diagonal Hessian terms only: every term >= 0
        q = np.zeros((res ** dim * C, K))
        q[:, 0] = np.abs(r.normal(size=q.shape[0]))
        q[:, 1 + dim:1 + 2 * dim] = np.abs(r.normal(size=(q.shape[0], dim)))
        q = q.reshape(-1)
        fq, _, _, _ = oracle.query(dim, res, 2, C, q, pts, want_grad=False)
        np.testing.assert_allclose(oracle.query_absscale(dim, res, 2, C, q, pts), fq.reshape(-1, C), rtol=1e-12)



# --------------------------------------------------------------------------
# The spatial-gradient tolerance scale:
# sum_i |d w_i / d x_a| sum_k |theta_ik phi_k| + w_i sum_k |theta_ik d phi_k / d x_a|
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,order,C", [(3, 2, 1), (3, 1, 3), (2, 2, 2), (3, 0, 1)])
def test_gradscale_bounds_the_spatial_gradient_and_is_exact_for_coherent_terms(dim, order, C):
    """G_a is never below |d f / d x_a| (triangle inequality over the terms of Eq. 4 differentiated), scales
    linearly with the coefficients, and equals |d f / d x_a| for an order-0 field whose vertex values are +|r|
    at odd and -|r| at even coordinates along a: inside a cell the two corners along a then carry opposite
    values and opposite weight slopes, so every term of the sum has the same sign."""
    res = 6
    r = rng(90 + dim + order)
    K = W.n_coefs(dim, order)
    coefs = r.normal(size=res ** dim * C * K)
    pts = r.random((300, dim)).astype(np.float32)
    _, gx, _, _ = oracle.query(dim, res, order, C, coefs, pts)
    G = oracle.query_gradscale(dim, res, order, C, coefs, pts)
    assert G.shape == gx.shape
    assert (G >= np.abs(gx) - 1e-9 * (1 + G)).all()
    assert (G > 1.5 * np.abs(gx)).any()                 # random signs do cancel somewhere
    np.testing.assert_allclose(oracle.query_gradscale(dim, res, order, C, -2.0 * coefs, pts), 2.0 * G, rtol=1e-12)
    j = np.stack(np.meshgrid(*[np.arange(res)] * dim, indexing="ij")[::-1], -1).reshape(-1, dim)  # x fastest
    for a in range(dim):
        sign = np.where(j[:, a] % 2 == 1, 1.0, -1.0)
        f0 = (sign[:, None] * np.abs(r.normal(size=(res ** dim, C)))).reshape(-1)
        _, g0, _, _ = oracle.query(dim, res, 0, C, f0, pts)
        G0 = oracle.query_gradscale(dim, res, 0, C, f0, pts)
        np.testing.assert_allclose(G0[..., a], np.abs(g0[..., a]), rtol=1e-12)


# --------------------------------------------------------------------------
# BF16 rounding of the Adam moments (the BF16 / FP16 storage form)
# --------------------------------------------------------------------------
def test_bf16_round_matches_torch_conversion():
    """The oracle's rounding to BF16 equals torch's float32 -> bfloat16 conversion (nearest, ties to even) on
    FP32 values: random normals over many magnitudes, exact ties, BF16 subnormals and values that are already
    BF16."""
    r = rng(95)
    x = (r.standard_normal(4000) * 10.0 ** r.uniform(-30, 30, 4000)).astype(np.float32)
    bits = r.integers(0, 2 ** 16, 500, dtype=np.uint32) << np.uint32(16)
    ties = (bits | np.uint32(0x8000)).view(np.float32)                    # exactly half way between BF16 values
    sub = (r.standard_normal(500) * 1e-39).astype(np.float32)             # FP32 subnormals: BF16 subnormals too
    exact = bits.view(np.float32)
    x = np.concatenate([x, ties, sub, exact, np.float32([0.0, -0.0, 1.0, -2.5])])
    x = x[np.isfinite(x)]
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = oracle.bf16_round(x.astype(np.float64))
    np.testing.assert_array_equal(got, want)


def test_adam_with_bf16_moments_reduces_to_adam_when_moments_are_representable():
    """With gradients that keep every moment exactly representable in BF16 (a constant gradient 2^k: m and v
    are sums of few powers of two scaled by the betas only when the betas are powers of two), the BF16-moment
    step equals the plain step; with generic gradients the moments differ from plain Adam's by at most half a
    BF16 unit in the last place of the rounded value."""
    n = 64
    p = np.linspace(-1, 1, n)
    pa, pb = p.copy(), p.copy()
    ma, va, mb, vb = (np.zeros(n) for _ in range(4))
    for step in range(1, 4):
        g = np.full(n, 0.25)
        oracle.adam(pa, g.copy(), ma, va, 1e-2, 0.5, 0.75, 1e-8, step)
        oracle.adam(pb, g.copy(), mb, vb, 1e-2, 0.5, 0.75, 1e-8, step, bf16_moments=True)
        np.testing.assert_array_equal(ma, mb)
        np.testing.assert_array_equal(va, vb)
        np.testing.assert_array_equal(pa, pb)
    r = rng(96)
    m0, v0 = r.normal(size=n), r.random(n)
    g = r.normal(size=n)
    mc, vc, md, vd = m0.copy(), v0.copy(), m0.copy(), v0.copy()
    oracle.adam(p.copy(), g.copy(), mc, vc, 1e-2, step=3)
    oracle.adam(p.copy(), g.copy(), md, vd, 1e-2, step=3, bf16_moments=True)
    np.testing.assert_array_equal(md, oracle.bf16_round(mc))
    np.testing.assert_array_equal(vd, oracle.bf16_round(vc))
    assert (np.abs(md - mc) <= np.abs(mc) * 2.0 ** -8).all()
