"""Mesh extraction (marching tetrahedra), mesh sampling and the Chamfer distance against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from parity import to_dev

pytestmark = pytest.mark.gpu


def sphere_taylor(res, c, r):
    """Order-2 Taylor data (world units, exchange layout) of the sphere SDF |x - c| - r at every vertex."""
    h = 1.0 / (res - 1)
    idx = np.arange(res ** 3)
    X = np.stack([(idx // res ** d) % res for d in range(3)], 1) * h - np.asarray(c)
    d = np.linalg.norm(X, axis=1)
    n = X / d[:, None]
    H = (np.eye(3)[None] - n[:, :, None] * n[:, None, :]) / d[:, None, None]
    out = np.zeros((res ** 3, 10))
    out[:, 0] = d - r
    out[:, 1:4] = n
    out[:, 4:7] = H[:, [0, 1, 2], [0, 1, 2]]
    out[:, 7:10] = np.stack([H[:, 0, 1], H[:, 0, 2], H[:, 1, 2]], 1)
    return out.reshape(-1)


def iso_with_margin(vals, scale):
    """An iso level whose distance to every lattice value is at least 2e-4 scale, so the inside / outside
    decisions of the FP32 lattice and of the FP64 oracle agree (their values differ by about 1e-7 scale)."""
    for iso in np.linspace(-0.05, 0.05, 41) * scale:
        if np.abs(vals - iso).min() > 2e-4 * scale:
            return float(iso)
    raise AssertionError("no iso level with a margin")


def quantized_coefs(res, seed):
    """Order-0 coefficients in {-1.5, -0.5, 0.5, 1.5}: on the lattice of the grid's own vertices every value
    lies at least 0.5 from 0."""
    return np.random.default_rng(seed).choice([-1.5, -0.5, 0.5, 1.5], size=res ** 3)


@pytest.mark.parametrize("res,order,M", [(70, 0, 70), (5, 2, 11), (6, 1, 13), (4, 2, 9)])
def test_extract_mesh_matches_oracle(tg, res, order, M):
    """The same triangles in the same order (rows of 69 cubes span three warp chunks), positions within the
    interpolation error that the margin bounds, and the same facing. A quantized order-0 field on its own
    vertex lattice, and random order-1/2 fields (many surface components, faces on the domain boundary)."""
    if M == res:
        coefs = quantized_coefs(res, 22)
    else:
        coefs = W.init_coefs(3, res, order, 1, seed=21 + order, std=0.5)
    g = tg.tg_create(3, res, order, 1, "f32")
    tg.tg_set_coefs(g, to_dev(coefs))
    vals = oracle.lattice_values(res, order, 1, coefs.astype(np.float64), M)
    iso = iso_with_margin(vals, np.abs(vals).max())
    want = oracle.marching_tets(M, vals, iso)
    got, count = tg.tg_extract_mesh(g, M, iso)
    assert count == want.shape[0] > 0
    got = got.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-4)
    ng = np.cross(got[:, 1] - got[:, 0], got[:, 2] - got[:, 0])
    nw = np.cross(want[:, 1] - want[:, 0], want[:, 2] - want[:, 0])
    big = np.linalg.norm(nw, axis=1) > 1e-6
    assert ((ng * nw).sum(1)[big] > 0).all()


def test_extract_mesh_capacity_and_empty(tg):
    coefs = W.init_coefs(3, 9, 2, 1, seed=30, std=0.5)
    g = tg.tg_create(3, 9, 2, 1, "f32")
    tg.tg_set_coefs(g, to_dev(coefs))
    full, count = tg.tg_extract_mesh(g, 20, 0.0)
    part, count2 = tg.tg_extract_mesh(g, 20, 0.0, max_tris=count // 3)
    assert count2 == count and part.shape[0] == count // 3
    assert torch.equal(part, full[:count // 3])
    high = float(np.abs(coefs).sum()) + 1.0            # above every value of the field
    empty, c0 = tg.tg_extract_mesh(g, 20, high)
    assert c0 == 0 and empty.shape[0] == 0
    pts = tg.tg_sample_mesh(empty, 16, seed=1)
    assert not pts.any()


def test_sphere_mesh_is_closed_and_accurate(tg):
    """The Taylor data of a sphere SDF (order 2, 33^3): the extracted surface at M = 97 is closed and
    consistently oriented, and its area and enclosed volume are those of the sphere within 1 %."""
    res, M, c, r = 33, 97, (0.5, 0.47, 0.52), 0.31
    g = tg.tg_create(3, res, 2, 1, "f32")
    tg.tg_set_coefs(g, to_dev(sphere_taylor(res, c, r)))
    T, count = tg.tg_extract_mesh(g, M, 0.0)
    T = T.cpu().numpy().astype(np.float64)
    area = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1).sum()
    vol = (T[:, 0] * np.cross(T[:, 1], T[:, 2])).sum() / 6.0
    assert abs(area / (4 * np.pi * r * r) - 1) < 0.01
    assert abs(vol / (4 / 3 * np.pi * r ** 3) - 1) < 0.01
    # closed and oriented: every directed edge once, and its reverse once (bit-identical shared vertices)
    V = T.astype(np.float32).view(np.int32).reshape(-1, 3, 3)
    e = np.concatenate([np.concatenate([V[:, a], V[:, b]], 1) for a, b in ((0, 1), (1, 2), (2, 0))])
    fwd = {tuple(x) for x in e}
    assert len(fwd) == e.shape[0]
    rev = {tuple(np.concatenate([x[3:], x[:3]])) for x in e}
    assert fwd == rev


def test_sample_mesh_matches_oracle(tg):
    vals = oracle.lattice_values(24, 0, 1, quantized_coefs(24, 31), 24)
    T = oracle.marching_tets(24, vals, 0.0).astype(np.float32)
    n = 5000
    got = tg.tg_sample_mesh(to_dev(T), n, seed=11).cpu().numpy()
    want = oracle.sample_mesh(T, n, seed=11)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-6)


@pytest.mark.parametrize("nA,nB", [(5000, 7000), (3000, 1), (1, 2049), (0, 100)])
def test_chamfer_matches_oracle(tg, nA, nB):
    r = np.random.default_rng(nA + nB)
    A = r.random((nA, 3)).astype(np.float32)
    B = r.random((nB, 3)).astype(np.float32)
    got = tg.tg_chamfer(to_dev(A), to_dev(B))
    want = oracle.chamfer(A, B) if nA else (0.0, 0.0)
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-12)
