"""GPU parity of differentiable ray marching (Sec. 3.3, Eq. 9 - Eq. 11) with the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from parity import to_dev

pytestmark = pytest.mark.gpu


def rays(n, seed=5):
    o, d = W.random_rays(seed, n, radius=1.3, spread=0.45)
    # add an axis-aligned ray, a ray that starts inside the cube and a miss
    extra_o = np.array([[-0.5, 0.37, 0.61], [0.4, 0.5, 0.6], [2.0, 2.0, 2.0]], np.float32)
    extra_d = np.array([[1, 0, 0], [0.6, 0.0, 0.8], [1, 0, 0]], np.float32)
    return np.concatenate([o, extra_o]), np.concatenate([d, extra_d])


def grids(tg, res, dtype="f32", seed=3):
    dco = W.init_coefs(3, res, 2, 1, seed=seed, std=1.0) + 0.5
    cco = W.init_coefs(3, res, 1, 3, seed=seed + 1, std=0.8)
    dg = tg.tg_create(3, res, 2, 1, dtype)
    cg = tg.tg_create(3, res, 1, 3, dtype)
    tg.tg_set_coefs(dg, to_dev(dco))
    tg.tg_set_coefs(cg, to_dev(cco))
    return dg, cg, dco, cco


@pytest.mark.parametrize("S", [32, 100, 256, 384, 512])      # up to 8 and up to 16 samples a lane
def test_render_forward_matches_oracle(tg, S):
    res = 10
    dg, cg, dco, cco = grids(tg, res)
    o, d = rays(200)
    rgb = tg.tg_render_rays(dg, cg, to_dev(o), to_dev(d), S=S, seed=9).cpu().numpy()
    ref = oracle.render(res, 2, dco, 1, cco, o, d, S, seed=9)
    np.testing.assert_allclose(rgb, ref, atol=1e-5)
    np.testing.assert_allclose(rgb[-1], [1, 1, 1])              # the miss renders the background


def test_render_homogeneous_closed_form(tg):
    res, S = 6, 64
    f0, g0 = 0.7, np.array([-0.3, 0.1, 0.9])
    dg = tg.tg_create(3, res, 0, 1, "f32")
    cg = tg.tg_create(3, res, 0, 3, "f32")
    tg.tg_set_coefs(dg, to_dev(np.full(res ** 3, f0, np.float32)))
    tg.tg_set_coefs(cg, to_dev(np.tile(g0, res ** 3).astype(np.float32)))
    o, d = rays(50, seed=8)
    rgb = tg.tg_render_rays(dg, cg, to_dev(o), to_dev(d), S=S, seed=3, bg=1.0).cpu().numpy()
    sigma = math.log1p(math.exp(f0))
    c = 1 / (1 + np.exp(-g0))
    for r in range(o.shape[0]):
        hit, n, f = oracle.ray_box(o[r].astype(np.float64), d[r].astype(np.float64))
        if not hit:
            np.testing.assert_allclose(rgb[r], 1.0); continue
        t0 = n + float(W.uniform(3, r, 0)) * (f - n) / S
        T = math.exp(-sigma * (f - t0))
        np.testing.assert_allclose(rgb[r], c * (1 - T) + T, atol=2e-5)


@pytest.mark.parametrize("dtype,S", [("f32", 48), ("bf16", 48), ("f32", 256), ("bf16", 256), ("f32", 400)])
def test_render_training_gradients_match_oracle(tg, dtype, S):
    """Both coefficient gradients against the oracle's (Eq. 10 - Eq. 11 differentiated) at the scale-aware
    1e-4: |gpu - oracle| <= 1e-4 max(|oracle|, A), A the magnitude of the terms of that gradient. S = 256 is the
    configured sample count (8 samples per lane)."""
    res = 16
    dg, cg, dco, cco = grids(tg, res, dtype)
    dq = tg.tg_get_coefs(dg, which=0).cpu().numpy().astype(np.float64)
    cq = tg.tg_get_coefs(cg, which=0).cpu().numpy().astype(np.float64)
    o, d = rays(60, seed=11)
    R = o.shape[0]
    target = np.random.default_rng(2).random((R, 3)).astype(np.float32)
    batch = tg.tg_batch_create(3, res, R * S)
    dgrad = torch.zeros(dg.n_coefs, device="cuda")
    cgrad = torch.zeros(cg.n_coefs, device="cuda")
    loss = torch.zeros(1, device="cuda")
    rgb = tg.tg_render_rays(dg, cg, to_dev(o), to_dev(d), S=S, seed=4, target=to_dev(target), batch=batch,
                            density_grad=dgrad, color_grad=cgrad, loss_sum=loss)
    torch.cuda.synchronize()
    assert tg.tg_batch_timeouts(batch) == 0
    ref_rgb, ref_loss, ref_dg, ref_cg, abs_dg, abs_cg = oracle.render(res, 2, dq, 1, cq, o, d, S, seed=4,
                                                                      target=target, want_abs=True)
    np.testing.assert_allclose(rgb.cpu().numpy(), ref_rgb, atol=1e-5)
    np.testing.assert_allclose(loss.item() / R, ref_loss, rtol=1e-4, atol=1e-7)
    for name, got, ref, A in (("density", dgrad.cpu().numpy(), ref_dg, abs_dg),
                              ("colour", cgrad.cpu().numpy(), ref_cg, abs_cg)):
        tol = 1e-4 * np.maximum(np.abs(ref), A) + 1e-30
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (name, int(bad.sum()), np.argwhere(bad)[:5].ravel().tolist())
        assert (A > 0).sum() > 100                      # the rays touch many coefficients


def test_render_rejects_bad_arguments(tg):
    dg, cg, _, _ = grids(tg, 6)
    o, d = rays(4)
    with pytest.raises(tg.TGError):
        tg.tg_render_rays(dg, cg, to_dev(o), to_dev(d), S=513)
    with pytest.raises(tg.TGError):
        tg.tg_render_rays(cg, dg, to_dev(o), to_dev(d), S=16)


def test_benchmark_ground_truth_renderer_matches_oracle(tg):
    """bench.py renders the blob scene's training targets on the GPU; they follow the oracle's quadrature."""
    import bench
    scene = W.blob_scene(4)
    o, d = W.camera_rays(100, 16, 16, cams=[3, 57])
    o = np.concatenate([o, np.array([[2.0, 2.0, 2.0]], np.float32)])          # plus a ray that misses the cube
    d = np.concatenate([d, np.array([[0.0, 0.0, 1.0]], np.float32)])
    got = bench.blob_gt(scene, to_dev(o), to_dev(d), n_samples=256).cpu().numpy()
    ref = oracle.render_blobs(scene, o, d, n_samples=256)
    np.testing.assert_allclose(got, ref, atol=2e-4)
    np.testing.assert_allclose(got[-1], [1, 1, 1])
