"""The torch.autograd front end: TaylorGridField and TaylorRadianceField.

The coefficient gradients autograd produces come from the library's backward
kernels; they are checked against central differences (exact up to rounding,
because f is linear in the coefficients), against the direct C-ABI calls and
against the FP64 oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from parity import check_coef_grad, to_dev

pytestmark = pytest.mark.gpu


def field(tg, res, order, C=1, dtype="f32", binned_min_points=1 << 16):
    from paper_2402_14415_gb300.autograd import TaylorGridField
    m = TaylorGridField(3, res, order, C, dtype, seed=3, init_std=0.5, binned_min_points=binned_min_points)
    return m


@pytest.mark.parametrize("binned_min", [1 << 30, 1])        # point-parallel kernels, then the binned ones
def test_coefficient_gradient_equals_central_differences(tg, binned_min):
    res, order = 12, 2
    m = field(tg, res, order, binned_min_points=binned_min)
    pts = to_dev(W.uniform_points(21, 20000))
    w = torch.randn((pts.shape[0], 1), device="cuda")
    loss = (w * m(pts)).sum()
    loss.backward()
    g = m.coefs.grad.clone()
    d = torch.randn_like(g)
    eps = 1e-2                                 # any step is exact for a linear function; rounding sets the floor
    with torch.no_grad():
        base = m.coefs.detach().clone()
        m.coefs.copy_(base + eps * d)
        fp = m(pts)
        lp = (w.double() * fp.double()).sum().item()
        m.coefs.copy_(base - eps * d)
        fm = m(pts)
        lm = (w.double() * fm.double()).sum().item()
        m.coefs.copy_(base)
    fd = (lp - lm) / (2 * eps)
    an = float((g.double() * d.double()).sum())
    # FP32 rounding of f (relative 1e-6 of its magnitude) divided by the step bounds the difference
    floor = 1e-6 * float((w.abs() * (fp.abs() + fm.abs())).sum()) / (2 * eps)
    assert abs(an - fd) <= 1e-4 * abs(fd) + floor, (an, fd, floor)


def test_eikonal_style_loss_matches_c_abi_and_oracle(tg):
    res, order = 10, 2
    m = field(tg, res, order, binned_min_points=1)
    pts_np = W.uniform_points(22, 30000)
    pts = to_dev(pts_np)
    f, gx = m(pts, want_grad=True)
    loss = (f[:, 0] - 0.1).abs().mean() + 0.1 * ((gx[:, 0].norm(dim=-1) - 1) ** 2).mean()
    uf, ug = torch.autograd.grad(loss, [f, gx], retain_graph=True)
    loss.backward()
    got = m.coefs.grad.clone()
    direct = torch.zeros_like(got)
    tg.tg_query_backward(m.grid, pts, uf.contiguous(), direct, dL_dgradx=ug.contiguous())
    torch.testing.assert_close(got, direct, rtol=1e-4, atol=1e-4 * float(direct.abs().max()))
    check_coef_grad(got.cpu().numpy(), 3, res, order, 1, pts_np, uf.cpu().numpy(), ug.cpu().numpy())


def test_point_gradient_is_the_spatial_gradient(tg):
    res, order = 9, 2
    m = field(tg, res, order)
    x = W.uniform_points(23, 4000) * 0.98 + 0.01
    pts = to_dev(x).requires_grad_(True)
    f = m(pts)
    f.sum().backward()
    _, gx = tg.tg_query(m.grid, to_dev(x), want_grad=True)
    torch.testing.assert_close(pts.grad, gx[:, 0], rtol=0, atol=0)
    # and against central differences of the field inside the cell
    h = 1e-3
    with torch.no_grad():
        for e in range(3):
            dx = np.zeros(3, dtype=np.float32); dx[e] = h
            fp = tg.tg_query(m.grid, to_dev(x + dx))[:, 0]
            fm = tg.tg_query(m.grid, to_dev(x - dx))[:, 0]
            fd = ((fp - fm) / (2 * h)).cpu().numpy()
            same_cell = (np.floor((x[:, e] + h) * (res - 1)) == np.floor((x[:, e] - h) * (res - 1)))
            err = np.abs(fd - pts.grad[:, e].cpu().numpy())[same_cell]
            assert np.percentile(err, 99) < 2e-2 * np.abs(fd).max(), np.percentile(err, 99)


def test_adam_step_through_the_module_matches_c_abi(tg):
    res, order = 8, 1
    a = field(tg, res, order)
    b = tg.tg_create(3, res, order, 1, "f32")
    tg.tg_set_coefs(b, a.coefs.detach().clone())
    pts = to_dev(W.uniform_points(24, 5000))
    a(pts).pow(2).sum().backward()
    g = a.coefs.grad.clone()
    a.adam_step(lr=1e-2, step=1)
    tg.tg_adam_step(b, g, lr=1e-2, step=1)
    torch.testing.assert_close(a.coefs.detach(), tg.tg_get_coefs(b, which=1), rtol=0, atol=0)
    assert float(a.coefs.grad.abs().max()) == 0.0           # the fused step zeroes the gradient


def test_bf16_storage_follows_an_outside_optimiser(tg):
    m = field(tg, 8, 2, dtype="bf16")
    opt = torch.optim.SGD(m.parameters(), lr=0.1)
    pts = to_dev(W.uniform_points(25, 5000))
    m(pts).sum().backward()
    opt.step()
    m.refresh_storage()
    stored = tg.tg_get_coefs(m.grid, which=0)
    torch.testing.assert_close(stored, m.coefs.detach().to(torch.bfloat16).float(), rtol=0, atol=0)


def test_render_autograd_matches_the_fused_training_call(tg):
    from paper_2402_14415_gb300.autograd import TaylorRadianceField
    res, S, R = 12, 64, 300
    fld = TaylorRadianceField(res, dtype="f32", seed=5, init_std=0.3, max_samples=R * S)
    o, d = W.random_rays(7, R)
    ro, rd = to_dev(o), to_dev(d)
    target = torch.rand((R, 3), device="cuda")
    rgb = fld(ro, rd, S=S, seed=9)
    loss = ((rgb - target) ** 2).sum(1).mean()
    loss.backward()
    batch = tg.tg_batch_create(3, res, R * S)
    dg = torch.zeros(fld.density.grid.n_coefs, device="cuda")
    cg = torch.zeros(fld.color.grid.n_coefs, device="cuda")
    lsum = torch.zeros(1, device="cuda")
    rgb2 = tg.tg_render_rays(fld.density.grid, fld.color.grid, ro, rd, S=S, seed=9, target=target, batch=batch,
                             density_grad=dg, color_grad=cg, loss_sum=lsum)
    torch.testing.assert_close(rgb, rgb2, rtol=0, atol=0)
    np.testing.assert_allclose(loss.item(), lsum.item() / R, rtol=1e-5)
    for got, ref in ((fld.density.coefs.grad, dg), (fld.color.coefs.grad, cg)):
        torch.testing.assert_close(got, ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))
