"""Canary padding around every caller-owned output buffer: each call writes only inside the buffer it is given.

A buffer is the middle of a larger allocation whose 64 leading and trailing 32-bit words hold a NaN
pattern; after the call (and a synchronize) the pattern must be intact. Sizes are ragged so that
vectorised tails are exercised.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from parity import to_dev

pytestmark = pytest.mark.gpu

PAD = 64                                      # 32-bit words: keeps the view 256-byte aligned
CANARY = 0x7FC0DEAD                           # a NaN bit pattern


class Padded:
    """A device buffer of `shape` with canary words before and after it."""

    def __init__(self, shape, dtype=torch.float32, fill=0.0):
        words = int(np.prod(shape)) * (2 if dtype == torch.float64 else 1)
        self.raw = torch.full((words + 2 * PAD,), CANARY, device="cuda", dtype=torch.int32)
        self.t = self.raw[PAD:PAD + words].view(dtype).view(shape)
        self.t.fill_(fill)

    def intact(self):
        torch.cuda.synchronize()
        r = self.raw.cpu()
        return bool((r[:PAD] == CANARY).all() and (r[-PAD:] == CANARY).all())


def test_query_paths_write_only_their_buffers(tg):
    res, N = 22, 300001                          # ragged: 16-byte vector tails, above the binning threshold
    g = tg.tg_create(3, res, 2, 1, "f32", seed=1, init_std=0.5)
    P = to_dev(W.uniform_points(60, N))
    U = torch.randn((N, 1), device="cuda")
    out, gx = Padded((N, 1)), Padded((N, 1, 3))
    tg.tg_query(g, P, out=out.t, grad_x=gx.t)                       # binned inside the call
    assert out.intact() and gx.intact()
    out2 = Padded((1001, 1))
    tg.tg_query(g, P[:1001], out=out2.t)                            # point-parallel
    assert out2.intact()
    grad = Padded((g.n_coefs,))
    tg.tg_query_backward(g, P, U, grad.t)
    assert grad.intact()
    batch = tg.tg_batch_create(3, res, N)
    tg.tg_batch_bin(batch, P)
    for binned in (False, True):
        o = Padded((N, 1))
        tg.tg_query_binned(g, batch, out=o.t, binned_order=binned)
        assert o.intact()
        gr = Padded((g.n_coefs,))
        tg.tg_query_backward_binned(g, batch, U, gr.t, binned_order=binned, deterministic=binned)
        assert gr.intact()


def test_optimiser_regulariser_and_mesh_calls_write_only_their_buffers(tg):
    g = tg.tg_create(3, 13, 2, 1, "f32", seed=2, init_std=0.5)
    for step_fn in (tg.tg_adam_step, tg.tg_adam_step_lazy):
        grad = Padded((g.n_coefs,), fill=0.5)
        step_fn(g, grad.t, lr=1e-3, step=1)
        assert grad.intact()
    grad, loss = Padded((g.n_coefs,)), Padded((1,))
    tg.tg_tv_step(g, 1e-3, grad.t, loss.t)
    assert grad.intact() and loss.intact()
    _, count = tg.tg_extract_mesh(g, 17, 0.0, max_tris=0)
    assert count > 10
    tris = Padded((count // 2, 3, 3))                                # capacity below the count
    n = torch.zeros(1, device="cuda", dtype=torch.int64)
    lib = tg.load()
    assert lib.tg_extract_mesh(g.handle, 17, ctypes.c_float(0.0), tris.t.data_ptr(), count // 2, n.data_ptr(),
                               None) == 0
    assert tris.intact() and int(n.item()) == count
    pts = Padded((777, 3))
    lib.tg_sample_mesh(tris.t.data_ptr(), n.data_ptr(), count // 2, 777, 5, pts.t.data_ptr(), None)
    assert pts.intact()
    sums = Padded((2,), dtype=torch.float64)
    A, B = torch.rand((333, 3), device="cuda"), torch.rand((555, 3), device="cuda")
    assert lib.tg_chamfer(A.data_ptr(), 333, B.data_ptr(), 555, sums.t.data_ptr(), None) == 0
    assert sums.intact()


def test_sdf_and_render_calls_write_only_their_buffers(tg):
    shape = W.union_shape(1)
    dsh = tg.DeviceShape(shape.spheres, shape.boxes, shape.area_cdf())
    g = tg.tg_create(3, 24, 2, 1, "f32", seed=3, init_std=1e-3)
    batch = tg.tg_batch_create(3, 24, 5003)
    grad, loss = Padded((g.n_coefs,)), Padded((2,))
    tg.tg_sdf_step(g, batch, dsh, grad.t, loss.t, n=5003, seed=1, step=0, lambda_eik=0.1, k_weight=50.0)
    assert grad.intact() and loss.intact()
    pts = Padded((5003, 3))
    tg.tg_sample_sdf_points(dsh, 1, 0, 5003, out=pts.t)
    assert pts.intact()
    dens = tg.tg_create(3, 20, 2, 1, "bf16", seed=4, init_std=0.1)
    col = tg.tg_create(3, 20, 1, 3, "bf16", seed=5, init_std=0.1)
    R, S = 301, 24
    o, d = W.random_rays(6, R)
    O, D = to_dev(o), to_dev(d)
    tgt = torch.rand((R, 3), device="cuda")
    rb = tg.tg_batch_create(3, 20, R * S)
    rgb, dg, cg, ls = Padded((R, 3)), Padded((dens.n_coefs,)), Padded((col.n_coefs,)), Padded((1,))
    tg.tg_render_rays(dens, col, O, D, S, seed=2, target=tgt, batch=rb, density_grad=dg.t, color_grad=cg.t,
                      loss_sum=ls.t, out=rgb.t)
    assert rgb.intact() and dg.intact() and cg.intact() and ls.intact()
