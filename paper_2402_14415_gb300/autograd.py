"""torch.autograd front end of the TaylorGrid library.

`TaylorGridField` is a torch module around one library grid. Its `coefs`
parameter is a zero-copy view of the grid's FP32 master coefficients
(exchange layout), so the gradient torch accumulates in `coefs.grad` is the
coefficient gradient of Sec. 3.1's direct optimisation, computed by the
library's backward kernels (`tg_query_backward`, or the binned backward for
large 3-D batches). `TaylorRadianceField` pairs a density and a colour grid and
renders rays (Eq. 9 - Eq. 10); its backward calls `tg_render_rays_backward`,
which recomputes every sample instead of keeping per-sample intermediates.

Every operation runs in the CUDA library; this module only arranges
arguments and tensors. There is no CPU path.
"""
from __future__ import annotations

import torch

from . import binding as B

_ELEM = {B.TG_F32: 4, B.TG_BF16: 2, B.TG_F16: 2}


class _DeviceArray:
    """__cuda_array_interface__ of a library-owned FP32 array (kept alive by `owner`)."""

    def __init__(self, ptr: int, n: int, owner):
        self.owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def master_view(grid: B.Grid) -> torch.Tensor:
    """The grid's FP32 master coefficients as a torch tensor sharing their memory."""
    info = grid.info()
    return torch.as_tensor(_DeviceArray(info.master, grid.n_coefs, grid), device="cuda")


def binned_supported(grid: B.Grid) -> bool:
    """Whether the brick-binned kernels accept this grid (3-D, TMA row rules)."""
    if grid.dim != 3:
        return False
    nv, elem = grid.K * grid.channels, _ELEM[grid.dtype]
    row = (9 * nv * elem + 15) // 16 * 16 // elem
    return (grid.res * nv * elem) % 16 == 0 and row <= 256


class TaylorGridField(torch.nn.Module):
    """A TaylorGrid (Sec. 3.1) as a module: f(x) (and optionally grad_x f) with autograd.

    Batches of at least `binned_min_points` points on a 3-D grid go through the
    brick-binned kernels (binned once in the forward and reused by the
    backward); smaller ones through the point-parallel kernels.
    """

    def __init__(self, dim: int, res: int, order: int, channels: int = 1, dtype: str = "f32", seed: int = 0,
                 init_std: float = 1e-3, binned_min_points: int = 1 << 16):
        super().__init__()
        self.grid = B.tg_create(dim, res, order, channels, dtype, seed=seed, init_std=init_std)
        self.coefs = torch.nn.Parameter(master_view(self.grid))
        self.binned = binned_supported(self.grid)
        self.binned_min_points = binned_min_points
        self._batch = None
        self._bin_gen = 0

    # --- batches ------------------------------------------------------------
    def _bin(self, pts: torch.Tensor) -> int:
        N = pts.shape[0]
        if self._batch is None or self._batch.max_points < N:
            self._batch = B.tg_batch_create(3, self.grid.res, N)
        B.tg_batch_bin(self._batch, pts)
        self._bin_gen += 1
        return self._bin_gen

    def use_binned(self, n: int) -> bool:
        return self.binned and n >= self.binned_min_points

    # --- storage ------------------------------------------------------------
    @torch.no_grad()
    def refresh_storage(self):
        """After an optimiser outside the library changed `coefs`, round them into the stored copy."""
        B.tg_set_coefs(self.grid, self.coefs)

    @torch.no_grad()
    def adam_step(self, lr: float, step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        """Fused Adam on `coefs` with `coefs.grad` (which it zeroes), refreshing the stored copy."""
        if self.coefs.grad is None:
            return
        B.tg_adam_step(self.grid, self.coefs.grad, lr, step, beta1, beta2, eps)

    def forward(self, pts: torch.Tensor, want_grad: bool = False):
        return _QueryFn.apply(pts, self.coefs, self, want_grad)


class _QueryFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pts, coefs, mod: TaylorGridField, want_grad: bool):
        pts = pts.detach().contiguous()
        N = pts.shape[0]
        need_gx = want_grad or ctx.needs_input_grad[0]
        binned = mod.use_binned(N)
        if binned:
            gen = mod._bin(pts)
            out, gx = B.tg_query_binned(mod.grid, mod._batch, want_grad=True) if need_gx else \
                (B.tg_query_binned(mod.grid, mod._batch), None)
        else:
            gen = 0
            out, gx = B.tg_query(mod.grid, pts, want_grad=True) if need_gx else (B.tg_query(mod.grid, pts), None)
        ctx.mod, ctx.binned, ctx.gen, ctx.want_grad = mod, binned, gen, want_grad
        ctx.save_for_backward(pts, gx if ctx.needs_input_grad[0] else None)
        return (out, gx) if want_grad else out

    @staticmethod
    def backward(ctx, *grads):
        pts, gx = ctx.saved_tensors
        mod = ctx.mod
        dL_df = grads[0]
        dL_dgx = grads[1] if ctx.want_grad else None
        N, C = pts.shape[0], mod.grid.channels
        if dL_df is None:
            dL_df = torch.zeros((N, C), device=pts.device)
        dL_df = dL_df.reshape(N, C).contiguous().float()
        if dL_dgx is not None:
            dL_dgx = dL_dgx.reshape(N, C, mod.grid.dim).contiguous().float()
        grad_pts = grad_coefs = None
        if ctx.needs_input_grad[1]:
            grad_coefs = torch.zeros(mod.grid.n_coefs, device=pts.device)
            if ctx.binned:
                if mod._bin_gen != ctx.gen:                # the module's batch was re-binned since
                    mod._bin(pts)
                    ctx.gen = mod._bin_gen
                B.tg_query_backward_binned(mod.grid, mod._batch, dL_df, grad_coefs, dL_dgradx=dL_dgx)
            else:
                B.tg_query_backward(mod.grid, pts, dL_df, grad_coefs, dL_dgradx=dL_dgx)
        if ctx.needs_input_grad[0]:
            if dL_dgx is not None and bool(torch.any(dL_dgx != 0)):
                raise NotImplementedError("TaylorGridField: second derivatives with respect to the points "
                                          "(a loss on grad_x f that needs d/dx) are not implemented")
            inside = ((pts >= 0) & (pts <= 1)).float()       # queries clamp to the domain
            grad_pts = (dL_df.unsqueeze(-1) * gx).sum(1) * inside
        return grad_pts, grad_coefs, None, None


class TaylorRadianceField(torch.nn.Module):
    """Density (1 channel, sigma = softplus(f)) and colour (3 channels, sigmoid) grids rendered along rays.

    Eq. 10 in the forward; the backward recomputes every sample
    (`tg_render_rays_backward`) and scatters both coefficient gradients.
    """

    def __init__(self, res: int, density_order: int = 2, color_order: int = 1, dtype: str = "bf16", seed: int = 0,
                 init_std: float = 1e-3, max_samples: int = 8192 * 256):
        super().__init__()
        self.density = TaylorGridField(3, res, density_order, 1, dtype, seed=seed, init_std=init_std)
        self.color = TaylorGridField(3, res, color_order, 3, dtype, seed=seed + 1, init_std=init_std)
        self._batch = B.tg_batch_create(3, res, max_samples)

    def forward(self, rays_o, rays_d, S: int, seed: int = 0, ray_base: int = 0, bg: float = 1.0):
        return _RenderFn.apply(rays_o, rays_d, self.density.coefs, self.color.coefs, self, S, seed, ray_base, bg)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rays_o, rays_d, dcoefs, ccoefs, field: TaylorRadianceField, S, seed, ray_base, bg):
        rays_o, rays_d = rays_o.detach().contiguous(), rays_d.detach().contiguous()
        rgb = B.tg_render_rays(field.density.grid, field.color.grid, rays_o, rays_d, S=S, seed=seed,
                               ray_base=ray_base, bg=bg)
        ctx.field, ctx.S, ctx.seed, ctx.ray_base, ctx.bg = field, S, seed, ray_base, bg
        ctx.save_for_backward(rays_o, rays_d)
        return rgb

    @staticmethod
    def backward(ctx, dL_drgb):
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            raise NotImplementedError("TaylorRadianceField: gradients with respect to the rays are not implemented")
        rays_o, rays_d = ctx.saved_tensors
        f = ctx.field
        dgrad = torch.zeros(f.density.grid.n_coefs, device=rays_o.device)
        cgrad = torch.zeros(f.color.grid.n_coefs, device=rays_o.device)
        B.tg_render_rays_backward(f.density.grid, f.color.grid, rays_o, rays_d, dL_drgb.contiguous().float(), ctx.S,
                                  f._batch, dgrad, cgrad, seed=ctx.seed, ray_base=ctx.ray_base, bg=ctx.bg)
        return None, None, dgrad, cgrad, None, None, None, None, None
