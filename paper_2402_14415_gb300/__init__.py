"""GB300-native TaylorGrid field engine (arXiv 2402.14415).

The CUDA library ``libtaylorgrid.so`` (sources in ``csrc/``, ABI in
``include/taylorgrid.h``) holds every kernel of the path; this package is
its thin Python binding (``binding``, ctypes argument marshalling), the
torch.autograd front end over the same calls (``autograd``: TaylorGridField,
TaylorRadianceField) and a small SDF fitting loop (``fit``). There is no CPU
fallback.
"""
from .binding import (  # noqa: F401
    DeviceShape, Server, tg_render_rays, tg_sample_sdf_points, tg_sdf_error, tg_sdf_eval_target, tg_sdf_step,
    TG_BF16, TG_F16, TG_F32, Batch, Grid, TGError, exported_symbols, load, tg_adam_step, tg_adam_step_lazy,
    tg_batch_bin,
    tg_batch_create, tg_batch_gather, tg_batch_order, tg_batch_scatter, tg_batch_points, tg_batch_timeouts,
    tg_grid_timeouts, tg_noalloc_timeouts, tg_inject_alloc_failures, tg_measure_fp32_peak,
    TG_ORDER_BINNED, TG_ORDER_INPUT, tg_create, tg_get_coefs, tg_locate, tg_query, tg_query_backward,
    tg_query_backward_binned, tg_query_binned, tg_query_noalloc, tg_load, tg_render_rays_backward, tg_resample,
    tg_save, tg_sdf_iou, tg_set_coefs, tg_tv_step, tg_extract_mesh, tg_sample_mesh, tg_chamfer,
)


def build(force: bool = False, verbose: bool = False) -> str:
    from .builder import build as _build
    return _build(force=force, verbose=verbose)
