// Internal interface of the SDF fitting pieces (tg_sdf.cu) used by the server.
#pragma once

#include "tg_binned.cuh"

namespace tg {

struct ShapeView {
    int ns, nb;
    const float *sph, *box, *cdf;
};

tg_status shape_view(const tg_shape *s, ShapeView *v, const char *who);

// One SDF fitting step; with step_dev != nullptr the sampler reads the step
// index on the device (for replayable CUDA graphs).
tg_status sdf_step_impl(const tg_grid *g, tg_batch *bt, const ShapeView &s, const float *pts, int64_t N,
                        uint64_t seed, int64_t step, const int64_t *step_dev, float lambda_eik, float k_weight,
                        float *coef_grad, float *loss_sums, cudaStream_t cs);

// sum |f - d| over points into err_sum; skipped on the device when *gate == 0.
tg_status sdf_error_impl(const tg_grid *g, const ShapeView &s, const float *pts, int64_t N, float *err_sum,
                         const int *gate, cudaStream_t cs, unsigned long long *iou = nullptr);

}  // namespace tg
