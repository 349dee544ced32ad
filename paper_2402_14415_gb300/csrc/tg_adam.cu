// Fused Adam step over every coefficient of a grid (one HBM pass).
// Reads master, gradient and both moments; writes master, moments, the
// BF16/FP16 stored copy, and zeroes the gradient for the next step.
#include "tg_adam.cuh"

namespace tg {

// Vectorised body over n4 = n / 4 float4 groups, scalar tail handled by block 0.
// T: stored copy (float: none); M: moment storage (FP32, or BF16 rounded to
// nearest even after every update, the arithmetic in FP32).
template <typename T, bool LAZY = false, typename M = float>
__global__ void __launch_bounds__(256)
adam_kernel(float *__restrict__ p, float *__restrict__ g, M *__restrict__ m, M *__restrict__ v,
            T *__restrict__ shadow, int64_t n, AdamCoef a, const int64_t *__restrict__ step_dev, float lr)
{
    if (step_dev) {   // bias corrections of the 1-based step *step_dev + 1, read on the device
        const float t = (float)(*step_dev + 1);
        a.step_size = lr / (1.0f - powf(a.beta1, t));
        a.inv_sqrt_bc2 = rsqrtf(1.0f - powf(a.beta2, t));
    }
    const int64_t n4 = n >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float4 *p4 = reinterpret_cast<float4 *>(p);
    float4 *g4 = reinterpret_cast<float4 *>(g);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n4; j += stride) {
        const float4 gg = __ldcs(g4 + j);
        if (LAZY && gg.x == 0.f && gg.y == 0.f && gg.z == 0.f && gg.w == 0.f) continue;
        float4 pp = p4[j], mm = Moments<M>::load(m, j), vv = Moments<M>::load(v, j);
        if (LAZY) {
            adam_lazy_one(pp.x, gg.x, mm.x, vv.x, a);
            adam_lazy_one(pp.y, gg.y, mm.y, vv.y, a);
            adam_lazy_one(pp.z, gg.z, mm.z, vv.z, a);
            adam_lazy_one(pp.w, gg.w, mm.w, vv.w, a);
        } else {
            adam_one(pp.x, gg.x, mm.x, vv.x, a);
            adam_one(pp.y, gg.y, mm.y, vv.y, a);
            adam_one(pp.z, gg.z, mm.z, vv.z, a);
            adam_one(pp.w, gg.w, mm.w, vv.w, a);
        }
        p4[j] = pp;
        Moments<M>::store(m, j, mm);
        Moments<M>::store(v, j, vv);
        __stcs(g4 + j, make_float4(0.f, 0.f, 0.f, 0.f));
        if (shadow) store4<T>(shadow, 4 * j, pp.x, pp.y, pp.z, pp.w);
    }
    if (blockIdx.x == 0) {
        for (int64_t j = 4 * n4 + threadIdx.x; j < n; j += blockDim.x) {
            if (LAZY && g[j] == 0.f) continue;
            float pp = p[j], mm = Moments<M>::get(m, j), vv = Moments<M>::get(v, j);
            adam_one(pp, g[j], mm, vv, a);
            p[j] = pp;
            Moments<M>::put(m, j, mm);
            Moments<M>::put(v, j, vv);
            g[j] = 0.0f;
            if (shadow) shadow[j] = from_f32<T>(pp);
        }
    }
}

tg_status ensure_adam_state(tg_grid *g)
{
    if (g->adam_m) return TG_OK;
    const size_t mb = (size_t)g->ncoef * moment_bytes(g) + 16;
    tg_status st = dev_alloc(&g->adam_m, mb, "tg_adam_step: cudaMalloc(m)");
    if (st == TG_OK) st = dev_alloc(&g->adam_v, mb, "tg_adam_step: cudaMalloc(v)");
    if (st == TG_OK) st = cuda_status(cudaMemset(g->adam_m, 0, mb), "tg_adam_step: zero m");
    if (st == TG_OK) st = cuda_status(cudaMemset(g->adam_v, 0, mb), "tg_adam_step: zero v");
    if (st == TG_OK) st = cuda_status(cudaDeviceSynchronize(), "tg_adam_step: init moments");
    if (st != TG_OK) {
        cudaFree(g->adam_m); cudaFree(g->adam_v);
        g->adam_m = g->adam_v = nullptr;
    }
    return st;
}

}  // namespace tg

using namespace tg;

namespace tg {


// Adam over all coefficients; with step_dev the 0-based step index is read on
// the device (for replayable CUDA graphs) and prm->step is ignored.
tg_status adam_launch(tg_grid *g, float *grad, const tg_adam *prm, const int64_t *step_dev, cudaStream_t s, bool lazy)
{
    tg_status st = ensure_adam_state(g);
    if (st != TG_OK) return st;
    const double step = step_dev ? 1.0 : (double)prm->step;
    const double b1t = 1.0 - pow((double)prm->beta1, step);
    const double b2t = 1.0 - pow((double)prm->beta2, step);
    AdamCoef a;
    a.beta1 = prm->beta1; a.beta2 = prm->beta2;
    a.one_m_b1 = 1.0f - prm->beta1; a.one_m_b2 = 1.0f - prm->beta2;
    a.step_size = (float)((double)prm->lr / b1t);
    a.inv_sqrt_bc2 = (float)(1.0 / sqrt(b2t));
    a.eps = prm->eps;
    const int64_t n4 = g->ncoef / 4;
    int per_sm = blocks_per_sm((const void *)adam_kernel<float>, 256, 0);
    int64_t need = (n4 + 255) / 256;
    int64_t cap = (int64_t)num_sms() * per_sm;
    unsigned nb = (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
#define TG_ADAM(T, L, SH)                                                                                       \
    (g->lp_moments ? adam_kernel<T, L, __nv_bfloat16><<<nb, 256, 0, s>>>(                                       \
                         g->master, grad, (__nv_bfloat16 *)g->adam_m, (__nv_bfloat16 *)g->adam_v, SH, g->ncoef, a, \
                         step_dev, prm->lr)                                                                     \
                   : adam_kernel<T, L, float><<<nb, 256, 0, s>>>(g->master, grad, (float *)g->adam_m,             \
                                                                 (float *)g->adam_v, SH, g->ncoef, a, step_dev, \
                                                                 prm->lr))
    if (g->dtype == TG_F32) {
        if (lazy) TG_ADAM(float, true, nullptr);
        else TG_ADAM(float, false, nullptr);
    } else if (g->dtype == TG_BF16) {
        if (lazy) TG_ADAM(__nv_bfloat16, true, (__nv_bfloat16 *)g->store);
        else TG_ADAM(__nv_bfloat16, false, (__nv_bfloat16 *)g->store);
    } else {
        if (lazy) TG_ADAM(__half, true, (__half *)g->store);
        else TG_ADAM(__half, false, (__half *)g->store);
    }
#undef TG_ADAM
    return launch_status(lazy ? "tg_adam_step_lazy" : "tg_adam_step");
}

}  // namespace tg

static tg_status adam_entry(tg_grid *g, float *grad, const tg_adam *prm, tg_stream stream, bool lazy)
{
    const char *name = lazy ? "tg_adam_step_lazy" : "tg_adam_step";
    if (!g || !grad || !prm) return fail(TG_EINVAL, "%s: NULL argument", name);
    if (prm->step < 1) return fail(TG_EINVAL, "%s: step must be >= 1", name);
    if (!(prm->beta1 >= 0.f && prm->beta1 < 1.f && prm->beta2 >= 0.f && prm->beta2 < 1.f && prm->eps >= 0.f))
        return fail(TG_EINVAL, "%s: betas must lie in [0,1) and eps >= 0", name);
    if (((uintptr_t)grad & 15) != 0) return fail(TG_EINVAL, "%s: coef_grad must be 16-byte aligned", name);
    return adam_launch(g, grad, prm, nullptr, (cudaStream_t)stream, lazy);
}

extern "C" tg_status tg_adam_step(tg_grid *g, float *grad, const tg_adam *prm, tg_stream stream)
{
    return adam_entry(g, grad, prm, stream, false);
}

extern "C" tg_status tg_adam_step_lazy(tg_grid *g, float *grad, const tg_adam *prm, tg_stream stream)
{
    return adam_entry(g, grad, prm, stream, true);
}
