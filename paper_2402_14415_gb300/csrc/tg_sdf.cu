// SDF fitting (Sec. 3.2): analytic targets, the device sampler of fit
// batches, the per-point loss (Eq. 6 with w = 1, eikonal term of Eq. 8) and
// the fitting step that composes binning, the binned forward with spatial
// gradients, the loss and the binned backward - all in binned order.
#include "tg_records.cuh"
#include "tg_sdf.cuh"

namespace tg {

tg_status shape_view(const tg_shape *s, ShapeView *v, const char *who)
{
    if (!s) return fail(TG_EINVAL, "%s: shape is NULL", who);
    if (s->n_spheres < 0 || s->n_boxes < 0 || s->n_spheres + s->n_boxes < 1 || s->n_spheres + s->n_boxes > 1024)
        return fail(TG_EINVAL, "%s: the shape needs 1..1024 members", who);
    if ((s->n_spheres && !s->spheres) || (s->n_boxes && !s->boxes)) return fail(TG_EINVAL, "%s: NULL member array", who);
    v->ns = s->n_spheres; v->nb = s->n_boxes; v->sph = s->spheres; v->box = s->boxes; v->cdf = s->area_cdf;
    return TG_OK;
}

__global__ void sdf_target_kernel(ShapeView s, const float *__restrict__ pts, int64_t N, float *__restrict__ d)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        d[n] = sdf_union(s, clamp01(pts[3 * n]), clamp01(pts[3 * n + 1]), clamp01(pts[3 * n + 2]));
}

// The fit batch of `step`, the same points as sample_sdf_point. The uniform
// half is one pass. For the surface half every lane runs a queue of its points
// with one candidate draw per iteration and moves to its next point as soon as
// the current one is accepted (or has used its 8 draws), so a lane whose point
// was accepted at once does not wait for the warp's slowest point.
__global__ void sdf_sample_kernel(ShapeView s, uint64_t seed, int64_t step, const int64_t *__restrict__ step_dev,
                                  int64_t N, float jitter, float *__restrict__ pts)
{
    constexpr uint64_t SLOTS = 16;
    if (step_dev) step = *step_dev;
    const int64_t n_uni = N / 2;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t base = (uint64_t)step * 256ull;
    const uint64_t key_u = stream_key(seed, base + 255ull);
    for (int64_t j = tid; j < n_uni; j += stride) {
        const uint64_t b = (uint64_t)j * SLOTS;
        pts[3 * j] = clamp01(uniform_k(key_u, b));
        pts[3 * j + 1] = clamp01(uniform_k(key_u, b + 1));
        pts[3 * j + 2] = clamp01(uniform_k(key_u, b + 2));
    }
    int64_t j = n_uni + tid;
    int a = 0;
    while (j < N) {
        const uint64_t b = (uint64_t)j * SLOTS;
        const uint64_t key = stream_key(seed, base + (uint64_t)a);
        float cand[3];
        surface_candidate(s, uniform_k(key, b), uniform_k(key, b + 1), uniform_k(key, b + 8), uniform_k(key, b + 9),
                          cand);
        const bool accepted = sdf_union(s, cand[0], cand[1], cand[2]) > -1e-6f;
        if (accepted || a == 7) {
            float p[3];
            if (accepted) {
                p[0] = cand[0]; p[1] = cand[1]; p[2] = cand[2];
            } else {
                p[0] = uniform_k(key_u, b); p[1] = uniform_k(key_u, b + 1); p[2] = uniform_k(key_u, b + 2);
            }
            finish_surface_point(key_u, j, jitter, p, pts + 3 * j);
            j += stride;
            a = 0;
        } else {
            ++a;
        }
    }
}

__device__ __forceinline__ float block_sum(float v, float *tmp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) tmp[wid] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += tmp[w];
    return s;
}

// Per-point loss in binned order (sdf_point_upstream): the upstreams of the
// L1 term with Eq. 7's weight and of the eikonal term, and the block's loss sums.
__global__ void __launch_bounds__(256)
sdf_loss_kernel(ShapeView s, const float4 *__restrict__ sorted, int64_t N, const float *__restrict__ f,
                const float *__restrict__ g, float lambda, float k_weight, float inv_n, float *__restrict__ uf,
                float *__restrict__ ug, float *__restrict__ sums)
{
    __shared__ float tmp[32];
    float l1 = 0.f, eik = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = sorted[p];
        const float d = sdf_union(s, clamp01(q.x), clamp01(q.y), clamp01(q.z));
        float gp[3], u[3], a, e;
        if (g) { gp[0] = g[3 * p]; gp[1] = g[3 * p + 1]; gp[2] = g[3 * p + 2]; }
        sdf_point_upstream(f[p], g ? gp : nullptr, d, lambda, k_weight, inv_n, uf + p, u, &a, &e);
        l1 += a;
        eik += e;
        if (g) {
            ug[3 * p] = u[0];
            ug[3 * p + 1] = u[1];
            ug[3 * p + 2] = u[2];
        }
    }
    const float a = block_sum(l1, tmp);
    if (threadIdx.x == 0) atomicAdd(sums, a);
    if (g) {
        const float b = block_sum(eik, tmp);
        if (threadIdx.x == 0) atomicAdd(sums + 1, b);
    }
}

// Sum of |f - d| over points, with f from a point-parallel gather; with iou
// also the point counts of (f < 0 and d < 0) and (f < 0 or d < 0).
template <typename T, int ORDER>
__global__ void __launch_bounds__(256)
sdf_error_kernel(ShapeView s, const T *__restrict__ coefs, int res, const float *__restrict__ pts, int64_t N,
                 float *__restrict__ err, const int *__restrict__ gate, unsigned long long *__restrict__ iou,
                 float *__restrict__ partials)
{
    if (gate && *gate == 0) return;
    __shared__ float tmp[32];
    unsigned inter = 0, uni = 0;
    constexpr int K = Basis<3, ORDER>::K;
    const float scale = (float)(res - 1);
    float acc = 0.f;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float x[3] = {pts[3 * n], pts[3 * n + 1], pts[3 * n + 2]};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        const int64_t v0 = base_vertex<3>(c, res);
        const PointTables3<ORDER> P(t, 1.0f / scale);
        float f = 0.f;
        for_corners<0>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            float th[K];
            load_block<T, K>(coefs + (v0 + corner_offset<3>(I, res)) * K, th);
            f = fmaf(P.template weight<I>(), P.template value<I>(th), f);
        });
        const float d = sdf_union(s, clamp01(x[0]), clamp01(x[1]), clamp01(x[2]));
        acc += fabsf(f - d);
        inter += (f < 0.f && d < 0.f);
        uni += (f < 0.f || d < 0.f);
    }
    if (err || partials) {
        const float a = block_sum(acc, tmp);
        if (threadIdx.x == 0) {
            if (partials) partials[blockIdx.x] = a;     // summed in block order by sum_partials_kernel
            else atomicAdd(err, a);
        }
    }
    if (iou) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            inter += __shfl_xor_sync(0xffffffffu, inter, o);
            uni += __shfl_xor_sync(0xffffffffu, uni, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(iou, (unsigned long long)inter);
            atomicAdd(iou + 1, (unsigned long long)uni);
        }
    }
}

// The SDF step on the record path in one pass: for every binned record, f and
// grad f (Eq. 2 - Eq. 4), the target distance, the upstreams of the L1 /
// Eq. 7 term and of the eikonal term (sdf_point_upstream), and the coefficient
// gradient added with the warp-aggregated vector reductions of the records
// backward; the loss sums as sdf_loss_kernel forms them. Nothing per point
// goes through memory between the stages.
template <typename T, int ORDER, bool EIK>
__global__ void __launch_bounds__(256)
sdf_records_step_kernel(ShapeView s, const T *__restrict__ coefs, int res, const float4 *__restrict__ sorted,
                        int64_t N, float lambda, float k_weight, float inv_n, float *__restrict__ grad,
                        float *__restrict__ sums)
{
    __shared__ float tmp[32];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float l1 = 0.f, eik = 0.f;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < N; base += stride) {
        const int64_t p = base + lane;
        const unsigned valid = __ballot_sync(0xffffffffu, p < N);
        if (p >= N) break;
        const float4 q = sorted[p];
        const float x[3] = {q.x, q.y, q.z};
        float f[1], gu[1][3];
        point_eval<T, 3, ORDER, 1>(coefs, res, x, f, gu);
        const float d = sdf_union(s, clamp01(q.x), clamp01(q.y), clamp01(q.z));
        float uf[1], ug[1][3], a, e;
        sdf_point_upstream(f[0], EIK ? gu[0] : nullptr, d, lambda, k_weight, inv_n, uf, ug[0], &a, &e);
        l1 += a;
        eik += e;
        point_scatter<3, ORDER, 1>(res, x, uf, ug, EIK, lane, valid, grad);
    }
    const float a = block_sum(l1, tmp);
    if (threadIdx.x == 0) atomicAdd(sums, a);
    if (EIK) {
        const float b = block_sum(eik, tmp);
        if (threadIdx.x == 0) atomicAdd(sums + 1, b);
    }
}

static unsigned blocks_for(int64_t n, int per_sm = 8)
{
    int64_t need = (n + 255) / 256, cap = (int64_t)num_sms() * per_sm;
    return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

tg_status sdf_step_impl(const tg_grid *g, tg_batch *bt, const ShapeView &s, const float *pts, int64_t N,
                        uint64_t seed, int64_t step, const int64_t *step_dev, float lambda_eik, float k_weight,
                        float *coef_grad, float *loss_sums, cudaStream_t cs, bool deterministic)
{
    tg_status st;
    if ((st = ensure_stage(bt, 11 * N, "tg_sdf_step")) != TG_OK) return st;
    float *f = bt->stage, *gx = bt->stage + N, *uf = bt->stage + 4 * N, *ug = bt->stage + 5 * N;
    float *sampled = bt->stage + 8 * N;
    const bool eik = lambda_eik > 0.f;
    if (!pts) {
        sdf_sample_kernel<<<blocks_for(N), 256, 0, cs>>>(s, seed, step, step_dev, N, 0.01f, sampled);
        if ((st = launch_status("tg_sdf_step: sample")) != TG_OK) return st;
        pts = sampled;
    }
    if ((st = tg_batch_bin(bt, pts, N, cs)) != TG_OK) return st;
    if (!deterministic && g->C == 1 && use_records_path(N, bt->nbricks, eik, true)) {
        // few points per brick: forward, loss and backward in one pass over the records
        const unsigned nb = records_blocks(N);
        const float inv_n = 1.0f / (float)N;
#define TG_RS(T, O)                                                                                               \
    (eik ? (sdf_records_step_kernel<T, O, true><<<nb, 256, 0, cs>>>(s, (const T *)g->store, g->res, bt->sorted, N,  \
                                                                     lambda_eik, k_weight, inv_n, coef_grad,        \
                                                                     loss_sums), 0)                                 \
         : (sdf_records_step_kernel<T, O, false><<<nb, 256, 0, cs>>>(s, (const T *)g->store, g->res, bt->sorted, N, \
                                                                      lambda_eik, k_weight, inv_n, coef_grad,       \
                                                                      loss_sums), 0))
        if (g->dtype == TG_F32) {
            if (g->order == 0) TG_RS(float, 0); else if (g->order == 1) TG_RS(float, 1); else TG_RS(float, 2);
        } else if (g->dtype == TG_BF16) {
            if (g->order == 0) TG_RS(__nv_bfloat16, 0); else if (g->order == 1) TG_RS(__nv_bfloat16, 1); else TG_RS(__nv_bfloat16, 2);
        } else {
            if (g->order == 0) TG_RS(__half, 0); else if (g->order == 1) TG_RS(__half, 1); else TG_RS(__half, 2);
        }
#undef TG_RS
        return launch_status("tg_sdf_step: records step");
    }
    if ((st = tg_query_binned(g, bt, f, eik ? gx : nullptr, TG_ORDER_BINNED, cs)) != TG_OK) return st;
    sdf_loss_kernel<<<blocks_for(N), 256, 0, cs>>>(s, bt->sorted, N, f, eik ? gx : nullptr, lambda_eik, k_weight,
                                                   1.0f / (float)N, uf, ug, loss_sums);
    if ((st = launch_status("tg_sdf_step: loss")) != TG_OK) return st;
    return tg_query_backward_binned(g, bt, uf, eik ? ug : nullptr, coef_grad,
                                    TG_ORDER_BINNED | (deterministic ? TG_DETERMINISTIC : 0), cs);
}

// The per-block sums of sdf_error_kernel added in block order (a fixed order, so the
// evaluated error does not depend on which block finished first).
__global__ void sum_partials_kernel(const float *__restrict__ partials, int n, float *__restrict__ err,
                                    const int *__restrict__ gate)
{
    if (gate && *gate == 0) return;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += partials[i];
    *err += s;
}

int error_blocks(int64_t N) { return (int)blocks_for(N); }

tg_status sdf_error_impl(const tg_grid *g, const ShapeView &s, const float *pts, int64_t N, float *err_sum,
                         const int *gate, cudaStream_t cs, unsigned long long *iou, float *partials)
{
    const unsigned nb = blocks_for(N);
#define TG_ERR(T, O) \
    sdf_error_kernel<T, O><<<nb, 256, 0, cs>>>(s, (const T *)g->store, g->res, pts, N, err_sum, gate, iou, partials)
    if (g->dtype == TG_F32) {
        if (g->order == 0) TG_ERR(float, 0); else if (g->order == 1) TG_ERR(float, 1); else TG_ERR(float, 2);
    } else if (g->dtype == TG_BF16) {
        if (g->order == 0) TG_ERR(__nv_bfloat16, 0); else if (g->order == 1) TG_ERR(__nv_bfloat16, 1); else TG_ERR(__nv_bfloat16, 2);
    } else {
        if (g->order == 0) TG_ERR(__half, 0); else if (g->order == 1) TG_ERR(__half, 1); else TG_ERR(__half, 2);
    }
#undef TG_ERR
    tg_status st = launch_status("tg_sdf_error");
    if (st != TG_OK || !partials) return st;
    sum_partials_kernel<<<1, 1, 0, cs>>>(partials, (int)nb, err_sum, gate);
    return launch_status("tg_sdf_error: ordered sum");
}

}  // namespace tg

using namespace tg;

extern "C" {

tg_status tg_sdf_eval_target(const tg_shape *shape, const float *pts, int64_t N, float *d, tg_stream stream)
{
    ShapeView s;
    tg_status st = shape_view(shape, &s, "tg_sdf_eval_target");
    if (st != TG_OK) return st;
    if (N < 0) return fail(TG_EINVAL, "tg_sdf_eval_target: N < 0");
    if (N == 0) return TG_OK;
    if (!pts || !d) return fail(TG_EINVAL, "tg_sdf_eval_target: NULL pts or d");
    sdf_target_kernel<<<blocks_for(N), 256, 0, (cudaStream_t)stream>>>(s, pts, N, d);
    return launch_status("tg_sdf_eval_target");
}

tg_status tg_sample_sdf_points(const tg_shape *shape, uint64_t seed, int64_t step, int64_t N, float jitter,
                               float *pts, tg_stream stream)
{
    ShapeView s;
    tg_status st = shape_view(shape, &s, "tg_sample_sdf_points");
    if (st != TG_OK) return st;
    if (!s.cdf) return fail(TG_EINVAL, "tg_sample_sdf_points: area_cdf is NULL");
    if (N < 0 || step < 0) return fail(TG_EINVAL, "tg_sample_sdf_points: N and step must be >= 0");
    if (N == 0) return TG_OK;
    if (!pts) return fail(TG_EINVAL, "tg_sample_sdf_points: pts is NULL");
    sdf_sample_kernel<<<blocks_for(N), 256, 0, (cudaStream_t)stream>>>(s, seed, step, nullptr, N, jitter, pts);
    return launch_status("tg_sample_sdf_points");
}

tg_status tg_sdf_step(const tg_grid *g, tg_batch *bt, const tg_shape *shape, const float *pts, int64_t N,
                      uint64_t seed, int64_t step, float lambda_eik, float k_weight, float *coef_grad, float *loss_sums,
                      tg_stream stream)
{
    ShapeView s;
    tg_status st = shape_view(shape, &s, "tg_sdf_step");
    if (st != TG_OK) return st;
    if (!g || g->dim != 3 || g->C != 1) return fail(TG_EINVAL, "tg_sdf_step: needs a 3-D one-channel grid");
    if ((st = check_pair(g, bt, "tg_sdf_step")) != TG_OK) return st;
    if (N <= 0 || N > bt->max_points) return fail(TG_EINVAL, "tg_sdf_step: N outside [1, max_points]");
    if (!coef_grad || !loss_sums) return fail(TG_EINVAL, "tg_sdf_step: NULL coef_grad or loss_sums");
    if (!pts && !s.cdf) return fail(TG_EINVAL, "tg_sdf_step: sampling needs area_cdf");
    if (!(lambda_eik >= 0.f)) return fail(TG_EINVAL, "tg_sdf_step: lambda_eik must be >= 0");
    return sdf_step_impl(g, bt, s, pts, N, seed, step, nullptr, lambda_eik, k_weight, coef_grad, loss_sums,
                         (cudaStream_t)stream, false);
}

tg_status tg_sdf_error(const tg_grid *g, const tg_shape *shape, const float *pts, int64_t N, float *err_sum,
                       tg_stream stream)
{
    ShapeView s;
    tg_status st = shape_view(shape, &s, "tg_sdf_error");
    if (st != TG_OK) return st;
    if (!g || g->dim != 3 || g->C != 1) return fail(TG_EINVAL, "tg_sdf_error: needs a 3-D one-channel grid");
    if (N < 0) return fail(TG_EINVAL, "tg_sdf_error: N < 0");
    if (N == 0) return TG_OK;
    if (!pts || !err_sum) return fail(TG_EINVAL, "tg_sdf_error: NULL pts or err_sum");
    return sdf_error_impl(g, s, pts, N, err_sum, nullptr, (cudaStream_t)stream);
}

tg_status tg_sdf_iou(const tg_grid *g, const tg_shape *shape, const float *pts, int64_t N, uint64_t *counts,
                     tg_stream stream)
{
    ShapeView s;
    tg_status st = shape_view(shape, &s, "tg_sdf_iou");
    if (st != TG_OK) return st;
    if (!g || g->dim != 3 || g->C != 1) return fail(TG_EINVAL, "tg_sdf_iou: needs a 3-D one-channel grid");
    if (N < 0) return fail(TG_EINVAL, "tg_sdf_iou: N < 0");
    if (N == 0) return TG_OK;
    if (!pts || !counts) return fail(TG_EINVAL, "tg_sdf_iou: NULL pts or counts");
    return sdf_error_impl(g, s, pts, N, nullptr, nullptr, (cudaStream_t)stream,
                          reinterpret_cast<unsigned long long *>(counts));
}

}  // extern "C"
