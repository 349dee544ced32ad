// SDF fitting (Sec. 3.2): analytic targets, the device sampler of fit
// batches, the per-point loss (Eq. 6 with w = 1, eikonal term of Eq. 8) and
// the fitting step that composes binning, the binned forward with spatial
// gradients, the loss and the binned backward - all in binned order.
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

// Signed distance of the union (Eq. 5): sphere |x - c| - r; box: distance to
// the box surface, negative inside; union = minimum.
__device__ __forceinline__ float sdf_union(const ShapeView &s, float x, float y, float z)
{
    float best = INFINITY;
    for (int i = 0; i < s.ns; ++i) {
        const float *q = s.sph + 4 * i;
        const float dx = x - __ldg(q), dy = y - __ldg(q + 1), dz = z - __ldg(q + 2);
        best = fminf(best, sqrtf(dx * dx + dy * dy + dz * dz) - __ldg(q + 3));
    }
    for (int i = 0; i < s.nb; ++i) {
        const float *q = s.box + 6 * i;
        const float ex = fabsf(x - __ldg(q)) - __ldg(q + 3);
        const float ey = fabsf(y - __ldg(q + 1)) - __ldg(q + 4);
        const float ez = fabsf(z - __ldg(q + 2)) - __ldg(q + 5);
        const float ox = fmaxf(ex, 0.f), oy = fmaxf(ey, 0.f), oz = fmaxf(ez, 0.f);
        const float d = sqrtf(ox * ox + oy * oy + oz * oz) + fminf(fmaxf(ex, fmaxf(ey, ez)), 0.f);
        best = fminf(best, d);
    }
    return best;
}

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }

__global__ void sdf_target_kernel(ShapeView s, const float *__restrict__ pts, int64_t N, float *__restrict__ d)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        d[n] = sdf_union(s, clamp01(pts[3 * n]), clamp01(pts[3 * n + 1]), clamp01(pts[3 * n + 2]));
}

// An area-weighted surface point of one member from the uniforms u0, u1 (position),
// u8 (member), u9 (box face).
__device__ __forceinline__ void surface_candidate(const ShapeView &s, float u0, float u1, float u8, float u9, float *p)
{
    const int nm = s.ns + s.nb;
    int prim = 0;
    for (int i = 0; i < nm; ++i) prim += (__ldg(s.cdf + i) <= u8) ? 1 : 0;   // first entry > u8
    prim = min(prim, nm - 1);
    if (prim < s.ns) {
        const float *q = s.sph + 4 * prim;
        const float z = 1.f - 2.f * u0;
        const float r = sqrtf(fmaxf(0.f, 1.f - z * z));
        const float R = __ldg(q + 3);
        p[0] = __ldg(q) + R * r * cospif(2.f * u1);
        p[1] = __ldg(q + 1) + R * r * sinpif(2.f * u1);
        p[2] = __ldg(q + 2) + R * z;
    } else {
        const float *q = s.box + 6 * (prim - s.ns);
        const float c[3] = {__ldg(q), __ldg(q + 1), __ldg(q + 2)};
        const float h[3] = {__ldg(q + 3), __ldg(q + 4), __ldg(q + 5)};
        const float fa[3] = {h[1] * h[2], h[0] * h[2], h[0] * h[1]};
        const float tot = 2.f * (fa[0] + fa[1] + fa[2]);
        float run = 0.f;
        int face = 0;
        for (int f = 0; f < 6; ++f) {
            run += fa[f / 2];
            face += (run / tot <= u9) ? 1 : 0;
        }
        face = min(face, 5);
        const int ax = face / 2, a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
        p[ax] = c[ax] + ((face % 2 == 0) ? -h[ax] : h[ax]);
        p[a1] = c[a1] + (2.f * u0 - 1.f) * h[a1];
        p[a2] = c[a2] + (2.f * u1 - 1.f) * h[a2];
    }
}

__global__ void sdf_sample_kernel(ShapeView s, uint64_t seed, int64_t step, const int64_t *__restrict__ step_dev,
                                  int64_t N, float jitter, float *__restrict__ pts)
{
    constexpr uint64_t SLOTS = 16;
    if (step_dev) step = *step_dev;
    const int64_t n_uni = N / 2;
    const uint64_t base = (uint64_t)step * 256ull;
    const uint64_t key_u = stream_key(seed, base + 255ull);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = (uint64_t)j * SLOTS;
        float p[3] = {uniform_k(key_u, b), uniform_k(key_u, b + 1), uniform_k(key_u, b + 2)};
        if (j >= n_uni) {
            for (int a = 0; a < 8; ++a) {
                const uint64_t key = stream_key(seed, base + (uint64_t)a);
                float cand[3];
                surface_candidate(s, uniform_k(key, b), uniform_k(key, b + 1), uniform_k(key, b + 8),
                                  uniform_k(key, b + 9), cand);
                if (sdf_union(s, cand[0], cand[1], cand[2]) > -1e-6f) {
                    p[0] = cand[0]; p[1] = cand[1]; p[2] = cand[2];
                    break;
                }
            }
            if (jitter > 0.f) {
#pragma unroll
                for (int k = 0; k < 3; ++k) p[k] += jitter * normal_k(key_u, (uint64_t)j * (SLOTS / 2) + 2 + k);
            }
        }
        pts[3 * j] = clamp01(p[0]);
        pts[3 * j + 1] = clamp01(p[1]);
        pts[3 * j + 2] = clamp01(p[2]);
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

// Per-point loss in binned order: r = f - d(x), dL/df = sign(r) / N and, with
// an eikonal weight, dL/d(grad_x f) = lambda 2 (|g| - 1) g / |g| / N.
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
        const float r = f[p] - d;
        // Eq. 7: w = max(w'(f), w'(d)), w'(z) = 1 - |2 sigmoid(k z) - 1| = 2 e / (1 + e), e = exp(-|k z|);
        // a fixed weight of the residual (k <= 0: w = 1)
        float w = 1.f;
        if (k_weight > 0.f) {
            const float ef = expf(-fabsf(k_weight * f[p])), ed = expf(-fabsf(k_weight * d));
            w = fmaxf(2.f * ef / (1.f + ef), 2.f * ed / (1.f + ed));
        }
        l1 += w * fabsf(r);
        uf[p] = r > 0.f ? w * inv_n : (r < 0.f ? -w * inv_n : 0.f);
        if (g) {
            const float gx = g[3 * p], gy = g[3 * p + 1], gz = g[3 * p + 2];
            const float e = sqrtf(gx * gx + gy * gy + gz * gz);
            eik += (e - 1.f) * (e - 1.f);
            const float c = e < 1e-12f ? 0.f : lambda * 2.f * (e - 1.f) / e * inv_n;
            ug[3 * p] = c * gx;
            ug[3 * p + 1] = c * gy;
            ug[3 * p + 2] = c * gz;
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
                 float *__restrict__ err, const int *__restrict__ gate, unsigned long long *__restrict__ iou)
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
    if (err) {
        const float a = block_sum(acc, tmp);
        if (threadIdx.x == 0) atomicAdd(err, a);
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

static unsigned blocks_for(int64_t n, int per_sm = 8)
{
    int64_t need = (n + 255) / 256, cap = (int64_t)num_sms() * per_sm;
    return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

tg_status sdf_step_impl(const tg_grid *g, tg_batch *bt, const ShapeView &s, const float *pts, int64_t N,
                        uint64_t seed, int64_t step, const int64_t *step_dev, float lambda_eik, float k_weight,
                        float *coef_grad, float *loss_sums, cudaStream_t cs)
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
    if ((st = tg_query_binned(g, bt, f, eik ? gx : nullptr, TG_ORDER_BINNED, cs)) != TG_OK) return st;
    sdf_loss_kernel<<<blocks_for(N), 256, 0, cs>>>(s, bt->sorted, N, f, eik ? gx : nullptr, lambda_eik, k_weight,
                                                   1.0f / (float)N, uf, ug, loss_sums);
    if ((st = launch_status("tg_sdf_step: loss")) != TG_OK) return st;
    return tg_query_backward_binned(g, bt, uf, eik ? ug : nullptr, coef_grad, TG_ORDER_BINNED, cs);
}

tg_status sdf_error_impl(const tg_grid *g, const ShapeView &s, const float *pts, int64_t N, float *err_sum,
                         const int *gate, cudaStream_t cs, unsigned long long *iou)
{
    const unsigned nb = blocks_for(N);
#define TG_ERR(T, O) \
    sdf_error_kernel<T, O><<<nb, 256, 0, cs>>>(s, (const T *)g->store, g->res, pts, N, err_sum, gate, iou)
    if (g->dtype == TG_F32) {
        if (g->order == 0) TG_ERR(float, 0); else if (g->order == 1) TG_ERR(float, 1); else TG_ERR(float, 2);
    } else if (g->dtype == TG_BF16) {
        if (g->order == 0) TG_ERR(__nv_bfloat16, 0); else if (g->order == 1) TG_ERR(__nv_bfloat16, 1); else TG_ERR(__nv_bfloat16, 2);
    } else {
        if (g->order == 0) TG_ERR(__half, 0); else if (g->order == 1) TG_ERR(__half, 1); else TG_ERR(__half, 2);
    }
#undef TG_ERR
    return launch_status("tg_sdf_error");
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
                         (cudaStream_t)stream);
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
