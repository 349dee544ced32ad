// The server's batched training step: one launch per stage advances every
// running fit job of one (order, storage dtype) group by one step.
//
// The jobs' fit batches are concatenated (job j owns points [pbase, pbase +
// npts)). One point-parallel kernel samples each point from its job's target
// (the sampler of tg_sdf_step, by point index), evaluates f and grad f on the
// job's grid (Eq. 2 - Eq. 4), forms the loss upstreams (Eq. 6 with Eq. 7's
// weight, the eikonal term of Eq. 8) and scatters the coefficient gradient
// with warp-aggregated vector reductions into the job's gradient. One Adam
// launch covers the float4 groups of all jobs' coefficients; a lazy-Adam job
// instead has the fit kernel flag every vertex its points reach, and Adam
// visits the flagged vertices only (an unflagged vertex has a zero gradient,
// which lazy Adam leaves alone), so its cost follows the points, not the grid
// size. A gated launch
// evaluates the jobs whose evaluation step it is, and one thread per job
// keeps the step counter and status.
#include "tg_adam.cuh"
#include "tg_query.cuh"
#include "tg_serve.cuh"

namespace tg {

// Index of the last job whose start (pbase or gbase) is <= key; jobs sorted by it.
template <bool BY_GROUP>
__device__ __forceinline__ int find_job(const BatchJob *__restrict__ jobs, int n, int64_t key)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t start = BY_GROUP ? jobs[mid].gbase : jobs[mid].pbase;
        if (start <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Eq. 3 / Eq. 4 at one point of a 3-D one-channel grid: f and d f / d x.
template <typename T, int ORDER, bool GRAD>
__device__ __forceinline__ float point_value(const T *__restrict__ coefs, int res, const int *c, const float *t,
                                             float *gx)
{
    using B = Basis<3, ORDER>;
    constexpr int K = B::K;
    const float scale = (float)(res - 1), h = 1.0f / scale;
    const int64_t v0 = base_vertex<3>(c, res);
    float f = 0.f;
    if (GRAD) gx[0] = gx[1] = gx[2] = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float th[K];
        load_block<T, K>(coefs + (v0 + corner_offset<3>(i, res)) * K, th);
        float dw[3], dl[3], g[3];
        const float w = corner_weight<3>(i, t, dw);
#pragma unroll
        for (int d = 0; d < 3; ++d) dl[d] = (t[d] - (float)((i >> d) & 1)) * h;
        const float Tv = B::eval(th, dl, g);
        f = fmaf(w, Tv, f);
        if (GRAD) {
#pragma unroll
            for (int d = 0; d < 3; ++d) gx[d] = fmaf(dw[d] * scale, Tv, fmaf(w, g[d], gx[d]));
        }
    }
    return f;
}

__global__ void batch_prologue_kernel(const BatchJob *__restrict__ jobs, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    unsigned char *b = jobs[j].block;
    const int64_t t = *JobBlock::step(b) + 1;                     // the 1-based step being taken
    *JobBlock::gate(b) = (t % jobs[j].eval_every) == 0 ? 1 : 0;
    const float ft = (float)t;
    JobBlock::adam(b)[0] = jobs[j].lr / (1.0f - powf(0.9f, ft));   // lr / (1 - beta1^t)
    JobBlock::adam(b)[1] = rsqrtf(1.0f - powf(0.999f, ft));        // 1 / sqrt(1 - beta2^t)
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(256, 4)
batch_fit_kernel(const BatchJob *__restrict__ jobs, int njobs, int64_t total)
{
    constexpr int K = Basis<3, ORDER>::K;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t n = base + lane;
        const unsigned valid = __ballot_sync(0xffffffffu, n < total);
        if (n >= total) break;
        const int j = find_job<false>(jobs, njobs, n);
        const BatchJob &J = jobs[j];
        const int res = J.res;
        const float scale = (float)(res - 1);
        float x[3];
        sample_sdf_point(J.shape, J.seed, *JobBlock::step(J.block), J.npts, n - J.pbase, 0.01f, x);
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        const bool eik = J.lambda_eik > 0.f;
        float gx[3];
        const float f = eik ? point_value<T, ORDER, true>((const T *)J.store, res, c, t, gx)
                            : point_value<T, ORDER, false>((const T *)J.store, res, c, t, gx);
        const float d = sdf_union(J.shape, x[0], x[1], x[2]);
        float uf[1], ug[1][3], l1, le;
        sdf_point_upstream(f, eik ? gx : nullptr, d, J.lambda_eik, J.k_weight, 1.0f / (float)J.npts, uf, ug[0], &l1,
                           &le);
        // scatter: lanes of the warp with the same job and cell are summed into one reduction
        const int64_t v0 = base_vertex<3>(c, res);
        const unsigned long long key = ((unsigned long long)j << 40) | (unsigned long long)v0;
        const unsigned peers = __match_any_sync(valid, key);
        const int group = __popc(peers);
        const int max_group = __reduce_max_sync(valid, (unsigned)group);
        const bool leader = (__ffs(peers) - 1) == lane;
        float *grad = J.grad;
        if (J.touched) {
#pragma unroll
            for (int i = 0; i < 8; ++i) J.touched[v0 + corner_offset<3>(i, res)] = 1;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float ctr[K];
            corner_contrib<3, ORDER, 1>(i, t, scale, uf, ug, eik, ctr);
            if (max_group > 1) {
                for (int r = 1; r < max_group; ++r) {
                    const int src = r < group ? (int)__fns(peers, 0, r + 1) : lane;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float v = __shfl_sync(valid, ctr[k], src);
                        if (leader && r < group) ctr[k] += v;
                    }
                }
                if (!leader) continue;
            }
            red_block<K>(grad + (v0 + corner_offset<3>(i, res)) * K, ctr);
        }
    }
}

// Adam over the units of every job: float4 groups (a group past a job's end is handled element by element), or
// runs of 4 vertices of a job with touched flags.
template <typename T, typename M>
__global__ void __launch_bounds__(256)
batch_adam_kernel(const BatchJob *__restrict__ jobs, int njobs, int64_t total_groups)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total_groups; q += stride) {
        const int j = find_job<true>(jobs, njobs, q);
        const BatchJob &J = jobs[j];
        const int64_t k = q - J.gbase;
        const float *ac = JobBlock::adam(J.block);
        const AdamCoef a{0.9f, 0.999f, 1.0f - 0.9f, 1.0f - 0.999f, ac[0], ac[1], 1e-8f};
        float *p = J.master, *g = J.grad;
        M *m = (M *)J.m, *v = (M *)J.v;
        T *shadow = (T *)J.shadow;
        const bool lazy = J.lazy != 0;
        if (J.touched) {      // 4 vertices per unit; only the flagged ones are read
            const int64_t v0 = 4 * k;
            const int nvu = (int)min((int64_t)4, J.nv - v0);
            unsigned fl = 0u;
            if (nvu == 4) fl = *reinterpret_cast<const unsigned *>(J.touched + v0);
            else
                for (int i = 0; i < nvu; ++i) fl |= (unsigned)J.touched[v0 + i] << (8 * i);
            if (fl == 0u) continue;
            for (int i = 0; i < nvu; ++i) {
                if (((fl >> (8 * i)) & 0xffu) == 0u) continue;
                for (int64_t e = (v0 + i) * J.K; e < (v0 + i + 1) * J.K; ++e) {
                    const float ge = g[e];
                    if (ge == 0.f) continue;
                    float pp = p[e], mm = Moments<M>::get(m, e), vv = Moments<M>::get(v, e);
                    adam_one(pp, ge, mm, vv, a);
                    p[e] = pp;
                    Moments<M>::put(m, e, mm);
                    Moments<M>::put(v, e, vv);
                    g[e] = 0.0f;
                    if (shadow) shadow[e] = from_f32<T>(pp);
                }
            }
            if (nvu == 4) *reinterpret_cast<unsigned *>(J.touched + v0) = 0u;
            else
                for (int i = 0; i < nvu; ++i) J.touched[v0 + i] = 0;
            continue;
        }
        if (4 * k + 3 < J.ncoef) {
            const float4 gg = __ldcs(reinterpret_cast<float4 *>(g) + k);
            if (lazy && gg.x == 0.f && gg.y == 0.f && gg.z == 0.f && gg.w == 0.f) continue;
            float4 pp = reinterpret_cast<float4 *>(p)[k], mm = Moments<M>::load(m, k), vv = Moments<M>::load(v, k);
            if (lazy) {
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
            reinterpret_cast<float4 *>(p)[k] = pp;
            Moments<M>::store(m, k, mm);
            Moments<M>::store(v, k, vv);
            __stcs(reinterpret_cast<float4 *>(g) + k, make_float4(0.f, 0.f, 0.f, 0.f));
            if (shadow) store4<T>(shadow, 4 * k, pp.x, pp.y, pp.z, pp.w);
        } else {
            for (int64_t e = 4 * k; e < J.ncoef; ++e) {
                if (lazy && g[e] == 0.f) continue;
                float pp = p[e], mm = Moments<M>::get(m, e), vv = Moments<M>::get(v, e);
                adam_one(pp, g[e], mm, vv, a);
                p[e] = pp;
                Moments<M>::put(m, e, mm);
                Moments<M>::put(v, e, vv);
                g[e] = 0.0f;
                if (shadow) shadow[e] = from_f32<T>(pp);
            }
        }
    }
}

// Sum of |f - d| over the evaluation points of the jobs whose gate is set (blockIdx.y = job).
template <typename T, int ORDER>
__global__ void __launch_bounds__(256)
batch_eval_kernel(const BatchJob *__restrict__ jobs)
{
    const BatchJob &J = jobs[blockIdx.y];
    if (*JobBlock::gate(J.block) == 0) return;
    __shared__ float tmp[8];
    const int res = J.res;
    const float scale = (float)(res - 1);
    float acc = 0.f;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < J.n_eval; n += (int64_t)gridDim.x * blockDim.x) {
        const float x[3] = {J.eval_pts[3 * n], J.eval_pts[3 * n + 1], J.eval_pts[3 * n + 2]};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        const float f = point_value<T, ORDER, false>((const T *)J.store, res, c, t, nullptr);
        acc += fabsf(f - sdf_union(J.shape, clamp01(x[0]), clamp01(x[1]), clamp01(x[2])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) tmp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += tmp[w];
        atomicAdd(JobBlock::err(J.block), s);
    }
}

__global__ void batch_finalize_kernel(const BatchJob *__restrict__ jobs, int n, DevStatus *__restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const BatchJob &J = jobs[j];
    unsigned char *b = J.block;
    DevStatus *st = JobBlock::status(b);
    const int64_t s = *JobBlock::step(b) + 1;
    if (*JobBlock::gate(b)) {
        const float e = *JobBlock::err(b) / (float)J.n_eval;
        st->error = e;
        *JobBlock::err(b) = 0.f;
        if (e < J.tol) st->done = 1;
    }
    *JobBlock::step(b) = s;
    st->steps = s;
    if (s >= J.max_steps) st->done = 1;
    out[j] = *st;
}

template <typename T, typename M, int ORDER>
static tg_status batch_launch(const BatchJob *host, BatchJob *dev, int n, DevStatus *status_dev, cudaStream_t s)
{
    const BatchJob &last = host[n - 1];
    const int64_t total = last.pbase + last.npts;
    const int64_t groups = last.gbase + (last.touched ? (last.nv + 3) / 4 : (last.ncoef + 3) / 4);
    int64_t max_eval = 0;
    for (int j = 0; j < n; ++j) max_eval = host[j].n_eval > max_eval ? host[j].n_eval : max_eval;
    const int64_t cap = (int64_t)num_sms() * 8;
    auto blocks = [&](int64_t items) { const int64_t b = (items + 255) / 256; return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap)); };
    tg_status st;
    batch_prologue_kernel<<<(n + 31) / 32, 32, 0, s>>>(dev, n);
    if ((st = launch_status("server: batched prologue")) != TG_OK) return st;
    batch_fit_kernel<T, ORDER><<<blocks(total), 256, 0, s>>>(dev, n, total);
    if ((st = launch_status("server: batched step")) != TG_OK) return st;
    batch_adam_kernel<T, M><<<blocks(groups), 256, 0, s>>>(dev, n, groups);
    if ((st = launch_status("server: batched Adam")) != TG_OK) return st;
    const int64_t eb = (max_eval + 255) / 256;
    batch_eval_kernel<T, ORDER><<<dim3((unsigned)(eb < 64 ? (eb < 1 ? 1 : eb) : 64), (unsigned)n), 256, 0, s>>>(dev);
    if ((st = launch_status("server: batched evaluation")) != TG_OK) return st;
    batch_finalize_kernel<<<(n + 31) / 32, 32, 0, s>>>(dev, n, status_dev);
    return launch_status("server: batched finalize");
}

tg_status batch_step(const BatchJob *host, BatchJob *dev, int n, int order, tg_dtype dtype, DevStatus *status_dev,
                     cudaStream_t s)
{
    if (n <= 0) return TG_OK;
    tg_status st = cuda_status(cudaMemcpyAsync(dev, host, (size_t)n * sizeof(BatchJob), cudaMemcpyHostToDevice, s),
                               "server: job table");
    if (st != TG_OK) return st;
#define TG_BL(T, M, O) batch_launch<T, M, O>(host, dev, n, status_dev, s)
    if (dtype == TG_F32) {
        if (order == 0) return TG_BL(float, float, 0);
        if (order == 1) return TG_BL(float, float, 1);
        return TG_BL(float, float, 2);
    }
    if (dtype == TG_BF16) {
        if (order == 0) return TG_BL(__nv_bfloat16, __nv_bfloat16, 0);
        if (order == 1) return TG_BL(__nv_bfloat16, __nv_bfloat16, 1);
        return TG_BL(__nv_bfloat16, __nv_bfloat16, 2);
    }
    if (order == 0) return TG_BL(__half, __nv_bfloat16, 0);
    if (order == 1) return TG_BL(__half, __nv_bfloat16, 1);
    return TG_BL(__half, __nv_bfloat16, 2);
#undef TG_BL
}

}  // namespace tg
