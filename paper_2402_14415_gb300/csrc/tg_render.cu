// Differentiable ray marching through TaylorGrid density and colour fields
// (Sec. 3.3, Eq. 9 - Eq. 11).
//
// One warp per ray; lane l owns a contiguous run of the ray's S stratified
// samples. Each sample queries the density grid (sigma = softplus(f), Eq. 9)
// and the colour grid (c = sigmoid(f), 3 channels). The optical depth prefix
// of Eq. 10 and, for the backward, the prefix of T_i alpha_i c_i are warp
// scans over the lanes' partial sums, so the whole forward and the per-sample
// derivatives are computed in registers in one pass (nothing per sample is
// stored between a forward and a backward pass). The per-sample coefficient
// upstreams are then sent through the binned, atomic-free backward of both
// grids.
#include "tg_binned.cuh"

namespace tg {

constexpr int kMaxSamplesPerLane = 16;     // S <= 512

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.f / (1.f + expf(-x)); }

// Point-parallel field value of a 3-D grid (all channels) at x (Eq. 2 - Eq. 4).
template <typename T, int ORDER, int C>
__device__ __forceinline__ void field_value(const T *__restrict__ coefs, int res, const float *x, float *f)
{
    constexpr int K = Basis<3, ORDER>::K;
    constexpr int NV = K * C;
    const float scale = (float)(res - 1);
    int c[3];
    float t[3];
    locate<3>(x, res, scale, c, t);
    const int64_t v0 = base_vertex<3>(c, res);
    const PointTables3<ORDER> P(t, 1.0f / scale);
#pragma unroll
    for (int ch = 0; ch < C; ++ch) f[ch] = 0.f;
    for_corners<0>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        float th[NV];
        load_block<T, NV>(coefs + (v0 + corner_offset<3>(I, res)) * NV, th);
        const float w = P.template weight<I>();
#pragma unroll
        for (int ch = 0; ch < C; ++ch) f[ch] = fmaf(w, P.template value<I>(th + ch * K), f[ch]);
    });
}

// Ray / unit-cube slab intersection; false on a miss.
__device__ __forceinline__ bool ray_box(const float *o, const float *d, float &tn, float &tf)
{
    tn = 0.f;
    tf = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.f) {
            if (o[a] < 0.f || o[a] > 1.f) return false;
            continue;
        }
        float t0 = __fdiv_rn(0.f - o[a], d[a]), t1 = __fdiv_rn(1.f - o[a], d[a]);
        if (t0 > t1) { float s = t0; t0 = t1; t1 = s; }
        tn = fmaxf(tn, t0);
        tf = fminf(tf, t1);
    }
    return tf > tn;
}

__device__ __forceinline__ float warp_excl_scan(float v, float &total)
{
    const int lane = threadIdx.x & 31;
    float incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
}

// Sum of v over the lanes above this one (0 on lane 31): an inclusive suffix
// scan by shuffles down, then shifted by one lane.
__device__ __forceinline__ float warp_excl_suffix(float v)
{
    const int lane = threadIdx.x & 31;
    float incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl += u;
    }
    const float ex = __shfl_down_sync(0xffffffffu, incl, 1);
    return lane == 31 ? 0.f : ex;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// MPL: the most samples a lane holds (8 for S <= 256, 16 for S <= 512); the
// per-sample state lives in registers, so a smaller MPL leaves room for two
// blocks per SM.
template <typename TD, typename TC, int OD, int OC, int MPL>
__global__ void __launch_bounds__(256, MPL <= 8 ? 2 : 1)
render_kernel(const TD *__restrict__ dcoef, const TC *__restrict__ ccoef, int res, const float *__restrict__ ro,
              const float *__restrict__ rd, int64_t R, int S, uint64_t seed, uint64_t ray_base, float bg,
              float *__restrict__ rgb, const float *__restrict__ target, const float *__restrict__ dldc, float inv_r,
              float *__restrict__ loss, float *__restrict__ xs, float *__restrict__ ud, float *__restrict__ uc)
{
    const int lane = threadIdx.x & 31;
    const int m = (S + 31) / 32;                 // samples per lane
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); r < R; r += warps) {
        const float o[3] = {ro[3 * r], ro[3 * r + 1], ro[3 * r + 2]};
        const float d[3] = {rd[3 * r], rd[3 * r + 1], rd[3 * r + 2]};
        float tn, tf;
        const bool hit = ray_box(o, d, tn, tf);
        const uint64_t key = stream_key(seed, ray_base + (uint64_t)r);
        // sample positions by the FP32 rule t_i = tn + (i + xi_i) step, every operation rounded once
        const float step = hit ? __fdiv_rn(__fsub_rn(tf, tn), (float)S) : 0.f;
        // per-lane samples: optical depth tau = sigma delta, colour, raw field values (positions are
        // recomputed by the same FP32 operations where the backward needs them)
        float tau[MPL], col[MPL][3], fd[MPL], dlt[MPL];
        float lane_tau = 0.f;
#pragma unroll
        for (int k = 0; k < MPL; ++k) {
            const int i = lane * m + k;
            tau[k] = 0.f;
            fd[k] = 0.f;
            dlt[k] = 0.f;
            col[k][0] = col[k][1] = col[k][2] = 0.f;
            if (k < m && i < S && hit) {
                const float ti = __fadd_rn(tn, __fmul_rn(__fadd_rn((float)i, uniform_k(key, (uint64_t)i)), step));
                const float tnext =
                    (i + 1 < S) ? __fadd_rn(tn, __fmul_rn(__fadd_rn((float)(i + 1), uniform_k(key, (uint64_t)(i + 1))), step))
                                : tf;
                const float x[3] = {fmaf(ti, d[0], o[0]), fmaf(ti, d[1], o[1]), fmaf(ti, d[2], o[2])};
                float fc[3];
                field_value<TD, OD, 1>(dcoef, res, x, &fd[k]);
                field_value<TC, OC, 3>(ccoef, res, x, fc);
                dlt[k] = tnext - ti;
                tau[k] = softplus_f(fd[k]) * dlt[k];
#pragma unroll
                for (int a = 0; a < 3; ++a) col[k][a] = sigmoid_f(fc[a]);
                lane_tau += tau[k];
            }
        }
        float total_tau;
        const float before = warp_excl_scan(lane_tau, total_tau);
        // Eq. 10: T_i = exp(-sum_{j<i} tau_j), weight T_i (1 - exp(-tau_i))
        float acc[3] = {0.f, 0.f, 0.f}, run = before;
        float Ti[MPL];
#pragma unroll
        for (int k = 0; k < MPL; ++k) {
            Ti[k] = expf(-run);
            const float wgt = Ti[k] * -expm1f(-tau[k]);       // T_i alpha_i, alpha_i without the 1 - exp cancellation
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] = fmaf(wgt, col[k][a], acc[a]);
            run += tau[k];
        }
        const float T_end = expf(-total_tau);
        float Cr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Cr[a] = warp_sum(acc[a]) + T_end * bg;
        if (lane == 0 && rgb) {
            rgb[3 * r] = Cr[0]; rgb[3 * r + 1] = Cr[1]; rgb[3 * r + 2] = Cr[2];
        }
        if (!target && !dldc) continue;
        // dL/dC: given (dldc), or of Eq. 11, L = (1/R) sum_r ||C_r - C*_r||^2, dL/dC = 2 (C - C*) / R
        float g[3], l = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (dldc) {
                g[a] = dldc[3 * r + a];
            } else {
                const float e = Cr[a] - target[3 * r + a];
                g[a] = 2.f * e * inv_r;
                l += e * e;
            }
        }
        if (target && lane == 0) atomicAdd(loss, l);
        // behind_i = sum_{j>i} T_j alpha_j c_j + T_S bg, formed as a suffix sum (the lanes above this one,
        // then this lane's samples from the last one down) so it is never a difference of two sums
        float behind[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) behind[a] = warp_excl_suffix(acc[a]) + T_end * bg;
#pragma unroll
        for (int k = MPL - 1; k >= 0; --k) {
            const int i = lane * m + k;
            if (!(k < m && i < S)) continue;
            const float alpha = -expm1f(-tau[k]);
            const float Tn = Ti[k] * expf(-tau[k]);              // T_{i+1}
            const float delta_i = dlt[k];
            float dsig = 0.f, dfc[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float w = Ti[k] * alpha * col[k][a];
                dsig = fmaf(g[a], delta_i * (Tn * col[k][a] - behind[a]), dsig);
                dfc[a] = g[a] * Ti[k] * alpha * col[k][a] * (1.f - col[k][a]);
                behind[a] += w;                                  // sample i is behind sample i - 1
            }
            const int64_t sidx = r * S + i;
            if (hit) {
                const float ti = __fadd_rn(tn, __fmul_rn(__fadd_rn((float)i, uniform_k(key, (uint64_t)i)), step));
                xs[3 * sidx] = fmaf(ti, d[0], o[0]);
                xs[3 * sidx + 1] = fmaf(ti, d[1], o[1]);
                xs[3 * sidx + 2] = fmaf(ti, d[2], o[2]);
            } else {
                // a missed ray's samples carry zero upstream gradient; spread them over the cube (a
                // low-discrepancy sequence of the sample index) so the binned backward's bricks stay
                // balanced instead of stacking them in one cell
                const double sd = (double)sidx;
                xs[3 * sidx] = (float)(sd * 0.7548776662466927 - floor(sd * 0.7548776662466927));
                xs[3 * sidx + 1] = (float)(sd * 0.5698402909980532 - floor(sd * 0.5698402909980532));
                xs[3 * sidx + 2] = (float)(sd * 0.4301597090019468 - floor(sd * 0.4301597090019468));
            }
            ud[sidx] = hit ? dsig * sigmoid_f(fd[k]) : 0.f;      // d softplus / d f = sigmoid(f)
#pragma unroll
            for (int a = 0; a < 3; ++a) uc[3 * sidx + a] = hit ? dfc[a] : 0.f;
        }
    }
}

}  // namespace tg

using namespace tg;

static tg_status render_impl(const tg_grid *dg, const tg_grid *cg, const float *rays_o, const float *rays_d,
                             int64_t R, int S, uint64_t seed, uint64_t ray_base, float bg, float *rgb_out,
                             const float *target_rgb, const float *dldc, tg_batch *batch, float *density_grad,
                             float *color_grad, float *loss_sum, cudaStream_t s, const char *who)
{
    if (!dg || !cg) return fail(TG_EINVAL, "%s: NULL grid", who);
    if (dg->dim != 3 || cg->dim != 3 || dg->C != 1 || cg->C != 3)
        return fail(TG_EINVAL, "%s: needs a 3-D 1-channel density grid and a 3-D 3-channel colour grid", who);
    if (dg->res != cg->res) return fail(TG_EINVAL, "%s: the two grids must share res", who);
    if (R < 0 || S < 1 || S > 32 * kMaxSamplesPerLane) return fail(TG_EINVAL, "%s: R >= 0, 1 <= S <= 512", who);
    if (R == 0) return TG_OK;
    if (!rays_o || !rays_d || (!rgb_out && !dldc)) return fail(TG_EINVAL, "%s: NULL ray or output pointer", who);
    tg_status st;
    const int64_t NS = R * S;
    const bool train = target_rgb || dldc;
    float *xs = nullptr, *ud = nullptr, *uc = nullptr;
    if (train) {
        if (!batch || !density_grad || !color_grad || (target_rgb && !loss_sum))
            return fail(TG_EINVAL, "%s: the backward needs batch and both gradients (and loss_sum with a target)", who);
        if ((st = check_pair(dg, batch, who)) != TG_OK) return st;
        if (NS > batch->max_points) return fail(TG_EINVAL, "%s: R * S exceeds the batch's max_points", who);
        if ((st = ensure_aux(batch, 7 * NS, who)) != TG_OK) return st;
        xs = batch->aux; ud = batch->aux + 3 * NS; uc = batch->aux + 4 * NS;
    }
    const int warps_per_block = 8;
    int64_t need = (R + warps_per_block - 1) / warps_per_block;
    int64_t cap = (int64_t)num_sms() * 8;
    unsigned nb = (unsigned)(need < cap ? need : cap);
    const float inv_r = 1.0f / (float)R;
#define TG_RK2(TD, TC, OD, OC, MPL)                                                                             \
    render_kernel<TD, TC, OD, OC, MPL><<<nb, 256, 0, s>>>((const TD *)dg->store, (const TC *)cg->store, dg->res, \
                                                          rays_o, rays_d, R, S, seed, ray_base, bg, rgb_out,       \
                                                          target_rgb, dldc, inv_r, loss_sum, xs, ud, uc)
#define TG_RK(TD, TC, OD, OC) \
    do { if (S <= 256) TG_RK2(TD, TC, OD, OC, 8); else TG_RK2(TD, TC, OD, OC, 16); } while (0)
    const int key = dg->order * 10 + cg->order;
    if (dg->dtype == TG_F32 && cg->dtype == TG_F32) {
        if (key == 21) TG_RK(float, float, 2, 1); else if (key == 0) TG_RK(float, float, 0, 0);
        else if (key == 20) TG_RK(float, float, 2, 0); else if (key == 11) TG_RK(float, float, 1, 1);
        else return fail(TG_EINVAL, "%s: unsupported order pair %d/%d", who, dg->order, cg->order);
    } else if (dg->dtype == TG_BF16 && cg->dtype == TG_BF16) {
        if (key == 21) TG_RK(__nv_bfloat16, __nv_bfloat16, 2, 1); else if (key == 0) TG_RK(__nv_bfloat16, __nv_bfloat16, 0, 0);
        else if (key == 20) TG_RK(__nv_bfloat16, __nv_bfloat16, 2, 0); else if (key == 11) TG_RK(__nv_bfloat16, __nv_bfloat16, 1, 1);
        else return fail(TG_EINVAL, "%s: unsupported order pair %d/%d", who, dg->order, cg->order);
    } else {
        return fail(TG_EINVAL, "%s: both grids must be FP32 or both BF16", who);
    }
#undef TG_RK
#undef TG_RK2
    if ((st = launch_status(who)) != TG_OK || !train) return st;
    // coefficient gradients of both grids through the binned backward
    if ((st = tg_batch_bin(batch, xs, NS, s)) != TG_OK) return st;
    if ((st = tg_query_backward_binned(dg, batch, ud, nullptr, density_grad, TG_ORDER_INPUT, s)) != TG_OK) return st;
    return tg_query_backward_binned(cg, batch, uc, nullptr, color_grad, TG_ORDER_INPUT, s);
}

extern "C" tg_status tg_render_rays(const tg_grid *dg, const tg_grid *cg, const float *rays_o, const float *rays_d,
                                    int64_t R, int S, uint64_t seed, uint64_t ray_base, float bg, float *rgb_out,
                                    const float *target_rgb, tg_batch *batch, float *density_grad, float *color_grad,
                                    float *loss_sum, tg_stream stream)
{
    if (!rgb_out && R > 0) return fail(TG_EINVAL, "tg_render_rays: rgb_out is NULL");
    return render_impl(dg, cg, rays_o, rays_d, R, S, seed, ray_base, bg, rgb_out, target_rgb, nullptr, batch,
                       density_grad, color_grad, loss_sum, (cudaStream_t)stream, "tg_render_rays");
}

extern "C" tg_status tg_render_rays_backward(const tg_grid *dg, const tg_grid *cg, const float *rays_o,
                                             const float *rays_d, int64_t R, int S, uint64_t seed, uint64_t ray_base,
                                             float bg, const float *dL_drgb, tg_batch *batch, float *density_grad,
                                             float *color_grad, float *rgb_out, tg_stream stream)
{
    if (!dL_drgb && R > 0) return fail(TG_EINVAL, "tg_render_rays_backward: dL_drgb is NULL");
    return render_impl(dg, cg, rays_o, rays_d, R, S, seed, ray_base, bg, rgb_out, nullptr, dL_drgb, batch,
                       density_grad, color_grad, nullptr, (cudaStream_t)stream, "tg_render_rays_backward");
}
