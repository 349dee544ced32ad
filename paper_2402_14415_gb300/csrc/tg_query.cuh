// Point-parallel query kernels: one thread per point gathers the 2^D corner
// blocks straight from HBM (Eq. 2 - Eq. 4) and, for the backward pass,
// scatters the coefficient gradient with vector FP32 reductions.
#pragma once

#include "tg_internal.cuh"

namespace tg {

constexpr int kQueryThreads = 256;

// f(x) (Eq. 4 over the Eq. 3 series of the 2^D corners) and d f / d x in world units at one point.
template <typename T, int DIM, int ORDER, int C>
__device__ __forceinline__ void point_eval(const T *__restrict__ coefs, int res, const float *x, float *f,
                                           float (*gu)[DIM])
{
    using B = Basis<DIM, ORDER>;
    constexpr int K = B::K;
    constexpr int NV = K * C;
    const float scale = (float)(res - 1), h = 1.0f / (float)(res - 1);
    int c[DIM];
    float t[DIM];
    locate<DIM>(x, res, scale, c, t);
    const int64_t v0 = base_vertex<DIM>(c, res);
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        f[ch] = 0.0f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) gu[ch][d] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < (1 << DIM); ++i) {
        float th[NV];
        load_block<T, NV>(coefs + (v0 + corner_offset<DIM>(i, res)) * NV, th);
        float dw[DIM], dl[DIM];
        const float w = corner_weight<DIM>(i, t, dw);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            dl[d] = (t[d] - (float)((i >> d) & 1)) * h;          // x - v_i
            dw[d] *= scale;                                      // d w / d x
        }
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            float g[DIM];
            const float Tv = B::eval(th + ch * K, dl, g);        // Eq. 3
            f[ch] = fmaf(w, Tv, f[ch]);                          // Eq. 4
#pragma unroll
            for (int d = 0; d < DIM; ++d) gu[ch][d] = fmaf(dw[d], Tv, fmaf(w, g[d], gu[ch][d]));
        }
    }
}

// Forward: f(x) and, if gx != nullptr, d f / d x in world units.
template <typename T, int DIM, int ORDER, int C>
__global__ void __launch_bounds__(kQueryThreads)
query_fwd_kernel(const T *__restrict__ coefs, int res, const float *__restrict__ pts, int64_t N,
                 float *__restrict__ out, float *__restrict__ gx)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += stride) {
        float x[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = __ldg(pts + n * DIM + d);
        float f[C], gu[C][DIM];
        point_eval<T, DIM, ORDER, C>(coefs, res, x, f, gu);
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            out[n * C + ch] = f[ch];
            if (gx) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) gx[(n * C + ch) * DIM + d] = gu[ch][d];
            }
        }
    }
}

// Coefficient gradient of one corner for all channels: s = dL/dT_i and
// q = dL/d(grad_delta T_i), from the upstream value / spatial gradients.
template <int DIM, int ORDER, int C>
__device__ __forceinline__ void corner_contrib(int i, const float *t, float scale, const float *uf,
                                               const float (*ug)[DIM], bool has_g, float *ctr)
{
    using B = Basis<DIM, ORDER>;
    constexpr int K = B::K;
    const float h = 1.0f / scale;
    float dw[DIM], dl[DIM];
    const float w = corner_weight<DIM>(i, t, dw);
#pragma unroll
    for (int d = 0; d < DIM; ++d) dl[d] = (t[d] - (float)((i >> d) & 1)) * h;   // x - v_i
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
        float s = w * uf[ch];
        float q[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) q[d] = 0.0f;
        if (has_g) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const float gd = ug[ch][d];
                s = fmaf(dw[d] * scale, gd, s);          // d w / d x = (res - 1) d w / d t
                q[d] = w * gd;
            }
        }
        B::adjoint(s, q, dl, ctr + ch * K);
    }
}

// The coefficient gradient of one point (upstreams uf and, with has_g, ug)
// added into grad. Lanes of the warp (mask `valid`, all of which call this)
// whose points fall in the same cell are combined by the group leader before
// the vector reduction (warp-level match + shuffle); a warp with no shared
// cell reduces directly.
template <int DIM, int ORDER, int C>
__device__ __forceinline__ void point_scatter(int res, const float *x, const float *uf, const float (*ug)[DIM],
                                              bool has_g, int lane, unsigned valid, float *__restrict__ grad)
{
    constexpr int K = Basis<DIM, ORDER>::K;
    constexpr int NV = K * C;
    const float scale = (float)(res - 1);
    int c[DIM];
    float t[DIM];
    locate<DIM>(x, res, scale, c, t);
    const int64_t v0 = base_vertex<DIM>(c, res);
    const unsigned peers = __match_any_sync(valid, (unsigned long long)v0);
    const int group = __popc(peers);
    const int max_group = __reduce_max_sync(valid, (unsigned)group);
    const bool leader = (__ffs(peers) - 1) == lane;
#pragma unroll
    for (int i = 0; i < (1 << DIM); ++i) {
        float ctr[NV];
        corner_contrib<DIM, ORDER, C>(i, t, scale, uf, ug, has_g, ctr);
        if (max_group > 1) {
            // gather the r-th other member of each group into its leader
            for (int r = 1; r < max_group; ++r) {
                const int src = r < group ? (int)__fns(peers, 0, r + 1) : lane;
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    const float v = __shfl_sync(valid, ctr[k], src);
                    if (leader && r < group) ctr[k] += v;
                }
            }
            if (!leader) continue;
        }
        red_block<NV>(grad + (v0 + corner_offset<DIM>(i, res)) * NV, ctr);
    }
}

// Backward: scatter-add into grad, one point per thread.
template <int DIM, int ORDER, int C>
__global__ void __launch_bounds__(kQueryThreads)
query_bwd_kernel(int res, const float *__restrict__ pts, int64_t N, const float *__restrict__ dLdf,
                 const float *__restrict__ dLdg, float *__restrict__ grad)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool has_g = dLdg != nullptr;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < N; base += stride) {
        const int64_t n = base + lane;
        const unsigned valid = __ballot_sync(0xffffffffu, n < N);
        if (n >= N) break;
        float x[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = __ldg(pts + n * DIM + d);
        float uf[C], ug[C][DIM];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            uf[ch] = __ldg(dLdf + n * C + ch);
#pragma unroll
            for (int d = 0; d < DIM; ++d) ug[ch][d] = has_g ? __ldg(dLdg + (n * C + ch) * DIM + d) : 0.0f;
        }
        point_scatter<DIM, ORDER, C>(res, x, uf, ug, has_g, lane, valid, grad);
    }
}

}  // namespace tg
