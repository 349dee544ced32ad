// Internal definitions of the GB300 TaylorGrid library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/taylorgrid.h"

struct tg_grid {
    int dim, res, order, C, K;
    tg_dtype dtype;
    int device;
    int64_t nv;          // res^dim vertices
    int64_t ncoef;       // nv * C * K
    void *store;         // stored coefficients in the storage dtype (== master for FP32)
    float *master;       // FP32 master copy
    void *adam_m;        // Adam first moment (lazily allocated): FP32, or BF16 with lp_moments
    void *adam_v;        // Adam second moment
    bool lp_moments;     // BF16 moments (the BF16 / FP16 storage form), FP32 arithmetic
    struct tg_batch *auto_batch;   // binning scratch of large tg_query / tg_query_backward calls (lazy)
    cudaEvent_t auto_event;        // last use of auto_batch
};

namespace tg {

// Records a failure message for tg_last_error() and returns the status.
tg_status fail(tg_status s, const char *fmt, ...);
// Maps a CUDA error to TG_EDEVICE with a message; TG_OK for cudaSuccess.
tg_status cuda_status(cudaError_t e, const char *what);
// Checks the launch error of the previous kernel.
tg_status launch_status(const char *what);

// Every device allocation of the library goes through these two: cudaMalloc /
// cudaMallocAsync with the status mapped (TG_ENOMEM when the device is out of
// memory), after the failure-injection counter of tg_inject_alloc_failures.
tg_status dev_alloc(void **p, size_t bytes, const char *what);
tg_status dev_alloc_async(void **p, size_t bytes, cudaStream_t s, const char *what);

int num_sms();                      // SM count of the current device (cached per device)
constexpr int kBinChunksPerSm = 2;  // point chunks of the binning per SM (one histogram row each): two coarse-pass blocks share an SM
// Resident blocks per SM of a kernel at a launch shape (cached per device and kernel).
int blocks_per_sm(const void *kernel, int threads, size_t smem);

// The point-parallel query pair (one thread per point; tg_query.cu). tg_query /
// tg_query_backward use them for small, 2-D or captured batches.
tg_status query_point_parallel(const tg_grid *g, const float *pts, int64_t N, float *out, float *grad_x,
                               cudaStream_t s);
tg_status query_backward_point_parallel(const tg_grid *g, const float *pts, int64_t N, const float *dL_df,
                                        const float *dL_dgradx, float *coef_grad, cudaStream_t s);

// Adam over all coefficients (tg_adam.cu); with step_dev != nullptr the
// 0-based step index is read on the device and prm->step is ignored; lazy
// skips the entries whose gradient is 0 (tg_adam_step_lazy).
tg_status adam_launch(tg_grid *g, float *grad, const tg_adam *prm, const int64_t *step_dev, cudaStream_t s,
                      bool lazy = false);
tg_status ensure_adam_state(tg_grid *g);

inline int num_coefs(int dim, int order)
{
    return 1 + (order >= 1 ? dim : 0) + (order >= 2 ? dim * (dim + 1) / 2 : 0);
}

inline size_t storage_bytes(tg_dtype d) { return d == TG_F32 ? 4 : 2; }
// Bytes of one Adam moment: BF16 moments go with BF16 / FP16 storage.
inline size_t moment_bytes(const tg_grid *g) { return g->lp_moments ? 2 : 4; }

// ---------------------------------------------------------------------------
// Storage types
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Largest vector width (bytes, <= 16) that keeps every block of BYTES bytes,
// placed at an arbitrary multiple of BYTES, naturally aligned.
template <int BYTES> struct VecWidth {
    static constexpr int value = (BYTES % 16 == 0) ? 16 : (BYTES % 8 == 0) ? 8 : (BYTES % 4 == 0) ? 4 : 2;
};

// Loads NV consecutive values of type T (one vertex block) through the
// read-only path with the widest aligned vector loads, widened to FP32.
template <typename T, int NV>
__device__ __forceinline__ void load_block(const T *__restrict__ p, float *out)
{
    constexpr int BYTES = NV * (int)sizeof(T);
    constexpr int VW = VecWidth<BYTES>::value;
    constexpr int NW = BYTES / VW;
    if constexpr (VW == 16) {
        uint4 r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = __ldg(reinterpret_cast<const uint4 *>(p) + i);
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    } else if constexpr (VW == 8) {
        uint2 r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = __ldg(reinterpret_cast<const uint2 *>(p) + i);
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    } else if constexpr (VW == 4) {
        unsigned r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = __ldg(reinterpret_cast<const unsigned *>(p) + i);
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    } else {
        unsigned short r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    }
}

// Adds NV consecutive FP32 values into global memory with vector reductions
// (float4 / float2 atomics are native on sm_90 and later).
template <int NV>
__device__ __forceinline__ void red_block(float *p, const float *v)
{
    constexpr int VW = VecWidth<NV * 4>::value;
    if constexpr (VW == 16) {
#pragma unroll
        for (int i = 0; i < NV / 4; ++i)
            atomicAdd(reinterpret_cast<float4 *>(p) + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
    } else if constexpr (VW == 8) {
        // an 8-byte-aligned block of 8k + 2 floats: 16-byte vector reductions from
        // whichever of its first two elements is 16-byte aligned, and one 8-byte
        // one for the remaining pair (K = 10: 3 reductions a vertex instead of 5)
        if (reinterpret_cast<uintptr_t>(p) & 15) {
            atomicAdd(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
#pragma unroll
            for (int i = 0; i < (NV - 2) / 4; ++i)
                atomicAdd(reinterpret_cast<float4 *>(p + 2 + 4 * i),
                          make_float4(v[2 + 4 * i], v[3 + 4 * i], v[4 + 4 * i], v[5 + 4 * i]));
        } else {
#pragma unroll
            for (int i = 0; i < (NV - 2) / 4; ++i)
                atomicAdd(reinterpret_cast<float4 *>(p + 4 * i),
                          make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
            atomicAdd(reinterpret_cast<float2 *>(p + NV - 2), make_float2(v[NV - 2], v[NV - 1]));
        }
    } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) atomicAdd(p + i, v[i]);
    }
}

// ---------------------------------------------------------------------------
// Eq. 2: voxel lookup (normative FP32 index rule)
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void locate(const float *x, int res, float scale, int *c, float *t)
{
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        float xd = fminf(fmaxf(x[d], 0.0f), 1.0f);   // fmaxf(NaN, 0) = 0
        float u = __fmul_rn(xd, scale);
        int ci = min((int)floorf(u), res - 2);
        c[d] = ci;
        t[d] = __fsub_rn(u, (float)ci);
    }
}

// ---------------------------------------------------------------------------
// Eq. 1 / Eq. 3: the truncated series as a linear form in its coefficients,
// evaluated at the world offset delta = x - v_i.
// phi[k] = dT/dtheta_k at delta; dphi[k][d] = d phi_k / d delta_d.
// Basis order: 1, delta_d, delta_d^2 / 2, then delta_a delta_b for a < b in
// the order (x,y), (x,z), (y,z).
// ---------------------------------------------------------------------------
template <int DIM, int ORDER>
struct Basis {
    static constexpr int K = 1 + (ORDER >= 1 ? DIM : 0) + (ORDER >= 2 ? DIM * (DIM + 1) / 2 : 0);

    __device__ __forceinline__ static void value(const float *dl, float *phi)
    {
        phi[0] = 1.0f;
        if constexpr (ORDER >= 1) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) phi[1 + d] = dl[d];
        }
        if constexpr (ORDER >= 2) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) phi[1 + DIM + d] = 0.5f * dl[d] * dl[d];
            if constexpr (DIM == 3) {
                phi[7] = dl[0] * dl[1];
                phi[8] = dl[0] * dl[2];
                phi[9] = dl[1] * dl[2];
            } else {
                phi[5] = dl[0] * dl[1];
            }
        }
    }

    // Series value T = sum_k theta_k phi_k and its delta-gradient g + H delta.
    __device__ __forceinline__ static float eval(const float *th, const float *dl, float *grad)
    {
        float T = th[0];
#pragma unroll
        for (int d = 0; d < DIM; ++d) grad[d] = 0.0f;
        if constexpr (ORDER >= 1) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) { T = fmaf(th[1 + d], dl[d], T); grad[d] = th[1 + d]; }
        }
        if constexpr (ORDER >= 2) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const float hd = th[1 + DIM + d];
                T = fmaf(0.5f * hd, dl[d] * dl[d], T);
                grad[d] = fmaf(hd, dl[d], grad[d]);
            }
            if constexpr (DIM == 3) {
                const float hxy = th[7], hxz = th[8], hyz = th[9];
                T = fmaf(hxy, dl[0] * dl[1], T);
                T = fmaf(hxz, dl[0] * dl[2], T);
                T = fmaf(hyz, dl[1] * dl[2], T);
                grad[0] = fmaf(hxy, dl[1], fmaf(hxz, dl[2], grad[0]));
                grad[1] = fmaf(hxy, dl[0], fmaf(hyz, dl[2], grad[1]));
                grad[2] = fmaf(hxz, dl[0], fmaf(hyz, dl[1], grad[2]));
            } else {
                const float hxy = th[5];
                T = fmaf(hxy, dl[0] * dl[1], T);
                grad[0] = fmaf(hxy, dl[1], grad[0]);
                grad[1] = fmaf(hxy, dl[0], grad[1]);
            }
        }
        return T;
    }

    // acc_k += s phi_k(delta) (+ sum_d q_d dphi_k/ddelta_d when HAS_Q).
    template <bool HAS_Q>
    __device__ __forceinline__ static void accumulate(float s, const float *q, const float *dl, float *acc)
    {
        acc[0] += s;
        if constexpr (ORDER >= 1) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) acc[1 + d] = fmaf(s, dl[d], HAS_Q ? acc[1 + d] + q[d] : acc[1 + d]);
        }
        if constexpr (ORDER >= 2) {
            float hs = 0.5f * s;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                float a = fmaf(hs, dl[d] * dl[d], acc[1 + DIM + d]);
                acc[1 + DIM + d] = HAS_Q ? fmaf(q[d], dl[d], a) : a;
            }
            if constexpr (DIM == 3) {
                const float sx = s * dl[0];
                float a7 = fmaf(sx, dl[1], acc[7]), a8 = fmaf(sx, dl[2], acc[8]), a9 = fmaf(s * dl[1], dl[2], acc[9]);
                if constexpr (HAS_Q) {
                    a7 = fmaf(q[0], dl[1], fmaf(q[1], dl[0], a7));
                    a8 = fmaf(q[0], dl[2], fmaf(q[2], dl[0], a8));
                    a9 = fmaf(q[1], dl[2], fmaf(q[2], dl[1], a9));
                }
                acc[7] = a7; acc[8] = a8; acc[9] = a9;
            } else {
                float a5 = fmaf(s * dl[0], dl[1], acc[5]);
                if constexpr (HAS_Q) a5 = fmaf(q[0], dl[1], fmaf(q[1], dl[0], a5));
                acc[5] = a5;
            }
        }
    }

    // Adjoint of eval: given s = dL/dT and q = dL/d(grad T), returns
    // dL/dtheta_k = s phi_k + sum_d q_d dphi_k/ddelta_d.
    __device__ __forceinline__ static void adjoint(float s, const float *q, const float *dl, float *out)
    {
        out[0] = s;
        if constexpr (ORDER >= 1) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) out[1 + d] = fmaf(s, dl[d], q[d]);
        }
        if constexpr (ORDER >= 2) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) out[1 + DIM + d] = fmaf(0.5f * s, dl[d] * dl[d], q[d] * dl[d]);
            if constexpr (DIM == 3) {
                out[7] = fmaf(s, dl[0] * dl[1], fmaf(q[0], dl[1], q[1] * dl[0]));
                out[8] = fmaf(s, dl[0] * dl[2], fmaf(q[0], dl[2], q[2] * dl[0]));
                out[9] = fmaf(s, dl[1] * dl[2], fmaf(q[1], dl[2], q[2] * dl[1]));
            } else {
                out[5] = fmaf(s, dl[0] * dl[1], fmaf(q[0], dl[1], q[1] * dl[0]));
            }
        }
    }
};

// Multilinear weight of corner i (bits b_d = (i >> d) & 1) and its t-gradient
// (Eq. 4). Called from fully unrolled corner loops, so i folds to a constant.
template <int DIM>
__device__ __forceinline__ float corner_weight(int i, const float *t, float *dw)
{
    float w = 1.0f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) w *= ((i >> d) & 1) ? t[d] : 1.0f - t[d];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        float g = ((i >> d) & 1) ? 1.0f : -1.0f;
#pragma unroll
        for (int e = 0; e < DIM; ++e)
            if (e != d) g *= ((i >> e) & 1) ? t[e] : 1.0f - t[e];
        dw[d] = g;
    }
    return w;
}

// Linear index of the base vertex (lower corner) of cell c and the offset of corner i.
template <int DIM>
__device__ __forceinline__ int64_t base_vertex(const int *c, int res)
{
    if constexpr (DIM == 3) return (int64_t)c[0] + (int64_t)res * ((int64_t)c[1] + (int64_t)res * c[2]);
    else return (int64_t)c[0] + (int64_t)res * c[1];
}
template <int DIM>
__device__ __forceinline__ int64_t corner_offset(int i, int res)
{
    int64_t o = (i & 1);
    if (i & 2) o += res;
    if (DIM == 3 && (i & 4)) o += (int64_t)res * res;
    return o;
}

// ---------------------------------------------------------------------------
// 3-D point tables: everything of Eq. 3 / Eq. 4 that depends on the point
// but not on the corner's coefficients, computed once per point. For corner
// bits b, delta_d = u[b_d][d] = (t_d - b_d) h is the world offset x - v_i
// (h = 1 / (res - 1)); the series basis is
//   1, u[b_d][d], h[b_d][d] = u^2 / 2, p_ab[b_a][b_b] = u[b_a][a] u[b_b][b]
// and the blend weight is w = a[b_x][0] a[b_y][1] a[b_z][2], a[0] = 1 - t,
// a[1] = t. T_i and its adjoint then cost one FMA per coefficient.
// ---------------------------------------------------------------------------
template <int ORDER>
struct PointTables3 {
    float u[2][3];            // delta components (t - b) h
    float h[2][3];            // delta^2 / 2
    float pxy[2][2], pxz[2][2], pyz[2][2];
    float a[2][3];            // weight factors
    float wxy[2][2];          // a_x a_y

    __device__ __forceinline__ PointTables3(const float *t, float cell)
    {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            u[0][d] = t[d] * cell;
            u[1][d] = (t[d] - 1.0f) * cell;
            a[0][d] = 1.0f - t[d];
            a[1][d] = t[d];
            if (ORDER >= 2) {
                h[0][d] = 0.5f * u[0][d] * u[0][d];
                h[1][d] = 0.5f * u[1][d] * u[1][d];
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                wxy[i][j] = a[i][0] * a[j][1];
                if (ORDER >= 2) {
                    pxy[i][j] = u[i][0] * u[j][1];
                    pxz[i][j] = u[i][0] * u[j][2];
                    pyz[i][j] = u[i][1] * u[j][2];
                }
            }
    }

    template <int I>
    __device__ __forceinline__ float weight() const
    {
        return wxy[I & 1][(I >> 1) & 1] * a[(I >> 2) & 1][2];
    }

    // d w / d t_d for corner I (d w / d x_d = (res - 1) d w / d t_d).
    template <int I>
    __device__ __forceinline__ void dweight(float *dw) const
    {
        constexpr int bx = I & 1, by = (I >> 1) & 1, bz = (I >> 2) & 1;
        dw[0] = (bx ? 1.f : -1.f) * a[by][1] * a[bz][2];
        dw[1] = (by ? 1.f : -1.f) * a[bx][0] * a[bz][2];
        dw[2] = (bz ? 1.f : -1.f) * wxy[bx][by];
    }

    // T_i = sum_k theta_k phi_k(delta_i) (Eq. 1 / Eq. 3).
    template <int I>
    __device__ __forceinline__ float value(const float *th) const
    {
        constexpr int bx = I & 1, by = (I >> 1) & 1, bz = (I >> 2) & 1;
        float T = th[0];
        if constexpr (ORDER >= 1) {
            T = fmaf(th[1], u[bx][0], T);
            T = fmaf(th[2], u[by][1], T);
            T = fmaf(th[3], u[bz][2], T);
        }
        if constexpr (ORDER >= 2) {
            T = fmaf(th[4], h[bx][0], T);
            T = fmaf(th[5], h[by][1], T);
            T = fmaf(th[6], h[bz][2], T);
            T = fmaf(th[7], pxy[bx][by], T);
            T = fmaf(th[8], pxz[bx][bz], T);
            T = fmaf(th[9], pyz[by][bz], T);
        }
        return T;
    }

    // d T_i / d delta = g + H delta.
    template <int I>
    __device__ __forceinline__ void gradient(const float *th, float *g) const
    {
        constexpr int bx = I & 1, by = (I >> 1) & 1, bz = (I >> 2) & 1;
        if constexpr (ORDER == 0) {
            g[0] = g[1] = g[2] = 0.f;
        } else {
            g[0] = th[1]; g[1] = th[2]; g[2] = th[3];
            if constexpr (ORDER >= 2) {
                const float ux = u[bx][0], uy = u[by][1], uz = u[bz][2];
                g[0] = fmaf(th[4], ux, fmaf(th[7], uy, fmaf(th[8], uz, g[0])));
                g[1] = fmaf(th[5], uy, fmaf(th[7], ux, fmaf(th[9], uz, g[1])));
                g[2] = fmaf(th[6], uz, fmaf(th[8], ux, fmaf(th[9], uy, g[2])));
            }
        }
    }

    // acc_k += s phi_k(delta_i) (+ sum_d q_d d phi_k / d delta_d when HAS_Q).
    template <int I, bool HAS_Q>
    __device__ __forceinline__ void accumulate(float s, const float *q, float *acc) const
    {
        constexpr int bx = I & 1, by = (I >> 1) & 1, bz = (I >> 2) & 1;
        acc[0] += s;
        if constexpr (ORDER >= 1) {
            const float ux = u[bx][0], uy = u[by][1], uz = u[bz][2];
            acc[1] = fmaf(s, ux, HAS_Q ? acc[1] + q[0] : acc[1]);
            acc[2] = fmaf(s, uy, HAS_Q ? acc[2] + q[1] : acc[2]);
            acc[3] = fmaf(s, uz, HAS_Q ? acc[3] + q[2] : acc[3]);
            if constexpr (ORDER >= 2) {
                acc[4] = fmaf(s, h[bx][0], acc[4]);
                acc[5] = fmaf(s, h[by][1], acc[5]);
                acc[6] = fmaf(s, h[bz][2], acc[6]);
                acc[7] = fmaf(s, pxy[bx][by], acc[7]);
                acc[8] = fmaf(s, pxz[bx][bz], acc[8]);
                acc[9] = fmaf(s, pyz[by][bz], acc[9]);
                if constexpr (HAS_Q) {
                    acc[4] = fmaf(q[0], ux, acc[4]);
                    acc[5] = fmaf(q[1], uy, acc[5]);
                    acc[6] = fmaf(q[2], uz, acc[6]);
                    acc[7] = fmaf(q[0], uy, fmaf(q[1], ux, acc[7]));
                    acc[8] = fmaf(q[0], uz, fmaf(q[2], ux, acc[8]));
                    acc[9] = fmaf(q[1], uz, fmaf(q[2], uy, acc[9]));
                }
            }
        }
    }
};

// Compile-time loop over the 8 corners: F::template run<I>() for I = 0..7.
template <int I, typename F>
__device__ __forceinline__ void for_corners(F &&f)
{
    if constexpr (I < 8) {
        f(std::integral_constant<int, I>{});
        for_corners<I + 1>(f);
    }
}

// Counter-based generator: splitmix64 (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) { return mix64(mix64(seed) + stream); }
// U[0,1) with 24 bits from a precomputed stream key.
__device__ __forceinline__ float uniform_k(uint64_t key, uint64_t idx)
{
    return (float)(mix64(key + idx) >> 40) * (1.0f / 16777216.0f);
}
__device__ __forceinline__ float normal_k(uint64_t key, uint64_t idx)
{
    float ua = uniform_k(key, 2 * idx), ub = uniform_k(key, 2 * idx + 1);
    return sqrtf(-2.0f * log1pf(-ua)) * cospif(2.0f * ub);
}

}  // namespace tg

// Dispatch a runtime (dim, order, channels) to a templated functor call:
// F::template run<DIM, ORDER, C>(args...).
#define TG_DISPATCH_SHAPE(dim, order, C, ...)                                                     \
    [&]() -> tg_status {                                                                          \
        switch ((dim) * 100 + (order) * 10 + (C)) {                                               \
        case 301: return __VA_ARGS__(3, 0, 1); case 302: return __VA_ARGS__(3, 0, 2);             \
        case 303: return __VA_ARGS__(3, 0, 3); case 304: return __VA_ARGS__(3, 0, 4);             \
        case 311: return __VA_ARGS__(3, 1, 1); case 312: return __VA_ARGS__(3, 1, 2);             \
        case 313: return __VA_ARGS__(3, 1, 3); case 314: return __VA_ARGS__(3, 1, 4);             \
        case 321: return __VA_ARGS__(3, 2, 1); case 322: return __VA_ARGS__(3, 2, 2);             \
        case 323: return __VA_ARGS__(3, 2, 3); case 324: return __VA_ARGS__(3, 2, 4);             \
        case 201: return __VA_ARGS__(2, 0, 1); case 202: return __VA_ARGS__(2, 0, 2);             \
        case 203: return __VA_ARGS__(2, 0, 3); case 204: return __VA_ARGS__(2, 0, 4);             \
        case 211: return __VA_ARGS__(2, 1, 1); case 212: return __VA_ARGS__(2, 1, 2);             \
        case 213: return __VA_ARGS__(2, 1, 3); case 214: return __VA_ARGS__(2, 1, 4);             \
        case 221: return __VA_ARGS__(2, 2, 1); case 222: return __VA_ARGS__(2, 2, 2);             \
        case 223: return __VA_ARGS__(2, 2, 3); case 224: return __VA_ARGS__(2, 2, 4);             \
        default: return tg::fail(TG_EINVAL, "unsupported shape dim=%d order=%d channels=%d",      \
                                 (int)(dim), (int)(order), (int)(C));                             \
        }                                                                                         \
    }()
