// Adam's per-coefficient update and moment storage, shared by the grid-wide
// step (tg_adam.cu) and the server's batched step (tg_serve_batch.cu).
#pragma once

#include "tg_internal.cuh"

namespace tg {

struct AdamCoef {
    float beta1, beta2, one_m_b1, one_m_b2;
    float step_size;       // lr / (1 - beta1^t)
    float inv_sqrt_bc2;    // 1 / sqrt(1 - beta2^t)
    float eps;
};

__device__ __forceinline__ float adam_one(float &p, float g, float &m, float &v, const AdamCoef &a)
{
    m = fmaf(a.beta1, m, a.one_m_b1 * g);
    v = fmaf(a.beta2, v, a.one_m_b2 * g * g);
    const float denom = fmaf(sqrtf(v), a.inv_sqrt_bc2, a.eps);   // sqrt(v_hat) + eps
    p -= a.step_size * __fdividef(m, denom);
    return p;
}

template <typename T>
__device__ __forceinline__ void store4(T *dst, int64_t j, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void store4<float>(float *, int64_t, float, float, float, float) {}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16 *dst, int64_t j, float a, float b, float c, float d)
{
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&lo);
    u.y = *reinterpret_cast<unsigned *>(&hi);
    *reinterpret_cast<uint2 *>(dst + j) = u;
}
template <>
__device__ __forceinline__ void store4<__half>(__half *dst, int64_t j, float a, float b, float c, float d)
{
    __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&lo);
    u.y = *reinterpret_cast<unsigned *>(&hi);
    *reinterpret_cast<uint2 *>(dst + j) = u;
}

// LAZY: entries whose gradient is 0 keep parameter and moments; a group of
// four zero gradients costs only its 16-byte gradient read.
__device__ __forceinline__ void adam_lazy_one(float &p, float g, float &m, float &v, const AdamCoef &a)
{
    if (g != 0.0f) adam_one(p, g, m, v, a);
}

// Four moments from FP32 (float4) or BF16 (8-byte) storage, widened to FP32, and back.
template <typename M> struct Moments;
template <> struct Moments<float> {
    __device__ __forceinline__ static float4 load(const float *p, int64_t j) { return reinterpret_cast<const float4 *>(p)[j]; }
    __device__ __forceinline__ static void store(float *p, int64_t j, float4 v) { reinterpret_cast<float4 *>(p)[j] = v; }
    __device__ __forceinline__ static float get(const float *p, int64_t j) { return p[j]; }
    __device__ __forceinline__ static void put(float *p, int64_t j, float v) { p[j] = v; }
};
template <> struct Moments<__nv_bfloat16> {
    __device__ __forceinline__ static float4 load(const __nv_bfloat16 *p, int64_t j)
    {
        const uint2 u = reinterpret_cast<const uint2 *>(p)[j];
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
        const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
        return make_float4(a.x, a.y, b.x, b.y);
    }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, int64_t j, float4 v)
    {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&lo);
        u.y = *reinterpret_cast<unsigned *>(&hi);
        reinterpret_cast<uint2 *>(p)[j] = u;
    }
    __device__ __forceinline__ static float get(const __nv_bfloat16 *p, int64_t j) { return __bfloat162float(p[j]); }
    __device__ __forceinline__ static void put(__nv_bfloat16 *p, int64_t j, float v) { p[j] = __float2bfloat16_rn(v); }
};

}  // namespace tg
