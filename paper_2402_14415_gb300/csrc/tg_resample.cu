// Progressive resolution (Sec. 4.1 trains coarse to fine): the field of one
// 3-D grid re-expanded as the Taylor data of another. At every destination
// vertex (coordinates fl32(j / (res_dst - 1)), located in the source grid by
// Eq. 2) the destination series takes the value, the gradient and, at order
// 2, the Hessian of the blended source field f = sum_i w_i T_i (Eq. 4):
//   grad f = sum_i T_i grad w_i + w_i grad T_i
//   Hess f = sum_i T_i Hess w_i + grad w_i (grad T_i)^T + grad T_i (grad w_i)^T + w_i Hess T_i
// (world units: d w / dx = (res_src - 1) d w / dt; Hess w has only mixed terms).
// One thread per destination vertex; the destination's FP32 master is written
// in the exchange layout and its stored copy is rounded from it afterwards.
#include "tg_internal.cuh"

namespace tg {

template <typename TS, int OS>
__global__ void __launch_bounds__(256)
resample_kernel(const TS *__restrict__ src, int res_src, int C, float *__restrict__ dst, int res_dst, int order_dst)
{
    constexpr int KS = Basis<3, OS>::K;
    const int KD = order_dst == 0 ? 1 : (order_dst == 1 ? 4 : 10);     // coefficients per dst vertex and channel
    const int64_t nd = (int64_t)res_dst * res_dst * res_dst;
    const float s = (float)(res_src - 1), h = 1.0f / s;
    const float den = (float)(res_dst - 1);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nd; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t jx = v % res_dst, jy = (v / res_dst) % res_dst, jz = v / ((int64_t)res_dst * res_dst);
        const float x[3] = {__fdiv_rn((float)jx, den), __fdiv_rn((float)jy, den), __fdiv_rn((float)jz, den)};
        int c[3];
        float t[3];
        locate<3>(x, res_src, s, c, t);
        const int64_t v0 = base_vertex<3>(c, res_src);
        for (int ch = 0; ch < C; ++ch) {
            float f = 0.f, g[3] = {0.f, 0.f, 0.f}, H[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int b[3] = {i & 1, (i >> 1) & 1, i >> 2};
                float th[KS];
                load_block<TS, KS>(src + ((v0 + corner_offset<3>(i, res_src)) * C + ch) * KS, th);
                float a[3], dl[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    a[e] = b[e] ? t[e] : 1.f - t[e];
                    dl[e] = (t[e] - (float)b[e]) * h;
                }
                // T, grad T = g + H delta, Hess T = H of this vertex's series
                float H0[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
                float gT[3] = {0.f, 0.f, 0.f};
                float T = th[0];
                if constexpr (OS >= 1) {
#pragma unroll
                    for (int e = 0; e < 3; ++e) gT[e] = th[1 + e];
                }
                if constexpr (OS >= 2) {
                    H0[0][0] = th[4]; H0[1][1] = th[5]; H0[2][2] = th[6];
                    H0[0][1] = H0[1][0] = th[7];
                    H0[0][2] = H0[2][0] = th[8];
                    H0[1][2] = H0[2][1] = th[9];
                }
                if constexpr (OS >= 1) {
                    float q = 0.f;
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        float hd = 0.f;
#pragma unroll
                        for (int k = 0; k < 3; ++k) hd += H0[e][k] * dl[k];
                        q += dl[e] * (gT[e] + 0.5f * hd);
                        gT[e] += hd;
                    }
                    T += q;
                }
                const float w = a[0] * a[1] * a[2];
                const float sg[3] = {b[0] ? s : -s, b[1] ? s : -s, b[2] ? s : -s};
                const float gw[3] = {sg[0] * a[1] * a[2], sg[1] * a[0] * a[2], sg[2] * a[0] * a[1]};
                f = fmaf(w, T, f);
#pragma unroll
                for (int e = 0; e < 3; ++e) g[e] += gw[e] * T + w * gT[e];
                if (order_dst >= 2) {
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            float hw = 0.f;           // d^2 w / dx_e dx_k: mixed terms only
                            if (e != k) hw = sg[e] * sg[k] * a[3 - e - k];
                            H[e][k] += hw * T + gw[e] * gT[k] + gT[e] * gw[k] + w * H0[e][k];
                        }
                    }
                }
            }
            float *out = dst + (v * C + ch) * KD;
            out[0] = f;
            if (order_dst >= 1) {
                out[1] = g[0]; out[2] = g[1]; out[3] = g[2];
            }
            if (order_dst >= 2) {
                out[4] = H[0][0]; out[5] = H[1][1]; out[6] = H[2][2];
                out[7] = H[0][1]; out[8] = H[0][2]; out[9] = H[1][2];
            }
        }
    }
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_resample(const tg_grid *src, tg_grid *dst, tg_stream stream)
{
    if (!src || !dst) return fail(TG_EINVAL, "tg_resample: NULL grid");
    if (src->dim != 3 || dst->dim != 3) return fail(TG_EINVAL, "tg_resample: 3-D grids only");
    if (src->C != dst->C) return fail(TG_EINVAL, "tg_resample: the grids must have the same channels");
    if (src == dst) return fail(TG_EINVAL, "tg_resample: src and dst must differ");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nd = dst->nv;
    int64_t need = (nd + 255) / 256, cap = (int64_t)num_sms() * 8;
    const unsigned nb = (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
#define TG_RS(TS, OS) resample_kernel<TS, OS><<<nb, 256, 0, s>>>((const TS *)src->store, src->res, src->C, \
                                                                 dst->master, dst->res, dst->order)
#define TG_RS_ORDER(TS) \
    (src->order == 0 ? (TG_RS(TS, 0), 0) : src->order == 1 ? (TG_RS(TS, 1), 0) : (TG_RS(TS, 2), 0))
    if (src->dtype == TG_F32) TG_RS_ORDER(float);
    else if (src->dtype == TG_BF16) TG_RS_ORDER(__nv_bfloat16);
    else TG_RS_ORDER(__half);
#undef TG_RS_ORDER
#undef TG_RS
    tg_status st = launch_status("tg_resample");
    if (st != TG_OK) return st;
    return tg_set_coefs(dst, dst->master, stream);      // the stored copy from the new master
}
