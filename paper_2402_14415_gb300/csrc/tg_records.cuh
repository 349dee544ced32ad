// Point-parallel passes over a binned batch, for batches with few points per
// brick (Eq. 2 - Eq. 4 and their adjoint).
//
// The brick kernels stage a whole 9^3 coefficient tile per occupied brick
// (forward: a TMA load; backward: a TMA reduce-add of the tile) and run fixed
// per-brick phases over its 729 vertices, so below a few dozen points per
// brick their cost follows the number of bricks, not of points. These passes
// instead give every record of the batch (brick order) one thread that
// gathers, or scatters with vector FP32 reductions, its 8 corner blocks
// directly; consecutive threads hold points of one brick, so the corner
// blocks they touch share L2 lines, and lanes whose points share a cell are
// combined by their group leader before the reductions.
#pragma once

#include <stdlib.h>

#include "tg_query.cuh"

namespace tg {

// Average points per brick below which tg_query_binned / tg_query_backward_binned
// take these passes (the deterministic backward always takes the brick kernels).
// Measured on 128^3 and 256^3 order-2 grids with half uniform, half clustered
// points: for value-only passes the two paths cross near 48 points per brick;
// with spatial gradients (forward d f / d x, backward dL/d grad f) the brick
// kernels do more per point and the crossing is near 96.
constexpr int kRecordsMaxPerBrick = 48;
constexpr int kRecordsMaxPerBrickGrad = 96;

// Whether a brick tile of this grid can be moved by TMA: every row of res
// vertex blocks and the array start on 16-byte boundaries, and a box row of
// box_inner elements is whole 16-byte units of at most 256 elements.
inline bool brick_tma_ok(int res, int nv, int elem, int box_inner, const void *base)
{
    return ((size_t)res * nv * elem) % 16 == 0 && ((uintptr_t)base & 15) == 0 && (box_inner * elem) % 16 == 0 &&
           box_inner <= 256;
}

// The records path is chosen by the batch's average occupancy, and always where
// the grid's rows do not suit TMA; TG_BINNED_PATH=brick or =records in the
// environment forces one path (read at every call, for measurements and for
// tests of both paths).
inline bool use_records_path(int64_t n, int64_t nbricks, bool with_grad, bool tma_ok)
{
    if (!tma_ok) return true;
    const char *e = getenv("TG_BINNED_PATH");
    if (e && e[0] == 'b') return false;
    if (e && e[0] == 'r') return true;
    return n < (int64_t)(with_grad ? kRecordsMaxPerBrickGrad : kRecordsMaxPerBrick) * nbricks;
}

// Forward: f and optionally d f / d x of record n, written at its binned slot
// or (IN_ORDER) at its input index.
template <typename T, int ORDER, int C, bool IN_ORDER>
__global__ void __launch_bounds__(kQueryThreads)
records_fwd_kernel(const T *__restrict__ coefs, int res, const float4 *__restrict__ sorted, int64_t N,
                   float *__restrict__ out, float *__restrict__ gx)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += stride) {
        const float4 q = sorted[n];
        const float x[3] = {q.x, q.y, q.z};
        const int64_t dst = IN_ORDER ? (int64_t)__float_as_int(q.w) : n;
        float f[C], gu[C][3];
        point_eval<T, 3, ORDER, C>(coefs, res, x, f, gu);
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            out[dst * C + ch] = f[ch];
            if (gx) {
#pragma unroll
                for (int d = 0; d < 3; ++d) gx[(dst * C + ch) * 3 + d] = gu[ch][d];
            }
        }
    }
}

// Backward: the coefficient gradient of record n's upstreams (read at its
// binned slot or, IN_ORDER, at its input index) added into grad.
template <int ORDER, int C, bool IN_ORDER>
__global__ void __launch_bounds__(kQueryThreads)
records_bwd_kernel(int res, const float4 *__restrict__ sorted, int64_t N, const float *__restrict__ dLdf,
                   const float *__restrict__ dLdg, float *__restrict__ grad)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool has_g = dLdg != nullptr;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < N; base += stride) {
        const int64_t n = base + lane;
        const unsigned valid = __ballot_sync(0xffffffffu, n < N);
        if (n >= N) break;
        const float4 q = sorted[n];
        const float x[3] = {q.x, q.y, q.z};
        const int64_t m = IN_ORDER ? (int64_t)__float_as_int(q.w) : n;
        float uf[C], ug[C][3];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            uf[ch] = __ldg(dLdf + m * C + ch);
#pragma unroll
            for (int d = 0; d < 3; ++d) ug[ch][d] = has_g ? __ldg(dLdg + (m * C + ch) * 3 + d) : 0.0f;
        }
        point_scatter<3, ORDER, C>(res, x, uf, ug, has_g, lane, valid, grad);
    }
}

inline unsigned records_blocks(int64_t n)
{
    const int64_t b = (n + kQueryThreads - 1) / kQueryThreads, cap = (int64_t)num_sms() * 16;
    return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace tg
