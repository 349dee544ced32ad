// Total variation term of Sec. 3.2 (the form of Plenoxels) over a 3-D grid's
// FP32 master coefficients: for every vertex v and coefficient channel c,
//   n(v, c) = sqrt(D_x^2 + D_y^2 + D_z^2),  D_a = theta(v + e_a, c) - theta(v, c)
// (D_a = 0 past the upper faces), L_TV = sum_{v,c} n(v, c) / res^3.
//
// dL/dtheta(v, c) = [-(D_x + D_y + D_z)(v) / n(v) + sum_a D_a(v - e_a) / n(v - e_a)] / res^3
// is a gather over v and its three lower neighbours, so every thread owns its
// coefficients and no write is shared. Each norm is wanted by four vertices
// (v and its three upper neighbours); a thread owns one coefficient in kTvRows
// consecutive rows and walks them along z, so n(v - e_y) is its own previous
// row's norm (one extra for the row below the strip), n(v - e_z) its own
// previous plane's, and only n(v - e_x) is formed a second time: 2 + 1 / kTvRows
// norms per coefficient. The values of plane z that plane z + 1 reuses stay in
// registers, so a step loads 3 + 4 / kTvRows values of theta per coefficient.
//
// Mapping: a block is 256 consecutive floats of a row strip (the vertices
// x .. x + 256 / NV of rows y .. y + kTvRows - 1, all their channels), so every
// load of a warp - at a fixed offset of +-NV, +-res NV or +-res^2 NV floats
// from the thread's own coefficient - is one contiguous 128-byte span.
// Neighbouring strips and planes are read by the blocks that own them at about
// the same time and come from L2; HBM sees theta about once and the gradient
// read and written once: 12 bytes per coefficient. There is no shared-memory
// tile, so the occupancy does not depend on the number of coefficients per vertex.
#include "tg_internal.cuh"

namespace tg {

constexpr int kTvThreads = 256;
constexpr int kTvZ = 32;                       // planes per thread
constexpr int kTvRows = 4;                     // rows per thread

// 1 / sqrt(dx^2 + dy^2 + dz^2) (the approximate reciprocal square root of PTX,
// relative error below 2^-22), 0 where the sum is 0: a zero term contributes
// no gradient.
__device__ __forceinline__ float tv_rnorm(float n2)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(n2));
    return n2 > 0.f ? r : 0.f;
}

__global__ void __launch_bounds__(kTvThreads)
tv_kernel(const float *__restrict__ theta, int res, int nv, float scale, float *__restrict__ grad,
          float *__restrict__ loss)
{
    const int64_t R = (int64_t)res * nv;                           // floats per row
    const int64_t P = (int64_t)R * res;                            // floats per plane
    const int xi = blockIdx.x * kTvThreads + threadIdx.x;          // float index within a row
    const int y0 = blockIdx.y * kTvRows, zb = blockIdx.z * kTvZ, ze = min(zb + kTvZ, res);
    float lsum = 0.f;
    if (xi < R) {
        const int x = xi / nv;
        const bool hx = x + 1 < res, lx = x > 0;                   // v + e_x, v - e_x exist
        const bool below = y0 > 0;                                 // the row y0 - 1 exists
        int nr = res - y0;                                         // rows of the strip inside the grid
        nr = nr < kTvRows ? nr : kTvRows;
        const bool above = y0 + kTvRows < res;                     // the row y0 + kTvRows exists
        const float *col = theta + (int64_t)y0 * R + xi;           // row y0 at z = 0
        float *gcol = grad + (int64_t)y0 * R + xi;
        // plane z of the strip at v and v - e_x, and of row y0 - 1 at v (carried between planes)
        float a[kTvRows], am[kTvRows], qz[kTvRows], h = 0.f;
#pragma unroll
        for (int r = 0; r < kTvRows; ++r) {
            a[r] = am[r] = qz[r] = 0.f;
            if (r < nr) {
                const float *p = col + r * R + zb * P;
                a[r] = __ldg(p);
                if (lx) am[r] = __ldg(p - nv);
            }
        }
        if (below) h = __ldg(col - R + zb * P);
        if (zb > 0) {                                              // q_z = D_z / n of the plane below
            const float *p = col + (zb - 1) * P;
            float l[kTvRows + 1];
#pragma unroll
            for (int r = 0; r <= kTvRows; ++r) l[r] = (r < nr || (r == kTvRows && above)) ? __ldg(p + r * R) : 0.f;
#pragma unroll
            for (int r = 0; r < kTvRows; ++r) {
                if (r >= nr) continue;
                const float dx = hx ? __ldg(p + r * R + nv) - l[r] : 0.f;
                const float dy = (r + 1 < nr || (r + 1 == kTvRows && above)) ? l[r + 1] - l[r] : 0.f;
                const float dz = a[r] - l[r];
                qz[r] = dz * tv_rnorm(dx * dx + dy * dy + dz * dz);
            }
        }
        for (int z = zb; z < ze; ++z) {
            const bool hz = z + 1 < res;
            const float *p = col + z * P;
            float *gp = gcol + z * P;
            // plane z: v + e_x of the strip, row y0 - 1 at v + e_x, row y0 + kTvRows at v and v - e_x;
            // plane z + 1 at v and v - e_x; the gradient
            float ax[kTvRows], gold[kTvRows], b[kTvRows], bm[kTvRows];
#pragma unroll
            for (int r = 0; r < kTvRows; ++r) {
                ax[r] = (r < nr && hx) ? __ldg(p + r * R + nv) : 0.f;
                b[r] = (r < nr && hz) ? __ldg(p + r * R + P) : 0.f;
                bm[r] = (r < nr && hz && lx) ? __ldg(p + r * R + P - nv) : 0.f;
                gold[r] = r < nr ? gp[r * R] : 0.f;
            }
            const float hxv = (below && hx) ? __ldg(p - R + nv) : 0.f;
            const float hb = (below && hz) ? __ldg(p - R + P) : 0.f;
            const float t = above ? __ldg(p + kTvRows * R) : 0.f;
            const float tm = (above && lx) ? __ldg(p + kTvRows * R - nv) : 0.f;
            // q_y of the row below the strip
            float qy_prev = 0.f;
            if (below) {
                const float dx = hx ? hxv - h : 0.f, dy = a[0] - h, dz = hz ? hb - h : 0.f;
                qy_prev = dy * tv_rnorm(dx * dx + dy * dy + dz * dz);
            }
#pragma unroll
            for (int r = 0; r < kTvRows; ++r) {
                if (r >= nr) continue;
                const bool hy = r + 1 < nr || (r + 1 == kTvRows && above);
                const float up = r + 1 < kTvRows ? a[r + 1] : t;   // plane z at v + e_y and v - e_x + e_y
                const float upm = r + 1 < kTvRows ? am[r + 1] : tm;
                const float dx = hx ? ax[r] - a[r] : 0.f, dy = hy ? up - a[r] : 0.f, dz = hz ? b[r] - a[r] : 0.f;
                const float n2 = dx * dx + dy * dy + dz * dz;
                const float rv = tv_rnorm(n2);
                lsum = fmaf(n2, rv, lsum);
                float g = qy_prev + qz[r] - (dx + dy + dz) * rv;
                if (lx) {                                          // n(v - e_x): D_x = theta(v) - theta(v - e_x)
                    const float mx = a[r] - am[r], my = hy ? upm - am[r] : 0.f, mz = hz ? bm[r] - am[r] : 0.f;
                    g = fmaf(mx, tv_rnorm(mx * mx + my * my + mz * mz), g);
                }
                gp[r * R] = fmaf(scale, g, gold[r]);
                qy_prev = dy * rv;
                qz[r] = dz * rv;
            }
#pragma unroll
            for (int r = 0; r < kTvRows; ++r) {
                a[r] = b[r];
                am[r] = bm[r];
            }
            h = hb;
        }
    }
    if (!loss) return;
    __shared__ float part[kTvThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kTvThreads / 32; ++w) s += part[w];
        if (s != 0.f) atomicAdd(loss, s);
    }
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_tv_step(const tg_grid *g, float lambda, float *coef_grad, float *loss_sum, tg_stream stream)
{
    if (!g || !coef_grad) return fail(TG_EINVAL, "tg_tv_step: NULL grid or coef_grad");
    if (g->dim != 3) return fail(TG_EINVAL, "tg_tv_step: 3-D grids only");
    if (!(lambda >= 0.f)) return fail(TG_EINVAL, "tg_tv_step: lambda must be >= 0");
    const int64_t row = (int64_t)g->res * g->K * g->C;
    if (row >= ((int64_t)1 << 31) - kTvThreads) return fail(TG_EINVAL, "tg_tv_step: grid row too long");
    if (g->res > 65535) return fail(TG_EINVAL, "tg_tv_step: res above 65535");
    const double v = (double)g->res * g->res * g->res;
    const float scale = (float)(lambda / v);
    dim3 grid((unsigned)((row + kTvThreads - 1) / kTvThreads), (g->res + kTvRows - 1) / kTvRows,
              (g->res + kTvZ - 1) / kTvZ);
    tv_kernel<<<grid, kTvThreads, 0, (cudaStream_t)stream>>>(g->master, g->res, g->K * g->C, scale, coef_grad,
                                                            loss_sum);
    return launch_status("tg_tv_step");
}
