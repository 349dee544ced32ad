// Total variation term of Sec. 3.2 (the form of Plenoxels) over a 3-D grid's
// FP32 master coefficients: for every vertex v and coefficient channel c,
//   n(v, c) = sqrt(D_x^2 + D_y^2 + D_z^2),  D_a = theta(v + e_a, c) - theta(v, c)
// (D_a = 0 past the upper faces), L_TV = sum_{v,c} n(v, c) / res^3.
//
// dL/dtheta(v, c) = [-(D_x + D_y + D_z)(v) / n(v) + sum_a D_a(v - e_a) / n(v - e_a)] / res^3
// is a gather over v and its three lower neighbours, so every thread owns one
// vertex column and no write is shared. A block covers 32 x 8 vertices in x, y
// and marches along z with the planes z - 1, z, z + 1 (with a halo) in shared
// memory while plane z + 2 streams in through asynchronous copies, so each
// coefficient is read from HBM about once and the gradient is read and
// written once: 12 bytes per coefficient.
#include "tg_binned.cuh"

namespace tg {

constexpr int kTvX = 32, kTvY = 8, kTvZ = 32;
constexpr int kTvRows = kTvY + 2;               // y0 - 1 .. y0 + 8
constexpr int kTvCols = kTvX + 4;               // x0 - 2 .. x0 + 33 (the row start stays 16-byte aligned)
constexpr int kTvBufs = 4;                      // planes z - 1, z, z + 1 and the one streaming in

// Asynchronous 16-byte global -> shared copy of the first `bytes` (0..16)
// bytes of src; the rest of the 16 bytes is zero-filled.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes)
                 : "memory");
}
// Asynchronous 4-byte copy (bytes = 0 zero-fills).
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Asynchronous 8-byte copy (bytes = 0 or 4 zero-fills the rest).
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes)
                 : "memory");
}

// Starts copying plane z of the block's tile - rows y0 - 1 .. y0 + 8, vertices
// x0 - 2 .. x0 + 33, all NV coefficients, in the global vertex order - into dst
// in copies of W floats; everything outside the grid arrives as zeros.
// Alignment: a row starts at float (z res + y) res NV of a 16-byte aligned
// array and the tile at float (x0 - 2) NV of it, x0 a multiple of 32; W = 4
// needs res NV and 2 NV to be multiples of 4 (both offsets then are), W = 2 needs
// res NV even (then (x0 - 2) NV is even too). tv_copy_width picks W.
template <int NV, int W>
__device__ __forceinline__ void tv_fetch_plane(const float *__restrict__ theta, int res, int x0, int y0, int z,
                                               float *dst)
{
    constexpr int row_floats = kTvCols * NV;                       // a multiple of W
    constexpr int chunks = kTvRows * row_floats / W;
    const int tid = threadIdx.y * kTvX + threadIdx.x;
    const int64_t rowlen = (int64_t)res * NV;
    const int64_t x_begin = (int64_t)(x0 - 2) * NV;                // valid floats of a row: [0, rowlen)
    for (int i = tid; i < chunks; i += kTvX * kTvY) {
        const int row = i / (row_floats / W), k = i - row * (row_floats / W);
        const int y = y0 - 1 + row;
        const int64_t f0 = x_begin + (int64_t)W * k;               // first float of the chunk within its row
        int bytes = 0;
        const float *src = theta;
        if (z >= 0 && z < res && y >= 0 && y < res && f0 >= 0 && f0 < rowlen) {
            bytes = (int)(min((int64_t)W, rowlen - f0) * 4);
            src = theta + ((int64_t)z * res + y) * rowlen + f0;
        }
        if constexpr (W == 4) cp_async16(dst + W * i, src, bytes);
        else if constexpr (W == 2) cp_async8(dst + W * i, src, bytes);
        else cp_async4(dst + i, src, bytes);
    }
}

// 1 / sqrt(n2) for n2 > 0, else 0 (a zero term contributes no gradient).
__device__ __forceinline__ float tv_rnorm(float n2) { return n2 > 0.f ? rsqrtf(n2) : 0.f; }

template <int NV>
__device__ __forceinline__ void tv_load_grad(const float *p, float *g)
{
    if constexpr (NV % 2 == 0) {
#pragma unroll
        for (int c = 0; c < NV / 2; ++c) {
            const float2 v = reinterpret_cast<const float2 *>(p)[c];
            g[2 * c] = v.x;
            g[2 * c + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < NV; ++c) g[c] = p[c];
    }
}

template <int NV>
__device__ __forceinline__ void tv_store_grad(float *p, const float *g)
{
    if constexpr (NV % 2 == 0) {
#pragma unroll
        for (int c = 0; c < NV / 2; ++c) reinterpret_cast<float2 *>(p)[c] = make_float2(g[2 * c], g[2 * c + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < NV; ++c) p[c] = g[c];
    }
}

template <int NV, int W>
__global__ void __launch_bounds__(kTvX * kTvY)
tv_kernel(const float *__restrict__ theta, int res, float scale, float *__restrict__ grad, float *__restrict__ loss)
{
    extern __shared__ __align__(16) float sm[];
    constexpr int plane = kTvRows * kTvCols * NV;
    constexpr int RP = kTvCols * NV;                               // row pitch (floats)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * kTvX, y0 = blockIdx.y * kTvY, zb = blockIdx.z * kTvZ;
    const int ze = min(zb + kTvZ, res);
    // ring of kTvBufs planes: plane z lives in buffer (z - zb + 1) mod 4
    tv_fetch_plane<NV, W>(theta, res, x0, y0, zb - 1, sm);
    tv_fetch_plane<NV, W>(theta, res, x0, y0, zb, sm + plane);
    tv_fetch_plane<NV, W>(theta, res, x0, y0, zb + 1, sm + 2 * plane);
    cp_async_commit();
    tv_fetch_plane<NV, W>(theta, res, x0, y0, zb + 2, sm + 3 * plane);
    cp_async_commit();
    const int x = x0 + tx, y = y0 + ty;
    const bool in = x < res && y < res;
    const bool hx = x + 1 < res, hy = y + 1 < res;                 // the +x / +y neighbour exists
    const int64_t plane_stride = (int64_t)res * res * NV;
    float *gp = grad + ((int64_t)zb * res + y) * res * NV + (int64_t)x * NV;
    float gold[NV];
    if (in) tv_load_grad<NV>(gp, gold);
    cp_async_wait<1>();                                            // planes zb - 1 .. zb + 1 have landed
    __syncthreads();
    const int at = (ty + 1) * RP + (tx + 2) * NV;                  // this vertex's block inside a plane
    float lsum = 0.f;
    int cur = 1;                                                   // buffer of plane z
    for (int z = zb; z < ze; ++z) {
        const bool hz = z + 1 < res;
        const float *Pm = sm + ((cur + 3) & 3) * plane, *P0 = sm + cur * plane, *Pp = sm + ((cur + 1) & 3) * plane;
        if (in) {
            float gnew[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                const float *am = Pm + at + c, *a0 = P0 + at + c, *ap = Pp + at + c;
                const float t0 = a0[0];
                // this vertex's own term
                const float dx = hx ? a0[NV] - t0 : 0.f;
                const float dy = hy ? a0[RP] - t0 : 0.f;
                const float dz = hz ? ap[0] - t0 : 0.f;
                const float n2 = dx * dx + dy * dy + dz * dz;
                const float rn = tv_rnorm(n2);
                lsum += n2 * rn;
                float g = -(dx + dy + dz) * rn;
                if (x > 0) {            // u = v - e_x: D_x(u) = t0 - theta(u)
                    const float tu = a0[-NV];
                    const float ux = t0 - tu;
                    const float uy = hy ? a0[RP - NV] - tu : 0.f;
                    const float uz = hz ? ap[-NV] - tu : 0.f;
                    g += ux * tv_rnorm(ux * ux + uy * uy + uz * uz);
                }
                if (y > 0) {            // u = v - e_y
                    const float tu = a0[-RP];
                    const float ux = hx ? a0[NV - RP] - tu : 0.f;
                    const float uy = t0 - tu;
                    const float uz = hz ? ap[-RP] - tu : 0.f;
                    g += uy * tv_rnorm(ux * ux + uy * uy + uz * uz);
                }
                if (z > 0) {            // u = v - e_z
                    const float tu = am[0];
                    const float ux = hx ? am[NV] - tu : 0.f;
                    const float uy = hy ? am[RP] - tu : 0.f;
                    const float uz = t0 - tu;
                    g += uz * tv_rnorm(ux * ux + uy * uy + uz * uz);
                }
                gnew[c] = fmaf(scale, g, gold[c]);
            }
            tv_store_grad<NV>(gp, gnew);
            gp += plane_stride;
            if (z + 1 < ze) tv_load_grad<NV>(gp, gold);
        }
        __syncthreads();                                           // plane z - 1 is no longer read
        if (z + 3 <= ze) tv_fetch_plane<NV, W>(theta, res, x0, y0, z + 3, sm + ((cur + 3) & 3) * plane);
        cp_async_commit();
        cp_async_wait<1>();                                        // plane z + 2 has landed
        __syncthreads();
        cur = (cur + 1) & 3;
    }
    cp_async_wait<0>();
    if (!loss) return;
    __shared__ float part[kTvX * kTvY / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    const int tid = ty * kTvX + tx;
    if ((tid & 31) == 0) part[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < kTvX * kTvY / 32; ++w) s += part[w];
        atomicAdd(loss, s);
    }
}

// Floats per asynchronous copy such that every copy's global address is aligned to its size.
inline int tv_copy_width(int res, int nv)
{
    const int64_t row = (int64_t)res * nv;
    if (nv % 2 == 0 && row % 4 == 0) return 4;
    if (row % 2 == 0) return 2;
    return 1;
}

template <int NV, int W>
static tg_status tv_launch_w(const tg_grid *g, float scale, float *coef_grad, float *loss_sum, cudaStream_t s)
{
    const int smem = kTvBufs * kTvRows * kTvCols * NV * (int)sizeof(float);
    if (smem > 48 * 1024) {
        tg_status st = cuda_status(cudaFuncSetAttribute((const void *)tv_kernel<NV, W>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                                   "tg_tv_step: shared memory attribute");
        if (st != TG_OK) return st;
    }
    dim3 grid((g->res + kTvX - 1) / kTvX, (g->res + kTvY - 1) / kTvY, (g->res + kTvZ - 1) / kTvZ);
    tv_kernel<NV, W><<<grid, dim3(kTvX, kTvY), smem, s>>>(g->master, g->res, scale, coef_grad, loss_sum);
    return launch_status("tg_tv_step");
}

template <int NV>
static tg_status tv_launch(const tg_grid *g, float scale, float *coef_grad, float *loss_sum, cudaStream_t s)
{
    switch (tv_copy_width(g->res, NV)) {
    case 4: return tv_launch_w<NV, (NV % 2 == 0 ? 4 : 1)>(g, scale, coef_grad, loss_sum, s);
    case 2: return tv_launch_w<NV, 2>(g, scale, coef_grad, loss_sum, s);
    default: return tv_launch_w<NV, 1>(g, scale, coef_grad, loss_sum, s);
    }
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_tv_step(const tg_grid *g, float lambda, float *coef_grad, float *loss_sum, tg_stream stream)
{
    if (!g || !coef_grad) return fail(TG_EINVAL, "tg_tv_step: NULL grid or coef_grad");
    if (g->dim != 3) return fail(TG_EINVAL, "tg_tv_step: 3-D grids only");
    if (!(lambda >= 0.f)) return fail(TG_EINVAL, "tg_tv_step: lambda must be >= 0");
    const int nv = g->K * g->C;
    if (nv % 2 == 0 && ((uintptr_t)coef_grad & 7) != 0)
        return fail(TG_EINVAL, "tg_tv_step: coef_grad must be 8-byte aligned");
    const double v = (double)g->res * g->res * g->res;
    const float scale = (float)(lambda / v);
    cudaStream_t s = (cudaStream_t)stream;
    switch (nv) {
    case 1: return tv_launch<1>(g, scale, coef_grad, loss_sum, s);
    case 2: return tv_launch<2>(g, scale, coef_grad, loss_sum, s);
    case 3: return tv_launch<3>(g, scale, coef_grad, loss_sum, s);
    case 4: return tv_launch<4>(g, scale, coef_grad, loss_sum, s);
    case 8: return tv_launch<8>(g, scale, coef_grad, loss_sum, s);
    case 10: return tv_launch<10>(g, scale, coef_grad, loss_sum, s);
    case 12: return tv_launch<12>(g, scale, coef_grad, loss_sum, s);
    case 16: return tv_launch<16>(g, scale, coef_grad, loss_sum, s);
    case 20: return tv_launch<20>(g, scale, coef_grad, loss_sum, s);
    case 30: return tv_launch<30>(g, scale, coef_grad, loss_sum, s);
    case 40: return tv_launch<40>(g, scale, coef_grad, loss_sum, s);
    default: return fail(TG_EINVAL, "tg_tv_step: unsupported coefficient count %d", nv);
    }
}
