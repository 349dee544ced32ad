// Total variation term of Sec. 3.2 (the form of Plenoxels) over a 3-D grid's
// FP32 master coefficients: for every vertex v and coefficient channel c,
//   n(v, c) = sqrt(D_x^2 + D_y^2 + D_z^2),  D_a = theta(v + e_a, c) - theta(v, c)
// (D_a = 0 past the upper faces), L_TV = sum_{v,c} n(v, c) / res^3.
//
// dL/dtheta(v, c) = [-(D_x + D_y + D_z)(v) / n(v) + sum_a D_a(v - e_a) / n(v - e_a)] / res^3
// is a gather over v and its three lower neighbours, so every thread owns one
// vertex column and no write is shared. A block covers 32 x 8 vertices in x, y
// and marches along z with three planes (z - 1, z, z + 1, each with a one-
// vertex halo) in shared memory, so each coefficient is read from HBM about
// once and the gradient is read and written once: 12 bytes per coefficient.
#include "tg_internal.cuh"

namespace tg {

constexpr int kTvX = 32, kTvY = 8, kTvZ = 32;
constexpr int kTvPX = kTvX + 2, kTvPY = kTvY + 2;

__device__ __forceinline__ void tv_load_plane(const float *__restrict__ theta, int res, int nv, int x0, int y0, int z,
                                              float *dst)
{
    const int tid = threadIdx.y * kTvX + threadIdx.x;
    const int per_row = kTvPX * nv;
    const int64_t rowlen = (int64_t)res * nv;
    for (int i = tid; i < kTvPY * per_row; i += kTvX * kTvY) {
        const int row = i / per_row, rem = i - row * per_row;
        const int xv = rem / nv, c = rem - xv * nv;
        const int y = y0 - 1 + row, x = x0 - 1 + xv;
        float v = 0.f;
        if (z >= 0 && z < res && y >= 0 && y < res && x >= 0 && x < res)
            v = __ldg(theta + ((int64_t)z * res + y) * rowlen + (int64_t)x * nv + c);
        dst[(c * kTvPY + row) * kTvPX + xv] = v;
    }
}

__global__ void __launch_bounds__(kTvX * kTvY)
tv_kernel(const float *__restrict__ theta, int res, int nv, float scale, float *__restrict__ grad,
          float *__restrict__ loss)
{
    extern __shared__ float sm[];
    const int plane = nv * kTvPY * kTvPX;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * kTvX, y0 = blockIdx.y * kTvY, zb = blockIdx.z * kTvZ;
    const int ze = min(zb + kTvZ, res);
    float *P[3] = {sm, sm + plane, sm + 2 * plane};       // planes z - 1, z, z + 1
    tv_load_plane(theta, res, nv, x0, y0, zb - 1, P[0]);
    tv_load_plane(theta, res, nv, x0, y0, zb, P[1]);
    tv_load_plane(theta, res, nv, x0, y0, zb + 1, P[2]);
    __syncthreads();
    const int x = x0 + tx, y = y0 + ty;
    const bool in = x < res && y < res;
    const bool hx = x + 1 < res, hy = y + 1 < res;        // the +x / +y neighbour exists
    const int64_t rowlen = (int64_t)res * nv;
    const int at = (ty + 1) * kTvPX + (tx + 1);           // this vertex inside a plane slice
    float lsum = 0.f;
    for (int z = zb; z < ze; ++z) {
        const bool hz = z + 1 < res;
        if (in) {
            float *gp = grad + ((int64_t)z * res + y) * rowlen + (int64_t)x * nv;
            for (int c = 0; c < nv; ++c) {
                const float *am = P[0] + c * kTvPY * kTvPX, *a0 = P[1] + c * kTvPY * kTvPX,
                            *ap = P[2] + c * kTvPY * kTvPX;
                const float t0 = a0[at];
                // this vertex's own term
                const float dx = hx ? a0[at + 1] - t0 : 0.f;
                const float dy = hy ? a0[at + kTvPX] - t0 : 0.f;
                const float dz = hz ? ap[at] - t0 : 0.f;
                const float n = sqrtf(dx * dx + dy * dy + dz * dz);
                lsum += n;
                float g = n > 0.f ? -(dx + dy + dz) / n : 0.f;
                if (x > 0) {            // u = v - e_x: D_x(u) = t0 - theta(u)
                    const float tu = a0[at - 1];
                    const float ux = t0 - tu;
                    const float uy = hy ? a0[at - 1 + kTvPX] - tu : 0.f;
                    const float uz = hz ? ap[at - 1] - tu : 0.f;
                    const float nu = sqrtf(ux * ux + uy * uy + uz * uz);
                    if (nu > 0.f) g += ux / nu;
                }
                if (y > 0) {            // u = v - e_y
                    const float tu = a0[at - kTvPX];
                    const float ux = hx ? a0[at - kTvPX + 1] - tu : 0.f;
                    const float uy = t0 - tu;
                    const float uz = hz ? ap[at - kTvPX] - tu : 0.f;
                    const float nu = sqrtf(ux * ux + uy * uy + uz * uz);
                    if (nu > 0.f) g += uy / nu;
                }
                if (z > 0) {            // u = v - e_z
                    const float tu = am[at];
                    const float ux = hx ? am[at + 1] - tu : 0.f;
                    const float uy = hy ? am[at + kTvPX] - tu : 0.f;
                    const float uz = t0 - tu;
                    const float nu = sqrtf(ux * ux + uy * uy + uz * uz);
                    if (nu > 0.f) g += uz / nu;
                }
                gp[c] += scale * g;
            }
        }
        __syncthreads();                                  // plane z - 1 is no longer read
        float *t = P[0];
        P[0] = P[1];
        P[1] = P[2];
        P[2] = t;
        if (z + 1 < ze) tv_load_plane(theta, res, nv, x0, y0, z + 2, P[2]);
        __syncthreads();
    }
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

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_tv_step(const tg_grid *g, float lambda, float *coef_grad, float *loss_sum, tg_stream stream)
{
    if (!g || !coef_grad) return fail(TG_EINVAL, "tg_tv_step: NULL grid or coef_grad");
    if (g->dim != 3) return fail(TG_EINVAL, "tg_tv_step: 3-D grids only");
    if (!(lambda >= 0.f)) return fail(TG_EINVAL, "tg_tv_step: lambda must be >= 0");
    const int nv = g->K * g->C;
    const int smem = 3 * nv * kTvPY * kTvPX * (int)sizeof(float);
    if (smem > 48 * 1024) {
        tg_status st = cuda_status(cudaFuncSetAttribute((const void *)tv_kernel,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                                   "tg_tv_step: shared memory attribute");
        if (st != TG_OK) return st;
    }
    const double v = (double)g->res * g->res * g->res;
    dim3 grid((g->res + kTvX - 1) / kTvX, (g->res + kTvY - 1) / kTvY, (g->res + kTvZ - 1) / kTvZ);
    tv_kernel<<<grid, dim3(kTvX, kTvY), smem, (cudaStream_t)stream>>>(g->master, g->res, nv, (float)(lambda / v),
                                                                       coef_grad, loss_sum);
    return launch_status("tg_tv_step");
}
