// Brick-binned query path (3-D): counting sort of the points by 8^3-cell
// brick, then one thread block per brick that
//   forward:  TMA-loads the brick's 9^3 vertex blocks into shared memory and
//             evaluates Eq. 3 / Eq. 4 for its points from there;
//   backward: accumulates the coefficient gradient of its points in a shared
//             9^3 block and adds it to the global gradient with one TMA
//             bulk-tensor reduce-add (element-wise atomic at L2), so bricks
//             that share a face combine correctly without per-point atomics.
#include <cudaTypedefs.h>
#include <stdlib.h>

#include <mutex>

#include "tg_internal.cuh"
#include "tg_tma.cuh"

struct tg_batch {
    int dim, res;
    int nb[3];            // bricks per axis
    int64_t nbricks;
    int64_t max_points;
    int64_t n;            // points binned by the last tg_batch_bin
    int *counts;          // nbricks + 1
    int *offsets;         // nbricks + 1, exclusive prefix sum of counts
    int *cursor;          // nbricks, scatter cursors
    float4 *sorted;       // max_points: (x, y, z, original index as int bits)
    int *status;          // device word: non-zero after a bounded wait gave up
    int device;
};

namespace tg {

constexpr int kBrick = 8;            // cells per brick edge
constexpr int kBV = kBrick + 1;      // vertices per brick edge
constexpr int kBinThreads = 256;
constexpr int kBrickThreads = 256;

// Elements per brick row in the TMA box: the 9 vertex blocks padded to 16 bytes.
template <typename T, int NV>
struct BoxInner {
    static constexpr int bytes = (kBV * NV * (int)sizeof(T) + 15) / 16 * 16;
    static constexpr int value = bytes / (int)sizeof(T);
    static constexpr int tile_bytes = kBV * kBV * bytes;
};

inline int box_inner_host(int nv, int elem) { return ((kBV * nv * elem + 15) / 16 * 16) / elem; }

template <int DIM>
__device__ __forceinline__ int brick_of(const int *c, int nbx, int nby)
{
    return (c[0] / kBrick) + nbx * ((c[1] / kBrick) + nby * (c[2] / kBrick));
}

__global__ void __launch_bounds__(kBinThreads)
bin_count_kernel(const float *__restrict__ pts, int64_t N, int res, int nbx, int nby, int *__restrict__ counts)
{
    const float scale = (float)(res - 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x[3] = {__ldg(pts + 3 * n), __ldg(pts + 3 * n + 1), __ldg(pts + 3 * n + 2)};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        atomicAdd(counts + brick_of<3>(c, nbx, nby), 1);
    }
}

// Single-block exclusive scan of counts[0..n) into offsets[0..n]; cursor = offsets.
__global__ void __launch_bounds__(1024) bin_scan_kernel(const int *__restrict__ counts, int *__restrict__ offsets,
                                                        int *__restrict__ cursor, int n)
{
    __shared__ int warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    int local = 0;
    for (int j = lo; j < hi; ++j) local += counts[j];
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int run = incl - local + (wid > 0 ? warp_sums[wid - 1] : 0);
    for (int j = lo; j < hi; ++j) {
        offsets[j] = run;
        cursor[j] = run;
        run += counts[j];
    }
    if (tid == blockDim.x - 1) offsets[n] = run;
}

__global__ void __launch_bounds__(kBinThreads)
bin_scatter_kernel(const float *__restrict__ pts, int64_t N, int res, int nbx, int nby, int *__restrict__ cursor,
                   float4 *__restrict__ sorted)
{
    const float scale = (float)(res - 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x[3] = {__ldg(pts + 3 * n), __ldg(pts + 3 * n + 1), __ldg(pts + 3 * n + 2)};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        const int slot = atomicAdd(cursor + brick_of<3>(c, nbx, nby), 1);
        sorted[slot] = make_float4(x[0], x[1], x[2], __int_as_float((int)n));
    }
}

// Loads NV consecutive values of type T from shared memory, widened to FP32.
template <typename T, int NV>
__device__ __forceinline__ void load_block_smem(const T *p, float *out)
{
    constexpr int BYTES = NV * (int)sizeof(T);
    constexpr int VW = VecWidth<BYTES>::value;
    constexpr int NW = BYTES / VW;
    if constexpr (VW == 16) {
        uint4 r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = reinterpret_cast<const uint4 *>(p)[i];
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    } else if constexpr (VW == 8) {
        uint2 r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = reinterpret_cast<const uint2 *>(p)[i];
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    } else if constexpr (VW == 4) {
        unsigned r[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) r[i] = reinterpret_cast<const unsigned *>(p)[i];
        const T *tp = reinterpret_cast<const T *>(r);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(tp[j]);
    } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = to_f32<T>(p[j]);
    }
}

// Forward over one brick per block.
template <typename T, int ORDER, int C>
__global__ void __launch_bounds__(kBrickThreads)
brick_fwd_kernel(const __grid_constant__ CUtensorMap cmap, int res, int nbx, int nby,
                 const float4 *__restrict__ sorted, const int *__restrict__ offsets, float *__restrict__ out,
                 float *__restrict__ gx, int *__restrict__ status)
{
    using B = Basis<3, ORDER>;
    constexpr int K = B::K;
    constexpr int NV = K * C;
    constexpr int BXI = BoxInner<T, NV>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    uint64_t &bar = *reinterpret_cast<uint64_t *>(smem_raw + BoxInner<T, NV>::tile_bytes);

    const int b = blockIdx.x;
    const int p0 = offsets[b], p1 = offsets[b + 1];
    if (p0 == p1) return;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, BoxInner<T, NV>::tile_bytes);
        tma_load_3d(tile, &cmap, x0 * NV, y0, z0, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0)) {
        if (threadIdx.x == 0) atomicExch(status, 1);
        mbar_wait_bounded(&bar, 0);          // second bounded wait for the copy in flight
        return;
    }

    const float scale = (float)(res - 1);
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const float4 q = sorted[p];
        const int64_t n = __float_as_int(q.w);
        const float x[3] = {q.x, q.y, q.z};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        const int lrow = (c[2] - z0) * kBV + (c[1] - y0);
        const int lx = c[0] - x0;
        float f[C], gu[C][3];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            f[ch] = 0.f;
            gu[ch][0] = gu[ch][1] = gu[ch][2] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = lrow + ((i >> 2) & 1) * kBV + ((i >> 1) & 1);
            float th[NV];
            load_block_smem<T, NV>(tile + row * BXI + (lx + (i & 1)) * NV, th);
            float dw[3], dl[3];
            const float w = corner_weight<3>(i, t, dw);
#pragma unroll
            for (int d = 0; d < 3; ++d) dl[d] = t[d] - (float)((i >> d) & 1);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                float g[3];
                const float Tv = B::eval(th + ch * K, dl, g);
                f[ch] = fmaf(w, Tv, f[ch]);
#pragma unroll
                for (int d = 0; d < 3; ++d) gu[ch][d] = fmaf(dw[d], Tv, fmaf(w, g[d], gu[ch][d]));
            }
        }
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            out[n * C + ch] = f[ch];
            if (gx) {
#pragma unroll
                for (int d = 0; d < 3; ++d) gx[(n * C + ch) * 3 + d] = gu[ch][d] * scale;
            }
        }
    }
}

// Backward over one brick per block: shared accumulation, one TMA reduce-add.
template <int ORDER, int C>
__global__ void __launch_bounds__(kBrickThreads)
brick_bwd_kernel(const __grid_constant__ CUtensorMap gmap, int res, int nbx, int nby,
                 const float4 *__restrict__ sorted, const int *__restrict__ offsets, const float *__restrict__ dLdf,
                 const float *__restrict__ dLdg)
{
    constexpr int K = Basis<3, ORDER>::K;
    constexpr int NV = K * C;
    constexpr int BXI = BoxInner<float, NV>::value;
    constexpr int TILE = kBV * kBV * BXI;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *acc = reinterpret_cast<float *>(smem_raw);

    const int b = blockIdx.x;
    const int p0 = offsets[b], p1 = offsets[b + 1];
    if (p0 == p1) return;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    for (int j = threadIdx.x; j < TILE / 4; j += blockDim.x)
        reinterpret_cast<float4 *>(acc)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    const float scale = (float)(res - 1);
    const bool has_g = dLdg != nullptr;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const float4 q = sorted[p];
        const int64_t n = __float_as_int(q.w);
        const float x[3] = {q.x, q.y, q.z};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        float uf[C], ug[C][3];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            uf[ch] = __ldg(dLdf + n * C + ch);
#pragma unroll
            for (int d = 0; d < 3; ++d) ug[ch][d] = has_g ? __ldg(dLdg + (n * C + ch) * 3 + d) : 0.f;
        }
        const int lrow = (c[2] - z0) * kBV + (c[1] - y0);
        const int lx = c[0] - x0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float dw[3], dl[3];
            const float w = corner_weight<3>(i, t, dw);
#pragma unroll
            for (int d = 0; d < 3; ++d) dl[d] = t[d] - (float)((i >> d) & 1);
            float *dst = acc + (lrow + ((i >> 2) & 1) * kBV + ((i >> 1) & 1)) * BXI + (lx + (i & 1)) * NV;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                float s = w * uf[ch], qv[3] = {0.f, 0.f, 0.f};
                if (has_g) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float gd = ug[ch][d] * scale;
                        s = fmaf(dw[d], gd, s);
                        qv[d] = w * gd;
                    }
                }
                float ctr[K];
                Basis<3, ORDER>::adjoint(s, qv, dl, ctr);
#pragma unroll
                for (int k = 0; k < K; ++k) atomicAdd(dst + ch * K + k, ctr[k]);
            }
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tma_reduce_add_3d(&gmap, acc, x0 * NV, y0, z0);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a res^3 x NV coefficient (or gradient) array viewed as the
// 3-D tensor [z][y][x * NV] with a box of 9 x 9 brick rows.
static tg_status make_brick_map(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int elem, int res, int nv)
{
    auto fn = encode_fn();
    if (!fn) return fail(TG_EDEVICE, "cuTensorMapEncodeTiled is unavailable from the driver");
    const int bxi = box_inner_host(nv, elem);
    if (bxi > 256) return fail(TG_EINVAL, "binned path: a brick row of %d elements exceeds the TMA box limit", bxi);
    if (((size_t)res * nv * elem) % 16 != 0)
        return fail(TG_EINVAL, "binned path: res * K * channels * elem (%d * %d * %d) must be a multiple of 16 bytes",
                    res, nv, elem);
    if (((uintptr_t)base & 15) != 0) return fail(TG_EINVAL, "binned path: array must be 16-byte aligned");
    cuuint64_t dims[3] = {(cuuint64_t)res * nv, (cuuint64_t)res, (cuuint64_t)res};
    cuuint64_t strides[2] = {(cuuint64_t)res * nv * elem, (cuuint64_t)res * res * nv * elem};
    cuuint32_t box[3] = {(cuuint32_t)bxi, (cuuint32_t)kBV, (cuuint32_t)kBV};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TG_EINVAL, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TG_OK;
}

static tg_status set_smem(const void *kernel, int bytes)
{
    if (bytes <= 48 * 1024) return TG_OK;
    return cuda_status(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
                       "binned path: shared memory attribute");
}

template <typename T>
struct BinnedLaunch {
    template <int DIM, int ORDER, int C>
    static tg_status fwd(const tg_grid *g, const tg_batch *bt, float *out, float *gx, cudaStream_t s)
    {
        if constexpr (DIM != 3) {
            return fail(TG_EINVAL, "binned path is 3-D only");
        } else {
            constexpr int NV = Basis<3, ORDER>::K * C;
            CUtensorMap map;
            const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : (g->dtype == TG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
            tg_status st = make_brick_map(&map, g->store, dt, (int)sizeof(T), g->res, NV);
            if (st != TG_OK) return st;
            auto k = brick_fwd_kernel<T, ORDER, C>;
            const int smem = BoxInner<T, NV>::tile_bytes + 16;     // tile + mbarrier
            if ((st = set_smem((const void *)k, smem)) != TG_OK) return st;
            k<<<(unsigned)bt->nbricks, kBrickThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted,
                                                                 bt->offsets, out, gx, bt->status);
            return launch_status("tg_query_binned");
        }
    }
};

template <int DIM, int ORDER, int C>
static tg_status binned_bwd(const tg_grid *g, const tg_batch *bt, const float *uf, const float *ug, float *grad,
                            cudaStream_t s)
{
    if constexpr (DIM != 3) {
        return fail(TG_EINVAL, "binned path is 3-D only");
    } else {
        constexpr int NV = Basis<3, ORDER>::K * C;
        CUtensorMap map;
        tg_status st = make_brick_map(&map, grad, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->res, NV);
        if (st != TG_OK) return st;
        auto k = brick_bwd_kernel<ORDER, C>;
        const int smem = BoxInner<float, NV>::tile_bytes;
        if ((st = set_smem((const void *)k, smem)) != TG_OK) return st;
        k<<<(unsigned)bt->nbricks, kBrickThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted,
                                                             bt->offsets, uf, ug);
        return launch_status("tg_query_backward_binned");
    }
}

static tg_status check_pair(const tg_grid *g, const tg_batch *bt, const char *who)
{
    if (!g || !bt) return fail(TG_EINVAL, "%s: NULL grid or batch", who);
    if (g->dim != 3 || bt->res != g->res) return fail(TG_EINVAL, "%s: batch was created for another grid shape", who);
    return TG_OK;
}

}  // namespace tg

using namespace tg;

extern "C" {

tg_status tg_batch_create(int dim, int res, int64_t max_points, tg_batch **out)
{
    if (!out) return fail(TG_EINVAL, "tg_batch_create: out is NULL");
    *out = nullptr;
    if (dim != 3) return fail(TG_EINVAL, "tg_batch_create: the binned path is 3-D only");
    if (res < 2 || res > 2048) return fail(TG_EINVAL, "tg_batch_create: res %d out of range", res);
    if (max_points < 0 || max_points > (int64_t)INT32_MAX) return fail(TG_EINVAL, "tg_batch_create: max_points out of range");
    tg_batch *b = (tg_batch *)calloc(1, sizeof(tg_batch));
    if (!b) return fail(TG_ENOMEM, "tg_batch_create: host allocation failed");
    b->dim = dim; b->res = res; b->max_points = max_points;
    cudaGetDevice(&b->device);
    b->nbricks = 1;
    for (int d = 0; d < 3; ++d) {
        b->nb[d] = (res - 1 + kBrick - 1) / kBrick;
        b->nbricks *= b->nb[d];
    }
    tg_status st = cuda_status(cudaMalloc(&b->counts, (b->nbricks + 1) * sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMalloc(&b->offsets, (b->nbricks + 1) * sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMalloc(&b->cursor, b->nbricks * sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMalloc(&b->sorted, (max_points > 0 ? max_points : 1) * sizeof(float4)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMalloc(&b->status, sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMemset(b->offsets, 0, (b->nbricks + 1) * sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMemset(b->status, 0, sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaDeviceSynchronize(), "tg_batch_create");
    if (st != TG_OK) { tg_batch_destroy(b); return st; }
    *out = b;
    return TG_OK;
}

tg_status tg_batch_destroy(tg_batch *b)
{
    if (!b) return TG_OK;
    cudaFree(b->counts); cudaFree(b->offsets); cudaFree(b->cursor); cudaFree(b->sorted); cudaFree(b->status);
    free(b);
    return TG_OK;
}

tg_status tg_batch_bin(tg_batch *b, const float *pts, int64_t N, tg_stream stream)
{
    if (!b) return fail(TG_EINVAL, "tg_batch_bin: batch is NULL");
    if (N < 0 || N > b->max_points) return fail(TG_EINVAL, "tg_batch_bin: N=%lld outside [0, %lld]", (long long)N, (long long)b->max_points);
    if (N > 0 && !pts) return fail(TG_EINVAL, "tg_batch_bin: pts is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    tg_status st = cuda_status(cudaMemsetAsync(b->counts, 0, (b->nbricks + 1) * sizeof(int), s), "tg_batch_bin");
    if (st != TG_OK) return st;
    b->n = N;
    const int nbx = b->nb[0], nby = b->nb[1];
    if (N > 0) {
        int64_t need = (N + kBinThreads - 1) / kBinThreads;
        int64_t cap = (int64_t)num_sms() * blocks_per_sm((const void *)bin_count_kernel, kBinThreads, 0);
        unsigned nblk = (unsigned)(need < cap ? need : cap);
        bin_count_kernel<<<nblk, kBinThreads, 0, s>>>(pts, N, b->res, nbx, nby, b->counts);
        if ((st = launch_status("tg_batch_bin: count")) != TG_OK) return st;
    }
    bin_scan_kernel<<<1, 1024, 0, s>>>(b->counts, b->offsets, b->cursor, (int)b->nbricks);
    if ((st = launch_status("tg_batch_bin: scan")) != TG_OK) return st;
    if (N > 0) {
        int64_t need = (N + kBinThreads - 1) / kBinThreads;
        int64_t cap = (int64_t)num_sms() * blocks_per_sm((const void *)bin_scatter_kernel, kBinThreads, 0);
        unsigned nblk = (unsigned)(need < cap ? need : cap);
        bin_scatter_kernel<<<nblk, kBinThreads, 0, s>>>(pts, N, b->res, nbx, nby, b->cursor, b->sorted);
        if ((st = launch_status("tg_batch_bin: scatter")) != TG_OK) return st;
    }
    return TG_OK;
}

tg_status tg_query_binned(const tg_grid *g, const tg_batch *bt, float *out, float *grad_x, tg_stream stream)
{
    tg_status st = check_pair(g, bt, "tg_query_binned");
    if (st != TG_OK) return st;
    if (bt->n == 0) return TG_OK;
    if (!out) return fail(TG_EINVAL, "tg_query_binned: out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
#define TG_QB(D, O, C)                                                                           \
    (g->dtype == TG_F32    ? BinnedLaunch<float>::fwd<D, O, C>(g, bt, out, grad_x, s)            \
     : g->dtype == TG_BF16 ? BinnedLaunch<__nv_bfloat16>::fwd<D, O, C>(g, bt, out, grad_x, s)    \
                           : BinnedLaunch<__half>::fwd<D, O, C>(g, bt, out, grad_x, s))
    return TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_QB);
#undef TG_QB
}

tg_status tg_query_backward_binned(const tg_grid *g, const tg_batch *bt, const float *dL_df, const float *dL_dgradx,
                                   float *coef_grad, tg_stream stream)
{
    tg_status st = check_pair(g, bt, "tg_query_backward_binned");
    if (st != TG_OK) return st;
    if (bt->n == 0) return TG_OK;
    if (!dL_df || !coef_grad) return fail(TG_EINVAL, "tg_query_backward_binned: NULL dL_df or coef_grad");
    cudaStream_t s = (cudaStream_t)stream;
#define TG_BB(D, O, C) binned_bwd<D, O, C>(g, bt, dL_df, dL_dgradx, coef_grad, s)
    return TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_BB);
#undef TG_BB
}

tg_status tg_batch_timeouts(tg_batch *b, int *timed_out)
{
    if (!b || !timed_out) return fail(TG_EINVAL, "tg_batch_timeouts: NULL argument");
    int v = 0;
    tg_status st = cuda_status(cudaMemcpy(&v, b->status, sizeof(int), cudaMemcpyDeviceToHost), "tg_batch_timeouts");
    if (st != TG_OK) return st;
    *timed_out = v;
    if (v) cudaMemset(b->status, 0, sizeof(int));
    return TG_OK;
}

}  // extern "C"
