// Binning of a point batch by 8^3-cell brick (counting sort), and the batch API.
//
// With at most 32768 bricks each of G chunk blocks builds a shared-memory
// histogram of its slice of the points, a column scan over the chunks turns
// the histograms into per-chunk write cursors, and two place passes (coarse
// runs, then a fine scatter inside an L2-resident region) write every point
// into brick order using shared-memory atomics only. Larger grids, and
// batches of fewer than 128 points per brick, use global-atomic counting. Every binned record keeps its input index (in
// its fourth word), so the brick kernels can address per-point arrays in
// either order; the binning also writes the permutation itself (slot ->
// input index) for tg_batch_order and the row permutations.
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "tg_binned.cuh"

namespace tg {

constexpr int kBinThreads = 256;
constexpr int kHistThreads = 1024;
constexpr int kMaxSmemBins = 32768;   // 128 KB of shared counters
constexpr int kCoarse = 64;           // most bricks per coarse bin of the two-pass scatter
constexpr int kFineThreads = 512;

__device__ __forceinline__ void load_point3(const float *__restrict__ pts, int64_t n, float *x)
{
    x[0] = __ldg(pts + 3 * n);
    x[1] = __ldg(pts + 3 * n + 1);
    x[2] = __ldg(pts + 3 * n + 2);
}

__global__ void __launch_bounds__(kHistThreads)
bin_hist_kernel(const float *__restrict__ pts, int64_t N, int64_t chunk, int res, int nbx, int nby, int nbricks,
                int *__restrict__ hist)
{
    extern __shared__ int sh[];
    for (int j = threadIdx.x; j < nbricks; j += blockDim.x) sh[j] = 0;
    __syncthreads();
    const float scale = (float)(res - 1);
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = min(N, lo + chunk);
    for (int64_t n = lo + threadIdx.x; n < hi; n += blockDim.x) {
        float x[3], t[3];
        int c[3];
        load_point3(pts, n, x);
        locate<3>(x, res, scale, c, t);
        atomicAdd(sh + brick_of(c, nbx, nby), 1);
    }
    __syncthreads();
    int *dst = hist + (int64_t)blockIdx.x * nbricks;
    for (int j = threadIdx.x; j < nbricks; j += blockDim.x) dst[j] = sh[j];
}

// Block-wide exclusive scan of one int per thread; returns this thread's
// exclusive prefix and the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tmp, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tmp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        warp_tmp[lane] = w;
    }
    __syncthreads();
    total = warp_tmp[nw - 1];
    const int excl = incl - v + (wid > 0 ? warp_tmp[wid - 1] : 0);
    __syncthreads();
    return excl;
}

// Column scan: one thread per brick turns the G chunk histograms of its
// column into exclusive per-chunk offsets (in place) and writes the brick's
// total. Neighbouring threads read neighbouring bricks, so every row access
// of a warp is one coalesced segment; kColUnroll rows are loaded before any is
// used, so that many loads per thread are in flight (the histograms were just
// written and sit in L2).
constexpr int kColUnroll = 16;
__global__ void __launch_bounds__(kBinThreads)
bin_chunk_scan_kernel(int *__restrict__ hist, int G, int nbricks, int *__restrict__ totals)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbricks) return;
    int *col = hist + b;
    int carry = 0, g = 0;
    for (; g + kColUnroll <= G; g += kColUnroll) {
        int v[kColUnroll];
#pragma unroll
        for (int k = 0; k < kColUnroll; ++k) v[k] = col[(int64_t)(g + k) * nbricks];
#pragma unroll
        for (int k = 0; k < kColUnroll; ++k) {
            col[(int64_t)(g + k) * nbricks] = carry;
            carry += v[k];
        }
    }
    for (; g < G; ++g) {
        const int v = col[(int64_t)g * nbricks];
        col[(int64_t)g * nbricks] = carry;
        carry += v;
    }
    totals[b] = carry;
}

// Single-block exclusive scan of counts[0..n) into offsets[0..n] (offsets[n] =
// total) and optionally cursor; each thread owns a contiguous run of 16 per
// tile, moved as four 16-byte vectors where the run is whole and all three
// arrays start on a 16-byte boundary (scalar accesses otherwise).
__global__ void __launch_bounds__(1024)
bin_scan_kernel(const int *__restrict__ counts, int *__restrict__ offsets, int *__restrict__ cursor, int n)
{
    __shared__ int warp_tmp[32];
    constexpr int PER = 16;
    const bool aligned = (((uintptr_t)counts | (uintptr_t)offsets | (uintptr_t)cursor) & 15) == 0;
    int carry = 0;
    const int per_tile = PER * blockDim.x;
    for (int base = 0; base < n; base += per_tile) {
        const int j0 = base + PER * threadIdx.x;
        const bool whole = aligned && j0 + PER <= n;
        int v[PER];
        int sum = 0;
        if (whole) {
#pragma unroll
            for (int k = 0; k < PER / 4; ++k) {
                const int4 q = reinterpret_cast<const int4 *>(counts + j0)[k];
                v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < PER; ++k) v[k] = (j0 + k < n) ? counts[j0 + k] : 0;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) sum += v[k];
        int total;
        int run = carry + block_exclusive_scan(sum, warp_tmp, total);
        int o[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            o[k] = run;
            run += v[k];
        }
        if (whole) {
#pragma unroll
            for (int k = 0; k < PER / 4; ++k) {
                const int4 q = make_int4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
                reinterpret_cast<int4 *>(offsets + j0)[k] = q;
                if (cursor) reinterpret_cast<int4 *>(cursor + j0)[k] = q;
            }
        } else {
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                if (j0 + k < n) {
                    offsets[j0 + k] = o[k];
                    if (cursor) cursor[j0 + k] = o[k];
                }
            }
        }
        carry += total;
    }
    if (threadIdx.x == 0) offsets[n] = carry;
}

// Both place passes work in tiles: a tile's records are counting-sorted by
// destination bin in shared memory, every bin reserves one run of slots, and
// the tile is then written out in its sorted order, so that consecutive
// threads store consecutive records of a run (coalesced lines instead of one
// L2 request per 16-byte record).
constexpr int kCoarseBins = kHistThreads;                     // most coarse bins: one thread each in the scan
static_assert(kCoarse % 32 == 0, "one warp lane per kCoarse / 32 bricks in the fine pass");

// Bricks per coarse bin: the widest power of two up to kCoarse that still
// gives the fine pass two blocks per SM, but no narrower than keeps the
// coarse bins within one thread each of the coarse pass's block.
static int coarse_width(int nbricks)
{
    int cw = kCoarse;
    while (cw > 1 && (nbricks + cw - 1) / cw < 2 * num_sms()) cw >>= 1;
    while ((nbricks + cw - 1) / cw > kCoarseBins) cw <<= 1;
    return cw;
}
// The coarse pass runs two blocks of 512 threads per SM (64 registers, 88 KB of
// shared memory each), one per point chunk, so that one block's load, count,
// scan and write phases overlap the other's: 0.377 ms for the whole binning of
// 2^24 points on 256^3, against 0.395 with one block of 1024 threads per SM.
constexpr int kCoarseThreads = 512;
constexpr int kCoarseTile = 8 * kCoarseThreads;               // records per coarse tile
constexpr int kFineTile = 4 * kFineThreads;                  // records per fine tile

struct CoarseSmem {
    float4 stage[kCoarseTile];
    unsigned short bin[kCoarseTile];
    int cur[kCoarseBins];      // this chunk's next slot in every coarse bin
    int cnt[kCoarseBins];
    int loff[kCoarseBins];
    int gbase[kCoarseBins];
    int warp_tmp[32];
};

struct FineSmem {
    float4 stage[kFineTile];
    unsigned char brick[kFineTile];
    int cur[kCoarse];
    int cnt[kCoarse];
    int loff[kCoarse];
    int gbase[kCoarse];
};

// Coarse place: every chunk block writes its points, grouped by coarse bin
// (kCoarse consecutive bricks), into the coarse array. A chunk's share of a
// coarse bin is one contiguous run, filled tile by tile.
__global__ void __launch_bounds__(kCoarseThreads, 2)
bin_coarse_place_kernel(const float *__restrict__ pts, int64_t N, int64_t chunk, int res, int nbx, int nby,
                        int nbricks, int cw, const int *__restrict__ hist, const int *__restrict__ offsets,
                        float4 *__restrict__ coarse)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CoarseSmem &S = *reinterpret_cast<CoarseSmem *>(smem_raw);
    const int ncoarse = (nbricks + cw - 1) / cw;
    const int *h = hist + (int64_t)blockIdx.x * nbricks;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int cb = wid; cb < ncoarse; cb += blockDim.x >> 5) {     // one warp per coarse bin
        int sum = 0;
        for (int j = lane; j < cw; j += 32) {
            const int b = cb * cw + j;
            if (b < nbricks) sum += __ldg(h + b);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) S.cur[cb] = __ldg(offsets + cb * cw) + sum;
    }
    const float scale = (float)(res - 1);
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = min(N, lo + chunk);
    constexpr int U = kCoarseTile / kCoarseThreads;
    for (int64_t t0 = lo; t0 < hi; t0 += kCoarseTile) {
        const int cnt = (int)min((int64_t)kCoarseTile, hi - t0);
        for (int j = threadIdx.x; j < ncoarse; j += blockDim.x) S.cnt[j] = 0;
        __syncthreads();
        float x[U][3];
        int key[U], rank[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kCoarseThreads;
            key[u] = -1;
            if (i < cnt) load_point3(pts, t0 + i, x[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kCoarseThreads;
            if (i < cnt) {
                int c[3];
                float t[3];
                locate<3>(x[u], res, scale, c, t);
                key[u] = brick_of(c, nbx, nby) / cw;
                rank[u] = atomicAdd(S.cnt + key[u], 1);
            }
        }
        __syncthreads();
        {   // tile offsets per bin (two bins per thread), and one run per bin reserved from the chunk's cursor
            const int b = 2 * threadIdx.x;
            const int v0 = b < ncoarse ? S.cnt[b] : 0, v1 = b + 1 < ncoarse ? S.cnt[b + 1] : 0;
            int total;
            const int ex = block_exclusive_scan(v0 + v1, S.warp_tmp, total);
            if (b < ncoarse) {
                S.loff[b] = ex;
                S.gbase[b] = S.cur[b];
                S.cur[b] += v0;
            }
            if (b + 1 < ncoarse) {
                S.loff[b + 1] = ex + v0;
                S.gbase[b + 1] = S.cur[b + 1];
                S.cur[b + 1] += v1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (key[u] < 0) continue;
            const int q = S.loff[key[u]] + rank[u];
            S.stage[q] = make_float4(x[u][0], x[u][1], x[u][2], __int_as_float((int)(t0 + threadIdx.x + u * kCoarseThreads)));
            S.bin[q] = (unsigned short)key[u];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += kCoarseThreads) {
            const int bkey = S.bin[q];
            coarse[S.gbase[bkey] + (q - S.loff[bkey])] = S.stage[q];
        }
        __syncthreads();
    }
}

// Fine place: one block per coarse bin scatters its records to their bricks,
// tile by tile, and records the permutation.
__global__ void __launch_bounds__(kFineThreads)
bin_fine_place_kernel(const float4 *__restrict__ coarse, int res, int nbx, int nby, int nbricks, int cw,
                      const int *__restrict__ offsets, float4 *__restrict__ sorted, int *__restrict__ perm)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FineSmem &S = *reinterpret_cast<FineSmem *>(smem_raw);
    const int b0 = blockIdx.x * cw;
    const int nb = min(cw, nbricks - b0);       // counters past nb stay zero
    for (int j = threadIdx.x; j < nb; j += blockDim.x) S.cur[j] = __ldg(offsets + b0 + j);
    const int lo = __ldg(offsets + b0), hi = __ldg(offsets + b0 + nb);
    const float scale = (float)(res - 1);
    constexpr int U = kFineTile / kFineThreads;
    const int lane = threadIdx.x & 31;
    // the next tile's records are loaded while this one is ranked, staged and written
    float4 q[U], qn[U];
    if (lo < hi) {
        const int cnt0 = min(kFineTile, hi - lo);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kFineThreads;
            if (i < cnt0) q[u] = coarse[lo + i];
        }
    }
    for (int t0 = lo; t0 < hi; t0 += kFineTile) {
        const int cnt = min(kFineTile, hi - t0);
        const int cnt1 = max(0, min(kFineTile, hi - (t0 + kFineTile)));
        for (int j = threadIdx.x; j < kCoarse; j += blockDim.x) S.cnt[j] = 0;
        __syncthreads();
        int key[U], rank[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kFineThreads;
            key[u] = -1;
            if (i < cnt) {
                const float x[3] = {q[u].x, q[u].y, q[u].z};
                int c[3];
                float t[3];
                locate<3>(x, res, scale, c, t);
                key[u] = brick_of(c, nbx, nby) - b0;
                rank[u] = atomicAdd(S.cnt + key[u], 1);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = threadIdx.x + u * kFineThreads;
            if (i < cnt1) qn[u] = coarse[t0 + kFineTile + i];
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // one warp: offsets of the kCoarse bricks in the tile, and their runs
            constexpr int PER = kCoarse / 32;
            int a[PER], sum = 0;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                a[k] = S.cnt[PER * lane + k];
                sum += a[k];
            }
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            int ex = incl - sum;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int j = PER * lane + k;
                S.loff[j] = ex;
                S.gbase[j] = S.cur[j];
                S.cur[j] += a[k];
                ex += a[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (key[u] < 0) continue;
            const int p = S.loff[key[u]] + rank[u];
            S.stage[p] = q[u];
            S.brick[p] = (unsigned char)key[u];
        }
        __syncthreads();
        for (int p = threadIdx.x; p < cnt; p += kFineThreads) {
            const int k = S.brick[p];
            const int slot = S.gbase[k] + (p - S.loff[k]);
            const float4 r = S.stage[p];
            sorted[slot] = r;
            perm[slot] = __float_as_int(r.w);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = qn[u];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBinThreads)
bin_count_kernel(const float *__restrict__ pts, int64_t N, int res, int nbx, int nby, int *__restrict__ counts)
{
    const float scale = (float)(res - 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x[3], t[3];
        int c[3];
        load_point3(pts, n, x);
        locate<3>(x, res, scale, c, t);
        atomicAdd(counts + brick_of(c, nbx, nby), 1);
    }
}

__global__ void __launch_bounds__(kBinThreads)
bin_scatter_kernel(const float *__restrict__ pts, int64_t N, int res, int nbx, int nby, int *__restrict__ cursor,
                   float4 *__restrict__ sorted, int *__restrict__ perm)
{
    const float scale = (float)(res - 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x[3], t[3];
        int c[3];
        load_point3(pts, n, x);
        locate<3>(x, res, scale, c, t);
        const int slot = atomicAdd(cursor + brick_of(c, nbx, nby), 1);
        sorted[slot] = make_float4(x[0], x[1], x[2], __int_as_float((int)n));
        perm[slot] = (int)n;
    }
}

// Per-point rows of `width` floats between the two orders. GATHER: binned
// from input, dst[p] = src[perm[p]]; otherwise SCATTER: dst[perm[p]] = src[p].
// WIDTH > 0 fixes the row width at compile time (1 and 3 are the common ones).
template <bool GATHER, int WIDTH>
__global__ void __launch_bounds__(256)
permute_rows_kernel(const int *__restrict__ perm, const float *__restrict__ src, int64_t N, int width,
                    float *__restrict__ dst)
{
    const int w = WIDTH > 0 ? WIDTH : width;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = __ldg(perm + p);
        const int64_t from = (GATHER ? n : p) * w, to = (GATHER ? p : n) * w;
        if (WIDTH > 0) {
#pragma unroll
            for (int j = 0; j < WIDTH; ++j) dst[to + j] = __ldg(src + from + j);
        } else {
            for (int j = 0; j < w; ++j) dst[to + j] = __ldg(src + from + j);
        }
    }
}

__global__ void __launch_bounds__(256)
batch_points_kernel(const float4 *__restrict__ sorted, int64_t N, float *__restrict__ pts)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = sorted[p];
        pts[3 * p] = q.x;
        pts[3 * p + 1] = q.y;
        pts[3 * p + 2] = q.z;
    }
}

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

tg_status make_brick_map(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int elem, int res, int nv,
                         int box_inner, int box_z)
{
    auto fn = encode_fn();
    if (!fn) return fail(TG_EDEVICE, "cuTensorMapEncodeTiled is unavailable from the driver");
    const int bxi = box_inner;
    if (bxi < kBV * nv || (bxi * elem) % 16 != 0) return fail(TG_EINVAL, "binned path: bad box row of %d elements", bxi);
    if (bxi > 256) return fail(TG_EINVAL, "binned path: a brick row of %d elements exceeds the TMA box limit", bxi);
    if (((size_t)res * nv * elem) % 16 != 0)
        return fail(TG_EINVAL, "binned path: res * K * channels * elem (%d * %d * %d) must be a multiple of 16 bytes",
                    res, nv, elem);
    if (((uintptr_t)base & 15) != 0) return fail(TG_EINVAL, "binned path: array must be 16-byte aligned");
    cuuint64_t dims[3] = {(cuuint64_t)res * nv, (cuuint64_t)res, (cuuint64_t)res};
    cuuint64_t strides[2] = {(cuuint64_t)res * nv * elem, (cuuint64_t)res * res * nv * elem};
    cuuint32_t box[3] = {(cuuint32_t)bxi, (cuuint32_t)kBV, (cuuint32_t)box_z};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TG_EINVAL, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TG_OK;
}

tg_status set_smem(const void *kernel, int bytes)
{
    if (bytes <= 48 * 1024) return TG_OK;
    return cuda_status(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
                       "binned path: shared memory attribute");
}

tg_status check_pair(const tg_grid *g, const tg_batch *bt, const char *who)
{
    if (!g || !bt) return fail(TG_EINVAL, "%s: NULL grid or batch", who);
    if (g->dim != 3 || bt->res != g->res) return fail(TG_EINVAL, "%s: batch was created for another grid shape", who);
    return TG_OK;
}

bool auto_bin_wanted(const tg_grid *g, int64_t N, const float *coef_grad, cudaStream_t s)
{
    if (g->dim != 3 || N < kAutoBinMin) return false;
    const int64_t nb = (int64_t)((g->res - 2) / kBrick + 1);
    if (N < 8 * nb * nb * nb) return false;
    const int nv = g->K * g->C, elem = g->dtype == TG_F32 ? 4 : 2;
    if (((int64_t)g->res * nv * elem) % 16 != 0 || ((int64_t)g->res * nv * 4) % 16 != 0) return false;
    if (box_inner_host(nv, elem) > 256 || box_inner_host(nv, 4) > 256) return false;
    if (coef_grad && ((uintptr_t)coef_grad & 15) != 0) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

tg_status with_auto_batch(const tg_grid *gc, const float *pts, int64_t N, cudaStream_t s,
                          tg_status (*op)(const tg_grid *, tg_batch *, void *, cudaStream_t), void *arg)
{
    static std::mutex mu;      // host-side bookkeeping and enqueueing only
    std::lock_guard<std::mutex> lock(mu);
    tg_grid *g = const_cast<tg_grid *>(gc);
    tg_status st = TG_OK;
    if (!g->auto_event &&
        (st = cuda_status(cudaEventCreateWithFlags(&g->auto_event, cudaEventDisableTiming), "query: binning event")) != TG_OK)
        return st;
    if (!g->auto_batch || g->auto_batch->max_points < N) {
        if (g->auto_batch) {
            cudaEventSynchronize(g->auto_event);
            tg_batch_destroy(g->auto_batch);
            g->auto_batch = nullptr;
        }
        if ((st = tg_batch_create(3, g->res, N, &g->auto_batch)) != TG_OK) return st;
    }
    if ((st = cuda_status(cudaStreamWaitEvent(s, g->auto_event, 0), "query: order the binning scratch")) != TG_OK)
        return st;
    st = tg_batch_bin(g->auto_batch, pts, N, s);
    if (st == TG_OK) st = op(gc, g->auto_batch, arg, s);
    const tg_status rec = cuda_status(cudaEventRecord(g->auto_event, s), "query: binning event");
    return st != TG_OK ? st : rec;
}

static unsigned grid_for(const void *kernel, int threads, int64_t N)
{
    int64_t need = (N + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * blocks_per_sm(kernel, threads, 0);
    return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

tg_status ensure_stage(tg_batch *bt, int64_t floats, const char *who)
{
    if (bt->stage_floats >= floats) return TG_OK;
    if (!bt->stage_owned && bt->stage)
        return fail(TG_EINVAL, "%s: the request needs %lld staging floats, the fixed scratch holds %lld", who,
                    (long long)floats, (long long)bt->stage_floats);
    float *p = nullptr;
    tg_status st = dev_alloc((void **)&p, (size_t)floats * sizeof(float), who);
    if (st != TG_OK) return st;
    if (bt->stage) {
        cudaDeviceSynchronize();
        cudaFree(bt->stage);
    }
    bt->stage = p;
    bt->stage_floats = floats;
    bt->stage_owned = true;
    return TG_OK;
}

tg_status ensure_aux(tg_batch *bt, int64_t floats, const char *who)
{
    if (bt->aux_floats >= floats) return TG_OK;
    float *p = nullptr;
    tg_status st = dev_alloc((void **)&p, (size_t)floats * sizeof(float), who);
    if (st != TG_OK) return st;
    if (bt->aux) {
        cudaDeviceSynchronize();
        cudaFree(bt->aux);
    }
    bt->aux = p;
    bt->aux_floats = floats;
    return TG_OK;
}

template <bool GATHER>
static tg_status permute_rows(const tg_batch *b, const float *src, int width, float *dst, cudaStream_t s,
                              const char *what)
{
    if (!b) return fail(TG_EINVAL, "%s: batch is NULL", what);
    if (width < 1 || width > 64) return fail(TG_EINVAL, "%s: width %d outside 1..64", what, width);
    if (b->n == 0) return TG_OK;
    if (!src || !dst) return fail(TG_EINVAL, "%s: NULL array", what);
    if (src == dst) return fail(TG_EINVAL, "%s: src and dst must not alias", what);
    if (width == 1) {
        auto k = permute_rows_kernel<GATHER, 1>;
        k<<<grid_for((const void *)k, 256, b->n), 256, 0, s>>>(b->perm, src, b->n, 1, dst);
    } else if (width == 3) {
        auto k = permute_rows_kernel<GATHER, 3>;
        k<<<grid_for((const void *)k, 256, b->n), 256, 0, s>>>(b->perm, src, b->n, 3, dst);
    } else {
        auto k = permute_rows_kernel<GATHER, 0>;
        k<<<grid_for((const void *)k, 256, b->n), 256, 0, s>>>(b->perm, src, b->n, width, dst);
    }
    return launch_status(what);
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
    b->G = b->nbricks <= kMaxSmemBins ? kBinChunksPerSm * num_sms() : 0;
    tg_status st = dev_alloc((void **)&b->counts, (b->nbricks + 1) * sizeof(int), "tg_batch_create");
    if (st == TG_OK) st = dev_alloc((void **)&b->offsets, (b->nbricks + 1) * sizeof(int), "tg_batch_create");
    if (st == TG_OK) st = dev_alloc((void **)&b->cursor, b->nbricks * sizeof(int), "tg_batch_create");
    if (st == TG_OK && b->G)
        st = dev_alloc((void **)&b->hist, (size_t)b->G * b->nbricks * sizeof(int), "tg_batch_create");
    if (st == TG_OK) st = dev_alloc((void **)&b->sorted, (max_points > 0 ? max_points : 1) * sizeof(float4), "tg_batch_create");
    if (st == TG_OK && b->G)
        st = dev_alloc((void **)&b->coarse, (max_points > 0 ? max_points : 1) * sizeof(float4), "tg_batch_create");
    if (st == TG_OK) st = dev_alloc((void **)&b->perm, (max_points > 0 ? max_points : 1) * sizeof(int), "tg_batch_create");
    b->stage_owned = true;        // staging for the fused training steps is allocated on first use
    if (st == TG_OK) st = dev_alloc((void **)&b->status, sizeof(int), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMemset(b->offsets, 0, (b->nbricks + 1) * sizeof(int)), "tg_batch_create");
    if (st == TG_OK) st = cuda_status(cudaMemset(b->status, 0, sizeof(int)), "tg_batch_create");
    if (st == TG_OK && b->G) {
        const int bytes = (int)(b->nbricks * sizeof(int));
        st = set_smem((const void *)bin_hist_kernel, bytes);
        if (st == TG_OK) st = set_smem((const void *)bin_coarse_place_kernel, (int)sizeof(CoarseSmem));
        if (st == TG_OK) st = set_smem((const void *)bin_fine_place_kernel, (int)sizeof(FineSmem));
    }
    if (st == TG_OK) st = cuda_status(cudaDeviceSynchronize(), "tg_batch_create");
    if (st != TG_OK) { tg_batch_destroy(b); return st; }
    *out = b;
    return TG_OK;
}

tg_status tg_batch_destroy(tg_batch *b)
{
    if (!b) return TG_OK;
    cudaFree(b->counts); cudaFree(b->offsets); cudaFree(b->cursor); cudaFree(b->hist); cudaFree(b->sorted);
    cudaFree(b->coarse);
    cudaFree(b->perm);
    if (b->stage_owned) cudaFree(b->stage);
    cudaFree(b->aux);
    cudaFree(b->status);
    free(b);
    return TG_OK;
}

tg_status tg_batch_bin(tg_batch *b, const float *pts, int64_t N, tg_stream stream)
{
    if (!b) return fail(TG_EINVAL, "tg_batch_bin: batch is NULL");
    if (N < 0 || N > b->max_points) return fail(TG_EINVAL, "tg_batch_bin: N=%lld outside [0, %lld]", (long long)N, (long long)b->max_points);
    if (N > 0 && !pts) return fail(TG_EINVAL, "tg_batch_bin: pts is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    b->n = N;
    const int nbx = b->nb[0], nby = b->nb[1];
    const int nbr = (int)b->nbricks;
    tg_status st;
    if (N == 0) return cuda_status(cudaMemsetAsync(b->offsets, 0, (b->nbricks + 1) * sizeof(int), s), "tg_batch_bin");
    // Below 128 points per brick the global-atomic counting sort is faster: its brick counters see little
    // contention, and it skips the histogram rows and the two-level scatter (2^20 points on 256^3:
    // 0.060 against 0.082 ms; 2^21 on 160^3, 262 points per brick: 0.106 against 0.087 ms).
    if (b->G && N >= 128 * b->nbricks) {
        // two point chunks per SM pay for their histogram rows (G x bricks ints, written and read back) only
        // on large batches: below 2^22 points one chunk per SM is faster
        const int G = N >= ((int64_t)1 << 22) ? b->G : std::max(1, b->G / kBinChunksPerSm);
        const int64_t chunk = (N + G - 1) / G;
        const int smem = nbr * (int)sizeof(int);
        bin_hist_kernel<<<G, kHistThreads, smem, s>>>(pts, N, chunk, b->res, nbx, nby, nbr, b->hist);
        if ((st = launch_status("tg_batch_bin: histogram")) != TG_OK) return st;
        bin_chunk_scan_kernel<<<(nbr + kBinThreads - 1) / kBinThreads, kBinThreads, 0, s>>>(b->hist, G, nbr,
                                                                                            b->counts);
        if ((st = launch_status("tg_batch_bin: chunk scan")) != TG_OK) return st;
        bin_scan_kernel<<<1, 1024, 0, s>>>(b->counts, b->offsets, nullptr, nbr);
        if ((st = launch_status("tg_batch_bin: scan")) != TG_OK) return st;
        const int cw = coarse_width(nbr);
        bin_coarse_place_kernel<<<G, kCoarseThreads, sizeof(CoarseSmem), s>>>(pts, N, chunk, b->res, nbx, nby, nbr,
                                                                               cw, b->hist, b->offsets, b->coarse);
        if ((st = launch_status("tg_batch_bin: coarse place")) != TG_OK) return st;
        bin_fine_place_kernel<<<(nbr + cw - 1) / cw, kFineThreads, sizeof(FineSmem), s>>>(
            b->coarse, b->res, nbx, nby, nbr, cw, b->offsets, b->sorted, b->perm);
        return launch_status("tg_batch_bin: fine place");
    }
    if ((st = cuda_status(cudaMemsetAsync(b->counts, 0, (b->nbricks + 1) * sizeof(int), s), "tg_batch_bin")) != TG_OK)
        return st;
    bin_count_kernel<<<grid_for((const void *)bin_count_kernel, kBinThreads, N), kBinThreads, 0, s>>>(
        pts, N, b->res, nbx, nby, b->counts);
    if ((st = launch_status("tg_batch_bin: count")) != TG_OK) return st;
    bin_scan_kernel<<<1, 1024, 0, s>>>(b->counts, b->offsets, b->cursor, nbr);
    if ((st = launch_status("tg_batch_bin: scan")) != TG_OK) return st;
    bin_scatter_kernel<<<grid_for((const void *)bin_scatter_kernel, kBinThreads, N), kBinThreads, 0, s>>>(
        pts, N, b->res, nbx, nby, b->cursor, b->sorted, b->perm);
    return launch_status("tg_batch_bin: scatter");
}

tg_status tg_batch_order(const tg_batch *b, int32_t *idx, tg_stream stream)
{
    if (!b) return fail(TG_EINVAL, "tg_batch_order: batch is NULL");
    if (b->n == 0) return TG_OK;
    if (!idx) return fail(TG_EINVAL, "tg_batch_order: idx is NULL");
    return cuda_status(cudaMemcpyAsync(idx, b->perm, (size_t)b->n * sizeof(int), cudaMemcpyDeviceToDevice,
                                       (cudaStream_t)stream), "tg_batch_order");
}

tg_status tg_batch_points(const tg_batch *b, float *pts, tg_stream stream)
{
    if (!b) return fail(TG_EINVAL, "tg_batch_points: batch is NULL");
    if (b->n == 0) return TG_OK;
    if (!pts) return fail(TG_EINVAL, "tg_batch_points: pts is NULL");
    batch_points_kernel<<<grid_for((const void *)batch_points_kernel, 256, b->n), 256, 0, (cudaStream_t)stream>>>(
        b->sorted, b->n, pts);
    return launch_status("tg_batch_points");
}

tg_status tg_batch_gather(const tg_batch *b, const float *src, int width, float *dst, tg_stream stream)
{
    return permute_rows<true>(b, src, width, dst, (cudaStream_t)stream, "tg_batch_gather");
}

tg_status tg_batch_scatter(const tg_batch *b, const float *src, int width, float *dst, tg_stream stream)
{
    return permute_rows<false>(b, src, width, dst, (cudaStream_t)stream, "tg_batch_scatter");
}

tg_status tg_batch_timeouts(tg_batch *b, int *timed_out)
{
    if (!b || !timed_out) return fail(TG_EINVAL, "tg_batch_timeouts: NULL argument");
    // every stream's launches, non-blocking streams included, have finished before the flag is read
    tg_status st = cuda_status(cudaDeviceSynchronize(), "tg_batch_timeouts: wait for the device");
    if (st != TG_OK) return st;
    int v = 0;
    if ((st = cuda_status(cudaMemcpy(&v, b->status, sizeof(int), cudaMemcpyDeviceToHost), "tg_batch_timeouts")) != TG_OK)
        return st;
    *timed_out = v;
    if (v) st = cuda_status(cudaMemset(b->status, 0, sizeof(int)), "tg_batch_timeouts: clear");
    return st;
}

tg_status tg_grid_timeouts(tg_grid *g, int *timed_out)
{
    if (!g || !timed_out) return fail(TG_EINVAL, "tg_grid_timeouts: NULL argument");
    *timed_out = 0;
    if (!g->auto_batch) return cuda_status(cudaDeviceSynchronize(), "tg_grid_timeouts: wait for the device");
    return tg_batch_timeouts(g->auto_batch, timed_out);
}

}  // extern "C"
