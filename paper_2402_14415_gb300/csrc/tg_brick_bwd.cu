// Brick-binned coefficient gradient: the adjoint of Eq. 2 - Eq. 4.
//
// One block per 8^3-cell brick. The brick's points are staged in shared
// memory with their upstream gradients (read at the binned slot, or at the
// input index every binned record carries) and counting-sorted by cell; the
// vertex-centric gather (tg_gather.cuh) then sums every vertex's
// contributions in registers, without atomics, into a shared 9^3 tile, and
// one TMA bulk-tensor reduce-add (element-wise atomic at L2) adds the tile to
// the global gradient, which also combines the faces neighbouring bricks share.
// A brick whose points fit one round stores the tile instead of zeroing it
// and adding to it.
#include <stdlib.h>

#include "tg_bwd_fast.cuh"
#include "tg_records.cuh"

namespace tg {

constexpr int kBwdThreads = 256;
constexpr int kPChunk = 1024;                        // points staged per round
constexpr int kPPT = kPChunk / kBwdThreads;          // 4 staged points per thread

template <int ORDER, int C, bool HAS_G, bool DET = false>
struct BwdLayout {
    static constexpr int NV = Basis<3, ORDER>::K * C;
    static constexpr int BXI = BoxInner<float, NV>::value;
    static constexpr int tile_floats = (kBV * kBV * BXI + 31) / 32 * 32;
    static constexpr int rec_floats = kPChunk * GatherRec<C, HAS_G>::stride;
    static constexpr int key_ints = DET ? kPChunk : 0;             // input index of every staged record
    static constexpr int bytes = (tile_floats + rec_floats + GatherInts::total + key_ints) * 4;
};

// Deterministic mode: bricks run in 8 launches, one per parity class (bx, by,
// bz mod 2) - bricks of one class share no vertex, so every gradient element
// receives at most one reduce-add per launch, in a fixed class order - and
// the points of every cell are ordered by input index before the gather, so
// each vertex sums its terms in a fixed order. A brick of more than kPChunk
// points takes its rounds by input index: round r holds the records whose
// index lies in (k_{r-1}, k_r], k_r the ((r + 1) kPChunk)-th smallest index of
// the brick, so what a round contains does not depend on the binned order.
struct DetClass {
    int px, py, pz;       // parity of the bricks of this launch
    int ncx, ncy;         // bricks of the class along x and y
};

// Number of the brick's n records whose input index lies in (lo, hi], summed
// over the block (every thread gets it). warp_sum: kBwdThreads / 32 ints.
__device__ __forceinline__ int det_count(const float4 *__restrict__ recs, int n, int lo, int hi, int *warp_sum)
{
    int c = 0;
    for (int j = threadIdx.x; j < n; j += kBwdThreads) {
        const int k = __float_as_int(recs[j].w);
        c += k > lo && k <= hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __syncthreads();                                   // the previous call's sums have been read
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    int total = 0;
#pragma unroll
    for (int w = 0; w < kBwdThreads / 32; ++w) total += warp_sum[w];
    return total;
}

// The smallest index T > lo such that (lo, T] holds kPChunk of the brick's
// records (more than kPChunk have an index above lo): a binary search on counts.
__device__ __forceinline__ int det_round_end(const float4 *__restrict__ recs, int n, int lo, int *warp_sum)
{
    int a = lo + 1, b = 0x7fffffff - 1;                 // the answer lies in [a, b]
    while (a < b) {
        const int m = a + (b - a) / 2;
        if (det_count(recs, n, lo, m, warp_sum) >= kPChunk) b = m;
        else a = m + 1;
    }
    return a;
}

template <int ORDER, int C, bool HAS_G, bool IN_ORDER, bool DET>
__global__ void __launch_bounds__(kBwdThreads)
brick_bwd_kernel(const __grid_constant__ CUtensorMap gmap, int res, int nbx, int nby,
                 const float4 *__restrict__ sorted, const int *__restrict__ offsets, const float *__restrict__ dLdf,
                 const float *__restrict__ dLdg, DetClass cls)
{
    using L = BwdLayout<ORDER, C, HAS_G, DET>;
    using R = GatherRec<C, HAS_G>;
    constexpr int NV = L::NV;
    constexpr int BXI = L::BXI;
    constexpr int RS = R::stride;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);
    float *rec = tile + L::tile_floats;
    int *ints = reinterpret_cast<int *>(rec + L::rec_floats);
    int *cell_cur = ints + GatherInts::cell_cur;
    int *rec_key = ints + GatherInts::total;                       // DET: input index per staged record

    int b = blockIdx.x;
    if (DET) {
        const int i = blockIdx.x % cls.ncx, j = (blockIdx.x / cls.ncx) % cls.ncy, k = blockIdx.x / (cls.ncx * cls.ncy);
        b = (2 * i + cls.px) + nbx * ((2 * j + cls.py) + nby * (2 * k + cls.pz));
    }
    const int p0 = offsets[b], p1 = offsets[b + 1];
    if (p0 == p1) return;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    const float scale = (float)(res - 1);
    const int tid = threadIdx.x;

    const bool single = p1 - p0 <= kPChunk;
    if (single) {   // the round stores every vertex block; only the row padding needs zeros
        constexpr int PAD = BXI - kBV * NV;
        for (int j = tid; j < kBV * kBV * PAD; j += kBwdThreads) tile[(j / PAD) * BXI + kBV * NV + j % PAD] = 0.f;
    } else {
        for (int j = tid; j < L::tile_floats / 4; j += kBwdThreads)
            reinterpret_cast<float4 *>(tile)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    const bool det_multi = DET && !single;
    int kprev = -1;                                   // deterministic rounds: indices above kprev are left
    for (int base = p0; base < p1; base += kPChunk) {
        const int cnt = min(kPChunk, p1 - base);
        int kend = 0x7fffffff;                        // deterministic rounds: this round's last index
        if (det_multi && p1 - base > kPChunk) kend = det_round_end(sorted + p0, p1 - p0, kprev, ints + GatherInts::warp_tmp);
        for (int j = tid; j < kBrickCells; j += kBwdThreads) cell_cur[j] = 0;
        __syncthreads();
        if (det_multi) {   // the round's records: two passes over the brick, counting then placing
            for (int j = tid; j < p1 - p0; j += kBwdThreads) {
                const float4 q = sorted[p0 + j];
                const int key = __float_as_int(q.w);
                if (key <= kprev || key > kend) continue;
                const float x[3] = {q.x, q.y, q.z};
                int c[3];
                float t[3];
                locate<3>(x, res, scale, c, t);
                atomicAdd(cell_cur + (c[0] - x0) + kBrick * ((c[1] - y0) + kBrick * (c[2] - z0)), 1);
            }
            __syncthreads();
            gather_scan_cells<kBwdThreads>(ints);
            for (int j = tid; j < p1 - p0; j += kBwdThreads) {
                const float4 q = sorted[p0 + j];
                const int key = __float_as_int(q.w);
                if (key <= kprev || key > kend) continue;
                const int64_t n = IN_ORDER ? (int64_t)key : (int64_t)(p0 + j);
                const float x[3] = {q.x, q.y, q.z};
                int c[3];
                float v[RS];
                locate<3>(x, res, scale, c, v);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) v[3 + ch] = __ldg(dLdf + n * C + ch);
                if constexpr (HAS_G) {
#pragma unroll
                    for (int i = 0; i < 3 * C; ++i) v[3 + C + i] = __ldg(dLdg + n * 3 * C + i);
                }
#pragma unroll
                for (int i = R::fields; i < RS; ++i) v[i] = 0.f;
                const int pos = atomicAdd(cell_cur + (c[0] - x0) + kBrick * ((c[1] - y0) + kBrick * (c[2] - z0)), 1);
#pragma unroll
                for (int i = 0; i < RS; i += 4)
                    *reinterpret_cast<float4 *>(rec + pos * RS + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                rec_key[pos] = key;
            }
            kprev = kend;
        }
        int my_lc[kPPT], my_key[kPPT];
        float my_t[kPPT][3];
        float my_u[kPPT][R::fields - 3];             // upstream gradients, loaded before the cell scan
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int i = tid + r * kBwdThreads;
            my_lc[r] = -1;
            if (i < cnt && !det_multi) {
                const float4 q = sorted[base + i];
                const int64_t n = IN_ORDER ? (int64_t)__float_as_int(q.w) : (int64_t)(base + i);
                my_key[r] = __float_as_int(q.w);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) my_u[r][ch] = __ldg(dLdf + n * C + ch);
                if constexpr (HAS_G) {
#pragma unroll
                    for (int j = 0; j < 3 * C; ++j) my_u[r][C + j] = __ldg(dLdg + n * 3 * C + j);
                }
                const float x[3] = {q.x, q.y, q.z};
                int c[3];
                locate<3>(x, res, scale, c, my_t[r]);
                my_lc[r] = (c[0] - x0) + kBrick * ((c[1] - y0) + kBrick * (c[2] - z0));
                atomicAdd(cell_cur + my_lc[r], 1);
            }
        }
        __syncthreads();
        if (!det_multi) gather_scan_cells<kBwdThreads>(ints);
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            if (my_lc[r] < 0) continue;
            const int pos = atomicAdd(cell_cur + my_lc[r], 1);
            float v[RS];
            v[0] = my_t[r][0]; v[1] = my_t[r][1]; v[2] = my_t[r][2];
#pragma unroll
            for (int j = 0; j < R::fields - 3; ++j) v[3 + j] = my_u[r][j];
#pragma unroll
            for (int j = R::fields; j < RS; ++j) v[j] = 0.f;
#pragma unroll
            for (int j = 0; j < RS; j += 4)
                *reinterpret_cast<float4 *>(rec + pos * RS + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            if (DET) rec_key[pos] = my_key[r];
        }
        __syncthreads();
        if (DET) {   // order every cell's records by input index (cells hold a handful of points)
            const int *off = ints + GatherInts::cell_off;
            for (int c = tid; c < kBrickCells; c += kBwdThreads) {
                const int lo = off[c], hi = off[c + 1];
                for (int a = lo + 1; a < hi; ++a) {
                    const int key = rec_key[a];
                    float4 rv[RS / 4];
#pragma unroll
                    for (int j = 0; j < RS / 4; ++j) rv[j] = reinterpret_cast<const float4 *>(rec + a * RS)[j];
                    int z = a;
                    while (z > lo && rec_key[z - 1] > key) {
                        rec_key[z] = rec_key[z - 1];
#pragma unroll
                        for (int j = 0; j < RS / 4; ++j)
                            reinterpret_cast<float4 *>(rec + z * RS)[j] = reinterpret_cast<const float4 *>(rec + (z - 1) * RS)[j];
                        --z;
                    }
                    rec_key[z] = key;
#pragma unroll
                    for (int j = 0; j < RS / 4; ++j) reinterpret_cast<float4 *>(rec + z * RS)[j] = rv[j];
                }
            }
            __syncthreads();
        }
        if (single) gather_round<ORDER, C, HAS_G, kBwdThreads, BXI, true>(rec, ints, tile, scale);
        else gather_round<ORDER, C, HAS_G, kBwdThreads, BXI, false>(rec, ints, tile, scale);
        __syncthreads();
    }

    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
        tma_reduce_add_3d(&gmap, tile, x0 * NV, y0, z0);
        bulk_commit();
        bulk_wait_read_all();
    }
}

// TG_BWD_GATHER=1 in the environment selects the vertex-centric gather kernel for value upstreams too
// (the pair-list kernel's predecessor), for comparisons.
static bool list_kernel_disabled()
{
    static const bool off = [] {
        const char *e = getenv("TG_BWD_GATHER");
        return e && e[0] == '1';
    }();
    return off;
}

template <int ORDER, int C, bool HAS_G, bool IN_ORDER>
static tg_status launch_bwd(const CUtensorMap &map, const tg_grid *g, const tg_batch *bt, const float *uf,
                            const float *ug, bool det, cudaStream_t s)
{
    if constexpr (!HAS_G) {
        if (!det && !list_kernel_disabled()) {   // value upstreams: the descriptor-driven gather
            auto k = brick_bwd_fast_kernel<ORDER, C, IN_ORDER>;
            const int smem = FastLayout<ORDER, C>::bytes;
            tg_status st = set_smem((const void *)k, smem);
            if (st != TG_OK) return st;
            k<<<(unsigned)bt->nbricks, kFThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted,
                                                             bt->offsets, uf);
            return launch_status("tg_query_backward_binned");
        }
    }
    if (!det) {
        auto k = brick_bwd_kernel<ORDER, C, HAS_G, IN_ORDER, false>;
        const int smem = BwdLayout<ORDER, C, HAS_G, false>::bytes;
        tg_status st = set_smem((const void *)k, smem);
        if (st != TG_OK) return st;
        k<<<(unsigned)bt->nbricks, kBwdThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted,
                                                           bt->offsets, uf, ug, DetClass{});
        return launch_status("tg_query_backward_binned");
    }
    auto k = brick_bwd_kernel<ORDER, C, HAS_G, IN_ORDER, true>;
    const int smem = BwdLayout<ORDER, C, HAS_G, true>::bytes;
    tg_status st = set_smem((const void *)k, smem);
    if (st != TG_OK) return st;
    for (int cl = 0; cl < 8; ++cl) {           // the 8 parity classes, in a fixed order
        DetClass c{cl & 1, (cl >> 1) & 1, cl >> 2, 0, 0};
        c.ncx = (bt->nb[0] - c.px + 1) / 2;
        c.ncy = (bt->nb[1] - c.py + 1) / 2;
        const int ncz = (bt->nb[2] - c.pz + 1) / 2;
        const int64_t blocks = (int64_t)c.ncx * c.ncy * ncz;
        if (blocks == 0) continue;
        k<<<(unsigned)blocks, kBwdThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted, bt->offsets, uf,
                                                      ug, c);
        if ((st = launch_status("tg_query_backward_binned (deterministic)")) != TG_OK) return st;
    }
    return TG_OK;
}

template <int DIM, int ORDER, int C>
static tg_status binned_bwd(const tg_grid *g, const tg_batch *bt, const float *uf, const float *ug, float *grad,
                            bool in_order, bool det, cudaStream_t s)
{
    if constexpr (DIM != 3) {
        return fail(TG_EINVAL, "binned path is 3-D only");
    } else {
        constexpr int NVr = Basis<3, ORDER>::K * C;
        const bool tma_ok = brick_tma_ok(g->res, NVr, 4, BoxInner<float, NVr>::value, grad);
        if (!det && use_records_path(bt->n, bt->nbricks, ug != nullptr, tma_ok)) {   // few points per brick
            // (or rows TMA cannot move): one thread per record
            const unsigned blocks = records_blocks(bt->n);
            if (in_order)
                records_bwd_kernel<ORDER, C, true><<<blocks, kQueryThreads, 0, s>>>(g->res, bt->sorted, bt->n, uf, ug,
                                                                                    grad);
            else
                records_bwd_kernel<ORDER, C, false><<<blocks, kQueryThreads, 0, s>>>(g->res, bt->sorted, bt->n, uf, ug,
                                                                                     grad);
            return launch_status("tg_query_backward_binned");
        }
        constexpr int NV = Basis<3, ORDER>::K * C;
        CUtensorMap map;
        tg_status st = make_brick_map(&map, grad, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->res, NV,
                                      BoxInner<float, NV>::value, kBV);
        if (st != TG_OK) return st;
        if (ug) return in_order ? launch_bwd<ORDER, C, true, true>(map, g, bt, uf, ug, det, s)
                                : launch_bwd<ORDER, C, true, false>(map, g, bt, uf, ug, det, s);
        return in_order ? launch_bwd<ORDER, C, false, true>(map, g, bt, uf, nullptr, det, s)
                        : launch_bwd<ORDER, C, false, false>(map, g, bt, uf, nullptr, det, s);
    }
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_query_backward_binned(const tg_grid *g, const tg_batch *bt_in, const float *dL_df,
                                              const float *dL_dgradx, float *coef_grad, int flags, tg_stream stream)
{
    tg_status st = check_pair(g, bt_in, "tg_query_backward_binned");
    if (st != TG_OK) return st;
    if ((flags & ~(TG_ORDER_BINNED | TG_DETERMINISTIC)) != 0)
        return fail(TG_EINVAL, "tg_query_backward_binned: bad flags");
    tg_batch *bt = const_cast<tg_batch *>(bt_in);
    if (bt->n == 0) return TG_OK;
    if (!dL_df || !coef_grad) return fail(TG_EINVAL, "tg_query_backward_binned: NULL dL_df or coef_grad");
    cudaStream_t s = (cudaStream_t)stream;
    const bool in_order = (flags & TG_ORDER_BINNED) == 0, det = (flags & TG_DETERMINISTIC) != 0;
#define TG_BB(D, O, C) binned_bwd<D, O, C>(g, bt, dL_df, dL_dgradx, coef_grad, in_order, det, s)
    return TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_BB);
#undef TG_BB
}
