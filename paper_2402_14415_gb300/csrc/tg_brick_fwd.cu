// Brick-binned forward query (Eq. 2 - Eq. 4): one block per 8^3-cell brick
// TMA-loads the brick's 9^3 vertex blocks into shared memory with one 3-D
// tiled copy and, while the copy is in flight, counting-sorts the brick's
// points by cell in shared memory, so that the lanes of a warp evaluate
// neighbouring cells and their corner reads from the tile fall into distinct
// banks. Each point is evaluated with per-point delta tables (one FMA per
// coefficient and corner). Outputs go straight to the caller's order: the
// binned slot, or the input index that every binned record carries.
#include "tg_gather.cuh"
#include "tg_records.cuh"

namespace tg {

constexpr int kFwdThreads = 256;

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

// Points sorted per round. The one-channel value kernel takes 512: it fits 48
// registers, so 5 blocks share an SM. The kernels that write spatial gradients
// or several channels need more registers, which then set their occupancy,
// and take 1024.
template <bool WIDE>
__host__ __device__ constexpr int fwd_chunk() { return WIDE ? 1024 : 512; }

template <typename T, int NV, int CHUNK>
struct FwdLayout {
    static constexpr int row = BoxInner<T, NV>::value;                 // tile row pitch (elements)
    static constexpr int tile_bytes = BoxInner<T, NV>::tile_bytes;
    static constexpr int bar_off = (tile_bytes + 15) / 16 * 16;
    static constexpr int ints_off = bar_off + 16;                    // cell counters + scan workspace
    static constexpr int rec_off = (ints_off + SortInts::total * 4 + 15) / 16 * 16;
    static constexpr int bytes = rec_off + CHUNK * 16;
};

template <typename T, int ORDER, int C, bool WANT_GRAD, bool IN_ORDER>
__global__ void __launch_bounds__(kFwdThreads, (WANT_GRAD || C > 1) ? 0 : 5)
brick_fwd_kernel(const __grid_constant__ CUtensorMap cmap, int res, int nbx, int nby,
                 const float4 *__restrict__ sorted, const int *__restrict__ offsets, float *__restrict__ out,
                 float *__restrict__ gx, int *__restrict__ status)
{
    constexpr int K = Basis<3, ORDER>::K;
    constexpr int NV = K * C;
    constexpr int kFwdChunk = fwd_chunk<WANT_GRAD || (C > 1)>();
    constexpr int kFwdPPT = kFwdChunk / kFwdThreads;
    // Cell order of the sort. With 40-byte FP32 blocks (one channel, order 2)
    // read as five 8-byte words and a tile row of 92 words, cells taken y
    // fastest put a half-warp's reads of rows y .. y + 7 (a 28-bank shift per
    // row) and of the next x (a 10-bank shift) into distinct banks; x fastest
    // gave about 1.9 times the conflict-free wavefronts, y fastest 1.5
    // (0.376 -> 0.334 ms at 2^24 points on 256^3). 20-byte BF16 / FP16 blocks
    // read as five 4-byte words with the 52-word row of box_row_bytes: about
    // 1.4 times with y fastest, against 2.4 for x fastest in 48-word rows.
    constexpr bool kYFirst = NV == 10;
    using L = FwdLayout<T, NV, kFwdChunk>;
    constexpr int BXI = L::row;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    uint64_t &bar = *reinterpret_cast<uint64_t *>(smem_raw + L::bar_off);
    int *ints = reinterpret_cast<int *>(smem_raw + L::ints_off);
    int *cell_cur = ints + SortInts::cell_cur;
    float4 *recs = reinterpret_cast<float4 *>(smem_raw + L::rec_off);

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
        mbar_arrive_expect_tx(&bar, L::tile_bytes);
        tma_load_3d(tile, &cmap, x0 * NV, y0, z0, &bar);
    }

    const float scale = (float)(res - 1), h = 1.0f / (float)(res - 1);
    bool waited = false;
    for (int base = p0; base < p1; base += kFwdChunk) {
        const int cnt = min(kFwdChunk, p1 - base);
        // counting sort of this round's points by cell (x fastest)
        for (int j = threadIdx.x; j < kBrickCells; j += kFwdThreads) cell_cur[j] = 0;
        __syncthreads();
        float4 q[kFwdPPT];
        int lc[kFwdPPT];
#pragma unroll
        for (int r = 0; r < kFwdPPT; ++r) {
            const int i = threadIdx.x + r * kFwdThreads;
            lc[r] = -1;
            if (i < cnt) {
                q[r] = sorted[base + i];
                const float x[3] = {q[r].x, q[r].y, q[r].z};
                int c[3];
                float t[3];
                locate<3>(x, res, scale, c, t);
                lc[r] = kYFirst ? (c[1] - y0) + kBrick * ((c[0] - x0) + kBrick * (c[2] - z0))
                                : (c[0] - x0) + kBrick * ((c[1] - y0) + kBrick * (c[2] - z0));
                if (!IN_ORDER) q[r].w = __int_as_float(base + i);      // output slot: the binned slot
                atomicAdd(cell_cur + lc[r], 1);
            }
        }
        __syncthreads();
        gather_scan_cells<kFwdThreads, SortInts>(ints);
#pragma unroll
        for (int r = 0; r < kFwdPPT; ++r)
            if (lc[r] >= 0) recs[atomicAdd(cell_cur + lc[r], 1)] = q[r];
        __syncthreads();
        if (!waited) {
            waited = true;
            if (!mbar_wait_bounded(&bar, 0)) {
                if (threadIdx.x == 0) atomicExch(status, 1);
                mbar_wait_bounded(&bar, 0);          // second bounded wait for the copy in flight
                return;
            }
        }
        for (int j = threadIdx.x; j < cnt; j += kFwdThreads) {
            const float4 qq = recs[j];
            const int64_t n = __float_as_int(qq.w);
            const float x[3] = {qq.x, qq.y, qq.z};
            int c[3];
            float t[3];
            locate<3>(x, res, scale, c, t);
            const PointTables3<ORDER> P(t, h);
            const T *cell = tile + ((c[2] - z0) * kBV + (c[1] - y0)) * BXI + (c[0] - x0) * NV;
            float f[C], gu[C][3];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                f[ch] = 0.f;
                gu[ch][0] = gu[ch][1] = gu[ch][2] = 0.f;
            }
            for_corners<0>([&](auto ic) {
                constexpr int I = decltype(ic)::value;
                constexpr int off = ((I >> 2) & 1) * kBV * BXI + ((I >> 1) & 1) * BXI + (I & 1) * NV;
                float th[NV];
                load_block_smem<T, NV>(cell + off, th);
                const float w = P.template weight<I>();
                float dw[3];
                if constexpr (WANT_GRAD) {
                    P.template dweight<I>(dw);
                    dw[0] *= scale; dw[1] *= scale; dw[2] *= scale;     // d w / d x
                }
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float Tv = P.template value<I>(th + ch * K);       // Eq. 3
                    f[ch] = fmaf(w, Tv, f[ch]);                               // Eq. 4
                    if constexpr (WANT_GRAD) {
                        float g[3];
                        P.template gradient<I>(th + ch * K, g);
#pragma unroll
                        for (int d = 0; d < 3; ++d) gu[ch][d] = fmaf(dw[d], Tv, fmaf(w, g[d], gu[ch][d]));
                    }
                }
            });
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                out[n * C + ch] = f[ch];
                if constexpr (WANT_GRAD) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) gx[(n * C + ch) * 3 + d] = gu[ch][d];
                }
            }
        }
        __syncthreads();                             // recs and counters are reused by the next round
    }
}

template <typename T>
struct BinnedFwd {
    template <bool WANT_GRAD, bool IN_ORDER, int ORDER, int C>
    static tg_status launch(const CUtensorMap &map, const tg_grid *g, const tg_batch *bt, float *out, float *gx,
                            cudaStream_t s)
    {
        constexpr int NV = Basis<3, ORDER>::K * C;
        auto k = brick_fwd_kernel<T, ORDER, C, WANT_GRAD, IN_ORDER>;
        const int smem = FwdLayout<T, NV, fwd_chunk<WANT_GRAD || (C > 1)>()>::bytes;
        tg_status st = set_smem((const void *)k, smem);
        if (st != TG_OK) return st;
        k<<<(unsigned)bt->nbricks, kFwdThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted, bt->offsets,
                                                           out, gx, bt->status);
        return launch_status("tg_query_binned");
    }

    template <int DIM, int ORDER, int C>
    static tg_status run(const tg_grid *g, const tg_batch *bt, float *out, float *gx, bool in_order, cudaStream_t s)
    {
        if constexpr (DIM != 3) {
            return fail(TG_EINVAL, "binned path is 3-D only");
        } else {
            constexpr int NVr = Basis<3, ORDER>::K * C;
            const bool tma_ok = brick_tma_ok(g->res, NVr, (int)sizeof(T), BoxInner<T, NVr>::value, g->store);
            if (use_records_path(bt->n, bt->nbricks, gx != nullptr, tma_ok)) {   // few points per brick
                // (or rows TMA cannot move): one thread per record
                const T *coefs = reinterpret_cast<const T *>(g->store);
                const unsigned blocks = records_blocks(bt->n);
                if (in_order)
                    records_fwd_kernel<T, ORDER, C, true><<<blocks, kQueryThreads, 0, s>>>(coefs, g->res, bt->sorted,
                                                                                           bt->n, out, gx);
                else
                    records_fwd_kernel<T, ORDER, C, false><<<blocks, kQueryThreads, 0, s>>>(coefs, g->res, bt->sorted,
                                                                                            bt->n, out, gx);
                return launch_status("tg_query_binned");
            }
            constexpr int NV = Basis<3, ORDER>::K * C;
            CUtensorMap map;
            const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : (g->dtype == TG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
            tg_status st = make_brick_map(&map, g->store, dt, (int)sizeof(T), g->res, NV, BoxInner<T, NV>::value, kBV);
            if (st != TG_OK) return st;
            if (gx) return in_order ? launch<true, true, ORDER, C>(map, g, bt, out, gx, s)
                                    : launch<true, false, ORDER, C>(map, g, bt, out, gx, s);
            return in_order ? launch<false, true, ORDER, C>(map, g, bt, out, nullptr, s)
                            : launch<false, false, ORDER, C>(map, g, bt, out, nullptr, s);
        }
    }
};

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_query_binned(const tg_grid *g, const tg_batch *bt_in, float *out, float *grad_x, int flags,
                                     tg_stream stream)
{
    tg_status st = check_pair(g, bt_in, "tg_query_binned");
    if (st != TG_OK) return st;
    if (flags != TG_ORDER_INPUT && flags != TG_ORDER_BINNED) return fail(TG_EINVAL, "tg_query_binned: bad flags");
    tg_batch *bt = const_cast<tg_batch *>(bt_in);
    if (bt->n == 0) return TG_OK;
    if (!out) return fail(TG_EINVAL, "tg_query_binned: out is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const bool in_order = flags == TG_ORDER_INPUT;
#define TG_QB(D, O, C)                                                                            \
    (g->dtype == TG_F32    ? BinnedFwd<float>::run<D, O, C>(g, bt, out, grad_x, in_order, s)            \
     : g->dtype == TG_BF16 ? BinnedFwd<__nv_bfloat16>::run<D, O, C>(g, bt, out, grad_x, in_order, s)    \
                           : BinnedFwd<__half>::run<D, O, C>(g, bt, out, grad_x, in_order, s))
    st = TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_QB);
#undef TG_QB
    return st;
}
