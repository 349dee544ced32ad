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
#include "tg_gather.cuh"

namespace tg {

constexpr int kBwdThreads = 256;
constexpr int kPChunk = 1024;                        // points staged per round
constexpr int kPPT = kPChunk / kBwdThreads;          // 4 staged points per thread

template <int ORDER, int C, bool HAS_G>
struct BwdLayout {
    static constexpr int NV = Basis<3, ORDER>::K * C;
    static constexpr int BXI = BoxInner<float, NV>::value;
    static constexpr int tile_floats = (kBV * kBV * BXI + 31) / 32 * 32;
    static constexpr int rec_floats = kPChunk * GatherRec<C, HAS_G>::stride;
    static constexpr int bytes = (tile_floats + rec_floats + GatherInts::total) * 4;
};

template <int ORDER, int C, bool HAS_G, bool IN_ORDER>
__global__ void __launch_bounds__(kBwdThreads)
brick_bwd_kernel(const __grid_constant__ CUtensorMap gmap, int res, int nbx, int nby,
                 const float4 *__restrict__ sorted, const int *__restrict__ offsets, const float *__restrict__ dLdf,
                 const float *__restrict__ dLdg)
{
    using L = BwdLayout<ORDER, C, HAS_G>;
    using R = GatherRec<C, HAS_G>;
    constexpr int NV = L::NV;
    constexpr int BXI = L::BXI;
    constexpr int RS = R::stride;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);
    float *rec = tile + L::tile_floats;
    int *ints = reinterpret_cast<int *>(rec + L::rec_floats);
    int *cell_cur = ints + GatherInts::cell_cur;

    const int b = blockIdx.x;
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

    for (int base = p0; base < p1; base += kPChunk) {
        const int cnt = min(kPChunk, p1 - base);
        for (int j = tid; j < kBrickCells; j += kBwdThreads) cell_cur[j] = 0;
        __syncthreads();
        int my_lc[kPPT];
        float my_t[kPPT][3];
        float my_u[kPPT][R::fields - 3];             // upstream gradients, loaded before the cell scan
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int i = tid + r * kBwdThreads;
            my_lc[r] = -1;
            if (i < cnt) {
                const float4 q = sorted[base + i];
                const int64_t n = IN_ORDER ? (int64_t)__float_as_int(q.w) : (int64_t)(base + i);
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
        gather_scan_cells<kBwdThreads>(ints);
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
        }
        __syncthreads();
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

template <int ORDER, int C, bool HAS_G, bool IN_ORDER>
static tg_status launch_bwd(const CUtensorMap &map, const tg_grid *g, const tg_batch *bt, const float *uf,
                            const float *ug, cudaStream_t s)
{
    auto k = brick_bwd_kernel<ORDER, C, HAS_G, IN_ORDER>;
    const int smem = BwdLayout<ORDER, C, HAS_G>::bytes;
    tg_status st = set_smem((const void *)k, smem);
    if (st != TG_OK) return st;
    k<<<(unsigned)bt->nbricks, kBwdThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted, bt->offsets,
                                                       uf, ug);
    return launch_status("tg_query_backward_binned");
}

template <int DIM, int ORDER, int C>
static tg_status binned_bwd(const tg_grid *g, const tg_batch *bt, const float *uf, const float *ug, float *grad,
                            bool in_order, cudaStream_t s)
{
    if constexpr (DIM != 3) {
        return fail(TG_EINVAL, "binned path is 3-D only");
    } else {
        constexpr int NV = Basis<3, ORDER>::K * C;
        CUtensorMap map;
        tg_status st = make_brick_map(&map, grad, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->res, NV,
                                      BoxInner<float, NV>::value, kBV);
        if (st != TG_OK) return st;
        if (ug) return in_order ? launch_bwd<ORDER, C, true, true>(map, g, bt, uf, ug, s)
                                : launch_bwd<ORDER, C, true, false>(map, g, bt, uf, ug, s);
        return in_order ? launch_bwd<ORDER, C, false, true>(map, g, bt, uf, nullptr, s)
                        : launch_bwd<ORDER, C, false, false>(map, g, bt, uf, nullptr, s);
    }
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_query_backward_binned(const tg_grid *g, const tg_batch *bt_in, const float *dL_df,
                                              const float *dL_dgradx, float *coef_grad, int flags, tg_stream stream)
{
    tg_status st = check_pair(g, bt_in, "tg_query_backward_binned");
    if (st != TG_OK) return st;
    if (flags != TG_ORDER_INPUT && flags != TG_ORDER_BINNED)
        return fail(TG_EINVAL, "tg_query_backward_binned: bad flags");
    tg_batch *bt = const_cast<tg_batch *>(bt_in);
    if (bt->n == 0) return TG_OK;
    if (!dL_df || !coef_grad) return fail(TG_EINVAL, "tg_query_backward_binned: NULL dL_df or coef_grad");
    cudaStream_t s = (cudaStream_t)stream;
    const bool in_order = flags == TG_ORDER_INPUT;
#define TG_BB(D, O, C) binned_bwd<D, O, C>(g, bt, dL_df, dL_dgradx, coef_grad, in_order, s)
    return TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_BB);
#undef TG_BB
}
