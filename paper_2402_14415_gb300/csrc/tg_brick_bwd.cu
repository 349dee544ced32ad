// Brick-binned coefficient gradient: the adjoint of Eq. 2 - Eq. 4.
//
// One block of four warps per 8^3-cell brick. The brick's points are staged
// in shared memory and counting-sorted by cell. Warp w owns the z-slab of
// cell layers {2w, 2w+1} and a private accumulator for the three vertex planes
// those cells touch. Each lane takes a contiguous, cell-aligned segment of
// the slab's cell-sorted points, so two lanes never hold points of the same
// cell; for a fixed corner index all lanes therefore target distinct
// vertices, and the accumulation is a plain shared-memory read-add-write with
// a warp barrier between corners - no atomics. Each warp finally adds its
// 3-plane block to the global gradient with one TMA bulk-tensor reduce-add
// (element-wise atomic at L2), which also combines the planes and faces that
// neighbouring slabs and bricks share.
#include "tg_binned.cuh"

namespace tg {

constexpr int kBwdWarps = 4;
constexpr int kBwdThreads = 32 * kBwdWarps;
constexpr int kSlabLayers = kBrick / kBwdWarps;         // 2 cell layers per warp
constexpr int kSlabPlanes = kSlabLayers + 1;            // 3 vertex planes per warp
constexpr int kSlabCells = kSlabLayers * kBrick * kBrick;
constexpr int kPChunk = 512;                            // points staged per round
constexpr int kPPT = kPChunk / kBwdThreads;             // 4 staged points per thread

// Staged point record: t (3), dL/df (C), with a spatial-gradient upstream
// dL/d(grad_x f) scaled to grid units (3 C), the local cell id; padded to 16 B.
template <int C, bool HAS_G>
struct BwdRec {
    static constexpr int fields = 3 + C + (HAS_G ? 3 * C : 0) + 1;
    static constexpr int stride = (fields + 3) / 4 * 4;
    static constexpr int cell = fields - 1;
};

template <int ORDER, int C, bool HAS_G>
struct BwdLayout {
    static constexpr int NV = Basis<3, ORDER>::K * C;
    static constexpr int BXI = BoxInner<float, NV>::value;
    // Each slab is the shared-memory source of a TMA tensor copy, which must
    // start on a 128-byte boundary: the slab stride is padded to 32 floats.
    static constexpr int slab_floats = (kSlabPlanes * kBV * BXI + 31) / 32 * 32;
    static constexpr int rec_floats = kPChunk * BwdRec<C, HAS_G>::stride;
    static constexpr int ints = 2 * kBrickCells + 1 + 32 + 3;
    static constexpr int bytes = (kBwdWarps * slab_floats + rec_floats + ints) * 4;
};

template <typename T, int N>
__device__ __forceinline__ void lds_block(const float *p, float *v)
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            float4 a = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = a.z; v[4 * i + 3] = a.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            float2 a = reinterpret_cast<const float2 *>(p)[i];
            v[2 * i] = a.x; v[2 * i + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = p[i];
    }
}

template <typename T, int N>
__device__ __forceinline__ void sts_block(float *p, const float *v)
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<float2 *>(p)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) p[i] = v[i];
    }
}

// Block-wide exclusive scan of one int per thread (kBwdThreads threads).
__device__ __forceinline__ int block_scan_excl(int v, int *warp_tmp, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tmp[wid] = incl;
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kBwdWarps; ++w) {
        const int s = warp_tmp[w];
        if (w < wid) before += s;
        total += s;
    }
    __syncthreads();
    return before + incl - v;
}

template <int ORDER, int C, bool HAS_G>
__global__ void __launch_bounds__(kBwdThreads)
brick_bwd_kernel(const __grid_constant__ CUtensorMap gmap, int res, int nbx, int nby,
                 const float4 *__restrict__ sorted, const int *__restrict__ offsets, const float *__restrict__ dLdf,
                 const float *__restrict__ dLdg)
{
    using L = BwdLayout<ORDER, C, HAS_G>;
    using R = BwdRec<C, HAS_G>;
    constexpr int K = Basis<3, ORDER>::K;
    constexpr int NV = L::NV;
    constexpr int BXI = L::BXI;
    constexpr int RS = R::stride;
    static_assert((L::slab_floats * 4) % 128 == 0, "TMA source slabs must stay 128-byte aligned");
    static_assert((kBwdWarps * L::slab_floats * 4) % 16 == 0, "records must stay 16-byte aligned");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *slabs = reinterpret_cast<float *>(smem_raw);
    float *rec = slabs + kBwdWarps * L::slab_floats;
    int *cell_cur = reinterpret_cast<int *>(rec + L::rec_floats);
    int *cell_off = cell_cur + kBrickCells;          // kBrickCells + 1
    int *warp_tmp = cell_off + kBrickCells + 1;      // 32

    const int b = blockIdx.x;
    const int p0 = offsets[b], p1 = offsets[b + 1];
    if (p0 == p1) return;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    const float scale = (float)(res - 1);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float *slab = slabs + wid * L::slab_floats;

    for (int j = tid; j < kBwdWarps * L::slab_floats / 4; j += kBwdThreads)
        reinterpret_cast<float4 *>(slabs)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    bool slab_used = false;

    for (int base = p0; base < p1; base += kPChunk) {
        const int cnt = min(kPChunk, p1 - base);
        for (int j = tid; j < kBrickCells; j += kBwdThreads) cell_cur[j] = 0;
        __syncthreads();
        // 1. locate the staged points and count them per cell
        int my_lc[kPPT];
        float my_t[kPPT][3];
        int my_n[kPPT];
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            const int i = tid + r * kBwdThreads;
            my_lc[r] = -1;
            if (i < cnt) {
                const float4 q = sorted[base + i];
                const float x[3] = {q.x, q.y, q.z};
                int c[3];
                locate<3>(x, res, scale, c, my_t[r]);
                my_n[r] = __float_as_int(q.w);
                my_lc[r] = (c[0] - x0) + kBrick * ((c[1] - y0) + kBrick * (c[2] - z0));
                atomicAdd(cell_cur + my_lc[r], 1);
            }
        }
        __syncthreads();
        // 2. exclusive scan of the 512 cell counts (4 consecutive cells per thread)
        {
            int v[4], sum = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) { v[k] = cell_cur[4 * tid + k]; sum += v[k]; }
            int total;
            int run = block_scan_excl(sum, warp_tmp, total);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                cell_off[4 * tid + k] = run;
                cell_cur[4 * tid + k] = run;
                run += v[k];
            }
            if (tid == 0) cell_off[kBrickCells] = total;
        }
        __syncthreads();
        // 3. place the point records in cell order
#pragma unroll
        for (int r = 0; r < kPPT; ++r) {
            if (my_lc[r] < 0) continue;
            const int pos = atomicAdd(cell_cur + my_lc[r], 1);
            const int64_t n = my_n[r];
            float v[RS];
            v[0] = my_t[r][0]; v[1] = my_t[r][1]; v[2] = my_t[r][2];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) v[3 + ch] = __ldg(dLdf + n * C + ch);
            if constexpr (HAS_G) {
#pragma unroll
                for (int j = 0; j < 3 * C; ++j) v[3 + C + j] = __ldg(dLdg + n * 3 * C + j) * scale;
            }
            v[R::cell] = __int_as_float(my_lc[r]);
#pragma unroll
            for (int j = R::fields; j < RS; ++j) v[j] = 0.f;
            sts_block<float, RS>(rec + pos * RS, v);
        }
        __syncthreads();
        // 4. slab accumulation: lane segments aligned to cell boundaries
        {
            const int lo = cell_off[wid * kSlabCells], hi = cell_off[(wid + 1) * kSlabCells];
            const int n = hi - lo;
            slab_used |= n > 0;
            int s = lo + (lane * n) / 32;
            if (s < hi) {
                const int c = __float_as_int(rec[s * RS + R::cell]);
                if (cell_off[c] != s) s = cell_off[c + 1];
            }
            int e = __shfl_down_sync(0xffffffffu, s, 1);
            if (lane == 31) e = hi;
            const int len = max(0, e - s);
            const int steps = __reduce_max_sync(0xffffffffu, (unsigned)len);
            for (int j = 0; j < steps; ++j) {
                const bool active = j < len;
                const float *r = rec + (active ? s + j : lo) * RS;
                float t[3] = {r[0], r[1], r[2]};
                const int lc = __float_as_int(r[R::cell]);
                const int lx = lc & 7, ly = (lc >> 3) & 7, lz = (lc >> 6) - kSlabLayers * wid;
                const PointTables3<ORDER> P(t);
                float *cellp = slab + (lz * kBV + ly) * BXI + lx * NV;
                for_corners<0>([&](auto ic) {
                    constexpr int I = decltype(ic)::value;
                    constexpr int off = ((I >> 2) & 1) * kBV * BXI + ((I >> 1) & 1) * BXI + (I & 1) * NV;
                    if (active) {
                        const float w = P.template weight<I>();
                        float dw[3];
                        if constexpr (HAS_G) P.template dweight<I>(dw);
                        float acc[NV];
                        lds_block<float, NV>(cellp + off, acc);
#pragma unroll
                        for (int ch = 0; ch < C; ++ch) {
                            float sv = w * r[3 + ch];
                            float q[3];
                            if constexpr (HAS_G) {
                                const float *g = r + 3 + C + 3 * ch;
                                sv = fmaf(dw[0], g[0], fmaf(dw[1], g[1], fmaf(dw[2], g[2], sv)));
                                q[0] = w * g[0]; q[1] = w * g[1]; q[2] = w * g[2];
                            }
                            P.template accumulate<I, HAS_G>(sv, q, acc + ch * K);
                        }
                        sts_block<float, NV>(cellp + off, acc);
                    }
                    __syncwarp();
                });
            }
        }
        __syncthreads();
    }

    // Add this warp's 3-plane block to the global gradient.
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0 && slab_used) {
        tma_reduce_add_3d(&gmap, slab, x0 * NV, y0, z0 + kSlabLayers * wid);
        bulk_commit();
        bulk_wait_read_all();
    }
}

template <int DIM, int ORDER, int C>
static tg_status binned_bwd(const tg_grid *g, const tg_batch *bt, const float *uf, const float *ug, float *grad,
                            cudaStream_t s)
{
    if constexpr (DIM != 3) {
        return fail(TG_EINVAL, "binned path is 3-D only");
    } else {
        constexpr int NV = Basis<3, ORDER>::K * C;
        CUtensorMap map;
        tg_status st = make_brick_map(&map, grad, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->res, NV, kSlabPlanes);
        if (st != TG_OK) return st;
        if (ug) {
            auto k = brick_bwd_kernel<ORDER, C, true>;
            const int smem = BwdLayout<ORDER, C, true>::bytes;
            if ((st = set_smem((const void *)k, smem)) != TG_OK) return st;
            k<<<(unsigned)bt->nbricks, kBwdThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted,
                                                               bt->offsets, uf, ug);
        } else {
            auto k = brick_bwd_kernel<ORDER, C, false>;
            const int smem = BwdLayout<ORDER, C, false>::bytes;
            if ((st = set_smem((const void *)k, smem)) != TG_OK) return st;
            k<<<(unsigned)bt->nbricks, kBwdThreads, smem, s>>>(map, g->res, bt->nb[0], bt->nb[1], bt->sorted,
                                                               bt->offsets, uf, nullptr);
        }
        return launch_status("tg_query_backward_binned");
    }
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_query_backward_binned(const tg_grid *g, const tg_batch *bt, const float *dL_df,
                                              const float *dL_dgradx, float *coef_grad, tg_stream stream)
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
