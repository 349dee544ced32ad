// Vertex-centric coefficient-gradient gather over one brick (the adjoint of
// Eq. 2 - Eq. 4) for the binned backward, and the block scans and cell sort
// that the binned forward shares with it.
//
// The brick's staged points are sorted by cell in shared memory. Every
// thread owns whole vertices: for a vertex it walks the points of its (up to)
// eight incident cells - four contiguous ranges of the cell-sorted records,
// one per incident cell row - and accumulates w_i phi_k(delta_i) s (+ the
// spatial-gradient terms) in registers. No two threads ever write the same
// vertex, so nothing is atomic. Vertices are counting-sorted by their load
// (points in incident cells) before they are dealt to threads, so the lanes
// of a warp carry nearly equal work.
#pragma once

#include "tg_binned.cuh"

namespace tg {

constexpr int kBrickVerts = kBV * kBV * kBV;   // 729
constexpr int kMaxLoadBins = 64;               // vertex loads >= 63 share the last bin

// Staged point record: t (3), s = dL/df (C) and, with a spatial-gradient
// upstream, g = dL/d(grad_x f) (3 C, world units); padded to 16 bytes.
template <int C, bool HAS_G>
struct GatherRec {
    static constexpr int fields = 3 + C + (HAS_G ? 3 * C : 0);
    static constexpr int stride = (fields + 3) / 4 * 4;
};

// Shared-memory integer workspace of the gather (counts, offsets, vertex order).
struct GatherInts {
    static constexpr int cell_cur = 0;                          // kBrickCells
    static constexpr int cell_off = cell_cur + kBrickCells;     // kBrickCells + 1
    static constexpr int vload_bins = cell_off + kBrickCells + 1 + 3;   // kMaxLoadBins
    static constexpr int vorder = vload_bins + kMaxLoadBins;    // kBrickVerts
    static constexpr int warp_tmp = vorder + kBrickVerts + 3;   // 32
    static constexpr int total = warp_tmp + 32;
};

// Block-wide exclusive scan of one int per thread; returns the prefix and the total.
template <int NT>
__device__ __forceinline__ int gather_block_scan(int v, int *warp_tmp, int &total)
{
    constexpr int NW = NT / 32;
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
    for (int w = 0; w < NW; ++w) {
        const int s = warp_tmp[w];
        if (w < wid) before += s;
        total += s;
    }
    __syncthreads();
    return before + incl - v;
}

// Integer workspace of a cell sort alone (the forward's).
struct SortInts {
    static constexpr int cell_cur = 0;                          // kBrickCells
    static constexpr int cell_off = cell_cur + kBrickCells;     // kBrickCells + 1
    static constexpr int warp_tmp = cell_off + kBrickCells + 1 + 3;   // 32
    static constexpr int total = warp_tmp + 32;
};

// Scan of the 512 cell counts in ints[cell_cur] into ints[cell_off] and back
// into ints[cell_cur] (as placement cursors). All NT threads take part.
template <int NT, typename LAY = GatherInts>
__device__ __forceinline__ void gather_scan_cells(int *ints)
{
    static_assert(kBrickCells % NT == 0, "");
    constexpr int CPT = kBrickCells / NT;
    int *cur = ints + LAY::cell_cur, *off = ints + LAY::cell_off;
    int v[CPT], sum = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) { v[k] = cur[CPT * threadIdx.x + k]; sum += v[k]; }
    int total;
    int run = gather_block_scan<NT>(sum, ints + LAY::warp_tmp, total);
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        off[CPT * threadIdx.x + k] = run;
        cur[CPT * threadIdx.x + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) off[kBrickCells] = total;
    __syncthreads();
}

// Load of vertex v: the points of its incident cells in this round.
__device__ __forceinline__ int vertex_load(int v, const int *off)
{
    const int vx = v % kBV, vy = (v / kBV) % kBV, vz = v / (kBV * kBV);
    const int xlo = max(vx - 1, 0), xhi = min(vx, kBrick - 1);
    int n = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int cy = vy - (r & 1), cz = vz - (r >> 1);
        if (cy >= 0 && cz >= 0 && cy < kBrick && cz < kBrick) {
            const int row = kBrick * (cy + kBrick * cz);
            n += off[row + xhi + 1] - off[row + xlo];
        }
    }
    return n;
}

// Counting sort of the 729 vertices by load into ints[vorder] (heaviest first).
template <int NT>
__device__ __forceinline__ void gather_order_vertices(int *ints)
{
    int *bins = ints + GatherInts::vload_bins, *order = ints + GatherInts::vorder;
    const int *off = ints + GatherInts::cell_off;
    for (int j = threadIdx.x; j < kMaxLoadBins; j += NT) bins[j] = 0;
    __syncthreads();
    constexpr int VPT = (kBrickVerts + NT - 1) / NT;
    int key[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        const int v = threadIdx.x + k * NT;
        key[k] = -1;
        if (v < kBrickVerts) {
            key[k] = kMaxLoadBins - 1 - min(vertex_load(v, off), kMaxLoadBins - 1);   // heavy first
            atomicAdd(bins + key[k], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of the 64 bins by one warp
        int a = bins[2 * threadIdx.x], b = bins[2 * threadIdx.x + 1];
        int incl = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)threadIdx.x >= o) incl += u;
        }
        const int ex = incl - a - b;
        bins[2 * threadIdx.x] = ex;
        bins[2 * threadIdx.x + 1] = ex + a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        if (key[k] >= 0) order[atomicAdd(bins + key[k], 1)] = threadIdx.x + k * NT;
    }
    __syncthreads();
}

// Accumulates into acc[NV] the contributions of all staged points of the
// incident cells of vertex v (local coordinates).
template <int ORDER, int C, bool HAS_G>
__device__ __forceinline__ void gather_vertex(int v, const float *rec, const int *off, float scale, float *acc)
{
    const float h = 1.0f / scale;
    constexpr int K = Basis<3, ORDER>::K;
    constexpr int RS = GatherRec<C, HAS_G>::stride;
    const int vx = v % kBV, vy = (v / kBV) % kBV, vz = v / (kBV * kBV);
    const int xlo = max(vx - 1, 0), xhi = min(vx, kBrick - 1);
    // The four incident cell rows r = (by, bz): point ranges [lo_r, lo_r + len_r)
    // and the first point of cell vx in each (points before it have bx = 1).
    int lo[4], len[4], mid[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int cy = vy - (r & 1), cz = vz - (r >> 1);
        lo[r] = len[r] = mid[r] = 0;
        if (cy >= 0 && cz >= 0 && cy < kBrick && cz < kBrick) {
            const int row = kBrick * (cy + kBrick * cz);
            lo[r] = off[row + xlo];
            len[r] = off[row + xhi + 1] - lo[r];
            mid[r] = off[row + vx];                   // = end of the row when vx = 8
        }
    }
    const int e0 = len[0], e1 = e0 + len[1], e2 = e1 + len[2], total = e2 + len[3];
    // One flat loop over the four ranges keeps a lane's trip count equal to
    // its (load-balanced) total.
    for (int j = 0; j < total; ++j) {
        const int r = (j < e0) ? 0 : (j < e1) ? 1 : (j < e2) ? 2 : 3;
        const int start = r == 0 ? 0 : r == 1 ? e0 : r == 2 ? e1 : e2;
        const int p = (r == 0 ? lo[0] : r == 1 ? lo[1] : r == 2 ? lo[2] : lo[3]) + (j - start);
        const int pm = r == 0 ? mid[0] : r == 1 ? mid[1] : r == 2 ? mid[2] : mid[3];
        const bool bx = p < pm, by = r & 1, bz = r >> 1;
        const float *q = rec + p * RS;
        const float4 tq = *reinterpret_cast<const float4 *>(q);
        const float t0 = tq.x, t1 = tq.y, t2 = tq.z;
        const float a0 = bx ? t0 : 1.f - t0;
        const float a1 = by ? t1 : 1.f - t1;
        const float a2 = bz ? t2 : 1.f - t2;
        const float w = a0 * a1 * a2;
        const float dl[3] = {(bx ? t0 - 1.f : t0) * h, (by ? t1 - 1.f : t1) * h, (bz ? t2 - 1.f : t2) * h};
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            float s = w * (ch == 0 ? tq.w : q[3 + ch]);
            float g[3];
            if constexpr (HAS_G) {
                const float *gp = q + 3 + C + 3 * ch;
                const float dw0 = (bx ? scale : -scale) * a1 * a2;     // d w / d x
                const float dw1 = (by ? scale : -scale) * a0 * a2;
                const float dw2 = (bz ? scale : -scale) * a0 * a1;
                s = fmaf(dw0, gp[0], fmaf(dw1, gp[1], fmaf(dw2, gp[2], s)));
                g[0] = w * gp[0]; g[1] = w * gp[1]; g[2] = w * gp[2];
            }
            Basis<3, ORDER>::template accumulate<HAS_G>(s, g, dl, acc + ch * K);
        }
    }
}

// One gather round: all NT threads take the vertices in load order and add
// their sums into the shared tile (row stride BXI floats, vertex stride NV),
// or, with ASSIGN (the brick's only round), store them over whatever the tile
// held - every vertex of the tile is written, empty ones with zeros.
template <int ORDER, int C, bool HAS_G, int NT, int BXI, bool ASSIGN>
__device__ __forceinline__ void gather_round(const float *rec, int *ints, float *tile, float scale)
{
    constexpr int NV = Basis<3, ORDER>::K * C;
    constexpr bool PAIRS = NV % 2 == 0 && BXI % 2 == 0;     // vertex blocks are 8-byte aligned
    gather_order_vertices<NT>(ints);
    const int *order = ints + GatherInts::vorder, *off = ints + GatherInts::cell_off;
    for (int j = threadIdx.x; j < kBrickVerts; j += NT) {
        const int v = order[j];
        float acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.f;
        gather_vertex<ORDER, C, HAS_G>(v, rec, off, scale, acc);
        float *d = tile + (v / kBV) * BXI + (v % kBV) * NV;
        if constexpr (PAIRS) {
            float2 *d2 = reinterpret_cast<float2 *>(d);
#pragma unroll
            for (int k = 0; k < NV / 2; ++k) {
                float2 o = make_float2(acc[2 * k], acc[2 * k + 1]);
                if (!ASSIGN) {
                    const float2 e = d2[k];
                    o.x += e.x;
                    o.y += e.y;
                }
                d2[k] = o;
            }
        } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) d[k] = ASSIGN ? acc[k] : d[k] + acc[k];
        }
    }
}

}  // namespace tg
