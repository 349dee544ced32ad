// Vertex-centric coefficient gradient over one brick for value upstreams
// dL/df (the adjoint of Eq. 2 - Eq. 4 without a spatial-gradient upstream,
// outside the deterministic mode).
//
// A round of at most kFCap points of the brick:
//   1. locates every point and ranks it within its cell (one shared atomic),
//   2. scans the 512 cell counts in place into cell offsets and stores the
//      point's record (brick-local grid coordinates u - x0, s) at its
//      cell-sorted slot,
//   3. packs, per cell row and vertex x-position, (first slot, points of the
//      two cells beside x) into one word - one thread per cell row, from the
//      row's nine offsets - so that a vertex finds each of its four incident
//      cell rows in one load, and counting-sorts the vertices by load (heavy
//      first) so that the lanes of a warp walk lists of nearly equal length,
//   4. lets every thread walk its vertices' four row ranges as one flat loop,
//      accumulating s w_i phi_k = s A_x A_y A_z (1, U_x, U_y, U_z, U_x^2/2,
//      U_y^2/2, U_z^2/2, U_x U_y, U_x U_z, U_y U_z) in registers. With the
//      local coordinate l of the point and the vertex coordinate v,
//      d = l - v = t - b exactly (both lie on the FP32 grid of u), so
//      A = 1 - |d| (= 1 - t or t, exact where t - b is) and U = d h need no
//      corner bits; the sums are taken in d and scaled by h, h^2 / 2 or h^2
//      once per vertex,
//   5. stores the sums as the 9^3 tile for one TMA bulk-tensor reduce-add into
//      the gradient.
#pragma once

#include "tg_gather.cuh"

namespace tg {

constexpr int kFThreads = 256;
constexpr int kFCap = 640;                                   // points per round
constexpr int kFPPT = (kFCap + kFThreads - 1) / kFThreads;   // staged points per thread
constexpr int kFVPT = (kBrickVerts + kFThreads - 1) / kFThreads;   // vertices per thread (3)

template <int ORDER, int C>
struct FastLayout {
    static constexpr int K = Basis<3, ORDER>::K;
    static constexpr int NV = K * C;
    static constexpr int BXI = BoxInner<float, NV>::value;
    static constexpr int tile_floats = (kBV * kBV * BXI + 31) / 32 * 32;
    static constexpr int RS = 4 + (C > 1 ? (C + 3) / 4 * 4 : 0);   // record floats: l (3) and s (C = 1), or l + s block
    static constexpr int rec = tile_floats;                          // float offsets
    static constexpr int wtab = rec + kFCap * RS;                    // 64 cell rows x 9 x-positions (row pitch 12)
    static constexpr int cells = wtab + kBrick * kBrick * 12;        // 512 + 1 (+3) counts, then offsets
    static constexpr int bins = cells + kBrickCells + 4;             // 64
    static constexpr int warp_tmp = bins + kMaxLoadBins;             // 32
    static constexpr int order = warp_tmp + 32;                      // 729 ushorts
    static constexpr int words = order + (kBrickVerts + 7) / 2;
    static constexpr int bytes = words * 4;
};

template <int ORDER, int C, bool IN_ORDER>
__global__ void __launch_bounds__(kFThreads, 4)
brick_bwd_fast_kernel(const __grid_constant__ CUtensorMap gmap, int res, int nbx, int nby,
                      const float4 *__restrict__ sorted, const int *__restrict__ offsets,
                      const float *__restrict__ dLdf)
{
    using L = FastLayout<ORDER, C>;
    constexpr int K = L::K, NV = L::NV, BXI = L::BXI, RS = L::RS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    float *tile = sm;
    float *rec = sm + L::rec;
    unsigned *wtab = reinterpret_cast<unsigned *>(sm + L::wtab);
    int *cells = reinterpret_cast<int *>(sm + L::cells);
    int *bins = reinterpret_cast<int *>(sm + L::bins);
    int *warp_tmp = reinterpret_cast<int *>(sm + L::warp_tmp);
    unsigned short *order = reinterpret_cast<unsigned short *>(sm + L::order);

    const int b = blockIdx.x;
    const int p0 = offsets[b], p1 = offsets[b + 1];
    if (p0 == p1) return;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    const float scale = (float)(res - 1), h = 1.0f / scale;
    const int tid = threadIdx.x;
    const bool single = p1 - p0 <= kFCap;

    // the row padding of the tile is never written by the gather
    {
        constexpr int PAD = BXI - kBV * NV;
        if constexpr (PAD > 0) {
            for (int j = tid; j < kBV * kBV * PAD; j += kFThreads) tile[(j / PAD) * BXI + kBV * NV + j % PAD] = 0.f;
        }
        if (!single)
            for (int j = tid; j < kBV * kBV * BXI; j += kFThreads) tile[j] = 0.f;
    }

    for (int base = p0; base < p1; base += kFCap) {
        const int cnt = min(kFCap, p1 - base);
        for (int j = tid; j < kBrickCells; j += kFThreads) cells[j] = 0;
        if (tid < kMaxLoadBins) bins[tid] = 0;
        __syncthreads();
        // 1. locate and rank within the cell
        float pt[kFPPT][3], ps[kFPPT][C];
        int plc[kFPPT], prk[kFPPT];
#pragma unroll
        for (int r = 0; r < kFPPT; ++r) {
            const int i = tid + r * kFThreads;
            plc[r] = -1;
            if (i < cnt) {
                const float4 q = sorted[base + i];
                const int64_t n = IN_ORDER ? (int64_t)__float_as_int(q.w) : (int64_t)(base + i);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) ps[r][ch] = __ldg(dLdf + n * C + ch);
                const float x[3] = {q.x, q.y, q.z};
                int c[3];
                float t[3];
                locate<3>(x, res, scale, c, t);
                // local coordinate (c - x0) + t: exact, it is u - x0 on the FP32 grid of u
                pt[r][0] = (float)(c[0] - x0) + t[0];
                pt[r][1] = (float)(c[1] - y0) + t[1];
                pt[r][2] = (float)(c[2] - z0) + t[2];
                plc[r] = (c[0] - x0) + kBrick * ((c[1] - y0) + kBrick * (c[2] - z0));
                prk[r] = atomicAdd(cells + plc[r], 1);
            }
        }
        __syncthreads();
        // 2. counts -> offsets in place, records at their cell-sorted slots
        {
            static_assert(kBrickCells == 2 * kFThreads, "two cells per thread");
            const int c0 = cells[2 * tid], c1 = cells[2 * tid + 1];
            int total;
            const int ex = gather_block_scan<kFThreads>(c0 + c1, warp_tmp, total);   // synchronises
            cells[2 * tid] = ex;
            cells[2 * tid + 1] = ex + c0;
            if (tid == 0) cells[kBrickCells] = total;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kFPPT; ++r) {
            if (plc[r] < 0) continue;
            const int p = cells[plc[r]] + prk[r];
            float *d = rec + p * RS;
            *reinterpret_cast<float4 *>(d) = make_float4(pt[r][0], pt[r][1], pt[r][2], C == 1 ? ps[r][0] : 0.f);
            if constexpr (C > 1) {
#pragma unroll
                for (int ch = 0; ch < C; ++ch) d[4 + ch] = ps[r][ch];
            }
        }
        // 3. row words (one thread per cell row), then vertex loads for the sort
        if (tid < kBrick * kBrick) {
            const int *row = cells + kBrick * tid;
            const int4 o0 = *reinterpret_cast<const int4 *>(row), o1 = *reinterpret_cast<const int4 *>(row + 4);
            const int o[kBV] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w, row[kBrick]};
            unsigned *wr = wtab + 12 * tid;
#pragma unroll
            for (int vx = 0; vx < kBV; ++vx) {
                const int lo = o[vx > 0 ? vx - 1 : 0];                      // cells vx - 1 and vx
                const int hi = o[vx < kBrick ? vx + 1 : kBrick];
                wr[vx] = (unsigned)lo | ((unsigned)(hi - lo) << 16);
            }
        }
        __syncthreads();
        int vkey[kFVPT], vrank[kFVPT];
#pragma unroll
        for (int k = 0; k < kFVPT; ++k) {
            const int v = tid + k * kFThreads;
            vkey[k] = -1;
            if (v >= kBrickVerts) continue;
            const int vz = v / (kBV * kBV), vy = (v / kBV) % kBV, vx = v % kBV;
            int load = 0;
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int cy = vy - (rr & 1), cz = vz - (rr >> 1);
                if ((unsigned)cy < (unsigned)kBrick && (unsigned)cz < (unsigned)kBrick) {
                    load += (int)(wtab[12 * (cy + kBrick * cz) + vx] >> 16);
                }
            }
            vkey[k] = kMaxLoadBins - 1 - min(load, kMaxLoadBins - 1);          // heaviest first
            vrank[k] = atomicAdd(bins + vkey[k], 1);
        }
        __syncthreads();
        if (tid < 32) {   // bin starts
            const int a = bins[2 * tid], c = bins[2 * tid + 1];
            int incl = a + c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += u;
            }
            bins[2 * tid] = incl - a - c;
            bins[2 * tid + 1] = incl - c;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kFVPT; ++k)
            if (vkey[k] >= 0) order[bins[vkey[k]] + vrank[k]] = (unsigned short)(tid + k * kFThreads);
        __syncthreads();
        // 4. the flat walk over each vertex's four row ranges
#pragma unroll 1
        for (int jv = tid; jv < kBrickVerts; jv += kFThreads) {
            const int v = order[jv];
            const int vz = v / (kBV * kBV), vy = (v / kBV) % kBV, vx = v % kBV;
            unsigned dw[4];                     // the four incident cell rows (0: outside the brick)
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int cy = vy - (rr & 1), cz = vz - (rr >> 1);
                dw[rr] = ((unsigned)cy < (unsigned)kBrick && (unsigned)cz < (unsigned)kBrick)
                             ? wtab[12 * (cy + kBrick * cz) + vx] : 0u;
            }
            int st[4], dd[4];
            int run = 0;
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                st[rr] = run;
                dd[rr] = (int)(dw[rr] & 0xFFFFu) - run;    // slot = j + dd within range rr
                run += (int)(dw[rr] >> 16);
            }
            const int e0 = st[1], e1 = st[2], e2 = st[3], total = run;
            const float fvx = (float)vx, fvy = (float)vy, fvz = (float)vz;
            float acc[NV];
#pragma unroll
            for (int a = 0; a < NV; ++a) acc[a] = 0.f;
            for (int j = 0; j < total; ++j) {
                const bool P0 = j >= e0, P1 = j >= e1, P2 = j >= e2;
                const int d = P2 ? dd[3] : P1 ? dd[2] : P0 ? dd[1] : dd[0];
                const float *qp = rec + (j + d) * RS;
                const float4 q = *reinterpret_cast<const float4 *>(qp);
                const float dx = q.x - fvx, dy = q.y - fvy, dz = q.z - fvz;      // t - b per axis
                const float w = (1.f - fabsf(dx)) * (1.f - fabsf(dy)) * (1.f - fabsf(dz));
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float S = w * (C == 1 ? q.w : qp[4 + ch]);
                    float *ac = acc + ch * K;
                    ac[0] += S;
                    if constexpr (ORDER >= 1) {   // in grid units t - b; the powers of h are applied per vertex
                        const float sdx = S * dx, sdy = S * dy, sdz = S * dz;
                        ac[1] += sdx;
                        ac[2] += sdy;
                        ac[3] += sdz;
                        if constexpr (ORDER >= 2) {
                            ac[4] = fmaf(sdx, dx, ac[4]);          // twice the delta^2 / 2 terms
                            ac[5] = fmaf(sdy, dy, ac[5]);
                            ac[6] = fmaf(sdz, dz, ac[6]);
                            ac[7] = fmaf(sdx, dy, ac[7]);
                            ac[8] = fmaf(sdx, dz, ac[8]);
                            ac[9] = fmaf(sdy, dz, ac[9]);
                        }
                    }
                }
            }
            if constexpr (ORDER >= 1) {       // delta = (t - b) h: first-order sums take h, second-order h^2
                const float h2 = h * h, hh2 = 0.5f * h * h;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    acc[ch * K + 1] *= h;
                    acc[ch * K + 2] *= h;
                    acc[ch * K + 3] *= h;
                    if constexpr (ORDER >= 2) {
                        acc[ch * K + 4] *= hh2;
                        acc[ch * K + 5] *= hh2;
                        acc[ch * K + 6] *= hh2;
                        acc[ch * K + 7] *= h2;
                        acc[ch * K + 8] *= h2;
                        acc[ch * K + 9] *= h2;
                    }
                }
            }
            float *dst = tile + (v / kBV) * BXI + (v % kBV) * NV;
            if constexpr (NV % 2 == 0 && BXI % 2 == 0) {
                float2 *d2 = reinterpret_cast<float2 *>(dst);
#pragma unroll
                for (int a = 0; a < NV / 2; ++a) {
                    float2 o = make_float2(acc[2 * a], acc[2 * a + 1]);
                    if (!single) {
                        const float2 e = d2[a];
                        o.x += e.x;
                        o.y += e.y;
                    }
                    d2[a] = o;
                }
            } else {
#pragma unroll
                for (int a = 0; a < NV; ++a) dst[a] = single ? acc[a] : dst[a] + acc[a];
            }
        }
        __syncthreads();                        // the round's records and descriptors are dead
    }
    // 5. one reduce-add of the tile
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
        tma_reduce_add_3d(&gmap, tile, x0 * NV, y0, z0);
        bulk_commit();
        bulk_wait_read_all();
    }
}

}  // namespace tg
