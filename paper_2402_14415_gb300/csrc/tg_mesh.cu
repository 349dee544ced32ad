// Mesh extraction and the surface metric of Sec. 4.1 (Chamfer distance).
//
// tg_extract_mesh samples channel 0 of a 3-D grid on an M^3 lattice (Eq. 2 -
// Eq. 4 at x = (i, j, k) / (M - 1)) and triangulates the level set
// {f = iso} by marching tetrahedra: every lattice cube is cut into the six
// tetrahedra around its main diagonal (one per order in which a monotone path
// from corner 0 to corner 7 visits the axes), so neighbouring cubes cut their
// common faces alike and no case table is needed. A tetrahedron with one
// vertex on its own side gives one triangle, a 2 : 2 split a quad (two
// triangles); triangles face increasing f. Crossings are interpolated from the
// lower-indexed end of each lattice edge, so the tetrahedra that share an edge
// produce the same point and the mesh closes.
//
// The output order is fixed: cubes row by row (k, j, then i), tetrahedra in a
// fixed order. A count pass gives every row of M - 1 cubes its triangle count
// (one warp per row), one block scans the rows, and the write pass recomputes
// each row warp by warp, 32 cubes at a time, placing a cube's triangles at its
// row offset plus a warp scan of the counts before it.
//
// tg_sample_mesh draws area-weighted points on a triangle soup (running FP64
// area, binary search), tg_chamfer sums squared nearest-neighbour distances
// between two point sets by brute force, tiled through shared memory.
#include "tg_internal.cuh"

namespace tg {

constexpr int kMeshThreads = 256;
constexpr int kScanThreads = 1024;
constexpr uint64_t kMeshStream = 0x4D455348ull;     // generator stream of the mesh sampler

// Corner q of a cube sits at offset (q & 1, q >> 1 & 1, q >> 2); the six
// tetrahedra around the diagonal 0 - 7, packed 4 bits per corner.
__device__ __forceinline__ int tet_corner(int tt, int a)
{
    constexpr uint32_t kTets[6] = {0x7310u, 0x7510u, 0x7320u, 0x7620u, 0x7540u, 0x7640u};
    return (kTets[tt] >> (4 * a)) & 15;
}

// The field (channel 0) at the lattice points, i fastest.
template <typename T, int ORDER, int C>
__global__ void __launch_bounds__(kMeshThreads)
lattice_kernel(const T *__restrict__ coefs, int res, int M, float *__restrict__ vals)
{
    using B = Basis<3, ORDER>;
    constexpr int K = B::K, NV = K * C;
    const int64_t n = (int64_t)M * M * M;
    const float scale = (float)(res - 1), h = 1.0f / (float)(res - 1), den = (float)(M - 1);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % M), j = (int)((idx / M) % M), k = (int)(idx / ((int64_t)M * M));
        const float x[3] = {__fdiv_rn((float)i, den), __fdiv_rn((float)j, den), __fdiv_rn((float)k, den)};
        int c[3];
        float t[3];
        locate<3>(x, res, scale, c, t);
        const int64_t v0 = base_vertex<3>(c, res);
        float f = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float th[K];
            load_block<T, K>(coefs + (v0 + corner_offset<3>(q, res)) * NV, th);
            float dw[3], dl[3], g[3];
            const float w = corner_weight<3>(q, t, dw);
#pragma unroll
            for (int d = 0; d < 3; ++d) dl[d] = (t[d] - (float)((q >> d) & 1)) * h;
            f = fmaf(w, B::eval(th, dl, g), f);
        }
        vals[idx] = f;
    }
}

struct MtCube {
    int c[8][3];
    float f[8];
};

__device__ __forceinline__ void mt_load(const float *vals, int M, int i, int j, int k, MtCube &q)
{
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        q.c[a][0] = i + (a & 1);
        q.c[a][1] = j + ((a >> 1) & 1);
        q.c[a][2] = k + (a >> 2);
        q.f[a] = __ldg(vals + q.c[a][0] + (int64_t)M * (q.c[a][1] + (int64_t)M * q.c[a][2]));
    }
}

// Triangles of one tetrahedron from its inside count (0..4).
__device__ __forceinline__ int mt_tris(int nin) { return (nin == 1 || nin == 3) ? 1 : (nin == 2 ? 2 : 0); }

__device__ __forceinline__ int mt_cube_count(const MtCube &q, float iso)
{
    int n = 0;
#pragma unroll
    for (int tt = 0; tt < 6; ++tt) {
        int nin = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) nin += q.f[tet_corner(tt, a)] < iso;
        n += mt_tris(nin);
    }
    return n;
}

// Crossing of the iso level on the lattice edge between corners a and b,
// interpolated from the edge's lower-indexed end.
__device__ __forceinline__ void mt_cross(const MtCube &q, int a, int b, float iso, float den, float *p)
{
    if (b < a) { const int s = a; a = b; b = s; }   // corner order = lattice index order within a cube
    const float fa = q.f[a], fb = q.f[b];
    const float t = __fdiv_rn(iso - fa, fb - fa);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float ca = (float)q.c[a][d], cb = (float)q.c[b][d];
        p[d] = __fdiv_rn(ca + t * (cb - ca), den);
    }
}

__device__ __forceinline__ float mt_orient(const float *a, const float *b, const float *c, const float *dir)
{
    const float u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
    const float v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
    return (u1 * v2 - u2 * v1) * dir[0] + (u2 * v0 - u0 * v2) * dir[1] + (u0 * v1 - u1 * v0) * dir[2];
}

__device__ __forceinline__ void mt_put(float *tris, int64_t slot, int64_t max_tris, const float *a, const float *b,
                                       const float *c)
{
    if (slot >= max_tris) return;
    float *o = tris + 9 * slot;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        o[d] = a[d];
        o[3 + d] = b[d];
        o[6 + d] = c[d];
    }
}

// Writes the cube's triangles from slot on; M - 1 = den (the lattice spacing is 1 / den).
__device__ void mt_cube_write(const MtCube &q, float iso, float den, float *tris, int64_t slot, int64_t max_tris)
{
    for (int tt = 0; tt < 6; ++tt) {
        int v[4], in[4], nin = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[a] = tet_corner(tt, a);
            in[a] = q.f[v[a]] < iso;
            nin += in[a];
        }
        if (nin == 0 || nin == 4) continue;
        float pos[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) pos[a][d] = __fdiv_rn((float)q.c[v[a]][d], den);
        if (nin == 1 || nin == 3) {
            int o = 0;                                             // the vertex on its own side
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (in[a] == (nin == 1)) o = a;
            float e[3][3], cen[3] = {0.f, 0.f, 0.f}, dir[3];
            int m = 0;
            for (int a = 0; a < 4; ++a) {
                if (a == o) continue;
                mt_cross(q, v[o], v[a], iso, den, e[m]);
                for (int d = 0; d < 3; ++d) cen[d] += e[m][d] / 3.0f;
                ++m;
            }
            for (int d = 0; d < 3; ++d) dir[d] = nin == 1 ? cen[d] - pos[o][d] : pos[o][d] - cen[d];
            if (mt_orient(e[0], e[1], e[2], dir) < 0.f) mt_put(tris, slot, max_tris, e[0], e[2], e[1]);
            else mt_put(tris, slot, max_tris, e[0], e[1], e[2]);
            ++slot;
        } else {
            int ii[2], oo[2], ni = 0, no = 0;
            for (int a = 0; a < 4; ++a) {
                if (in[a]) ii[ni++] = a;
                else oo[no++] = a;
            }
            float qd[4][3], dir[3];
            mt_cross(q, v[ii[0]], v[oo[0]], iso, den, qd[0]);
            mt_cross(q, v[ii[0]], v[oo[1]], iso, den, qd[1]);
            mt_cross(q, v[ii[1]], v[oo[1]], iso, den, qd[2]);
            mt_cross(q, v[ii[1]], v[oo[0]], iso, den, qd[3]);
            for (int d = 0; d < 3; ++d)
                dir[d] = 0.5f * (pos[oo[0]][d] + pos[oo[1]][d]) - 0.5f * (pos[ii[0]][d] + pos[ii[1]][d]);
            if (mt_orient(qd[0], qd[1], qd[2], dir) < 0.f) {      // both halves follow (q0 q1 q2)
                mt_put(tris, slot, max_tris, qd[0], qd[3], qd[2]);
                mt_put(tris, slot + 1, max_tris, qd[0], qd[2], qd[1]);
            } else {
                mt_put(tris, slot, max_tris, qd[0], qd[1], qd[2]);
                mt_put(tris, slot + 1, max_tris, qd[0], qd[2], qd[3]);
            }
            slot += 2;
        }
    }
}

// One warp per row (j, k) of M - 1 cubes: the row's triangle count.
__global__ void __launch_bounds__(kMeshThreads)
mt_count_kernel(const float *__restrict__ vals, int M, float iso, int *__restrict__ row_count)
{
    const int64_t rows = (int64_t)(M - 1) * (M - 1);
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int j = (int)(row % (M - 1)), k = (int)(row / (M - 1));
    int n = 0;
    for (int i = lane; i < M - 1; i += 32) {
        MtCube q;
        mt_load(vals, M, i, j, k, q);
        n += mt_cube_count(q, iso);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) row_count[row] = n;
}

// Exclusive scan of n counts (int or double) by one block into off[0..n), total into *total.
template <typename IN, typename OUT>
__global__ void __launch_bounds__(kScanThreads)
scan_one_block_kernel(const IN *__restrict__ in, int64_t n, const int64_t *__restrict__ n_dev, int64_t n_cap,
                      OUT *__restrict__ off, OUT *__restrict__ total)
{
    __shared__ OUT warp_sum[kScanThreads / 32];
    if (n_dev) n = min(*n_dev, n_cap);
    const int64_t per = (n + kScanThreads - 1) / kScanThreads;
    const int64_t b = threadIdx.x * per, e = min(b + per, n);
    OUT s = 0;
    for (int64_t x = b; x < e; ++x) s += (OUT)in[x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    OUT incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const OUT u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {
        OUT v = lane < kScanThreads / 32 ? warp_sum[lane] : (OUT)0;
        OUT vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const OUT u = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += u;
        }
        if (lane < kScanThreads / 32) warp_sum[lane] = vi - v;     // exclusive warp offsets
        if (lane == 31) *total = vi;
    }
    __syncthreads();
    OUT run = warp_sum[w] + incl - s;
    for (int64_t x = b; x < e; ++x) {
        off[x] = run;
        run += (OUT)in[x];
    }
}

// One warp per row: 32 cubes at a time, each lane's triangles at the row
// offset plus the warp's exclusive scan of the counts.
__global__ void __launch_bounds__(kMeshThreads)
mt_write_kernel(const float *__restrict__ vals, int M, float iso, const int64_t *__restrict__ row_off,
                float *__restrict__ tris, int64_t max_tris)
{
    const int64_t rows = (int64_t)(M - 1) * (M - 1);
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int j = (int)(row % (M - 1)), k = (int)(row / (M - 1));
    const float den = (float)(M - 1);
    int64_t base = row_off[row];
    for (int i0 = 0; i0 < M - 1; i0 += 32) {
        const int i = i0 + lane;
        MtCube q;
        int n = 0;
        if (i < M - 1) {
            mt_load(vals, M, i, j, k, q);
            n = mt_cube_count(q, iso);
        }
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (n > 0) mt_cube_write(q, iso, den, tris, base + incl - n, max_tris);
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Area of every triangle (FP64), 0 past the count.
__global__ void __launch_bounds__(kMeshThreads)
tri_area_kernel(const float *__restrict__ tris, const int64_t *__restrict__ n_dev, int64_t cap,
                double *__restrict__ area)
{
    const int64_t n = min(*n_dev, cap);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float *p = tris + 9 * t;
        const double u0 = (double)p[3] - p[0], u1 = (double)p[4] - p[1], u2 = (double)p[5] - p[2];
        const double v0 = (double)p[6] - p[0], v1 = (double)p[7] - p[1], v2 = (double)p[8] - p[2];
        const double cx = u1 * v2 - u2 * v1, cy = u2 * v0 - u0 * v2, cz = u0 * v1 - u1 * v0;
        area[t] = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    }
}

// Sample s: the first triangle whose inclusive running area exceeds
// U(3 s) times the total, then the point at barycentric (1 - sqrt r1,
// sqrt r1 (1 - r2), sqrt r1 r2) with r1 = U(3 s + 1), r2 = U(3 s + 2).
__global__ void __launch_bounds__(kMeshThreads)
sample_mesh_kernel(const float *__restrict__ tris, const int64_t *__restrict__ n_dev, int64_t cap,
                   const double *__restrict__ excl, const double *__restrict__ area, const double *__restrict__ total,
                   int64_t N, uint64_t seed, float *__restrict__ out)
{
    const uint64_t key = stream_key(seed, kMeshStream);
    const int64_t T = min(*n_dev, cap);
    const double tot = *total;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        if (T <= 0) {
            out[3 * s] = out[3 * s + 1] = out[3 * s + 2] = 0.f;
            continue;
        }
        const double u0 = (double)(mix64(key + 3 * (uint64_t)s) >> 40) * (1.0 / 16777216.0);
        const double r1 = (double)(mix64(key + 3 * (uint64_t)s + 1) >> 40) * (1.0 / 16777216.0);
        const double r2 = (double)(mix64(key + 3 * (uint64_t)s + 2) >> 40) * (1.0 / 16777216.0);
        const double target = u0 * tot;
        int64_t lo = 0, hi = T - 1;
        while (lo < hi) {                         // first t with excl[t] + area[t] > target
            const int64_t mid = (lo + hi) >> 1;
            if (excl[mid] + area[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        const float *p = tris + 9 * lo;
        const double sr = sqrt(r1), a = 1.0 - sr, b = sr * (1.0 - r2), c = sr * r2;
#pragma unroll
        for (int d = 0; d < 3; ++d) out[3 * s + d] = (float)(a * p[d] + b * p[3 + d] + c * p[6 + d]);
    }
}

constexpr int kChamferTile = 2048;

// sum over p in P of min over q in Q of |p - q|^2 (FP32 distances, FP64 sum).
__global__ void __launch_bounds__(kMeshThreads)
chamfer_kernel(const float *__restrict__ P, int64_t nP, const float *__restrict__ Q, int64_t nQ,
               double *__restrict__ sum)
{
    __shared__ float4 tile[kChamferTile];
    __shared__ double part[kMeshThreads / 32];
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool have = p < nP;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (have) {
        px = P[3 * p];
        py = P[3 * p + 1];
        pz = P[3 * p + 2];
    }
    float best = INFINITY;
    for (int64_t q0 = 0; q0 < nQ; q0 += kChamferTile) {
        const int cnt = (int)min((int64_t)kChamferTile, nQ - q0);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            const float *s = Q + 3 * (q0 + j);
            tile[j] = make_float4(s[0], s[1], s[2], 0.f);
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float4 q = tile[j];
            const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
            best = fminf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
    }
    double v = (have && nQ > 0) ? (double)best : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kMeshThreads / 32; ++w) s += part[w];
        atomicAdd(sum, s);
    }
}

template <typename T, int ORDER, int C>
static tg_status launch_lattice(const tg_grid *g, int M, float *vals, cudaStream_t s)
{
    const int64_t n = (int64_t)M * M * M;
    const int64_t need = (n + kMeshThreads - 1) / kMeshThreads, cap = (int64_t)num_sms() * 16;
    lattice_kernel<T, ORDER, C><<<(unsigned)(need < cap ? need : cap), kMeshThreads, 0, s>>>(
        (const T *)g->store, g->res, M, vals);
    return launch_status("tg_extract_mesh (field lattice)");
}

template <int ORDER, int C>
static tg_status lattice_dtype(const tg_grid *g, int M, float *vals, cudaStream_t s)
{
    if (g->dtype == TG_F32) return launch_lattice<float, ORDER, C>(g, M, vals, s);
    if (g->dtype == TG_BF16) return launch_lattice<__nv_bfloat16, ORDER, C>(g, M, vals, s);
    return launch_lattice<__half, ORDER, C>(g, M, vals, s);
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_extract_mesh(const tg_grid *g, int M, float iso, float *tris, int64_t max_tris,
                                     int64_t *n_tris, tg_stream stream)
{
    if (!g || !n_tris || (max_tris > 0 && !tris)) return fail(TG_EINVAL, "tg_extract_mesh: NULL argument");
    if (g->dim != 3) return fail(TG_EINVAL, "tg_extract_mesh: 3-D grids only");
    if (M < 2 || M > 2048) return fail(TG_EINVAL, "tg_extract_mesh: M must lie in [2, 2048]");
    if (max_tris < 0) return fail(TG_EINVAL, "tg_extract_mesh: max_tris < 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nl = (int64_t)M * M * M, rows = (int64_t)(M - 1) * (M - 1);
    float *vals = nullptr;
    int *row_count = nullptr;
    int64_t *row_off = nullptr;
    tg_status st = dev_alloc_async((void **)&vals, nl * sizeof(float), s, "tg_extract_mesh: lattice");
    if (st == TG_OK)
        st = dev_alloc_async((void **)&row_count, rows * sizeof(int), s, "tg_extract_mesh: counts");
    if (st == TG_OK)
        st = dev_alloc_async((void **)&row_off, rows * sizeof(int64_t), s, "tg_extract_mesh: offsets");
    if (st == TG_OK) {
#define TG_LAT(D, O, C) lattice_dtype<O, C>(g, M, vals, s)
        st = TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_LAT);
#undef TG_LAT
    }
    const unsigned row_blocks = (unsigned)((rows * 32 + kMeshThreads - 1) / kMeshThreads);
    if (st == TG_OK) {
        mt_count_kernel<<<row_blocks, kMeshThreads, 0, s>>>(vals, M, iso, row_count);
        st = launch_status("tg_extract_mesh (count)");
    }
    if (st == TG_OK) {
        scan_one_block_kernel<int, int64_t><<<1, kScanThreads, 0, s>>>(row_count, rows, nullptr, 0, row_off, n_tris);
        st = launch_status("tg_extract_mesh (scan)");
    }
    if (st == TG_OK) {
        mt_write_kernel<<<row_blocks, kMeshThreads, 0, s>>>(vals, M, iso, row_off, tris, max_tris);
        st = launch_status("tg_extract_mesh (write)");
    }
    if (vals) cudaFreeAsync(vals, s);
    if (row_count) cudaFreeAsync(row_count, s);
    if (row_off) cudaFreeAsync(row_off, s);
    return st;
}

extern "C" tg_status tg_sample_mesh(const float *tris, const int64_t *n_tris, int64_t max_tris, int64_t N,
                                    uint64_t seed, float *pts, tg_stream stream)
{
    if (!n_tris || (N > 0 && !pts) || (max_tris > 0 && !tris)) return fail(TG_EINVAL, "tg_sample_mesh: NULL argument");
    if (N < 0 || max_tris < 0) return fail(TG_EINVAL, "tg_sample_mesh: negative size");
    if (N == 0) return TG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t cap = max_tris > 0 ? max_tris : 1;
    double *area = nullptr, *excl = nullptr, *total = nullptr;
    tg_status st = dev_alloc_async((void **)&area, cap * sizeof(double), s, "tg_sample_mesh: areas");
    if (st == TG_OK) st = dev_alloc_async((void **)&excl, cap * sizeof(double), s, "tg_sample_mesh: scan");
    if (st == TG_OK) st = dev_alloc_async((void **)&total, sizeof(double), s, "tg_sample_mesh: total");
    if (st == TG_OK && max_tris > 0) {
        const int64_t need = (max_tris + kMeshThreads - 1) / kMeshThreads, lim = (int64_t)num_sms() * 16;
        tri_area_kernel<<<(unsigned)(need < lim ? need : lim), kMeshThreads, 0, s>>>(tris, n_tris, max_tris, area);
        st = launch_status("tg_sample_mesh (areas)");
    }
    if (st == TG_OK) {
        scan_one_block_kernel<double, double><<<1, kScanThreads, 0, s>>>(area, max_tris, n_tris, max_tris, excl,
                                                                         total);
        st = launch_status("tg_sample_mesh (scan)");
    }
    if (st == TG_OK) {
        const int64_t need = (N + kMeshThreads - 1) / kMeshThreads, lim = (int64_t)num_sms() * 16;
        sample_mesh_kernel<<<(unsigned)(need < lim ? need : lim), kMeshThreads, 0, s>>>(
            tris, n_tris, max_tris, excl, area, total, N, seed, pts);
        st = launch_status("tg_sample_mesh (sample)");
    }
    if (area) cudaFreeAsync(area, s);
    if (excl) cudaFreeAsync(excl, s);
    if (total) cudaFreeAsync(total, s);
    return st;
}

extern "C" tg_status tg_chamfer(const float *A, int64_t nA, const float *B, int64_t nB, double *sums,
                                tg_stream stream)
{
    if (!sums || (nA > 0 && !A) || (nB > 0 && !B)) return fail(TG_EINVAL, "tg_chamfer: NULL argument");
    if (nA < 0 || nB < 0) return fail(TG_EINVAL, "tg_chamfer: negative size");
    cudaStream_t s = (cudaStream_t)stream;
    if (nA > 0) {
        chamfer_kernel<<<(unsigned)((nA + kMeshThreads - 1) / kMeshThreads), kMeshThreads, 0, s>>>(A, nA, B, nB, sums);
        tg_status st = launch_status("tg_chamfer");
        if (st != TG_OK) return st;
    }
    if (nB > 0) {
        chamfer_kernel<<<(unsigned)((nB + kMeshThreads - 1) / kMeshThreads), kMeshThreads, 0, s>>>(B, nB, A, nA,
                                                                                                   sums + 1);
        return launch_status("tg_chamfer");
    }
    return TG_OK;
}
