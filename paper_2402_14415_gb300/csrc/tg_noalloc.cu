// tg_query_noalloc: the brick-binned forward query for callers that cannot
// allocate device memory. All of its scratch (brick counters, offsets, write
// cursors, the sorted point records, the permutation and a status word) lives
// in one file-scope device array of fixed size; the call itself never
// allocates. tg_noalloc_timeouts reads and clears the status word.
#include <stddef.h>

#include <mutex>

#include "tg_binned.cuh"

namespace tg {

constexpr int64_t kNoallocMaxPoints = (int64_t)1 << 18;     // 262144 points per call
constexpr int64_t kNoallocMaxBricks = 32768;                // res <= 257

struct NoallocScratch {      // every array starts on a 16-byte boundary
    int counts[kNoallocMaxBricks + 4];
    int offsets[kNoallocMaxBricks + 4];
    int cursor[kNoallocMaxBricks];
    int status[4];
    float4 sorted[kNoallocMaxPoints];
    int perm[kNoallocMaxPoints];
};

// The vector paths of the scans and the float4 records need every array on a
// 16-byte boundary (a misaligned layout once raised a misaligned-address fault).
static_assert(kNoallocMaxBricks % 4 == 0 && kNoallocMaxPoints % 4 == 0, "array sizes must keep 16-byte alignment");
static_assert(offsetof(NoallocScratch, counts) % 16 == 0, "counts");
static_assert(offsetof(NoallocScratch, offsets) % 16 == 0, "offsets");
static_assert(offsetof(NoallocScratch, cursor) % 16 == 0, "cursor");
static_assert(offsetof(NoallocScratch, status) % 16 == 0, "status");
static_assert(offsetof(NoallocScratch, sorted) % 16 == 0, "sorted");
static_assert(offsetof(NoallocScratch, perm) % 16 == 0, "perm");

// About 5.6 MB; every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a stand-in).
static tg_status scratch_address(NoallocScratch **out)
{
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    tg_status st = cuda_status(cudaGetDevice(&dev), "tg_query_noalloc: cudaGetDevice");
    if (st != TG_OK) return st;
    if (dev < 0 || dev >= 64) return fail(TG_EINVAL, "tg_query_noalloc: device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        st = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch), "tg_query_noalloc: cudaGetSymbolAddress");
        if (st != TG_OK) return st;
        addr[dev] = p;
    }
    *out = reinterpret_cast<NoallocScratch *>(addr[dev]);
    return TG_OK;
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_query_noalloc(const tg_grid *g, const float *pts, int64_t N, float *out, float *grad_x,
                                      tg_stream stream)
{
    if (!g) return fail(TG_EINVAL, "tg_query_noalloc: grid is NULL");
    if (g->dim != 3) return fail(TG_EINVAL, "tg_query_noalloc: 3-D grids only");
    if (N < 0) return fail(TG_EINVAL, "tg_query_noalloc: N < 0");
    if (N > kNoallocMaxPoints)
        return fail(TG_EINVAL, "tg_query_noalloc: N = %lld exceeds the fixed scratch limit of %lld points",
                    (long long)N, (long long)kNoallocMaxPoints);
    if (N == 0) return TG_OK;
    if (!pts || !out) return fail(TG_EINVAL, "tg_query_noalloc: NULL pts or out");
    int dev = -1;
    tg_status st = cuda_status(cudaGetDevice(&dev), "tg_query_noalloc: cudaGetDevice");
    if (st != TG_OK) return st;
    if (dev != g->device)     // the scratch and the coefficients must be on one GPU
        return fail(TG_EINVAL, "tg_query_noalloc: the grid lives on device %d but device %d is current", g->device,
                    dev);
    tg_batch b = {};
    b.dim = 3;
    b.res = g->res;
    b.nbricks = 1;
    for (int d = 0; d < 3; ++d) {
        b.nb[d] = (g->res - 1 + kBrick - 1) / kBrick;
        b.nbricks *= b.nb[d];
    }
    if (b.nbricks > kNoallocMaxBricks)
        return fail(TG_EINVAL, "tg_query_noalloc: res = %d needs %lld bricks, over the fixed limit of %lld",
                    g->res, (long long)b.nbricks, (long long)kNoallocMaxBricks);
    NoallocScratch *s = nullptr;
    st = scratch_address(&s);
    if (st != TG_OK) return st;
    b.max_points = kNoallocMaxPoints;
    b.G = 0;                       // global-atomic binning: needs no per-chunk histogram
    b.counts = s->counts;
    b.offsets = s->offsets;
    b.cursor = s->cursor;
    b.hist = nullptr;
    b.sorted = s->sorted;
    b.perm = s->perm;
    b.stage = nullptr;             // the input-order forward writes straight to out / grad_x
    b.stage_floats = 0;
    b.stage_owned = false;
    b.status = s->status;
    b.device = dev;
    st = tg_batch_bin(&b, pts, N, stream);     // clears the brick counters before counting
    if (st != TG_OK) return st;
    return tg_query_binned(g, &b, out, grad_x, TG_ORDER_INPUT, stream);
}

extern "C" tg_status tg_noalloc_timeouts(int *timed_out)
{
    if (!timed_out) return fail(TG_EINVAL, "tg_noalloc_timeouts: timed_out is NULL");
    NoallocScratch *s = nullptr;
    tg_status st = scratch_address(&s);
    if (st != TG_OK) return st;
    if ((st = cuda_status(cudaDeviceSynchronize(), "tg_noalloc_timeouts: wait for the device")) != TG_OK) return st;
    int v = 0;
    if ((st = cuda_status(cudaMemcpy(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost), "tg_noalloc_timeouts")) !=
        TG_OK)
        return st;
    *timed_out = v;
    if (v) st = cuda_status(cudaMemset(s->status, 0, sizeof(int)), "tg_noalloc_timeouts: clear");
    return st;
}
