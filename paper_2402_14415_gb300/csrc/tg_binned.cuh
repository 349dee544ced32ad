// Shared definitions of the brick-binned query path (3-D).
#pragma once

#include <cudaTypedefs.h>

#include "tg_internal.cuh"
#include "tg_tma.cuh"

struct tg_batch {
    int dim, res;
    int nb[3];            // bricks per axis
    int64_t nbricks;
    int64_t max_points;
    int64_t n;            // points binned by the last tg_batch_bin
    int G;                // chunk blocks of the histogram binning (0: global-atomic binning)
    int *counts;          // nbricks + 1 (global-atomic binning) / per-brick totals
    int *offsets;         // nbricks + 1, exclusive prefix sum of the brick counts
    int *cursor;          // nbricks, scatter cursors (global-atomic binning)
    int *hist;            // G x nbricks chunk histograms, then chunk cursors
    float4 *sorted;       // max_points: (x, y, z, original index as int bits)
    float4 *coarse;       // max_points: the same records grouped by coarse bin (histogram binning)
    int *perm;            // max_points: original index of every binned slot
    float *stage;         // binned-order per-point staging of the fused training steps (grown on demand)
    int64_t stage_floats; // capacity of stage
    bool stage_owned;     // stage was allocated by the batch (false: caller-provided scratch)
    float *aux;           // per-sample workspace of the renderer (grown on demand)
    int64_t aux_floats;
    int *status;          // device word: non-zero after a bounded wait gave up
    int device;
};

namespace tg {

constexpr int kBrick = 8;                              // cells per brick edge
constexpr int kBV = kBrick + 1;                        // vertices per brick edge
constexpr int kBrickCells = kBrick * kBrick * kBrick;  // 512

// Bytes of one brick row in a TMA box: the 9 vertex blocks padded to 16 bytes.
// 16-bit order-2 blocks (20 bytes) take a 208-byte row instead of 192: a
// 52-word row pitch shifts consecutive rows by 20 banks, against 16 for 48
// words (every second row on the same banks), which with cells sorted y
// fastest spreads the forward's tile reads over more banks; the box reads 16
// bytes of the next vertices it does not use.
constexpr int box_row_bytes(int nv, int elem)
{
    return (elem == 2 && nv == 10) ? 208 : (kBV * nv * elem + 15) / 16 * 16;
}

// Elements per brick row in a TMA box.
template <typename T, int NV>
struct BoxInner {
    static constexpr int bytes = box_row_bytes(NV, (int)sizeof(T));
    static constexpr int value = bytes / (int)sizeof(T);
    static constexpr int tile_bytes = kBV * kBV * bytes;   // a full 9 x 9 x 9 brick
};

inline int box_inner_host(int nv, int elem) { return box_row_bytes(nv, elem) / elem; }

__device__ __forceinline__ int brick_of(const int *c, int nbx, int nby)
{
    return (c[0] / kBrick) + nbx * ((c[1] / kBrick) + nby * (c[2] / kBrick));
}

// Tensor map of a res^3 x nv array (coefficients or gradient) viewed as the
// 3-D tensor [z][y][x * nv], with a box of box_z planes of 9 brick rows.
// 3-D tensor map of a res^3 grid of nv-element vertex blocks viewed as
// [z][y][x * nv], with a box of `box_inner` elements x 9 rows x box_z planes
// (box_inner >= 9 nv, a multiple of 16 bytes, at most 256).
tg_status make_brick_map(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int elem, int res, int nv,
                         int box_inner, int box_z);

// Opts a kernel in to more than 48 KB of dynamic shared memory.
tg_status set_smem(const void *kernel, int bytes);

tg_status check_pair(const tg_grid *g, const tg_batch *bt, const char *who);

// Makes bt->stage hold at least `floats` floats (grows a batch-owned buffer
// synchronously; a caller-provided buffer that is too small is an error).
tg_status ensure_stage(tg_batch *bt, int64_t floats, const char *who);
tg_status ensure_aux(tg_batch *bt, int64_t floats, const char *who);

// Large 3-D batches of tg_query / tg_query_backward are binned into a
// grid-owned batch and served by the binned kernels (input order).
// auto_bin_wanted: at least kAutoBinMin points and 8 per brick on average, a
// grid the binned path accepts (with FP32 gradients for the backward, which
// must be 16-byte aligned), and a stream that is not capturing.
constexpr int64_t kAutoBinMin = (int64_t)1 << 18;
bool auto_bin_wanted(const tg_grid *g, int64_t N, const float *coef_grad, cudaStream_t s);
// Bins pts into the grid's batch (creating or growing it: a synchronous
// allocation), runs op(batch) on stream s and orders the batch's next use after
// this one with an event. Calls on one grid from several threads are
// serialised on the host; their GPU work is ordered through the event.
tg_status with_auto_batch(const tg_grid *g, const float *pts, int64_t N, cudaStream_t s,
                          tg_status (*op)(const tg_grid *, tg_batch *, void *, cudaStream_t), void *arg);

}  // namespace tg
