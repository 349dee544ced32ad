/*
 * taylorgrid.h - C ABI of the GB300 TaylorGrid field engine.
 *
 * TaylorGrid (arXiv 2402.14415, Sec. 3.1) stores at every vertex of a dense
 * grid V_T a truncated Taylor series S(v) of the field: the value, the
 * gradient and, at order 2, the Hessian. A query point x is evaluated by
 * finding its voxel (Eq. 2), evaluating the series of each of the 2^D corner
 * vertices at the offset x - v_i (Eq. 1, Eq. 3) and blending the 2^D values
 * with trilinear (bilinear in 2-D) weights (Eq. 4). The grid is optimised
 * directly: the loss gradient is scattered back onto the coefficients.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Domain [0,1]^D with D = dim in {2, 3}; `res` >= 2 vertices per axis,
 *    vertex j at x = j / (res - 1).
 *  - K = C(D + order, order) coefficients per vertex and channel, stored in
 *    this order (true Hessian entries; the 1/2 of Eq. 1 applies to the
 *    diagonal only and each off-diagonal entry appears once):
 *        3-D: f, g_x, g_y, g_z, H_xx, H_yy, H_zz, H_xy, H_xz, H_yz
 *        2-D: f, g_x, g_y, H_xx, H_yy, H_xy
 *    Derivatives are taken with respect to the world coordinates x, as in
 *    Eq. 1: the offset of Eq. 3 is delta = x - v_i = (t - b_i) / (res - 1).
 *  - Exchange layout (tg_set_coefs / tg_get_coefs / coefficient gradients):
 *    FP32 [vertex][channel][k], vertex = x + res (y + res z). The library's
 *    device layout of the stored coefficients is the same order, in the
 *    grid's storage dtype.
 *  - Index rule of Eq. 2 (bit-exact, normative): clamp each coordinate to
 *    [0,1] (NaN becomes 0), u = fl32(x * (res - 1)) as one round-to-nearest
 *    FP32 multiply, c = min(floor(u), res - 2), t = fl32(u - c). A point on an
 *    interior face belongs to the upper cell; x = 1 lies in cell res - 2, t = 1.
 *  - All evaluation, blending and gradient accumulation is FP32.
 *  - Pointers marked (device) are device memory owned by the caller unless a
 *    call says otherwise; (host) pointers are host memory. Every call that
 *    takes a `tg_stream` (a cudaStream_t; NULL = the legacy default stream)
 *    only enqueues work on that stream and returns without synchronising.
 *  - Every call returns a tg_status and never aborts. A failed call leaves
 *    its outputs unspecified; tg_last_error() describes the last failure of
 *    the calling thread.
 */
#ifndef TAYLORGRID_H
#define TAYLORGRID_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TG_API __attribute__((visibility("default")))
#else
#define TG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TG_OK = 0,
    TG_EINVAL = 1,     /* an argument is out of range or a pointer is NULL */
    TG_ENOMEM = 2,     /* device allocation failed */
    TG_EBUDGET = 3,    /* admission refused: the request can never fit the HBM budget */
    TG_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
    TG_EDEVICE = 5,    /* a CUDA call or kernel launch failed */
    TG_ENOTFOUND = 6,  /* unknown job or handle */
    TG_EBUSY = 7       /* the object is in use (e.g. a grid still referenced by a job) */
} tg_status;

typedef enum { TG_F32 = 0, TG_BF16 = 1, TG_F16 = 2 } tg_dtype;

typedef void *tg_stream;            /* cudaStream_t */
typedef struct tg_grid tg_grid;     /* opaque, library-owned */

/* Human-readable name of a status code (static storage). */
TG_API const char *tg_status_string(tg_status s);

/* Description of the last failure on the calling thread (static, per thread). */
TG_API const char *tg_last_error(void);

/* Host-side fault injection for tests of the failure paths (no paper
 * counterpart): after this call the next `pass` device allocations made by
 * the library succeed and the `fail` allocations after them report TG_ENOMEM
 * without reaching the CUDA allocator; fail = 0 switches injection off.
 * Process-wide. The GPU never sees a fault: the failing call returns
 * TG_ENOMEM and frees what it had allocated. Errors: TG_EINVAL (negative). */
TG_API tg_status tg_inject_alloc_failures(int pass, int fail);

/* Measured FP32 FMA throughput of the current device (no paper counterpart):
 * the denominator of the ALU roofline beside the measured HBM copy peak. A
 * kernel of independent fused multiply-add chains, one resident wave of blocks
 * per SM, is timed with CUDA events after one warm-up launch; *tflops receives
 * 2 x FMAs / seconds / 1e12. Synchronous: it waits for the device, allocates
 * and frees 4 bytes. Errors: TG_EINVAL (NULL), TG_ENOMEM, TG_EDEVICE. */
TG_API tg_status tg_measure_fp32_peak(double *tflops);

/* ---------------------------------------------------------------------------
 * Grid storage V_T (Sec. 3.1: "a dense grid G of size w x d x h", each vertex
 * storing the low-order Taylor series).
 * ------------------------------------------------------------------------ */

/* Create a res^dim grid of order `order` (0, 1 or 2) with `channels`
 * (1..4) independent series per vertex, stored in `dtype`. When dtype is
 * BF16 or FP16 an FP32 master copy is kept for the optimiser and the stored
 * copy is its round-to-nearest image. Coefficients are initialised to
 * N(0, init_std^2) drawn from the counter-based generator
 * (seed, stream 0xC0EF, index j) in exchange-layout order, on the current
 * device, and the call synchronises the device before returning.
 * Errors: TG_EINVAL for a bad shape or NULL `out`, TG_ENOMEM. */
TG_API tg_status tg_create(int dim, int res, int order, int channels, tg_dtype dtype,
                    uint64_t seed, float init_std, tg_grid **out);

/* Free a grid and everything it owns (coefficients, master, Adam state).
 * The caller must ensure no enqueued work still uses it. NULL is a no-op. */
TG_API tg_status tg_destroy(tg_grid *grid);

typedef struct {
    int dim, res, order, channels, K;
    tg_dtype dtype;
    int64_t n_vertices;     /* res^dim */
    int64_t n_coefs;        /* n_vertices * channels * K */
    size_t bytes;           /* device bytes held (storage + master + Adam state) */
    const void *coefs;      /* (device) stored coefficients, storage dtype, exchange order */
    const float *master;    /* (device) FP32 master (same as coefs for TG_F32) */
} tg_grid_info;

TG_API tg_status tg_get_info(const tg_grid *grid, tg_grid_info *info);

/* Load FP32 coefficients (device, exchange layout, n_coefs floats) into the
 * master copy and the stored copy (rounded to the storage dtype). `src` may be
 * the grid's own master (tg_grid_info.master), e.g. after an optimiser outside
 * the library updated it in place: then only the stored copy is refreshed. */
TG_API tg_status tg_set_coefs(tg_grid *grid, const float *src, tg_stream stream);

/* Read coefficients into `dst` (device, n_coefs floats). which = 0: the
 * stored copy, widened to FP32 (what queries use); which = 1: the FP32 master;
 * which = 2 / 3: Adam's first / second moment widened to FP32 (TG_EINVAL
 * before the first Adam step). FP32 grids keep FP32 moments; BF16 and FP16
 * grids keep them in BF16 (the FP32 master and FP32 arithmetic stay). */
TG_API tg_status tg_get_coefs(const tg_grid *grid, float *dst, int which, tg_stream stream);

/* Progressive resolution (Sec. 4.1 trains coarse to fine): overwrites dst's
 * coefficients with the Taylor data of src's field (Eq. 4) at dst's vertices
 * - the value, the world-unit gradient and, at order 2, the Hessian of the
 * blended field, including the blend weights' derivatives - for any dst res
 * and order (3-D grids with the same channels). A dst vertex's coordinates
 * are fl32(j / (res_dst - 1)) and it takes the src cell of Eq. 2's rule, so a
 * vertex on a src face takes the upper cell's one-sided derivatives. Writes
 * dst's FP32 master and rounds its stored copy; dst's Adam state is left as
 * is (a fresh grid has none). A src quadratic field is reproduced exactly.
 * Errors: TG_EINVAL (NULL or 2-D grid, channel mismatch, src == dst), TG_EDEVICE. */
TG_API tg_status tg_resample(const tg_grid *src, tg_grid *dst, tg_stream stream);

/* Checkpoint / resume (synchronous; host files). tg_save writes the grid's
 * shape, its FP32 master coefficients and, if the grid has taken an Adam
 * step, Adam's two moments: format "TGCK", u32 version 1, i32 dim, res,
 * order, channels, dtype, has_adam, i64 n_coefs, then n_coefs floats per
 * array (little-endian). tg_load creates a grid on the current device from
 * such a file (the stored BF16/FP16 copy is rounded from the master), so a fit
 * resumes where it stopped; the caller keeps its own Adam step counter.
 * Errors: TG_EINVAL (NULL argument, unreadable / malformed / truncated file),
 * TG_ENOMEM, TG_EDEVICE. */
TG_API tg_status tg_save(const tg_grid *grid, const char *path);
TG_API tg_status tg_load(const char *path, tg_grid **out);

/* ---------------------------------------------------------------------------
 * Field query, Eq. 2 - Eq. 4.
 * ------------------------------------------------------------------------ */

/* Eq. 2 alone: the voxel of each point under the index rule above.
 * Writes cells (device, N x dim int32, lower-corner vertex coordinates) and,
 * if t is not NULL, the local coordinates (device, N x dim FP32). These are
 * exactly the indices and offsets every query kernel uses. */
TG_API tg_status tg_locate(int dim, int res, const float *pts, int64_t N, int32_t *cells, float *t,
                    tg_stream stream);

/* Forward query of N points (device, N x dim FP32, row-major). Writes
 * out (device, N x channels) = f(x) and, if grad_x is not NULL, the spatial
 * gradient in world units (device, N x channels x dim) = d f / d x, which is
 * the blend derivative of Eq. 4 plus the series derivative g + H delta of
 * each corner, times (res - 1). Points are clamped to the domain.
 * Large 3-D batches (N >= 2^18 and at least 8 points per 8^3-cell brick on
 * average, on a grid the binned calls below accept, outside stream capture)
 * are binned into a batch the grid owns and evaluated by the binned kernels;
 * the first such call allocates that batch (36 bytes per point, synchronously)
 * and later larger calls grow it. Calls on one grid from several streams are
 * ordered through an event; the results equal the point-parallel ones up to
 * FP32 rounding. Everything else runs one thread per point.
 * N = 0 is a no-op. Errors: TG_EINVAL (NULL grid/pts/out with N > 0,
 * N < 0), TG_ENOMEM, TG_EDEVICE (launch failure). */
TG_API tg_status tg_query(const tg_grid *grid, const float *pts, int64_t N,
                   float *out, float *grad_x, tg_stream stream);

/* Coefficient gradient of the query (direct grid optimisation: the field is
 * linear in the coefficients, f = A theta, so this computes A^T). Given the
 * upstream gradients dL_df (device, N x channels) and optionally dL_dgradx
 * (device, N x channels x dim, world units; NULL = none), ADDS
 *   dL/dtheta_{v,c,k} += sum_n w_i(x_n) phi_k(delta_i) dL_df[n,c]
 *                        + sum_d dL_dgradx[n,c,d] d/dx_d (w_i phi_k(delta_i))
 * (v the i-th corner of x_n's cell, delta_i = x_n - v in world units, phi_k
 * the basis 1, delta_d, delta_d^2 / 2, delta_a delta_b of Eq. 1) into
 * coef_grad (device, FP32, n_coefs, exchange layout) with FP32 reductions at
 * L2; consecutive points that share a cell are first combined inside the
 * warp. The summation order is not fixed, so results vary at FP32 rounding.
 * Large batches are binned as in tg_query (when coef_grad is 16-byte
 * aligned) and scattered by the binned backward.
 * The caller zeroes coef_grad (tg_adam_step does so after using it).
 * Errors as tg_query. */
TG_API tg_status tg_query_backward(const tg_grid *grid, const float *pts, int64_t N,
                            const float *dL_df, const float *dL_dgradx,
                            float *coef_grad, tg_stream stream);

/* ---------------------------------------------------------------------------
 * Brick-binned query path. The paper gives no kernel design; this is the
 * GB300 path for large batches: points are counting-sorted by the 8^D-cell
 * brick that holds their voxel, then each thread block stages one brick of
 * coefficients in shared memory and evaluates (forward) or accumulates
 * (backward) its points there, so the grid is streamed about once per pass
 * instead of gathered per point. Results equal tg_query / tg_query_backward.
 * ------------------------------------------------------------------------ */
typedef struct tg_batch tg_batch;   /* opaque; owns the scratch of one binned batch */

/* Create a batch able to hold up to max_points points for grids of the
 * given dim and res (the brick count depends on res). Allocates device
 * scratch (about 36 bytes per point plus 12 bytes per brick, and 4 bytes per
 * brick for each of the per-SM binning histograms). */
TG_API tg_status tg_batch_create(int dim, int res, int64_t max_points, tg_batch **out);
TG_API tg_status tg_batch_destroy(tg_batch *batch);

/* Bin N points (device, N x dim). The batch keeps a sorted copy of the points
 * and the permutation; `pts` may be reused by the caller afterwards. */
TG_API tg_status tg_batch_bin(tg_batch *batch, const float *pts, int64_t N, tg_stream stream);

/* Order of the per-point arrays of the two calls below. */
#define TG_ORDER_INPUT 0    /* the caller's original point order */
#define TG_ORDER_BINNED 1   /* the batch's binned order (see tg_batch_order / tg_batch_points) */
/* OR'd into the backward's flags: bitwise reproducible coefficient gradients.
 * The brick kernels run in 8 launches, one per parity class of bricks (bricks
 * of a class share no vertex), and each cell's points are ordered by input
 * index before the gather, so every gradient element sums the same terms in
 * the same order on every run. A brick holding more than 1024 of the batch's
 * points is processed in rounds of 1024 taken by input index (the 1024
 * smallest, the next 1024, ...), found by a binary search over the brick per
 * round, so such bricks cost more than in the default mode. */
#define TG_DETERMINISTIC 2

/* Same outputs as tg_query / tg_query_backward for the points last binned.
 * With TG_ORDER_INPUT the per-point arrays (out, grad_x, dL_df, dL_dgradx)
 * are in the caller's original order: each binned record carries its input
 * index, and the kernels write the outputs (or read the upstream gradients)
 * at that index. With TG_ORDER_BINNED they are in binned order (slot p of
 * tg_batch_order), which keeps those accesses within each brick's range -
 * use it when the per-point work around the query (a loss, a sampler) can
 * run in that order too. Neither order needs scratch beyond the batch.
 * Kernels: with at least 48 points per brick on average (96 when spatial
 * gradients are asked for or given) one block per brick stages the brick's
 * coefficient (or gradient) tile through shared memory; below that, or where
 * a grid row of res x K x channels elements is not a whole number of 16-byte
 * units, one thread per binned record gathers (or reduces into) its 8 corner
 * blocks directly. The deterministic backward always takes the brick form.
 * TG_BINNED_PATH=brick or =records in the environment (read at every call)
 * forces one form, for measurements and tests.
 * Errors: TG_EINVAL (shape or order flag), TG_EDEVICE. */
TG_API tg_status tg_query_binned(const tg_grid *grid, const tg_batch *batch,
                                 float *out, float *grad_x, int order_flags, tg_stream stream);
TG_API tg_status tg_query_backward_binned(const tg_grid *grid, const tg_batch *batch,
                                          const float *dL_df, const float *dL_dgradx,
                                          float *coef_grad, int order_flags, tg_stream stream);

/* The original index of every binned slot (device, N int32): slot p holds
 * input point idx[p]. */
TG_API tg_status tg_batch_order(const tg_batch *batch, int32_t *idx, tg_stream stream);

/* The binned points in binned order (device, N x 3 FP32). */
TG_API tg_status tg_batch_points(const tg_batch *batch, float *pts, tg_stream stream);

/* Move per-point rows of `width` floats (1..64) between the two orders of
 * the points last binned. tg_batch_gather: dst (device, N x width, binned
 * order) [p] = src (device, N x width, input order) [idx[p]].
 * tg_batch_scatter: dst (input order) [idx[p]] = src (binned order) [p].
 * idx is the order of tg_batch_order. Together with TG_ORDER_BINNED these
 * give the same results as TG_ORDER_INPUT, one launch per call; they let a
 * caller permute several arrays at once or keep them in binned order.
 * src and dst must not overlap. N = 0 is a no-op.
 * Errors: TG_EINVAL (NULL batch or array, width out of range, src == dst),
 * TG_EDEVICE. */
TG_API tg_status tg_batch_gather(const tg_batch *batch, const float *src, int width, float *dst, tg_stream stream);
TG_API tg_status tg_batch_scatter(const tg_batch *batch, const float *src, int width, float *dst, tg_stream stream);

/* The binned kernels wait on their TMA copies with a 2 s limit; a wait that
 * gives up sets a device flag instead of hanging. Waits for all work on the
 * current device (cudaDeviceSynchronize), then reads that flag into
 * *timed_out (non-zero = some launch on this batch since the last call gave
 * up, its outputs are invalid) and clears it. Not for use during capture. */
TG_API tg_status tg_batch_timeouts(tg_batch *batch, int *timed_out);

/* The same for the batch that tg_query / tg_query_backward bin large 3-D
 * batches into (owned by the grid): *timed_out = 0 when no call has binned. */
TG_API tg_status tg_grid_timeouts(tg_grid *grid, int *timed_out);

/* Binned forward query that allocates nothing (the paper has no counterpart;
 * this is a deployment convenience). Some callers cannot call cudaMalloc:
 * code embedded in a host framework that owns every device allocation, or a
 * latency-critical serving path that must never reach the allocator. For
 * them this call bins the N points (device, N x 3) and evaluates f (and, if
 * grad_x is not NULL, the world-unit spatial gradient) exactly like
 * tg_batch_bin + tg_query_binned, with all scratch held in one fixed array
 * of about 5.6 MB compiled into the library (every GPU that loads the
 * library keeps it until the process exits).
 * Limits: N <= 262144 points and res <= 257 (at most 32768 bricks); other
 * requests fail with TG_EINVAL and a message. 3-D grids only, with the same shape rules as tg_query_binned.
 * The grid's device must be the current device (TG_EINVAL otherwise).
 * A TMA wait that gives up is reported by tg_noalloc_timeouts, not by the
 * return status of this call (which only enqueues).
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.
 * Every call reuses the same array and leaves its contents behind (the call
 * clears what must start at zero), so calls whose GPU work overlaps - on two
 * streams, or from two threads - race and give wrong results: serialise them. */
TG_API tg_status tg_query_noalloc(const tg_grid *grid, const float *pts, int64_t N,
                                  float *out, float *grad_x, tg_stream stream);

/* Timeout report of tg_query_noalloc (allocates nothing either): waits for
 * all work on the current device, reads the fixed array's status word into
 * *timed_out (non-zero = a bounded TMA wait of some call on this device gave
 * up since the last read, and that call's outputs are invalid) and clears it.
 * Errors: TG_EINVAL (NULL), TG_EDEVICE. */
TG_API tg_status tg_noalloc_timeouts(int *timed_out);

/* ---------------------------------------------------------------------------
 * Optimiser. The paper fixes only the learning rate (Sec. 4.1, "fixed
 * learning rate of 0.003"); the engine uses Adam (Kingma & Ba 2015) with
 * bias correction and no weight decay, fused into one pass.
 * ------------------------------------------------------------------------ */
typedef struct {
    float lr;
    float beta1, beta2, eps;
    int64_t step;            /* 1-based step number used for bias correction */
} tg_adam;

/* One fused Adam step over every coefficient of the grid: reads the FP32
 * master, coef_grad (device, n_coefs) and the moments, writes master and
 * moments, refreshes the stored BF16/FP16 copy (round to nearest even) and
 * zeroes coef_grad. The first call on a grid allocates and zeroes the
 * moments (synchronously), so make it before any stream capture.
 * Errors: TG_EINVAL (NULL, step < 1), TG_ENOMEM, TG_EDEVICE. */
TG_API tg_status tg_adam_step(tg_grid *grid, float *coef_grad, const tg_adam *params, tg_stream stream);

/* Lazy (sparse) Adam: as tg_adam_step, but a coefficient whose gradient is
 * exactly 0 this step keeps its parameter and both moments (its moments do
 * not decay); the others take the update above with the bias corrections of
 * the global step. This changes the optimiser: a coefficient that no point
 * touches stops moving instead of coasting on its first moment. It is the
 * rule of torch.optim.SparseAdam except for the placement of eps, which here
 * is added to sqrt(v_hat) as in tg_adam_step. A group of four coefficients
 * with zero gradients costs only its 16-byte gradient read, so steps that
 * touch a small part of the grid move far fewer bytes. Zeroes coef_grad.
 * Errors as tg_adam_step. */
TG_API tg_status tg_adam_step_lazy(tg_grid *grid, float *coef_grad, const tg_adam *params, tg_stream stream);

/* ---------------------------------------------------------------------------
 * SDF fitting (Sec. 3.2). The target S is the zero level set of an analytic
 * signed distance (Eq. 5): a union of spheres and axis-aligned boxes.
 * ------------------------------------------------------------------------ */
typedef struct {
    int n_spheres;
    int n_boxes;
    const float *spheres;    /* (device) n_spheres x (cx, cy, cz, r) */
    const float *boxes;      /* (device) n_boxes x (cx, cy, cz, hx, hy, hz) */
    const float *area_cdf;   /* (device) n_spheres + n_boxes cumulative surface-area fractions, last = 1
                                (spheres first); used by the sampler only */
} tg_shape;

/* Signed distance of the union at N points (device, N x 3, clamped to
 * [0,1]^3 like a query) into d (device, N). */
TG_API tg_status tg_sdf_eval_target(const tg_shape *shape, const float *pts, int64_t N, float *d,
                                    tg_stream stream);

/* Fit batch of step `step`: the first N/2 points uniform in [0,1]^3, the rest
 * near the surface (an area-weighted surface point of a member, kept if it is
 * not inside another member, up to 8 attempts, else a uniform point; plus
 * N(0, jitter^2) noise per axis, clamped). Every draw is the counter-based
 * generator (seed, stream step*256 + a, index 16 j + slot); the same
 * definition is implemented by the input generator of the tests. */
TG_API tg_status tg_sample_sdf_points(const tg_shape *shape, uint64_t seed, int64_t step, int64_t N,
                                      float jitter, float *pts, tg_stream stream);

/* One SDF fitting step on a 3-D one-channel grid (Sec. 3.2):
 *   L = mean_P w(x) |f(x) - d(x)|  +  lambda_eik * mean_P (||grad_x f(x)|| - 1)^2
 * (Eq. 6, IGR's eikonal term of Eq. 8) with Eq. 7's adaptive weight
 *   w(x) = max(w'(f(x)), w'(d(x))),  w'(z) = 1 - |2 sigmoid(k_weight z) - 1|
 * held fixed in the gradient (k_weight <= 0: w = 1, the plain L1 loss; the
 * paper leaves k open). Add the total variation term with tg_tv_step. The points are `pts`
 * (device, N x 3) or, if pts is NULL, the fit batch of (seed, step) drawn on
 * the device. The points are binned into `batch` (created for the grid's
 * res, max_points >= N), the forward, the per-point loss and the backward run
 * in binned order, and dL/dtheta is ADDED to coef_grad (device, n_coefs).
 * loss_sums (device, 2 floats, accumulated) receives sum w |f - d| and
 * sum (||grad_x f|| - 1)^2 over the batch. sign(0) = 0; points whose spatial
 * gradient has norm below 1e-12 get no eikonal gradient.
 * The first call may grow the batch's staging buffer (11 floats per point). */
TG_API tg_status tg_sdf_step(const tg_grid *grid, tg_batch *batch, const tg_shape *shape, const float *pts,
                             int64_t N, uint64_t seed, int64_t step, float lambda_eik, float k_weight,
                             float *coef_grad, float *loss_sums, tg_stream stream);

/* Total variation term of Sec. 3.2 (the form of Plenoxels) on a 3-D grid's
 * FP32 master, over every vertex v and coefficient c of the exchange layout:
 *   n(v, c) = sqrt(D_x^2 + D_y^2 + D_z^2),  D_a = theta(v + e_a, c) - theta(v, c)
 * (D_a = 0 where v + e_a is outside the grid), L_TV = sum_{v,c} n(v, c) / res^3.
 * ADDS lambda * dL_TV/dtheta into coef_grad (device, FP32, n_coefs; a zero n
 * contributes nothing) and, if loss_sum (device, 1 float) is not NULL, adds
 * sum_{v,c} n(v, c) to it. One pass over the grid (a 3-D stencil).
 * Errors: TG_EINVAL (NULL grid or coef_grad, 2-D grid, lambda < 0), TG_EDEVICE. */
TG_API tg_status tg_tv_step(const tg_grid *grid, float lambda, float *coef_grad, float *loss_sum, tg_stream stream);

/* ---------------------------------------------------------------------------
 * Mesh extraction and the Chamfer distance (the surface metric of Sec. 4.1).
 * ------------------------------------------------------------------------ */
/* Triangulates the level set f = iso of channel 0 of a 3-D grid. The field is
 * sampled on the M^3 lattice x = (i, j, k) / (M - 1) (Eq. 2 - Eq. 4), and the
 * mesh is made by marching tetrahedra: each lattice cube is cut into the six
 * tetrahedra around its main diagonal, a lattice point is inside where its
 * value is below iso, crossings are linear on the lattice edges, and the
 * triangles face increasing f. The mesh of a level set that stays inside the
 * domain is closed. The triangles are written to tris (device, max_tris x 9
 * floats: x, y, z of the three vertices) in a fixed order: cubes with k, then
 * j, then i ascending, six tetrahedra per cube in a fixed order. Writes stop at
 * max_tris, and *n_tris (device, 1 int64) receives the full count, so a call
 * with max_tris = 0 (tris may be NULL) sizes the buffer. Allocates and frees
 * about 4 M^3 + 12 (M - 1)^2 bytes of scratch in stream order.
 * Errors: TG_EINVAL (NULL, 2-D grid, M outside [2, 2048]), TG_EDEVICE. */
TG_API tg_status tg_extract_mesh(const tg_grid *grid, int M, float iso, float *tris, int64_t max_tris,
                                 int64_t *n_tris, tg_stream stream);

/* N area-weighted points (device, N x 3) on the first min(*n_tris, max_tris)
 * triangles of tris (device, 9 floats each; n_tris a device int64, as
 * tg_extract_mesh writes it). Sample s takes u = U(3 s) times the total area
 * and the first triangle whose running area (summed in triangle order, FP64)
 * exceeds it, then r1 = U(3 s + 1), r2 = U(3 s + 2) and the point
 * (1 - sqrt r1) v0 + sqrt r1 (1 - r2) v1 + sqrt r1 r2 v2, where U is the
 * counter-based generator (seed, stream 0x4D455348). With no triangles the
 * points are 0. Errors: TG_EINVAL (NULL, negative sizes), TG_EDEVICE. */
TG_API tg_status tg_sample_mesh(const float *tris, const int64_t *n_tris, int64_t max_tris, int64_t N,
                                uint64_t seed, float *pts, tg_stream stream);

/* Adds sum_{a in A} min_{b in B} |a - b|^2 to sums[0] and
 * sum_{b in B} min_{a in A} |a - b|^2 to sums[1] (device, 2 doubles; the
 * caller zeroes them) for point sets A (device, nA x 3) and B (nB x 3); the
 * Chamfer distance is sums[0] / nA + sums[1] / nB. Exact nearest neighbours
 * (brute force, FP32 distances, FP64 sums). Errors: TG_EINVAL, TG_EDEVICE. */
TG_API tg_status tg_chamfer(const float *A, int64_t nA, const float *B, int64_t nB, double *sums,
                            tg_stream stream);

/* Accumulates sum_P |f(x) - d(x)| over N points (device, N x 3) into
 * err_sum (device, 1 float): the mean |SDF error| of a fit is err_sum / N.
 * 3-D one-channel grids. */
TG_API tg_status tg_sdf_error(const tg_grid *grid, const tg_shape *shape, const float *pts, int64_t N,
                              float *err_sum, tg_stream stream);

/* Volumetric IoU of the fitted shape (the paper's reconstruction metric,
 * measured on points instead of meshes): over N points (device, N x 3) adds
 * #{f(x) < 0 and d(x) < 0} to counts[0] and #{f(x) < 0 or d(x) < 0} to
 * counts[1] (device, 2 x uint64, accumulated); IoU = counts[0] / counts[1].
 * Uniform points in [0,1]^3 give the volume IoU. 3-D one-channel grids. */
TG_API tg_status tg_sdf_iou(const tg_grid *grid, const tg_shape *shape, const float *pts, int64_t N,
                            uint64_t *counts, tg_stream stream);

/* ---------------------------------------------------------------------------
 * Differentiable ray marching (Sec. 3.3, Eq. 9 - Eq. 11).
 * ------------------------------------------------------------------------ */

/* Renders R rays (rays_o, rays_d: device, R x 3, unit directions) through a
 * density grid (3-D, 1 channel, sigma = softplus(f), Eq. 9) and a colour grid
 * (3-D, 3 channels, c = sigmoid(f)) of the same res, with S (1..512)
 * stratified samples per ray inside the unit cube:
 *   t_i = near + (i + xi_i)(far - near)/S,  xi_i = U(seed, ray_base + r, i),
 *   delta_i = t_{i+1} - t_i (t_S = far),
 *   C(r) = sum_i T_i (1 - exp(-sigma_i delta_i)) c_i + T_S bg        (Eq. 10)
 * with T_i = exp(-sum_{j<i} sigma_j delta_j); a ray that misses the cube is
 * bg. Writes rgb_out (device, R x 3).
 * Training (target_rgb != NULL, device R x 3): adds sum_r ||C - C*||^2 into
 * loss_sum[0] (device; divide by R for the loss of Eq. 11) and ADDS the coefficient gradients of Eq. 11 into density_grad and
 * color_grad (device, FP32, each grid's n_coefs). The per-sample derivatives
 * come from the same pass; the samples are binned into `batch` (created for
 * the grids' res with max_points >= R * S) and scattered by the binned
 * backward. Both grids FP32 or both BF16; orders (2,1), (1,1), (2,0) or (0,0).
 * The first training call may grow the batch's workspace (7 floats per sample). */
TG_API tg_status tg_render_rays(const tg_grid *density, const tg_grid *color, const float *rays_o,
                                const float *rays_d, int64_t R, int S, uint64_t seed, uint64_t ray_base,
                                float bg, float *rgb_out, const float *target_rgb, tg_batch *batch,
                                float *density_grad, float *color_grad, float *loss_sum, tg_stream stream);

/* Backward of tg_render_rays for any upstream dL_drgb (device, R x 3), e.g.
 * from a loss computed outside the library. Recomputes every sample of every
 * ray - the same stratified samples as the forward for the same seed,
 * ray_base and bg, so nothing is stored between the two calls - and ADDS
 *   dL/dtheta = sum_r sum_a dL_drgb[r, a] dC_a(r)/dtheta
 * into density_grad and color_grad under the same rules as the training form
 * of tg_render_rays (batch, dtypes, orders). rgb_out may be NULL; otherwise
 * it receives the recomputed colours. */
TG_API tg_status tg_render_rays_backward(const tg_grid *density, const tg_grid *color, const float *rays_o,
                                         const float *rays_d, int64_t R, int S, uint64_t seed, uint64_t ray_base,
                                         float bg, const float *dL_drgb, tg_batch *batch, float *density_grad,
                                         float *color_grad, float *rgb_out, tg_stream stream);

/* ---------------------------------------------------------------------------
 * Fit / query server (continuous batching; no paper counterpart - the paper
 * fits one shape at a time). Fit jobs (Sec. 3.2 SDF fits) and query requests
 * arrive at any time. A tick (tg_server_step) retires finished work, admits
 * queued jobs while the sum of their device bytes stays within the budget,
 * and launches one training step of every running fit job:
 *  - running jobs that share order and storage dtype are advanced together,
 *    one launch per stage for all of them: one point-parallel kernel over the
 *    concatenation of their fit batches (sampler, f and grad f, the L1 /
 *    Eq. 7 / eikonal upstreams, the warp-aggregated coefficient gradient),
 *    one Adam launch over all their coefficients, a device-gated evaluation
 *    every eval_every steps and one thread per job for the step counter;
 *  - a job with TG_FIT_DETERMINISTIC or a TV term runs alone on its own
 *    stream as a CUDA graph captured at admission (sampler, binning, binned
 *    forward, loss, binned backward, TV, Adam, gated evaluation).
 * Step counters, errors and stop flags live in device memory; the host never
 * waits for the device inside a tick and reads progress from pinned status
 * words. A finished fit job's grid stays resident (for queries) until
 * tg_release.
 * ------------------------------------------------------------------------ */
typedef struct tg_server tg_server;
typedef int64_t tg_job_id;

typedef struct {
    int res, order;
    tg_dtype dtype;
    uint64_t seed;              /* sampler seed of the fit batches; evaluation points use seed + 1 */
    int n_spheres, n_boxes;     /* the target shape (host arrays, copied at submission) */
    const float *spheres;       /* (host) n_spheres x 4 */
    const float *boxes;         /* (host) n_boxes x 6 */
    const float *area_cdf;      /* (host) n_spheres + n_boxes */
    int64_t points_per_step;    /* fit batch size */
    int64_t eval_points;        /* evaluation points (fixed per job) */
    int eval_every;             /* evaluate the mean |SDF error| every this many steps */
    int max_steps;
    float tol;                  /* stop once the evaluated mean |SDF error| < tol */
    float lr, lambda_eik, init_std;
    float k_weight;             /* Eq. 7 adaptive weight (tg_sdf_step); <= 0: off */
    float lambda_tv;            /* total variation weight (tg_tv_step); 0: off */
    int flags;                  /* TG_FIT_DETERMINISTIC | TG_FIT_LAZY_ADAM */
} tg_fit_desc;

/* tg_fit_desc.flags. TG_FIT_DETERMINISTIC: the job trains alone on its own
 * stream with the bitwise-reproducible backward (TG_DETERMINISTIC) and an
 * evaluation summed in a fixed order, so its grid is the same bits whatever
 * else runs. TG_FIT_LAZY_ADAM: Adam as tg_adam_step_lazy (coefficients no
 * point touched keep parameter and moments). */
#define TG_FIT_DETERMINISTIC 1
#define TG_FIT_LAZY_ADAM 2

typedef enum {
    TG_JOB_QUEUED = 0,
    TG_JOB_RUNNING = 1,
    TG_JOB_DONE = 2,
    TG_JOB_FAILED = 3,
    TG_JOB_CANCELLED = 4
} tg_job_state;

typedef struct {
    int state;                  /* tg_job_state */
    int kind;                   /* 0 = fit, 1 = query */
    int64_t steps;              /* fit steps done */
    float error;                /* last evaluated mean |SDF error| (fit) */
    double t_submit, t_start, t_done;   /* seconds on the server's monotonic clock */
    int64_t points;             /* points processed (fit: steps x batch; query: N) */
    size_t bytes;               /* device bytes charged to the budget */
} tg_job_result;

/* budget_bytes: HBM admission budget; max_running: at most this many fit
 * jobs train at once (further admitted jobs wait in the queue). */
TG_API tg_status tg_server_create(size_t budget_bytes, int max_running, tg_server **out);
/* Waits for all device work of the server, then frees every job. */
TG_API tg_status tg_server_destroy(tg_server *server);

/* Enqueue a fit job. TG_EBUDGET if the job alone needs more than the budget;
 * TG_EINVAL for a bad description. The job id is returned in *id. */
TG_API tg_status tg_fit_job(tg_server *server, const tg_fit_desc *desc, tg_job_id *id);

/* Enqueue a query of N points (device, N x 3) against the grid of fit job
 * `grid_job` (queued, running or done but not released); out (device, N).
 * The query runs on the stream that trains the grid (the job's own, or its
 * group's), between two of its steps. */
TG_API tg_status tg_query_job(tg_server *server, tg_job_id grid_job, const float *pts, int64_t N, float *out,
                              tg_job_id *id);

/* One tick (see above). *pending (optional) = jobs queued or running. */
TG_API tg_status tg_server_step(tg_server *server, int *pending);

TG_API tg_status tg_poll(tg_server *server, tg_job_id id, tg_job_result *result);

/* The grid of a fit job (borrowed; valid until tg_release). */
TG_API tg_status tg_server_grid(tg_server *server, tg_job_id id, tg_grid **grid);

/* Frees a finished fit job's grid (or a finished query's record). TG_EBUSY if it is still running. */
TG_API tg_status tg_release(tg_server *server, tg_job_id id);

/* Cancels a job. A queued job leaves the queue at once. A running fit job
 * stops at its next step boundary (no kernel is interrupted): the server step
 * that sees its last step retired marks it TG_JOB_CANCELLED and frees its
 * scratch, while its grid - the fit so far - stays resident, and queries can
 * still use it, until tg_release. A query that has been launched cannot be
 * recalled (TG_EBUSY). Finished jobs are left as they are.
 * Errors: TG_EINVAL (NULL), TG_ENOTFOUND, TG_EBUSY. */
TG_API tg_status tg_cancel(tg_server *server, tg_job_id id);

/* Admission order of queued fit jobs: arrival order (default), or the job
 * with the fewest device bytes first (short jobs overtake long ones; queries
 * are always admitted first). */
#define TG_ADMIT_FIFO 0
#define TG_ADMIT_SMALLEST 1
TG_API tg_status tg_server_set_policy(tg_server *server, int policy);

/* Seconds on the server's monotonic clock (the clock of tg_job_result). */
TG_API double tg_server_time(const tg_server *server);

#ifdef __cplusplus
}
#endif

#endif /* TAYLORGRID_H */
