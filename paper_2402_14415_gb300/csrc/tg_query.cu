// C ABI of the query pair (tg_query / tg_query_backward): the point-parallel
// kernels, or, for large 3-D batches, binning into a grid-owned batch and the
// brick-binned kernels.
#include "tg_binned.cuh"
#include "tg_query.cuh"

namespace tg {

// Persistent grid size: all resident blocks of the kernel on every SM.
static unsigned persistent_blocks(const void *kernel, int threads, int64_t work_items)
{
    int64_t need = (work_items + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * blocks_per_sm(kernel, threads, 0);
    return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

template <typename T>
struct QueryLaunch {
    template <int DIM, int ORDER, int C>
    static tg_status fwd(const tg_grid *g, const float *pts, int64_t N, float *out, float *gx, cudaStream_t s)
    {
        auto k = query_fwd_kernel<T, DIM, ORDER, C>;
        unsigned nb = persistent_blocks((const void *)k, kQueryThreads, N);
        k<<<nb, kQueryThreads, 0, s>>>((const T *)g->store, g->res, pts, N, out, gx);
        return launch_status("tg_query");
    }
};

template <int DIM, int ORDER, int C>
static tg_status bwd(const tg_grid *g, const float *pts, int64_t N, const float *uf, const float *ug, float *grad,
                     cudaStream_t s)
{
    auto k = query_bwd_kernel<DIM, ORDER, C>;
    unsigned nb = persistent_blocks((const void *)k, kQueryThreads, N);
    k<<<nb, kQueryThreads, 0, s>>>(g->res, pts, N, uf, ug, grad);
    return launch_status("tg_query_backward");
}

}  // namespace tg

using namespace tg;

namespace tg {

tg_status query_point_parallel(const tg_grid *g, const float *pts, int64_t N, float *out, float *grad_x,
                               cudaStream_t s)
{
#define TG_Q(D, O, C)                                                                                          \
    (g->dtype == TG_F32    ? QueryLaunch<float>::fwd<D, O, C>(g, pts, N, out, grad_x, s)                       \
     : g->dtype == TG_BF16 ? QueryLaunch<__nv_bfloat16>::fwd<D, O, C>(g, pts, N, out, grad_x, s)               \
                           : QueryLaunch<__half>::fwd<D, O, C>(g, pts, N, out, grad_x, s))
    return TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_Q);
#undef TG_Q
}

tg_status query_backward_point_parallel(const tg_grid *g, const float *pts, int64_t N, const float *dL_df,
                                        const float *dL_dgradx, float *coef_grad, cudaStream_t s)
{
#define TG_B(D, O, C) bwd<D, O, C>(g, pts, N, dL_df, dL_dgradx, coef_grad, s)
    return TG_DISPATCH_SHAPE(g->dim, g->order, g->C, TG_B);
#undef TG_B
}

struct FwdArgs {
    float *out, *grad_x;
};
struct BwdArgs {
    const float *dL_df, *dL_dgradx;
    float *coef_grad;
};

static tg_status binned_fwd_op(const tg_grid *g, tg_batch *bt, void *a, cudaStream_t s)
{
    const FwdArgs *f = static_cast<const FwdArgs *>(a);
    return tg_query_binned(g, bt, f->out, f->grad_x, TG_ORDER_INPUT, s);
}

static tg_status binned_bwd_op(const tg_grid *g, tg_batch *bt, void *a, cudaStream_t s)
{
    const BwdArgs *b = static_cast<const BwdArgs *>(a);
    return tg_query_backward_binned(g, bt, b->dL_df, b->dL_dgradx, b->coef_grad, TG_ORDER_INPUT, s);
}

}  // namespace tg

extern "C" {

tg_status tg_query(const tg_grid *g, const float *pts, int64_t N, float *out, float *grad_x, tg_stream stream)
{
    if (!g) return fail(TG_EINVAL, "tg_query: grid is NULL");
    if (N < 0) return fail(TG_EINVAL, "tg_query: N < 0");
    if (N == 0) return TG_OK;
    if (!pts || !out) return fail(TG_EINVAL, "tg_query: NULL pts or out");
    cudaStream_t s = (cudaStream_t)stream;
    if (auto_bin_wanted(g, N, nullptr, s)) {
        FwdArgs a{out, grad_x};
        return with_auto_batch(g, pts, N, s, binned_fwd_op, &a);
    }
    return query_point_parallel(g, pts, N, out, grad_x, s);
}

tg_status tg_query_backward(const tg_grid *g, const float *pts, int64_t N, const float *dL_df,
                            const float *dL_dgradx, float *coef_grad, tg_stream stream)
{
    if (!g) return fail(TG_EINVAL, "tg_query_backward: grid is NULL");
    if (N < 0) return fail(TG_EINVAL, "tg_query_backward: N < 0");
    if (N == 0) return TG_OK;
    if (!pts || !dL_df || !coef_grad) return fail(TG_EINVAL, "tg_query_backward: NULL pts, dL_df or coef_grad");
    cudaStream_t s = (cudaStream_t)stream;
    if (auto_bin_wanted(g, N, coef_grad, s)) {
        BwdArgs a{dL_df, dL_dgradx, coef_grad};
        return with_auto_batch(g, pts, N, s, binned_bwd_op, &a);
    }
    return query_backward_point_parallel(g, pts, N, dL_df, dL_dgradx, coef_grad, s);
}

}  // extern "C"

namespace tg {

template <int DIM>
__global__ void locate_kernel(int res, const float *__restrict__ pts, int64_t N, int32_t *__restrict__ cells,
                              float *__restrict__ ts)
{
    const float scale = (float)(res - 1);
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        float x[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = pts[n * DIM + d];
        int c[DIM];
        float t[DIM];
        locate<DIM>(x, res, scale, c, t);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            cells[n * DIM + d] = c[d];
            if (ts) ts[n * DIM + d] = t[d];
        }
    }
}

}  // namespace tg

extern "C" tg_status tg_locate(int dim, int res, const float *pts, int64_t N, int32_t *cells, float *t,
                               tg_stream stream)
{
    if (dim != 2 && dim != 3) return fail(TG_EINVAL, "tg_locate: dim must be 2 or 3");
    if (res < 2) return fail(TG_EINVAL, "tg_locate: res must be >= 2");
    if (N < 0) return fail(TG_EINVAL, "tg_locate: N < 0");
    if (N == 0) return TG_OK;
    if (!pts || !cells) return fail(TG_EINVAL, "tg_locate: NULL pts or cells");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t need = (N + 255) / 256, cap = (int64_t)num_sms() * 8;
    unsigned nb = (unsigned)(need < cap ? need : cap);
    if (dim == 3) locate_kernel<3><<<nb, 256, 0, s>>>(res, pts, N, cells, t);
    else locate_kernel<2><<<nb, 256, 0, s>>>(res, pts, N, cells, t);
    return launch_status("tg_locate");
}
