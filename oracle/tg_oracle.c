/*
 * TaylorGrid oracle: a plain, slow, obviously-correct FP64 CPU statement of the
 * TaylorGrid method (arXiv 2402.14415), written from the paper.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code, header, table or constant generator with
 * the CUDA library.
 *
 * Conventions (readings of points the paper leaves open):
 *  - Domain [0,1]^D, `res` vertices per axis, vertex j at x = j/(res-1).
 *  - Offsets x - v_i (Eq. 3) are world coordinates, delta = (t - b_i) h with
 *    h = 1 / (res - 1): the stored series are the derivatives of f with
 *    respect to x, as Eq. 1 writes them.
 *  - Corner i has offset bits b_d = (i >> d) & 1 (x fastest).
 *  - Coefficients per vertex and channel, in this order:
 *      3-D: f, g_x, g_y, g_z, H_xx, H_yy, H_zz, H_xy, H_xz, H_yz   (K = 1 / 4 / 10)
 *      2-D: f, g_x, g_y, H_xx, H_yy, H_xy                           (K = 1 / 3 / 6)
 *    H holds the true Hessian entries; the symmetric H is assembled and the
 *    quadratic form of Eq. 1 evaluated as written.
 *  - Exchange layout of a grid: [vertex][channel][k], vertex = x + res*(y + res*z).
 *  - Index rule (Eq. 2, `query`): clamp x to [0,1]; u = fl32(x * (res-1));
 *    c = min(floor(u), res-2); t = fl32(u - c). The oracle runs exactly these
 *    FP32 operations and only then promotes t to FP64.
 *
 * Parity pins live in tests/test_oracle_pins.py. Functions without an
 * independent pin say "parity unpinned" in their comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TGO_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Sizes                                                                     */
/* ------------------------------------------------------------------------ */

/* Number of Taylor coefficients of a truncated series of order `order` in D
 * variables: C(D + order, order) (the value, D first derivatives and the
 * D(D+1)/2 distinct second derivatives; Sec. 3.1, Eq. 1). */
TGO_API int tgo_num_coefs(int dim, int order)
{
    int k = 1;
    if (order >= 1) k += dim;
    if (order >= 2) k += dim * (dim + 1) / 2;
    return k;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: query(x, V_T) -> the Taylor voxel that contains x                  */
/* ------------------------------------------------------------------------ */
TGO_API void tgo_locate(int dim, int res, const float *x, int *cell, double *t)
{
    for (int d = 0; d < dim; ++d) {
        float xd = x[d];
        xd = fmaxf(xd, 0.0f);             /* NaN -> 0 (fmax drops the NaN) */
        xd = fminf(xd, 1.0f);
        volatile float scale = (float)(res - 1);
        volatile float u = xd * scale;    /* one FP32 multiply, no contraction */
        int c = (int)floorf(u);
        if (c > res - 2) c = res - 2;
        if (c < 0) c = 0;
        volatile float tf = u - (float)c; /* FP32 subtraction */
        cell[d] = c;
        t[d] = (double)tf;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 / Eq. 3: the truncated series T'(delta; S(v)) of one vertex        */
/* ------------------------------------------------------------------------ */

/* Unpack the stored coefficients into f, the gradient g and the full
 * symmetric Hessian H (zero where the order does not reach). */
static void unpack(int dim, int order, const double *th, double *f, double g[3], double H[3][3])
{
    *f = th[0];
    for (int a = 0; a < 3; ++a) { g[a] = 0; for (int b = 0; b < 3; ++b) H[a][b] = 0; }
    if (order >= 1) for (int a = 0; a < dim; ++a) g[a] = th[1 + a];
    if (order >= 2) {
        const double *h = th + 1 + dim;
        for (int a = 0; a < dim; ++a) H[a][a] = h[a];
        if (dim == 3) {
            H[0][1] = H[1][0] = h[3];
            H[0][2] = H[2][0] = h[4];
            H[1][2] = H[2][1] = h[5];
        } else {
            H[0][1] = H[1][0] = h[2];
        }
    }
}

/* T = f + g^T delta + 1/2 delta^T H delta  (Eq. 1 truncated at the order). */
static double series_value(int dim, int order, const double *th, const double *delta)
{
    double f, g[3], H[3][3];
    unpack(dim, order, th, &f, g, H);
    double lin = 0, quad = 0;
    for (int a = 0; a < dim; ++a) lin += g[a] * delta[a];
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) quad += delta[a] * H[a][b] * delta[b];
    return f + lin + 0.5 * quad;
}

/* d T / d delta = g + H delta. */
static void series_gradient(int dim, int order, const double *th, const double *delta, double *out)
{
    double f, g[3], H[3][3];
    unpack(dim, order, th, &f, g, H);
    for (int a = 0; a < dim; ++a) {
        double s = g[a];
        for (int b = 0; b < dim; ++b) s += H[a][b] * delta[b];
        out[a] = s;
    }
}

/* dT/dtheta_k at delta, i.e. T with the unit coefficient vector e_k
 * (T is linear in its coefficients). */
static void series_jacobian(int dim, int order, const double *delta, double *phi)
{
    int K = tgo_num_coefs(dim, order);
    double e[10];
    for (int k = 0; k < K; ++k) {
        memset(e, 0, sizeof e);
        e[k] = 1.0;
        phi[k] = series_value(dim, order, e, delta);
    }
}

/* d/d delta_a of dT/dtheta_k. */
static void series_jacobian_grad(int dim, int order, const double *delta, double dphi[][3])
{
    int K = tgo_num_coefs(dim, order);
    double e[10], gr[3];
    for (int k = 0; k < K; ++k) {
        memset(e, 0, sizeof e);
        e[k] = 1.0;
        series_gradient(dim, order, e, delta, gr);
        for (int a = 0; a < 3; ++a) dphi[k][a] = a < dim ? gr[a] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 4: interp(x, v_L), the multilinear blend of the 2^D corner values     */
/* ------------------------------------------------------------------------ */
static double corner_weight(int dim, int i, const double *t)
{
    double w = 1.0;
    for (int d = 0; d < dim; ++d) w *= ((i >> d) & 1) ? t[d] : 1.0 - t[d];
    return w;
}

static double corner_weight_grad(int dim, int i, const double *t, int a)
{
    double w = 1.0;
    for (int d = 0; d < dim; ++d) {
        int b = (i >> d) & 1;
        if (d == a) w *= b ? 1.0 : -1.0;
        else w *= b ? t[d] : 1.0 - t[d];
    }
    return w;
}

static int64_t vertex_index(int dim, int res, const int *cell, int i)
{
    int64_t v = 0, stride = 1;
    for (int d = 0; d < dim; ++d) { v += (int64_t)(cell[d] + ((i >> d) & 1)) * stride; stride *= res; }
    return v;
}

/* Field value and spatial gradient d f / d x (world units) of every channel
 * for a given cell and local coordinate t (Eq. 3 + Eq. 4). The blend weights
 * depend on t = x (res - 1) - cell, so d w / d x = (res - 1) d w / d t. */
TGO_API void tgo_eval_cell(int dim, int res, int order, int C, const double *coefs,
                           const int *cell, const double *t, double *f_out, double *gx_out)
{
    int K = tgo_num_coefs(dim, order);
    double h = 1.0 / (double)(res - 1);
    for (int ch = 0; ch < C; ++ch) {
        double f = 0, gx[3] = {0, 0, 0};
        for (int i = 0; i < (1 << dim); ++i) {
            double delta[3] = {0, 0, 0}, dT[3];
            for (int d = 0; d < dim; ++d) delta[d] = (t[d] - (double)((i >> d) & 1)) * h;   /* x - v_i */
            const double *th = coefs + (vertex_index(dim, res, cell, i) * C + ch) * K;
            double Ti = series_value(dim, order, th, delta);   /* Eq. 3 */
            series_gradient(dim, order, th, delta, dT);
            double w = corner_weight(dim, i, t);
            f += w * Ti;                                        /* Eq. 4 */
            for (int a = 0; a < dim; ++a) gx[a] += corner_weight_grad(dim, i, t, a) / h * Ti + w * dT[a];
        }
        f_out[ch] = f;
        if (gx_out) for (int a = 0; a < dim; ++a) gx_out[ch * dim + a] = gx[a];
    }
}

/* d^2 w_i / dt_a dt_b of the multilinear weight (zero for a = b). */
static double corner_weight_hess(int dim, int i, const double *t, int a, int b)
{
    if (a == b) return 0.0;
    double w = 1.0;
    for (int d = 0; d < dim; ++d) {
        int bit = (i >> d) & 1;
        if (d == a || d == b) w *= bit ? 1.0 : -1.0;
        else w *= bit ? t[d] : 1.0 - t[d];
    }
    return w;
}

/* Progressive resolution (Sec. 4.1 trains coarse to fine): the field of a
 * 3-D grid `src` (res_src, order_src, C channels) re-expanded as the Taylor
 * data of a grid with res_dst vertices per axis and order order_dst. At every
 * dst vertex - coordinates fl32(j / (res_dst - 1)), located in src by Eq. 2 -
 * the dst series holds the value, the gradient and (order 2) the Hessian of
 * f = sum_i w_i T_i (Eq. 4):
 *   grad f = sum_i T_i grad w_i + w_i grad T_i
 *   Hess f = sum_i T_i Hess w_i + grad w_i (grad T_i)^T + grad T_i (grad w_i)^T + w_i Hess T_i
 * with derivatives in world units (d/dx = (res_src - 1) d/dt for w). Written
 * in the exchange layout and the basis order of the stored series. */
TGO_API void tgo_resample(int res_src, int order_src, int C, const double *src, int res_dst, int order_dst,
                          double *dst)
{
    const int dim = 3;
    const int Ks = tgo_num_coefs(dim, order_src), Kd = tgo_num_coefs(dim, order_dst);
    const double h = 1.0 / (double)(res_src - 1), s = (double)(res_src - 1);
    const int64_t nd = (int64_t)res_dst * res_dst * res_dst;
    #pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < nd; ++v) {
        const int64_t j[3] = {v % res_dst, (v / res_dst) % res_dst, v / ((int64_t)res_dst * res_dst)};
        float x[3];
        for (int a = 0; a < 3; ++a) {
            volatile float num = (float)j[a], den = (float)(res_dst - 1);
            x[a] = num / den;
        }
        int cell[3];
        double t[3];
        tgo_locate(dim, res_src, x, cell, t);
        for (int ch = 0; ch < C; ++ch) {
            double f = 0, g[3] = {0, 0, 0}, H[3][3] = {{0}};
            for (int i = 0; i < 8; ++i) {
                double delta[3], dT[3], f0, g0[3], H0[3][3];
                for (int a = 0; a < 3; ++a) delta[a] = (t[a] - (double)((i >> a) & 1)) * h;
                const double *th = src + (vertex_index(dim, res_src, cell, i) * C + ch) * Ks;
                const double T = series_value(dim, order_src, th, delta);
                series_gradient(dim, order_src, th, delta, dT);
                unpack(dim, order_src, th, &f0, g0, H0);
                const double w = corner_weight(dim, i, t);
                double gw[3];
                for (int a = 0; a < 3; ++a) gw[a] = corner_weight_grad(dim, i, t, a) * s;
                f += w * T;
                for (int a = 0; a < 3; ++a) {
                    g[a] += gw[a] * T + w * dT[a];
                    for (int b = 0; b < 3; ++b)
                        H[a][b] += corner_weight_hess(dim, i, t, a, b) * s * s * T + gw[a] * dT[b] + dT[a] * gw[b] +
                                   w * H0[a][b];
                }
            }
            double *out = dst + (v * C + ch) * Kd;
            out[0] = f;
            if (order_dst >= 1) for (int a = 0; a < 3; ++a) out[1 + a] = g[a];
            if (order_dst >= 2) {
                out[4] = H[0][0]; out[5] = H[1][1]; out[6] = H[2][2];
                out[7] = H[0][1]; out[8] = H[0][2]; out[9] = H[1][2];
            }
        }
    }
}

/* Forward query of N points: values (N x C), optional world-unit spatial
 * gradients (N x C x D), optional cells (N x D) and local coordinates. */
TGO_API void tgo_query(int dim, int res, int order, int C, const double *coefs, int64_t N,
                       const float *pts, double *out, double *grad_x, int32_t *cells, double *ts)
{
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        int cell[3]; double t[3], gx[16 * 3];
        tgo_locate(dim, res, pts + n * dim, cell, t);
        tgo_eval_cell(dim, res, order, C, coefs, cell, t, out + n * C, gx);
        if (grad_x) for (int j = 0; j < C * dim; ++j) grad_x[n * C * dim + j] = gx[j];
        if (cells) for (int d = 0; d < dim; ++d) cells[n * dim + d] = cell[d];
        if (ts) for (int d = 0; d < dim; ++d) ts[n * dim + d] = t[d];
    }
}

/* Coefficient gradient (direct grid optimisation, Sec. 3.1 / Sec. 3.3):
 * the field is linear in the coefficients, so dL/dtheta = J^T dL/df with
 * J_{n,(i,k)} = w_i(t) phi_k(delta_i), plus the same for the spatial gradient
 * with d/dx of (w_i phi_k). Accumulates into coef_grad; abs_grad (optional)
 * accumulates the sum of the absolute values of the individual terms of each
 * contribution (the magnitude FP32 rounding of that sum is relative to), for
 * the scale-aware tolerance. */
TGO_API void tgo_query_backward(int dim, int res, int order, int C, int64_t N, const float *pts,
                                const double *dL_df, const double *dL_dgx,
                                double *coef_grad, double *abs_grad)
{
    int K = tgo_num_coefs(dim, order);
    double h = 1.0 / (double)(res - 1);
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        int cell[3]; double t[3];
        tgo_locate(dim, res, pts + n * dim, cell, t);
        for (int i = 0; i < (1 << dim); ++i) {
            double delta[3] = {0, 0, 0}, phi[10], dphi[10][3];
            for (int d = 0; d < dim; ++d) delta[d] = (t[d] - (double)((i >> d) & 1)) * h;
            series_jacobian(dim, order, delta, phi);
            series_jacobian_grad(dim, order, delta, dphi);
            double w = corner_weight(dim, i, t), dw[3];
            for (int a = 0; a < dim; ++a) dw[a] = corner_weight_grad(dim, i, t, a) / h;   /* d w / d x */
            int64_t v = vertex_index(dim, res, cell, i);
            for (int ch = 0; ch < C; ++ch) {
                for (int k = 0; k < K; ++k) {
                    double c = w * phi[k] * dL_df[n * C + ch];
                    double mag = fabs(c);   /* sum of |terms|: the scale FP32 rounding acts on */
                    if (dL_dgx)
                        for (int a = 0; a < dim; ++a) {
                            double ga = dL_dgx[(n * C + ch) * dim + a];
                            c += ga * (dw[a] * phi[k] + w * dphi[k][a]);
                            mag += fabs(ga) * (fabs(dw[a] * phi[k]) + fabs(w * dphi[k][a]));
                        }
                    int64_t j = (v * C + ch) * K + k;
                    #pragma omp atomic
                    coef_grad[j] += c;
                    if (abs_grad) {
                        double a = mag;
                        #pragma omp atomic
                        abs_grad[j] += a;
                    }
                }
            }
        }
    }
}

/* Per-point scale of the forward value for the tolerance: sum_i w_i sum_k |theta phi_k|. */
TGO_API void tgo_query_absscale(int dim, int res, int order, int C, const double *coefs, int64_t N,
                                const float *pts, double *scale)
{
    int K = tgo_num_coefs(dim, order);
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        int cell[3]; double t[3];
        tgo_locate(dim, res, pts + n * dim, cell, t);
        for (int ch = 0; ch < C; ++ch) {
            double s = 0;
            for (int i = 0; i < (1 << dim); ++i) {
                double delta[3] = {0, 0, 0}, phi[10];
                for (int d = 0; d < dim; ++d) delta[d] = (t[d] - (double)((i >> d) & 1)) / (double)(res - 1);
                series_jacobian(dim, order, delta, phi);
                const double *th = coefs + (vertex_index(dim, res, cell, i) * C + ch) * K;
                double w = corner_weight(dim, i, t);
                for (int k = 0; k < K; ++k) s += w * fabs(th[k] * phi[k]);
            }
            scale[n * C + ch] = s;
        }
    }
}

/* Per-point, per-axis scale of the world-unit spatial gradient for the
 * tolerance: d f / d x_a = sum_i (d w_i / d x_a) T_i + w_i d T_i / d x_a
 * (Eq. 3 and Eq. 4 differentiated), so the magnitude of the terms its FP32
 * sum cancels is
 *   sum_i |d w_i / d x_a| sum_k |theta_k phi_k| + w_i sum_k |theta_k d phi_k / d delta_a|
 * with d w / d x = (res - 1) d w / d t and delta = x - v_i in world units. */
TGO_API void tgo_query_gradscale(int dim, int res, int order, int C, const double *coefs, int64_t N,
                                 const float *pts, double *scale)
{
    int K = tgo_num_coefs(dim, order);
    double h = 1.0 / (double)(res - 1);
    #pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        int cell[3]; double t[3];
        tgo_locate(dim, res, pts + n * dim, cell, t);
        for (int ch = 0; ch < C; ++ch) {
            double s[3] = {0, 0, 0};
            for (int i = 0; i < (1 << dim); ++i) {
                double delta[3] = {0, 0, 0}, phi[10], dphi[10][3];
                for (int d = 0; d < dim; ++d) delta[d] = (t[d] - (double)((i >> d) & 1)) * h;
                series_jacobian(dim, order, delta, phi);
                series_jacobian_grad(dim, order, delta, dphi);
                const double *th = coefs + (vertex_index(dim, res, cell, i) * C + ch) * K;
                double w = corner_weight(dim, i, t), tsum = 0;
                for (int k = 0; k < K; ++k) tsum += fabs(th[k] * phi[k]);
                for (int a = 0; a < dim; ++a) {
                    double dsum = 0;
                    for (int k = 0; k < K; ++k) dsum += fabs(th[k] * dphi[k][a]);
                    s[a] += fabs(corner_weight_grad(dim, i, t, a) / h) * tsum + w * dsum;
                }
            }
            for (int a = 0; a < dim; ++a) scale[(n * C + ch) * dim + a] = s[a];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Optimiser. The paper fixes only the learning rate (Sec. 4.1); the build   */
/* uses Adam (Kingma & Ba 2015, Algorithm 1) with bias correction, step >= 1. */
/* With bf16_moments, the step uses the new m and v as computed, and stores  */
/* them rounded to BF16 for the next step (the moment storage of the BF16 /   */
/* FP16 storage form); the rounding is pinned to torch's conversion.         */
/* ------------------------------------------------------------------------ */
/* Rounding to BF16 (8-bit significand, the exponent range of FP32), ties to
 * even: the storage of Adam's moments in the BF16 / FP16 storage form. Below
 * the smallest normal 2^-126 the spacing is 2^-133 (BF16 subnormals). */
TGO_API double tgo_bf16_round(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    if (fabs(x) < ldexp(1.0, -126)) return nearbyint(ldexp(x, 133)) * ldexp(1.0, -133);
    int e;
    const double f = frexp(x, &e);               /* x = f 2^e, 0.5 <= |f| < 1 */
    return ldexp(nearbyint(ldexp(f, 8)), e - 8);  /* default rounding mode: nearest, ties to even */
}

TGO_API void tgo_adam(int64_t n, double *p, double *g, double *m, double *v,
                      double lr, double beta1, double beta2, double eps, int64_t step, int bf16_moments)
{
    double bc1 = 1.0 - pow(beta1, (double)step);
    double bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t j = 0; j < n; ++j) {
        m[j] = beta1 * m[j] + (1.0 - beta1) * g[j];
        v[j] = beta2 * v[j] + (1.0 - beta2) * g[j] * g[j];
        double mhat = m[j] / bc1;
        double vhat = v[j] / bc2;
        p[j] -= lr * mhat / (sqrt(vhat) + eps);
        if (bf16_moments) { m[j] = tgo_bf16_round(m[j]); v[j] = tgo_bf16_round(v[j]); }   /* stored for the next step */
        g[j] = 0.0;
    }
}

/* Lazy (sparse) Adam: the update above applied only to the entries whose
 * gradient is nonzero; the others keep their parameter and both moments (no
 * decay). The bias corrections use the global step. */
TGO_API void tgo_adam_lazy(int64_t n, double *p, double *g, double *m, double *v,
                           double lr, double beta1, double beta2, double eps, int64_t step, int bf16_moments)
{
    double bc1 = 1.0 - pow(beta1, (double)step);
    double bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t j = 0; j < n; ++j) {
        if (g[j] == 0.0) continue;
        m[j] = beta1 * m[j] + (1.0 - beta1) * g[j];
        v[j] = beta2 * v[j] + (1.0 - beta2) * g[j] * g[j];
        p[j] -= lr * (m[j] / bc1) / (sqrt(v[j] / bc2) + eps);
        if (bf16_moments) { m[j] = tgo_bf16_round(m[j]); v[j] = tgo_bf16_round(v[j]); }
        g[j] = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* SDF targets (Sec. 3.2, Eq. 5): analytic signed distances                  */
/* ------------------------------------------------------------------------ */

/* sphere (cx,cy,cz,r): |x - c| - r;  box (cx,cy,cz,hx,hy,hz): distance to the
 * box surface, negative inside; the union is the minimum of the members. */
TGO_API double tgo_sdf_union(int ns, const float *sph, int nb, const float *box, const double *x)
{
    double best = INFINITY;
    for (int s = 0; s < ns; ++s) {
        const float *q = sph + 4 * s;
        double dx = x[0] - q[0], dy = x[1] - q[1], dz = x[2] - q[2];
        double d = sqrt(dx * dx + dy * dy + dz * dz) - q[3];
        if (d < best) best = d;
    }
    for (int b = 0; b < nb; ++b) {
        const float *q = box + 6 * b;
        double e[3], outside = 0, inside = -INFINITY;
        for (int a = 0; a < 3; ++a) {
            e[a] = fabs(x[a] - q[a]) - q[3 + a];
            if (e[a] > 0) outside += e[a] * e[a];
            if (e[a] > inside) inside = e[a];
        }
        double d = sqrt(outside) + (inside < 0 ? inside : 0.0);
        if (d < best) best = d;
    }
    return best;
}

/* The adaptive weight of Eq. 7: w'(z) = 1 - |2 sigmoid(k z) - 1|, which is 1
 * at z = 0 and falls towards 0 away from the surface; k <= 0 turns the
 * weighting off (w' = 1). */
TGO_API double tgo_adaptive_weight1(double k, double z)
{
    if (!(k > 0.0)) return 1.0;
    return 1.0 - fabs(2.0 / (1.0 + exp(-k * z)) - 1.0);
}

/* One SDF fitting step on given points (Sec. 3.2):
 *   L = mean_P w(x) |f(x) - d(x)|                   (Eq. 6; w of Eq. 7)
 *     + lambda_eik * mean_P (||grad_x f(x)|| - 1)^2  (IGR eikonal term, Eq. 8)
 * with w(x) = max(w'(f(x)), w'(d(x))) and d evaluated at the clamped point.
 * w only weights the residual: it is held fixed in the gradient (a weight
 * that followed f would reward pushing f away from the surface). With k <= 0,
 * w = 1 and the first term is the plain L1 loss. The gradient of L with
 * respect to the coefficients is accumulated into coef_grad. loss[0] = the
 * weighted reconstruction term, loss[1] = eikonal mean (unweighted),
 * loss[2] = mean |f - d|. sign(0) = 0; a zero spatial gradient
 * (norm < 1e-12) gets zero eikonal gradient. */
TGO_API void tgo_sdf_step(int res, int order, const double *coefs, int64_t N, const float *pts,
                          int ns, const float *sph, int nb, const float *box,
                          double lambda_eik, double k_weight, double *coef_grad, double *loss)
{
    const int dim = 3;
    double *f = (double *)malloc(sizeof(double) * N);
    double *gx = (double *)malloc(sizeof(double) * N * 3);
    double *dLdf = (double *)malloc(sizeof(double) * N);
    double *dLdg = (double *)malloc(sizeof(double) * N * 3);
    tgo_query(dim, res, order, 1, coefs, N, pts, f, gx, NULL, NULL);
    double rec = 0, l1 = 0, eik = 0;
    for (int64_t n = 0; n < N; ++n) {
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = fmin(fmax((double)pts[n * 3 + a], 0.0), 1.0);
        double d = tgo_sdf_union(ns, sph, nb, box, x);
        double r = f[n] - d;
        double w = fmax(tgo_adaptive_weight1(k_weight, f[n]), tgo_adaptive_weight1(k_weight, d));
        rec += w * fabs(r);
        l1 += fabs(r);
        dLdf[n] = w * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)N;
        double nrm = sqrt(gx[3 * n] * gx[3 * n] + gx[3 * n + 1] * gx[3 * n + 1] + gx[3 * n + 2] * gx[3 * n + 2]);
        eik += (nrm - 1.0) * (nrm - 1.0);
        for (int a = 0; a < 3; ++a)
            dLdg[3 * n + a] = nrm < 1e-12 ? 0.0 : lambda_eik * 2.0 * (nrm - 1.0) * gx[3 * n + a] / nrm / (double)N;
    }
    tgo_query_backward(dim, res, order, 1, N, pts, dLdf, lambda_eik != 0.0 ? dLdg : NULL, coef_grad, NULL);
    if (loss) { loss[0] = rec / (double)N; loss[1] = eik / (double)N; loss[2] = l1 / (double)N; }
    free(f); free(gx); free(dLdf); free(dLdg);
}

/* Total variation term of Sec. 3.2, in the form of Plenoxels, over a 3-D grid
 * of res^3 vertices with nv coefficients each (layout [vertex][nv]): for every
 * vertex v and coefficient c,
 *   n(v, c) = sqrt(D_x^2 + D_y^2 + D_z^2),  D_a = theta(v + e_a, c) - theta(v, c)
 * (D_a = 0 where v + e_a lies outside the grid), and
 *   L_TV = (1 / res^3) sum_{v, c} n(v, c).
 * Adds lambda * dL_TV/dtheta into coef_grad (when not NULL) and returns L_TV.
 * Where n = 0 the term contributes no gradient. */
TGO_API double tgo_tv(int res, int nv, const double *coefs, double lambda, double *coef_grad)
{
    const int64_t V = (int64_t)res * res * res;
    const double inv_v = 1.0 / (double)V;
    double total = 0.0;
    for (int64_t z = 0; z < res; ++z)
        for (int64_t y = 0; y < res; ++y)
            for (int64_t x = 0; x < res; ++x) {
                const int64_t v = x + res * (y + res * z);
                const int64_t nbr[3] = {x + 1 < res ? v + 1 : -1, y + 1 < res ? v + res : -1,
                                        z + 1 < res ? v + (int64_t)res * res : -1};
                for (int c = 0; c < nv; ++c) {
                    const double t0 = coefs[v * nv + c];
                    double D[3], n2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        D[a] = nbr[a] >= 0 ? coefs[nbr[a] * nv + c] - t0 : 0.0;
                        n2 += D[a] * D[a];
                    }
                    const double n = sqrt(n2);
                    total += n;
                    if (!coef_grad || n == 0.0) continue;
                    const double s = lambda * inv_v / n;       /* d n / d D_a = D_a / n */
                    for (int a = 0; a < 3; ++a) {
                        if (nbr[a] < 0) continue;
                        coef_grad[nbr[a] * nv + c] += s * D[a];
                        coef_grad[v * nv + c] -= s * D[a];
                    }
                }
            }
    return total * inv_v;
}

/* ------------------------------------------------------------------------ */
/* Counter-based generator (splitmix64, Steele/Lea/Flood 2014)               */
/* ------------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

TGO_API double tgo_uniform(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t k = mix64(mix64(mix64(seed) + stream) + idx);
    return (double)(k >> 40) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* Mesh extraction: marching tetrahedra over a lattice of field values       */
/* ------------------------------------------------------------------------ */
/* Every lattice cube (corner q at offset (q & 1, q >> 1 & 1, q >> 2)) is cut
 * into the six tetrahedra that share its main diagonal 0 - 7, one per order
 * in which a monotone path from corner 0 to corner 7 visits the axes, so
 * neighbouring cubes cut their common faces alike and the surface closes. */
static const int kTets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

/* The iso crossing on the lattice edge a - b, taken from its lower-indexed end
 * so that every tetrahedron sharing the edge gets the same point. */
static void mt_cross(int M, const int *a, const int *b, double fa, double fb, double iso, double *p)
{
    const int64_t ia = a[0] + (int64_t)M * (a[1] + (int64_t)M * a[2]);
    const int64_t ib = b[0] + (int64_t)M * (b[1] + (int64_t)M * b[2]);
    if (ia > ib) {
        const int *tc = a; a = b; b = tc;
        double tf = fa; fa = fb; fb = tf;
    }
    const double t = (iso - fa) / (fb - fa);
    for (int d = 0; d < 3; ++d) p[d] = (a[d] + t * (b[d] - a[d])) / (double)(M - 1);
}

/* Writes triangle (a, b, c), or (a, c, b) if its normal points against dir. */
static void mt_emit(double *tris, int64_t *n, int64_t max, const double *a, const double *b, const double *c,
                    const double *dir)
{
    double u[3], v[3];
    for (int d = 0; d < 3; ++d) { u[d] = b[d] - a[d]; v[d] = c[d] - a[d]; }
    const double nx = u[1] * v[2] - u[2] * v[1], ny = u[2] * v[0] - u[0] * v[2], nz = u[0] * v[1] - u[1] * v[0];
    const int flip = nx * dir[0] + ny * dir[1] + nz * dir[2] < 0.0;
    if (*n < max) {
        double *o = tris + 9 * *n;
        for (int d = 0; d < 3; ++d) {
            o[d] = a[d];
            o[3 + d] = flip ? c[d] : b[d];
            o[6 + d] = flip ? b[d] : c[d];
        }
    }
    ++*n;
}

/* Marching tetrahedra over the M^3 lattice vals[i + M (j + M k)] at
 * x = (i, j, k) / (M - 1): a lattice point is inside where its value, rounded
 * to FP32, is below iso (rounded likewise). Triangles are oriented toward
 * increasing values and written (9 doubles each, up to max_tris) in cube order
 * (k, then j, then i), the six tetrahedra in the order of kTets, a quad as the
 * two triangles (q0 q1 q2) (q0 q2 q3). Returns the number of triangles. */
TGO_API int64_t tgo_marching_tets(int M, const double *vals, double iso, double *tris, int64_t max_tris)
{
    int64_t n = 0;
    const float iso32 = (float)iso;
    for (int k = 0; k + 1 < M; ++k)
        for (int j = 0; j + 1 < M; ++j)
            for (int i = 0; i + 1 < M; ++i) {
                int cc[8][3];
                double f[8];
                for (int q = 0; q < 8; ++q) {
                    cc[q][0] = i + (q & 1); cc[q][1] = j + ((q >> 1) & 1); cc[q][2] = k + (q >> 2);
                    f[q] = (double)(float)vals[cc[q][0] + (int64_t)M * (cc[q][1] + (int64_t)M * cc[q][2])];
                }
                for (int tt = 0; tt < 6; ++tt) {
                    const int *tv = kTets[tt];
                    int in[4], nin = 0;
                    for (int a = 0; a < 4; ++a) { in[a] = (float)f[tv[a]] < iso32; nin += in[a]; }
                    if (nin == 0 || nin == 4) continue;
                    double pos[4][3];
                    for (int a = 0; a < 4; ++a)
                        for (int d = 0; d < 3; ++d) pos[a][d] = cc[tv[a]][d] / (double)(M - 1);
                    if (nin == 1 || nin == 3) {
                        int o = 0;                        /* the vertex on its own side */
                        for (int a = 0; a < 4; ++a)
                            if (in[a] == (nin == 1)) o = a;
                        double e[3][3], cen[3] = {0, 0, 0}, dir[3];
                        int m = 0;
                        for (int a = 0; a < 4; ++a) {
                            if (a == o) continue;
                            mt_cross(M, cc[tv[o]], cc[tv[a]], f[tv[o]], f[tv[a]], iso32, e[m]);
                            for (int d = 0; d < 3; ++d) cen[d] += e[m][d] / 3.0;
                            ++m;
                        }
                        for (int d = 0; d < 3; ++d) dir[d] = nin == 1 ? cen[d] - pos[o][d] : pos[o][d] - cen[d];
                        mt_emit(tris, &n, max_tris, e[0], e[1], e[2], dir);
                    } else {
                        int ii[2], oo[2], a_i = 0, a_o = 0;
                        for (int a = 0; a < 4; ++a) {
                            if (in[a]) ii[a_i++] = a;
                            else oo[a_o++] = a;
                        }
                        double q[4][3], dir[3];
                        const int pa[4][2] = {{ii[0], oo[0]}, {ii[0], oo[1]}, {ii[1], oo[1]}, {ii[1], oo[0]}};
                        for (int r = 0; r < 4; ++r)
                            mt_cross(M, cc[tv[pa[r][0]]], cc[tv[pa[r][1]]], f[tv[pa[r][0]]], f[tv[pa[r][1]]], iso32, q[r]);
                        for (int d = 0; d < 3; ++d)
                            dir[d] = 0.5 * (pos[oo[0]][d] + pos[oo[1]][d]) - 0.5 * (pos[ii[0]][d] + pos[ii[1]][d]);
                        /* both halves take the orientation of (q0 q1 q2); reversing it swaps q1 and q3 */
                        double u[3], v[3];
                        for (int d = 0; d < 3; ++d) { u[d] = q[1][d] - q[0][d]; v[d] = q[2][d] - q[0][d]; }
                        const double nx = u[1] * v[2] - u[2] * v[1], ny = u[2] * v[0] - u[0] * v[2],
                                     nz = u[0] * v[1] - u[1] * v[0];
                        if (nx * dir[0] + ny * dir[1] + nz * dir[2] < 0.0) {
                            double t3[3];
                            for (int d = 0; d < 3; ++d) { t3[d] = q[1][d]; q[1][d] = q[3][d]; q[3][d] = t3[d]; }
                        }
                        if (n < max_tris) {
                            double *o = tris + 9 * n;
                            for (int d = 0; d < 3; ++d) { o[d] = q[0][d]; o[3 + d] = q[1][d]; o[6 + d] = q[2][d]; }
                        }
                        ++n;
                        if (n < max_tris) {
                            double *o = tris + 9 * n;
                            for (int d = 0; d < 3; ++d) { o[d] = q[0][d]; o[3 + d] = q[2][d]; o[6 + d] = q[3][d]; }
                        }
                        ++n;
                    }
                }
            }
    return n;
}

/* Area-weighted points on a triangle soup (T x 9 floats): sample s takes
 * u = U(seed, stream, 3 s) times the total area and the first triangle whose
 * inclusive running area (summed in triangle order, FP64) exceeds it, then
 * r1 = U(.., 3 s + 1), r2 = U(.., 3 s + 2) and the point
 * (1 - sqrt r1) v0 + sqrt r1 (1 - r2) v1 + sqrt r1 r2 v2. */
TGO_API void tgo_sample_mesh(int64_t T, const float *tris, int64_t N, uint64_t seed, uint64_t stream, double *out)
{
    double *cum = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
    double run = 0.0;
    for (int64_t j = 0; j < T; ++j) {
        const float *t = tris + 9 * j;
        double u[3], v[3];
        for (int d = 0; d < 3; ++d) { u[d] = (double)t[3 + d] - t[d]; v[d] = (double)t[6 + d] - t[d]; }
        const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
        run += 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        cum[j] = run;
    }
    const uint64_t key = mix64(mix64(seed) + stream);
    for (int64_t s = 0; s < N; ++s) {
        const double u0 = (double)(mix64(key + 3 * (uint64_t)s) >> 40) * (1.0 / 16777216.0);
        const double r1 = (double)(mix64(key + 3 * (uint64_t)s + 1) >> 40) * (1.0 / 16777216.0);
        const double r2 = (double)(mix64(key + 3 * (uint64_t)s + 2) >> 40) * (1.0 / 16777216.0);
        const double target = u0 * run;
        int64_t lo = 0, hi = T - 1;              /* first j with cum[j] > target */
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (cum[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        const float *t = tris + 9 * lo;
        const double sr = sqrt(r1), a = 1.0 - sr, b = sr * (1.0 - r2), c = sr * r2;
        for (int d = 0; d < 3; ++d) out[3 * s + d] = a * t[d] + b * t[3 + d] + c * t[6 + d];
    }
    free(cum);
}

/* ------------------------------------------------------------------------ */
/* Volume rendering (Sec. 3.3, Eq. 9 - Eq. 11)                                */
/* ------------------------------------------------------------------------ */
static double softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }
static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Ray / unit-cube slab intersection. Returns 1 and [near, far] on a hit. */
TGO_API int tgo_ray_box(const double *o, const double *d, double *near_, double *far_)
{
    double tn = 0.0, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > 1.0) return 0;
            continue;
        }
        double t0 = (0.0 - o[a]) / d[a], t1 = (1.0 - o[a]) / d[a];
        if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
    }
    if (!(tf > tn)) return 0;
    *near_ = tn; *far_ = tf;
    return 1;
}

/* Sample positions of a ray, by a normative FP32 rule (as the index rule of
 * Eq. 2 is), so that both sides evaluate the same points: the slab test in
 * FP32 (IEEE division), step = fl32(fl32(far - near) / S),
 * t_i = fl32(near + fl32(fl32(i + xi_i) * step)), x = fma(t_i, d, o) rounded
 * once to FP32, and delta_i = fl32(t_{i+1} - t_i) with t_S = far. Returns 0
 * for a ray that misses the cube. */
static int ray_samples_f32(const float *o, const float *d, int S, uint64_t seed, uint64_t stream, float *xs,
                           double *del)
{
    float tn = 0.0f, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < 0.0f || o[a] > 1.0f) return 0;
            continue;
        }
        volatile float t0 = (0.0f - o[a]) / d[a], t1 = (1.0f - o[a]) / d[a];
        float lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
        if (lo > tn) tn = lo;
        if (hi < tf) tf = hi;
    }
    if (!(tf > tn)) return 0;
    volatile float span = tf - tn;
    volatile float step = span / (float)S;
    float tprev = 0.0f;
    for (int i = 0; i <= S; ++i) {
        float ti = tf;
        if (i < S) {
            volatile float k = (float)i + (float)tgo_uniform(seed, stream, (uint64_t)i);
            volatile float off = k * step;
            volatile float tt = tn + off;
            ti = tt;
            for (int a = 0; a < 3; ++a) xs[3 * i + a] = fmaf(ti, d[a], o[a]);
        }
        if (i > 0) {
            volatile float dl = ti - tprev;
            del[i - 1] = (double)dl;
        }
        tprev = ti;
    }
    return 1;
}

/* Render R rays through a density grid (order od, 1 channel, sigma =
 * softplus(f), Eq. 9) and a colour grid (order oc, 3 channels, c =
 * sigmoid(f)), both res^3, with S stratified samples per ray at the
 * positions of ray_samples_f32 (xi_i = U(seed, ray_base + r, i)):
 *   C = sum_i T_i (1 - exp(-sigma_i delta_i)) c_i + T_S * bg           (Eq. 10)
 * A ray that misses the cube renders bg. If `target` is given, the loss
 * (1/R) sum_r ||C_r - target_r||^2 (Eq. 11) is returned in *loss and its
 * gradient is accumulated into dgrad / cgrad (coefficient gradients of the
 * two grids). The per-sample derivatives are taken term by term from Eq. 10:
 *   dC/dc_i     = T_i alpha_i
 *   dC/dsigma_i = delta_i T_{i+1} c_i - delta_i (sum_{j>i} T_j alpha_j c_j + T_S bg)
 * dabs / cabs (optional) accumulate, per coefficient, the magnitude of the
 * terms of its gradient that FP32 rounding acts on: every difference above
 * (C - target, and the two parts of dC/dsigma_i) taken with both parts
 * positive, times |w_i phi_k| of the query's Jacobian. */
TGO_API void tgo_render(int res, int od, const double *dcoef, int oc, const double *ccoef,
                        int64_t R, int S, const float *rays_o, const float *rays_d,
                        uint64_t seed, uint64_t ray_base, double bg, double *rgb_out,
                        const float *target, double *dgrad, double *cgrad, double *loss,
                        double *dabs, double *cabs)
{
    double total = 0.0;
    double *sig = (double *)malloc(sizeof(double) * S);
    double *fs = (double *)malloc(sizeof(double) * S);
    double *col = (double *)malloc(sizeof(double) * S * 3);
    double *del = (double *)malloc(sizeof(double) * S);
    double *Tr = (double *)malloc(sizeof(double) * (S + 1));
    double *rest = (double *)malloc(sizeof(double) * (S + 1) * 3);
    float *xs = (float *)malloc(sizeof(float) * S * 3);
    const int64_t nd = (int64_t)res * res * res * tgo_num_coefs(3, od), nc = (int64_t)res * res * res * 3 * tgo_num_coefs(3, oc);
    double *scratch = (dabs || cabs) ? (double *)calloc((size_t)(nd > nc ? nd : nc), sizeof(double)) : NULL;
    for (int64_t r = 0; r < R; ++r) {
        double C[3] = {bg, bg, bg};
        int hit = ray_samples_f32(rays_o + 3 * r, rays_d + 3 * r, S, seed, ray_base + (uint64_t)r, xs, del);
        if (hit) {
            double fc[3];
            for (int i = 0; i < S; ++i) {
                double fd;
                int cell[3]; double t[3];
                tgo_locate(3, res, xs + 3 * i, cell, t);
                tgo_eval_cell(3, res, od, 1, dcoef, cell, t, &fd, NULL);
                tgo_eval_cell(3, res, oc, 3, ccoef, cell, t, fc, NULL);
                fs[i] = fd;
                sig[i] = softplus(fd);
                for (int a = 0; a < 3; ++a) col[3 * i + a] = sigmoid(fc[a]);
            }
            /* Eq. 10: T_i = exp(-sum_{j<i} sigma_j delta_j) */
            for (int i = 0; i <= S; ++i) {
                double acc = 0;
                for (int j = 0; j < i; ++j) acc += sig[j] * del[j];
                Tr[i] = exp(-acc);
            }
            for (int a = 0; a < 3; ++a) {
                double c = 0;
                for (int i = 0; i < S; ++i) c += Tr[i] * (1.0 - exp(-sig[i] * del[i])) * col[3 * i + a];
                C[a] = c + Tr[S] * bg;
            }
            if (target) {
                double g[3], gs[3];
                for (int a = 0; a < 3; ++a) {
                    g[a] = 2.0 * (C[a] - (double)target[3 * r + a]) / (double)R;
                    gs[a] = 2.0 * (fabs(C[a]) + fabs((double)target[3 * r + a])) / (double)R;
                }
                for (int a = 0; a < 3; ++a) {      /* rest_i = sum_{j>i} T_j alpha_j c_j + T_S bg */
                    rest[3 * S + a] = Tr[S] * bg;
                    for (int i = S - 1; i >= 0; --i)
                        rest[3 * i + a] = rest[3 * (i + 1) + a] + Tr[i] * (1.0 - exp(-sig[i] * del[i])) * col[3 * i + a];
                }
                for (int i = 0; i < S; ++i) {
                    double alpha = 1.0 - exp(-sig[i] * del[i]);
                    double dsig = 0, dsig_s = 0, dcol[3], dcol_s[3];
                    for (int a = 0; a < 3; ++a) {
                        const double behind = rest[3 * (i + 1) + a];
                        dsig += g[a] * (del[i] * Tr[i + 1] * col[3 * i + a] - del[i] * behind);
                        dsig_s += gs[a] * del[i] * (Tr[i + 1] * col[3 * i + a] + behind);
                        dcol[a] = g[a] * Tr[i] * alpha;
                        dcol_s[a] = gs[a] * Tr[i] * alpha;
                    }
                    /* chain through sigma = softplus(f) and c = sigmoid(f) into Eq. 3/4 */
                    double dfd = dsig * sigmoid(fs[i]), dfd_s = dsig_s * sigmoid(fs[i]);
                    double dfc[3], dfc_s[3];
                    for (int a = 0; a < 3; ++a) {
                        dfc[a] = dcol[a] * col[3 * i + a] * (1.0 - col[3 * i + a]);
                        dfc_s[a] = dcol_s[a] * col[3 * i + a] * (1.0 - col[3 * i + a]);
                    }
                    tgo_query_backward(3, res, od, 1, 1, xs + 3 * i, &dfd, NULL, dgrad, NULL);
                    tgo_query_backward(3, res, oc, 3, 1, xs + 3 * i, dfc, NULL, cgrad, NULL);
                    if (dabs) tgo_query_backward(3, res, od, 1, 1, xs + 3 * i, &dfd_s, NULL, scratch, dabs);
                    if (cabs) tgo_query_backward(3, res, oc, 3, 1, xs + 3 * i, dfc_s, NULL, scratch, cabs);
                }
            }
        }
        for (int a = 0; a < 3; ++a) rgb_out[3 * r + a] = C[a];
        if (target)
            for (int a = 0; a < 3; ++a) total += (C[a] - (double)target[3 * r + a]) * (C[a] - (double)target[3 * r + a]);
    }
    if (loss) *loss = total / (double)R;
    free(sig); free(fs); free(col); free(del); free(Tr); free(rest); free(xs); free(scratch);
}

/* Ground truth of the synthetic radiance scene (stand-in for Synthetic-NeRF,
 * Sec. 4.2): B anisotropic Gaussian blobs, density
 *   sigma(x) = sum_k a_k exp(-1/2 (x - mu_k)^T P_k (x - mu_k))   (P_k = inverse covariance)
 * and colour the density-weighted mean of the blobs' rgb, rendered with Eq. 10
 * by midpoint quadrature with n samples over the ray's [near, far] in the unit
 * cube (T_i = exp(-sum_{j<i} sigma_j delta)); a miss renders bg. */
TGO_API void tgo_render_blobs(int B, const double *mu, const double *icov, const double *amp, const double *rgb,
                              int64_t R, const float *rays_o, const float *rays_d, int n, double bg, double *out)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < R; ++r) {
        double o[3], d[3], nr, fr;
        for (int a = 0; a < 3; ++a) { o[a] = rays_o[3 * r + a]; d[a] = rays_d[3 * r + a]; }
        double C[3] = {bg, bg, bg};
        if (tgo_ray_box(o, d, &nr, &fr)) {
            double dt = (fr - nr) / (double)n, depth = 0.0, acc[3] = {0, 0, 0};
            for (int i = 0; i < n; ++i) {
                double t = nr + ((double)i + 0.5) * dt, x[3];
                for (int a = 0; a < 3; ++a) x[a] = o[a] + t * d[a];
                double sig = 0.0, col[3] = {0, 0, 0};
                for (int k = 0; k < B; ++k) {
                    double e[3], q = 0.0;
                    for (int a = 0; a < 3; ++a) e[a] = x[a] - mu[3 * k + a];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) q += e[a] * icov[9 * k + 3 * a + b] * e[b];
                    double s = amp[k] * exp(-0.5 * q);
                    sig += s;
                    for (int a = 0; a < 3; ++a) col[a] += s * rgb[3 * k + a];
                }
                double T = exp(-depth), alpha = 1.0 - exp(-sig * dt);
                for (int a = 0; a < 3; ++a) acc[a] += T * alpha * (sig > 0 ? col[a] / sig : 0.0);
                depth += sig * dt;
            }
            for (int a = 0; a < 3; ++a) C[a] = acc[a] + exp(-depth) * bg;
        }
        for (int a = 0; a < 3; ++a) out[3 * r + a] = C[a];
    }
}
