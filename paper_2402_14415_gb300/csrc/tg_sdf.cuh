// Internal interface of the SDF fitting pieces (tg_sdf.cu) used by the server.
#pragma once

#include "tg_binned.cuh"

namespace tg {

struct ShapeView {
    int ns, nb;
    const float *sph, *box, *cdf;
};

tg_status shape_view(const tg_shape *s, ShapeView *v, const char *who);

// Signed distance of the union (Eq. 5): sphere |x - c| - r; box: distance to
// the box surface, negative inside; union = minimum.
__device__ __forceinline__ float sdf_union(const ShapeView &s, float x, float y, float z)
{
    float best = INFINITY;
    for (int i = 0; i < s.ns; ++i) {
        const float *q = s.sph + 4 * i;
        const float dx = x - __ldg(q), dy = y - __ldg(q + 1), dz = z - __ldg(q + 2);
        best = fminf(best, sqrtf(dx * dx + dy * dy + dz * dz) - __ldg(q + 3));
    }
    for (int i = 0; i < s.nb; ++i) {
        const float *q = s.box + 6 * i;
        const float ex = fabsf(x - __ldg(q)) - __ldg(q + 3);
        const float ey = fabsf(y - __ldg(q + 1)) - __ldg(q + 4);
        const float ez = fabsf(z - __ldg(q + 2)) - __ldg(q + 5);
        const float ox = fmaxf(ex, 0.f), oy = fmaxf(ey, 0.f), oz = fmaxf(ez, 0.f);
        const float d = sqrtf(ox * ox + oy * oy + oz * oz) + fminf(fmaxf(ex, fmaxf(ey, ez)), 0.f);
        best = fminf(best, d);
    }
    return best;
}

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }

// An area-weighted surface point of one member from the uniforms u0, u1 (position),
// u8 (member), u9 (box face).
__device__ __forceinline__ void surface_candidate(const ShapeView &s, float u0, float u1, float u8, float u9, float *p)
{
    const int nm = s.ns + s.nb;
    int prim = 0;
    for (int i = 0; i < nm; ++i) prim += (__ldg(s.cdf + i) <= u8) ? 1 : 0;   // first entry > u8
    prim = min(prim, nm - 1);
    if (prim < s.ns) {
        const float *q = s.sph + 4 * prim;
        const float z = 1.f - 2.f * u0;
        const float r = sqrtf(fmaxf(0.f, 1.f - z * z));
        const float R = __ldg(q + 3);
        p[0] = __ldg(q) + R * r * cospif(2.f * u1);
        p[1] = __ldg(q + 1) + R * r * sinpif(2.f * u1);
        p[2] = __ldg(q + 2) + R * z;
    } else {
        const float *q = s.box + 6 * (prim - s.ns);
        const float c[3] = {__ldg(q), __ldg(q + 1), __ldg(q + 2)};
        const float h[3] = {__ldg(q + 3), __ldg(q + 4), __ldg(q + 5)};
        const float fa[3] = {h[1] * h[2], h[0] * h[2], h[0] * h[1]};
        const float tot = 2.f * (fa[0] + fa[1] + fa[2]);
        float run = 0.f;
        int face = 0;
        for (int f = 0; f < 6; ++f) {
            run += fa[f / 2];
            face += (run / tot <= u9) ? 1 : 0;
        }
        face = min(face, 5);
        const int ax = face / 2, a1 = (ax + 1) % 3;
        // axis ax is the face's normal, a1 takes u0 and the third axis u1; the
        // roles are selected per component so that every array index is a constant
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float along = k == ax ? ((face % 2 == 0) ? -h[k] : h[k])
                                        : (k == a1 ? (2.f * u0 - 1.f) * h[k] : (2.f * u1 - 1.f) * h[k]);
            p[k] = c[k] + along;
        }
    }
}

// Point j of the fit batch of `step` (N points): the first half uniform in the
// cube, the rest area-weighted on the target surface (a candidate inside
// another member is redrawn, up to 8 times) plus N(0, jitter^2) noise,
// clamped to the cube. Every draw comes from the counter-based generator, so
// any thread can produce any point.
__device__ __forceinline__ void sample_sdf_point(const ShapeView &s, uint64_t seed, int64_t step, int64_t N,
                                                 int64_t j, float jitter, float *out)
{
    constexpr uint64_t SLOTS = 16;
    const int64_t n_uni = N / 2;
    const uint64_t base = (uint64_t)step * 256ull;
    const uint64_t key_u = stream_key(seed, base + 255ull);
    const uint64_t b = (uint64_t)j * SLOTS;
    float p[3] = {uniform_k(key_u, b), uniform_k(key_u, b + 1), uniform_k(key_u, b + 2)};
    if (j >= n_uni) {
        for (int a = 0; a < 8; ++a) {
            const uint64_t key = stream_key(seed, base + (uint64_t)a);
            float cand[3];
            surface_candidate(s, uniform_k(key, b), uniform_k(key, b + 1), uniform_k(key, b + 8),
                              uniform_k(key, b + 9), cand);
            if (sdf_union(s, cand[0], cand[1], cand[2]) > -1e-6f) {
                p[0] = cand[0]; p[1] = cand[1]; p[2] = cand[2];
                break;
            }
        }
        if (jitter > 0.f) {
#pragma unroll
            for (int k = 0; k < 3; ++k) p[k] += jitter * normal_k(key_u, (uint64_t)j * (SLOTS / 2) + 2 + k);
        }
    }
    out[0] = clamp01(p[0]);
    out[1] = clamp01(p[1]);
    out[2] = clamp01(p[2]);
}

// The final position of surface point j: p (the accepted candidate, or the
// uniform fallback after 8 rejected ones) plus its jitter, clamped; the same
// operations as the end of sample_sdf_point.
__device__ __forceinline__ void finish_surface_point(uint64_t key_u, int64_t j, float jitter, float *p, float *out)
{
    constexpr uint64_t SLOTS = 16;
    if (jitter > 0.f) {
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] += jitter * normal_k(key_u, (uint64_t)j * (SLOTS / 2) + 2 + k);
    }
    out[0] = clamp01(p[0]);
    out[1] = clamp01(p[1]);
    out[2] = clamp01(p[2]);
}

// Upstream gradients of one point's loss terms (Eq. 6 with Eq. 7's weight,
// and the eikonal term of Eq. 8): r = f - d, dL/df = w sign(r) / N, and
// dL/d(grad_x f) = lambda 2 (|g| - 1) g / |g| / N (0 below |g| = 1e-12).
// w = max(w'(f), w'(d)), w'(z) = 2 e / (1 + e), e = exp(-|k z|); k <= 0: w = 1.
// Returns w |r| and (|g| - 1)^2 for the loss sums.
__device__ __forceinline__ void sdf_point_upstream(float f, const float *g, float d, float lambda, float k_weight,
                                                   float inv_n, float *uf, float *ug, float *l1, float *eik)
{
    const float r = f - d;
    float w = 1.f;
    if (k_weight > 0.f) {
        const float ef = expf(-fabsf(k_weight * f)), ed = expf(-fabsf(k_weight * d));
        w = fmaxf(2.f * ef / (1.f + ef), 2.f * ed / (1.f + ed));
    }
    *l1 = w * fabsf(r);
    *uf = r > 0.f ? w * inv_n : (r < 0.f ? -w * inv_n : 0.f);
    *eik = 0.f;
    ug[0] = ug[1] = ug[2] = 0.f;
    if (g) {
        const float e = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        *eik = (e - 1.f) * (e - 1.f);
        const float c = e < 1e-12f ? 0.f : lambda * 2.f * (e - 1.f) / e * inv_n;
        ug[0] = c * g[0];
        ug[1] = c * g[1];
        ug[2] = c * g[2];
    }
}

// One SDF fitting step; with step_dev != nullptr the sampler reads the step
// index on the device (for replayable CUDA graphs).
// deterministic: the bitwise-reproducible backward (TG_DETERMINISTIC).
tg_status sdf_step_impl(const tg_grid *g, tg_batch *bt, const ShapeView &s, const float *pts, int64_t N,
                        uint64_t seed, int64_t step, const int64_t *step_dev, float lambda_eik, float k_weight,
                        float *coef_grad, float *loss_sums, cudaStream_t cs, bool deterministic);

// sum |f - d| over points into err_sum; skipped on the device when *gate == 0.
// With partials (error_blocks(N) floats) the block sums are added in a fixed order.
tg_status sdf_error_impl(const tg_grid *g, const ShapeView &s, const float *pts, int64_t N, float *err_sum,
                         const int *gate, cudaStream_t cs, unsigned long long *iou = nullptr,
                         float *partials = nullptr);
int error_blocks(int64_t N);

}  // namespace tg
