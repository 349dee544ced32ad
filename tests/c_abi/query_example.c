/* A C caller of the TaylorGrid C ABI: no Python, no torch.
 *
 *   query_example host   argument checks only (no device call is made)
 *   query_example gpu    a 16^3 order-2 grid: query 4099 points, accumulate the
 *                        coefficient gradient of sum f, one Adam step; prints
 *                        the sum of f, of the gradient and of the updated
 *                        coefficients (%.17e) for comparison with other callers.
 *
 * Points come from a fixed 32-bit linear congruential sequence so that every
 * caller can reproduce them. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "taylorgrid.h"

#define CHECK(call)                                                                               \
    do {                                                                                          \
        tg_status st_ = (call);                                                                   \
        if (st_ != TG_OK) {                                                                       \
            fprintf(stderr, "%s: %s (%s)\n", #call, tg_status_string(st_), tg_last_error());      \
            return 1;                                                                             \
        }                                                                                         \
    } while (0)

static unsigned lcg_state = 12345u;
static float lcg01(void)
{
    lcg_state = lcg_state * 1664525u + 1013904223u;
    return (float)(lcg_state >> 8) * (1.0f / 16777216.0f);
}

static int host_checks(void)
{
    tg_grid *g = NULL;
    int bad = 0;
    bad |= tg_create(4, 8, 2, 1, TG_F32, 0, 0.0f, &g) != TG_EINVAL;      /* dim */
    bad |= tg_create(3, 1, 2, 1, TG_F32, 0, 0.0f, &g) != TG_EINVAL;      /* res */
    bad |= tg_create(3, 8, 3, 1, TG_F32, 0, 0.0f, &g) != TG_EINVAL;      /* order */
    bad |= tg_query(NULL, NULL, 0, NULL, NULL, NULL) != TG_EINVAL;
    bad |= tg_adam_step(NULL, NULL, NULL, NULL) != TG_EINVAL;
    printf("host checks %s\n", bad ? "FAILED" : "ok");
    return bad;
}

static int gpu_run(void)
{
    const int res = 16, order = 2, channels = 1;
    const int64_t N = 4099;
    tg_grid *g = NULL;
    tg_grid_info info;
    CHECK(tg_create(3, res, order, channels, TG_F32, 7, 0.5f, &g));
    CHECK(tg_get_info(g, &info));
    const int64_t nc = info.n_coefs;

    float *pts = (float *)malloc((size_t)N * 3 * sizeof(float));
    float *out = (float *)malloc((size_t)N * sizeof(float));
    float *ones = (float *)malloc((size_t)N * sizeof(float));
    float *host = (float *)malloc((size_t)nc * sizeof(float));
    for (int64_t i = 0; i < 3 * N; ++i) pts[i] = lcg01();
    for (int64_t i = 0; i < N; ++i) ones[i] = 1.0f;

    float *d_pts, *d_out, *d_up, *d_grad, *d_coef;
    if (cudaMalloc((void **)&d_pts, (size_t)N * 3 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&d_out, (size_t)N * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&d_up, (size_t)N * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&d_grad, (size_t)nc * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&d_coef, (size_t)nc * sizeof(float)) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(d_pts, pts, (size_t)N * 3 * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(d_up, ones, (size_t)N * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(d_grad, 0, (size_t)nc * sizeof(float));

    CHECK(tg_query(g, d_pts, N, d_out, NULL, NULL));
    CHECK(tg_query_backward(g, d_pts, N, d_up, NULL, d_grad, NULL));
    double sf = 0.0, sg = 0.0, sc = 0.0;
    cudaMemcpy(out, d_out, (size_t)N * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(host, d_grad, (size_t)nc * sizeof(float), cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < N; ++i) sf += out[i];
    for (int64_t i = 0; i < nc; ++i) sg += host[i];
    tg_adam adam = {1e-2f, 0.9f, 0.999f, 1e-8f, 1};
    CHECK(tg_adam_step(g, d_grad, &adam, NULL));
    CHECK(tg_get_coefs(g, d_coef, 1, NULL));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        fprintf(stderr, "device error\n");
        return 1;
    }
    cudaMemcpy(host, d_coef, (size_t)nc * sizeof(float), cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < nc; ++i) sc += host[i];
    printf("%.17e %.17e %.17e\n", sf, sg, sc);

    cudaFree(d_pts); cudaFree(d_out); cudaFree(d_up); cudaFree(d_grad); cudaFree(d_coef);
    free(pts); free(out); free(ones); free(host);
    CHECK(tg_destroy(g));
    return 0;
}

int main(int argc, char **argv)
{
    if (argc > 1 && strcmp(argv[1], "host") == 0) return host_checks();
    return gpu_run();
}
