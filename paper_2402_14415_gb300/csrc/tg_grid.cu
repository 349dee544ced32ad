// Grid storage V_T (Sec. 3.1): creation, coefficient exchange, status strings.
#include <atomic>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "tg_internal.cuh"

namespace tg {

static thread_local char g_err[512] = "";

tg_status fail(tg_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

tg_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TG_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(TG_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(TG_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

tg_status launch_status(const char *what) { return cuda_status(cudaGetLastError(), what); }

// Failure injection (tg_inject_alloc_failures): the next g_alloc_pass
// allocations go through, the g_alloc_fail after them report TG_ENOMEM.
static std::atomic<int> g_alloc_pass{0}, g_alloc_fail{0};

static bool injected_failure()
{
    if (g_alloc_fail.load() <= 0) return false;
    if (g_alloc_pass.fetch_sub(1) > 0) return false;
    g_alloc_pass.store(0);
    return g_alloc_fail.fetch_sub(1) > 0;
}

tg_status dev_alloc(void **p, size_t bytes, const char *what)
{
    *p = nullptr;
    if (injected_failure()) return fail(TG_ENOMEM, "%s: allocation of %zu bytes failed (injected)", what, bytes);
    return cuda_status(cudaMalloc(p, bytes), what);
}

tg_status dev_alloc_async(void **p, size_t bytes, cudaStream_t s, const char *what)
{
    *p = nullptr;
    if (injected_failure()) return fail(TG_ENOMEM, "%s: allocation of %zu bytes failed (injected)", what, bytes);
    return cuda_status(cudaMallocAsync(p, bytes, s), what);
}

int num_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cache[dev] = n;
    }
    return cache[dev];
}

int blocks_per_sm(const void *kernel, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_tuple(dev, kernel, threads, smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    cache[key] = n;
    return n;
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_kernel(float *__restrict__ master, T *__restrict__ store, int64_t n, uint64_t key, float std)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        float v = normal_k(key, (uint64_t)j) * std;
        master[j] = v;
        if (store) store[j] = from_f32<T>(v);
    }
}

template <typename T>
__global__ void narrow_kernel(const float *__restrict__ src, float *__restrict__ master, T *__restrict__ store, int64_t n)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        float v = src[j];
        if (master) master[j] = v;
        store[j] = from_f32<T>(v);
    }
}

template <typename T>
__global__ void widen_kernel(const T *__restrict__ store, float *__restrict__ dst, int64_t n)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = to_f32<T>(store[j]);
}

static unsigned elementwise_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace tg

using namespace tg;

extern "C" {

tg_status tg_inject_alloc_failures(int pass, int fail_count)
{
    if (pass < 0 || fail_count < 0) return fail(TG_EINVAL, "tg_inject_alloc_failures: negative count");
    g_alloc_fail.store(0);
    g_alloc_pass.store(pass);
    g_alloc_fail.store(fail_count);
    return TG_OK;
}

const char *tg_status_string(tg_status s)
{
    switch (s) {
    case TG_OK: return "TG_OK";
    case TG_EINVAL: return "TG_EINVAL";
    case TG_ENOMEM: return "TG_ENOMEM";
    case TG_EBUDGET: return "TG_EBUDGET";
    case TG_ETIMEOUT: return "TG_ETIMEOUT";
    case TG_EDEVICE: return "TG_EDEVICE";
    case TG_ENOTFOUND: return "TG_ENOTFOUND";
    case TG_EBUSY: return "TG_EBUSY";
    }
    return "TG_UNKNOWN";
}

const char *tg_last_error(void) { return tg::g_err; }

tg_status tg_create(int dim, int res, int order, int channels, tg_dtype dtype, uint64_t seed, float init_std,
                    tg_grid **out)
{
    if (!out) return fail(TG_EINVAL, "tg_create: out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(TG_EINVAL, "tg_create: dim must be 2 or 3 (got %d)", dim);
    if (order < 0 || order > 2) return fail(TG_EINVAL, "tg_create: order must be 0, 1 or 2 (got %d)", order);
    if (channels < 1 || channels > 4) return fail(TG_EINVAL, "tg_create: channels must be 1..4 (got %d)", channels);
    if (dtype != TG_F32 && dtype != TG_BF16 && dtype != TG_F16) return fail(TG_EINVAL, "tg_create: bad dtype %d", (int)dtype);
    if (res < 2 || res > (dim == 3 ? 2048 : 65536)) return fail(TG_EINVAL, "tg_create: res %d out of range", res);
    if (!(init_std >= 0.0f)) return fail(TG_EINVAL, "tg_create: init_std must be >= 0");

    tg_grid *g = (tg_grid *)calloc(1, sizeof(tg_grid));
    if (!g) return fail(TG_ENOMEM, "tg_create: host allocation failed");
    g->dim = dim; g->res = res; g->order = order; g->C = channels; g->dtype = dtype;
    g->lp_moments = dtype != TG_F32;      // the BF16 / FP16 storage form keeps Adam's moments in BF16
    g->K = num_coefs(dim, order);
    g->nv = 1;
    for (int d = 0; d < dim; ++d) g->nv *= res;
    g->ncoef = g->nv * channels * g->K;
    cudaGetDevice(&g->device);

    tg_status st = dev_alloc((void **)&g->master, (size_t)g->ncoef * 4 + 16, "tg_create: cudaMalloc(master)");
    if (st == TG_OK) {
        if (dtype == TG_F32) g->store = g->master;
        else st = dev_alloc((void **)&g->store, (size_t)g->ncoef * 2 + 16, "tg_create: cudaMalloc(store)");
    }
    if (st == TG_OK) {
        uint64_t key = 0;
        {   // host copy of the stream key (seed, 0xC0EF) of the generator
            auto mix = [](uint64_t z) {
                z += 0x9E3779B97F4A7C15ull;
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                return z ^ (z >> 31);
            };
            key = mix(mix(seed) + 0xC0EFull);
        }
        unsigned nb = elementwise_blocks(g->ncoef);
        if (dtype == TG_F32) init_kernel<float><<<nb, 256>>>(g->master, nullptr, g->ncoef, key, init_std);
        else if (dtype == TG_BF16) init_kernel<__nv_bfloat16><<<nb, 256>>>(g->master, (__nv_bfloat16 *)g->store, g->ncoef, key, init_std);
        else init_kernel<__half><<<nb, 256>>>(g->master, (__half *)g->store, g->ncoef, key, init_std);
        st = launch_status("tg_create: init kernel");
        if (st == TG_OK) st = cuda_status(cudaDeviceSynchronize(), "tg_create: init");
    }
    if (st != TG_OK) { tg_destroy(g); return st; }
    *out = g;
    return TG_OK;
}

tg_status tg_destroy(tg_grid *g)
{
    if (!g) return TG_OK;
    if (g->auto_event) cudaEventSynchronize(g->auto_event);
    if (g->auto_batch) tg_batch_destroy(g->auto_batch);
    if (g->auto_event) cudaEventDestroy(g->auto_event);
    if (g->store && g->store != g->master) cudaFree(g->store);
    if (g->master) cudaFree(g->master);
    if (g->adam_m) cudaFree(g->adam_m);
    if (g->adam_v) cudaFree(g->adam_v);
    free(g);
    return TG_OK;
}

tg_status tg_get_info(const tg_grid *g, tg_grid_info *info)
{
    if (!g || !info) return fail(TG_EINVAL, "tg_get_info: NULL argument");
    info->dim = g->dim; info->res = g->res; info->order = g->order; info->channels = g->C; info->K = g->K;
    info->dtype = g->dtype; info->n_vertices = g->nv; info->n_coefs = g->ncoef;
    size_t b = (size_t)g->ncoef * 4;
    if (g->dtype != TG_F32) b += (size_t)g->ncoef * 2;
    if (g->adam_m) b += (size_t)g->ncoef * 2 * moment_bytes(g);
    info->bytes = b;
    info->coefs = g->store;
    info->master = g->master;
    return TG_OK;
}

tg_status tg_set_coefs(tg_grid *g, const float *src, tg_stream stream)
{
    if (!g || !src) return fail(TG_EINVAL, "tg_set_coefs: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    tg_status st = TG_OK;
    if (src != g->master)      // src may be the master itself: then only the stored copy is refreshed
        st = cuda_status(cudaMemcpyAsync(g->master, src, (size_t)g->ncoef * 4, cudaMemcpyDeviceToDevice, s),
                         "tg_set_coefs: copy");
    if (st != TG_OK || g->dtype == TG_F32) return st;
    unsigned nb = elementwise_blocks(g->ncoef);
    if (g->dtype == TG_BF16) narrow_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>(g->master, nullptr, (__nv_bfloat16 *)g->store, g->ncoef);
    else narrow_kernel<__half><<<nb, 256, 0, s>>>(g->master, nullptr, (__half *)g->store, g->ncoef);
    return launch_status("tg_set_coefs: narrow kernel");
}

tg_status tg_get_coefs(const tg_grid *g, float *dst, int which, tg_stream stream)
{
    if (!g || !dst) return fail(TG_EINVAL, "tg_get_coefs: NULL argument");
    if (which < 0 || which > 3) return fail(TG_EINVAL, "tg_get_coefs: which must be 0, 1, 2 or 3");
    cudaStream_t s = (cudaStream_t)stream;
    if (which >= 2) {      // Adam's first (2) or second (3) moment, widened to FP32
        const void *src = which == 2 ? g->adam_m : g->adam_v;
        if (!src) return fail(TG_EINVAL, "tg_get_coefs: the grid has no Adam state yet");
        if (!g->lp_moments)
            return cuda_status(cudaMemcpyAsync(dst, src, (size_t)g->ncoef * 4, cudaMemcpyDeviceToDevice, s),
                               "tg_get_coefs: copy");
        widen_kernel<__nv_bfloat16><<<elementwise_blocks(g->ncoef), 256, 0, s>>>((const __nv_bfloat16 *)src, dst,
                                                                               g->ncoef);
        return launch_status("tg_get_coefs: widen kernel");
    }
    if (which == 1 || g->dtype == TG_F32)
        return cuda_status(cudaMemcpyAsync(dst, g->master, (size_t)g->ncoef * 4, cudaMemcpyDeviceToDevice, s),
                           "tg_get_coefs: copy");
    unsigned nb = elementwise_blocks(g->ncoef);
    if (g->dtype == TG_BF16) widen_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>((const __nv_bfloat16 *)g->store, dst, g->ncoef);
    else widen_kernel<__half><<<nb, 256, 0, s>>>((const __half *)g->store, dst, g->ncoef);
    return launch_status("tg_get_coefs: widen kernel");
}


/* Checkpoint format (little-endian): "TGCK", u32 version 1, i32 dim, res,
 * order, channels, dtype, has_adam, i64 n_coefs, then the FP32 master
 * (n_coefs floats) and, if has_adam, Adam's m and v (n_coefs floats each). */
tg_status tg_save(const tg_grid *g, const char *path)
{
    if (!g || !path) return fail(TG_EINVAL, "tg_save: NULL argument");
    const int32_t hdr[7] = {1, g->dim, g->res, g->order, g->C, (int32_t)g->dtype, g->adam_m ? 1 : 0};
    const int64_t n = g->ncoef;
    const size_t bytes = (size_t)n * 4;
    float *host = (float *)malloc(bytes);
    if (!host) return fail(TG_ENOMEM, "tg_save: host buffer");
    FILE *f = fopen(path, "wb");
    if (!f) {
        free(host);
        return fail(TG_EINVAL, "tg_save: cannot open %s for writing", path);
    }
    tg_status st = TG_OK;
    bool ok = fwrite("TGCK", 1, 4, f) == 4 && fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&n, 8, 1, f) == 1;
    const void *arrays[3] = {g->master, g->adam_m, g->adam_v};
    for (int a = 0; ok && st == TG_OK && a < (g->adam_m ? 3 : 1); ++a) {
        const bool lp = a > 0 && g->lp_moments;      // BF16 moments: the upper halves of FP32 words
        st = cuda_status(cudaMemcpy(host, arrays[a], lp ? (size_t)n * 2 : bytes, cudaMemcpyDeviceToHost), "tg_save: copy");
        if (st == TG_OK && lp) {
            const uint16_t *h16 = reinterpret_cast<const uint16_t *>(host);
            uint32_t *h32 = reinterpret_cast<uint32_t *>(host);
            for (int64_t k = n - 1; k >= 0; --k) h32[k] = (uint32_t)h16[k] << 16;     // back to front: in place
        }
        if (st == TG_OK) ok = fwrite(host, 1, bytes, f) == bytes;
    }
    if (fclose(f) != 0) ok = false;
    free(host);
    if (st != TG_OK) return st;
    return ok ? TG_OK : fail(TG_EINVAL, "tg_save: write to %s failed", path);
}

tg_status tg_load(const char *path, tg_grid **out)
{
    if (!path || !out) return fail(TG_EINVAL, "tg_load: NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(TG_EINVAL, "tg_load: cannot open %s", path);
    char magic[4];
    int32_t hdr[7];
    int64_t n = 0;
    if (fread(magic, 1, 4, f) != 4 || memcmp(magic, "TGCK", 4) != 0 || fread(hdr, sizeof(hdr), 1, f) != 1 ||
        fread(&n, 8, 1, f) != 1 || hdr[0] != 1) {
        fclose(f);
        return fail(TG_EINVAL, "tg_load: %s is not a TaylorGrid checkpoint (version 1)", path);
    }
    tg_grid *g = nullptr;
    tg_status st = tg_create(hdr[1], hdr[2], hdr[3], hdr[4], (tg_dtype)hdr[5], 0, 0.0f, &g);
    if (st != TG_OK) {
        fclose(f);
        return st;
    }
    if (g->ncoef != n) {
        fclose(f);
        tg_destroy(g);
        return fail(TG_EINVAL, "tg_load: %s holds %lld coefficients, its shape needs %lld", path, (long long)n,
                    (long long)g->ncoef);
    }
    const size_t bytes = (size_t)n * 4;
    float *host = (float *)malloc(bytes);
    if (!host) {
        fclose(f);
        tg_destroy(g);
        return fail(TG_ENOMEM, "tg_load: host buffer");
    }
    const int arrays = hdr[6] ? 3 : 1;
    if (hdr[6]) st = ensure_adam_state(g);
    void *dst[3] = {g->master, g->adam_m, g->adam_v};
    for (int a = 0; st == TG_OK && a < arrays; ++a) {
        const bool lp = a > 0 && g->lp_moments;
        if (fread(host, 1, bytes, f) != bytes) {
            st = fail(TG_EINVAL, "tg_load: %s is truncated", path);
            break;
        }
        if (lp) {      // FP32 -> BF16, round to nearest even (exact for moments saved from BF16)
            const uint32_t *h32 = reinterpret_cast<const uint32_t *>(host);
            uint16_t *h16 = reinterpret_cast<uint16_t *>(host);
            for (int64_t k = 0; k < n; ++k) {
                const uint32_t u = h32[k];
                const bool nan = (u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu) != 0;
                h16[k] = nan ? (uint16_t)((u >> 16) | 0x40u) : (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
            }
        }
        st = cuda_status(cudaMemcpy(dst[a], host, lp ? (size_t)n * 2 : bytes, cudaMemcpyHostToDevice), "tg_load: copy");
    }
    fclose(f);
    free(host);
    if (st == TG_OK) st = tg_set_coefs(g, g->master, nullptr);       // the stored copy from the master
    if (st == TG_OK) st = cuda_status(cudaDeviceSynchronize(), "tg_load");
    if (st != TG_OK) {
        tg_destroy(g);
        return st;
    }
    *out = g;
    return TG_OK;
}

}  // extern "C"
