// FP32 FMA throughput of the device: the ALU roofline's denominator.
#include "tg_internal.cuh"

namespace tg {

constexpr int kProbeChains = 8;      // independent accumulators per thread: enough to cover the FMA latency
constexpr int kProbeIters = 4096;

__global__ void __launch_bounds__(256) fma_probe_kernel(float a, float b, float *__restrict__ sink)
{
    float acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = (float)(threadIdx.x + c);
#pragma unroll 16
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c];
    if (s == 12345.678f) *sink = s;     // keeps the chains live; a and b make it (practically) never true
}

}  // namespace tg

using namespace tg;

extern "C" tg_status tg_measure_fp32_peak(double *tflops)
{
    if (!tflops) return fail(TG_EINVAL, "tg_measure_fp32_peak: tflops is NULL");
    float *sink = nullptr;
    tg_status st = dev_alloc((void **)&sink, sizeof(float), "tg_measure_fp32_peak");
    if (st != TG_OK) return st;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const unsigned blocks = (unsigned)(num_sms() * per_sm);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = cuda_status(cudaEventCreate(&e0), "tg_measure_fp32_peak: event");
    if (st == TG_OK) st = cuda_status(cudaEventCreate(&e1), "tg_measure_fp32_peak: event");
    float ms = 0.f;
    if (st == TG_OK) {
        fma_probe_kernel<<<blocks, 256>>>(0.999999f, 1e-7f, sink);             // warm-up
        cudaEventRecord(e0);
        fma_probe_kernel<<<blocks, 256>>>(0.999999f, 1e-7f, sink);
        cudaEventRecord(e1);
        st = launch_status("tg_measure_fp32_peak");
        if (st == TG_OK) st = cuda_status(cudaEventSynchronize(e1), "tg_measure_fp32_peak");
        if (st == TG_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1), "tg_measure_fp32_peak");
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (st != TG_OK) return st;
    const double fmas = (double)blocks * 256.0 * kProbeChains * kProbeIters;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return TG_OK;
}
