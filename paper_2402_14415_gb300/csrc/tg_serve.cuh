// Internal interface of the fit / query server: the device status block of a
// fit job and the batched training step that advances many jobs per launch.
#pragma once

#include "tg_sdf.cuh"

namespace tg {

struct DevStatus {
    long long steps;
    float error;
    int done;
};

// Device status block of a fit job (64 bytes): loss sums [2], error sum, gate,
// step counter, status, and the Adam coefficients of the step in flight.
struct JobBlock {
    __host__ __device__ static float *loss(unsigned char *b) { return reinterpret_cast<float *>(b); }
    __host__ __device__ static float *err(unsigned char *b) { return reinterpret_cast<float *>(b) + 2; }
    __host__ __device__ static int *gate(unsigned char *b) { return reinterpret_cast<int *>(b) + 3; }
    __host__ __device__ static int64_t *step(unsigned char *b) { return reinterpret_cast<int64_t *>(b + 16); }
    __host__ __device__ static DevStatus *status(unsigned char *b) { return reinterpret_cast<DevStatus *>(b + 32); }
    __host__ __device__ static float *adam(unsigned char *b) { return reinterpret_cast<float *>(b + 48); }   // [2]
    static constexpr int bytes = 64;
};

// One running fit job of a batched step (an entry of the device job table).
// Jobs of one batch share order and storage dtype.
struct BatchJob {
    const void *store;       // stored coefficients (the batch's storage type)
    float *master, *grad;    // FP32 master and gradient
    void *m, *v;             // Adam moments: FP32 (FP32 storage) or BF16
    void *shadow;            // the stored copy Adam refreshes (BF16 / FP16), or null
    unsigned char *block;    // JobBlock
    const float *eval_pts;   // n_eval x 3
    ShapeView shape;
    uint64_t seed;
    int64_t ncoef;
    int64_t pbase, npts;     // the job's points in the batch: [pbase, pbase + npts)
    int64_t gbase;           // its first unit of the Adam pass: ceil(ncoef / 4) float4 groups, or, with
                             // touched flags, ceil(nv / 4) runs of 4 vertices
    unsigned char *touched;  // lazy Adam: one flag per vertex, set by the fit kernel, cleared by Adam; or null
    int64_t nv;              // vertices (ncoef = nv * K)
    int K;
    int64_t n_eval;
    int res, eval_every, max_steps, lazy;
    float lambda_eik, k_weight, lr, tol;
};

// One training step of every job in jobs[0..n) (host table, copied to dev):
// sample -> f and grad f -> loss upstreams -> coefficient gradient (one fused
// point-parallel launch over all jobs' points), Adam over all jobs'
// coefficients (one launch), the gated evaluation and the step bookkeeping;
// then the jobs' DevStatus words are gathered into status_dev[0..n).
tg_status batch_step(const BatchJob *host, BatchJob *dev, int n, int order, tg_dtype dtype, DevStatus *status_dev,
                     cudaStream_t s);

}  // namespace tg
