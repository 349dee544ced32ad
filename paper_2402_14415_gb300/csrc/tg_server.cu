// Continuous-batching fit / query server.
//
// Running fit jobs that share order and storage dtype form a group; a tick
// advances every group by one step with one launch per stage for all of its
// jobs (tg_serve_batch.cu: a fused point-parallel kernel over the
// concatenated fit batches, one Adam launch over all their coefficients, a
// gated evaluation, the step bookkeeping), on the group's stream, and copies
// the jobs' status words to pinned host memory behind it. A job with
// TG_FIT_DETERMINISTIC or a TV term instead owns a stream and a CUDA graph of
// one step (sampler -> binning -> forward -> loss -> backward -> TV -> Adam ->
// gated evaluation -> finalize) captured at admission. Later ticks read the
// status only once the step's event has completed, so the host never blocks
// on the device inside a tick.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "tg_serve.cuh"

namespace tg {

__global__ void eval_gate_kernel(const int64_t *__restrict__ step, int eval_every, int *__restrict__ gate)
{
    *gate = ((*step + 1) % eval_every) == 0 ? 1 : 0;
}

__global__ void finalize_kernel(int64_t *__restrict__ step, const int *__restrict__ gate, float *__restrict__ err_sum,
                                float inv_eval, float tol, int max_steps, float *__restrict__ loss,
                                DevStatus *__restrict__ st)
{
    const int64_t s = *step + 1;
    if (*gate) {
        const float e = *err_sum * inv_eval;
        st->error = e;
        *err_sum = 0.f;
        if (e < tol) st->done = 1;
    }
    *step = s;
    st->steps = s;
    if (s >= max_steps) st->done = 1;
    loss[0] = 0.f;
    loss[1] = 0.f;
}

struct Job {
    tg_job_id id = 0;
    int kind = 0;                    // 0 fit, 1 query
    int state = TG_JOB_QUEUED;
    tg_fit_desc desc{};
    std::vector<float> sph, box, cdf;
    size_t bytes = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t steps = 0;
    float error = -1.f;
    // fit job device state
    tg_grid *grid = nullptr;
    tg_batch *batch = nullptr;
    float *grad = nullptr;
    float *shape_dev = nullptr;      // spheres | boxes | cdf
    float *eval_pts = nullptr;
    unsigned char *small = nullptr;  // loss[2], err, gate, step, status
    DevStatus *status_host = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool in_flight = false;
    bool cancel = false;             // stop at the next step boundary
    ShapeView sv{};
    // query
    tg_job_id grid_of = 0;
    const float *qpts = nullptr;
    float *qout = nullptr;
    int64_t qn = 0;

    float *partials = nullptr;       // deterministic evaluation: per-block error sums
    unsigned char *touched = nullptr;   // batched lazy-Adam job: one flag per vertex
    bool batched = false;            // advanced with its group (no own stream or graph)
    int group = -1;                  // group key of a batched job

    float *loss() { return JobBlock::loss(small); }
    float *err() { return JobBlock::err(small); }
    int *gate() { return JobBlock::gate(small); }
    int64_t *step() { return JobBlock::step(small); }
    DevStatus *status() { return JobBlock::status(small); }
};

// Running batched fit jobs of one (order, storage dtype): one step of all of
// them per tick, on the group's stream.
struct Group {
    int order = 0;
    tg_dtype dtype = TG_F32;
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    int cap = 0;
    BatchJob *table_host = nullptr;      // pinned
    BatchJob *table_dev = nullptr;
    DevStatus *status_host = nullptr;    // pinned
    DevStatus *status_dev = nullptr;
    std::vector<Job *> members;          // the jobs of the step in flight, in table order
    bool in_flight = false;
};

static void free_group(Group *g)
{
    if (g->stream) cudaStreamSynchronize(g->stream);
    cudaFreeHost(g->table_host); cudaFreeHost(g->status_host);
    cudaFree(g->table_dev); cudaFree(g->status_dev);
    if (g->event) cudaEventDestroy(g->event);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

static tg_status group_capacity(Group *g, int n)
{
    if (n <= g->cap) return TG_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    cudaFreeHost(g->table_host); cudaFreeHost(g->status_host);
    cudaFree(g->table_dev); cudaFree(g->status_dev);
    g->table_host = nullptr; g->status_host = nullptr; g->table_dev = nullptr; g->status_dev = nullptr;
    g->cap = 0;
    const int cap = std::max(n, 8);
    tg_status st = cuda_status(cudaMallocHost(&g->table_host, cap * sizeof(BatchJob)), "server: job table");
    if (st == TG_OK) st = cuda_status(cudaMallocHost(&g->status_host, cap * sizeof(DevStatus)), "server: status words");
    if (st == TG_OK) st = dev_alloc((void **)&g->table_dev, cap * sizeof(BatchJob), "server: job table");
    if (st == TG_OK) st = dev_alloc((void **)&g->status_dev, cap * sizeof(DevStatus), "server: status words");
    if (st == TG_OK) g->cap = cap;
    return st;
}

static bool runs_alone(const tg_fit_desc &d) { return (d.flags & TG_FIT_DETERMINISTIC) || d.lambda_tv > 0.f; }

static size_t fit_bytes(const tg_fit_desc &d)
{
    const int K = num_coefs(3, d.order);
    const size_t ncoef = (size_t)d.res * d.res * d.res * K;
    if (!runs_alone(d))    // batched: the grid, Adam state, gradient, evaluation points, status block, touched flags
        return (d.dtype == TG_F32 ? ncoef * (4 + 8 + 4) : ncoef * (4 + 4 + 4 + 2)) + (size_t)d.eval_points * 12 + 4096 +
               ((d.flags & TG_FIT_LAZY_ADAM) ? ncoef / K + 16 : 0);     // flags: an upper bound
    // master, Adam m + v (FP32, or BF16 for BF16 / FP16 storage), gradient, shadow
    size_t b = d.dtype == TG_F32 ? ncoef * (4 + 8 + 4) : ncoef * (4 + 4 + 4 + 2);
    const size_t nb = (size_t)((d.res - 2) / 8 + 1);
    const size_t bricks = nb * nb * nb;
    b += (size_t)d.points_per_step * (16 + 16 + 4 + 4 * 11);                  // records, coarse, perm, staging
    b += bricks * (3 * 4 + (bricks <= 32768 ? 4 * kBinChunksPerSm * num_sms() : 0));   // offsets, chunk histograms
    b += (size_t)d.eval_points * 12 + 4096;
    return b;
}

static void free_fit_scratch(Job *j)
{
    if (j->graph) cudaGraphExecDestroy(j->graph);
    j->graph = nullptr;
    if (j->batch) tg_batch_destroy(j->batch);
    j->batch = nullptr;
    cudaFree(j->grad); j->grad = nullptr;
    cudaFree(j->shape_dev); j->shape_dev = nullptr;
    cudaFree(j->eval_pts); j->eval_pts = nullptr;
    cudaFree(j->small); j->small = nullptr;
    cudaFree(j->partials); j->partials = nullptr;
    cudaFree(j->touched); j->touched = nullptr;
}

static void free_job(Job *j)
{
    if (j->stream) cudaStreamSynchronize(j->stream);
    free_fit_scratch(j);
    if (j->grid) tg_destroy(j->grid);
    j->grid = nullptr;
    if (j->status_host) cudaFreeHost(j->status_host);
    j->status_host = nullptr;
    if (j->event) cudaEventDestroy(j->event);
    j->event = nullptr;
    if (j->stream) cudaStreamDestroy(j->stream);
    j->stream = nullptr;
}

// Records one training step of a fit job on its stream (captured or direct).
static tg_status record_step(Job *j)
{
    const tg_fit_desc &d = j->desc;
    const bool det = (d.flags & TG_FIT_DETERMINISTIC) != 0;
    tg_status st = sdf_step_impl(j->grid, j->batch, j->sv, nullptr, d.points_per_step, d.seed, 0, j->step(),
                                 d.lambda_eik, d.k_weight, j->grad, j->loss(), j->stream, det);
    if (st != TG_OK) return st;
    if (d.lambda_tv > 0.f && (st = tg_tv_step(j->grid, d.lambda_tv, j->grad, nullptr, j->stream)) != TG_OK) return st;
    tg_adam prm{d.lr, 0.9f, 0.999f, 1e-8f, 1};
    if ((st = adam_launch(j->grid, j->grad, &prm, j->step(), j->stream, (d.flags & TG_FIT_LAZY_ADAM) != 0)) != TG_OK)
        return st;
    eval_gate_kernel<<<1, 1, 0, j->stream>>>(j->step(), d.eval_every, j->gate());
    if ((st = launch_status("server: eval gate")) != TG_OK) return st;
    if ((st = sdf_error_impl(j->grid, j->sv, j->eval_pts, d.eval_points, j->err(), j->gate(), j->stream, nullptr,
                             j->partials)) != TG_OK)
        return st;
    finalize_kernel<<<1, 1, 0, j->stream>>>(j->step(), j->gate(), j->err(), 1.0f / (float)d.eval_points, d.tol,
                                            d.max_steps, j->loss(), j->status());
    return launch_status("server: finalize");
}

// Admission: device state of a fit job. A batched job gets its grid, Adam
// state, gradient, status block, target and evaluation points, set up on the
// stream `s` (its group's); a job that runs alone also gets a stream, a point
// batch and its step captured as a CUDA graph.
static tg_status admit_fit(Job *j, cudaStream_t group_stream)
{
    const tg_fit_desc &d = j->desc;
    const bool alone = !j->batched;
    tg_status st = TG_OK;
    if (alone) {
        st = cuda_status(cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking), "server: stream");
        if (st == TG_OK) st = cuda_status(cudaEventCreateWithFlags(&j->event, cudaEventDisableTiming), "server: event");
        if (st == TG_OK) st = cuda_status(cudaMallocHost(&j->status_host, sizeof(DevStatus)), "server: pinned status");
    }
    if (st == TG_OK) st = tg_create(3, d.res, d.order, 1, d.dtype, d.seed, d.init_std, &j->grid);
    if (st == TG_OK && alone) st = tg_batch_create(3, d.res, d.points_per_step, &j->batch);
    if (st == TG_OK && alone) st = ensure_stage(j->batch, 11 * d.points_per_step, "server: staging");
    if (st == TG_OK && alone && (d.flags & TG_FIT_DETERMINISTIC))
        st = dev_alloc((void **)&j->partials, (size_t)error_blocks(d.eval_points) * 4, "server: evaluation sums");
    if (st == TG_OK) st = ensure_adam_state(j->grid);
    if (st == TG_OK) st = dev_alloc((void **)&j->grad, (size_t)j->grid->ncoef * 4 + 16, "server: gradient");
    if (st == TG_OK) st = dev_alloc((void **)&j->small, 64, "server: status block");
    // touched flags where a step reaches few of the vertices (8 corners a point against at least 16 vertices
    // a point): Adam then visits the flagged vertices only; on denser grids it streams every coefficient
    const bool flags = !alone && (d.flags & TG_FIT_LAZY_ADAM) && j->grid->nv >= 16 * d.points_per_step;
    if (st == TG_OK && flags)
        st = dev_alloc((void **)&j->touched, (size_t)j->grid->nv + 16, "server: touched flags");
    const size_t nsh = j->sph.size() + j->box.size() + j->cdf.size();
    if (st == TG_OK) st = dev_alloc((void **)&j->shape_dev, nsh * 4, "server: shape");
    if (st == TG_OK) st = dev_alloc((void **)&j->eval_pts, (size_t)d.eval_points * 12, "server: eval points");
    if (st != TG_OK) return st;
    cudaStream_t s = alone ? j->stream : group_stream;
    st = cuda_status(cudaMemsetAsync(j->grad, 0, (size_t)j->grid->ncoef * 4, s), "server: zero gradient");
    if (st == TG_OK) st = cuda_status(cudaMemsetAsync(j->small, 0, 64, s), "server: zero status");
    if (st == TG_OK && flags)
        st = cuda_status(cudaMemsetAsync(j->touched, 0, (size_t)j->grid->nv + 16, s), "server: zero flags");
    float *sp = j->shape_dev, *bp = sp + j->sph.size(), *cp = bp + j->box.size();
    if (st == TG_OK && !j->sph.empty())
        st = cuda_status(cudaMemcpyAsync(sp, j->sph.data(), j->sph.size() * 4, cudaMemcpyHostToDevice, s), "server: shape");
    if (st == TG_OK && !j->box.empty())
        st = cuda_status(cudaMemcpyAsync(bp, j->box.data(), j->box.size() * 4, cudaMemcpyHostToDevice, s), "server: shape");
    if (st == TG_OK)
        st = cuda_status(cudaMemcpyAsync(cp, j->cdf.data(), j->cdf.size() * 4, cudaMemcpyHostToDevice, s), "server: shape");
    if (st != TG_OK) return st;
    tg_shape shape{d.n_spheres, d.n_boxes, sp, bp, cp};
    if ((st = shape_view(&shape, &j->sv, "server")) != TG_OK) return st;
    if ((st = tg_sample_sdf_points(&shape, d.seed + 1, 0, d.eval_points, 0.01f, j->eval_pts, s)) != TG_OK) return st;
    if (!alone) return TG_OK;      // ordered before the group's next step by its stream
    if ((st = cuda_status(cudaStreamSynchronize(s), "server: admission")) != TG_OK) return st;
    // capture one step as a graph; fall back to direct launches if capture is refused
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const tg_status rec = record_step(j);
        const cudaError_t ec = cudaStreamEndCapture(s, &graph);
        if (rec == TG_OK && ec == cudaSuccess && graph &&
            cudaGraphInstantiate(&j->graph, graph, 0) == cudaSuccess) {
            cudaGraphDestroy(graph);
        } else {
            if (graph) cudaGraphDestroy(graph);
            j->graph = nullptr;
            cudaGetLastError();
        }
    } else {
        cudaGetLastError();
    }
    return TG_OK;
}

}  // namespace tg

using namespace tg;

struct tg_server {
    size_t budget = 0, used = 0;
    int max_running = 1;
    int policy = TG_ADMIT_FIFO;
    std::map<tg_job_id, Job *> jobs;
    std::map<int, Group *> groups;      // key: order * 8 + storage dtype
    std::deque<tg_job_id> queue;
    tg_job_id next = 1;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

extern "C" {

tg_status tg_server_create(size_t budget_bytes, int max_running, tg_server **out)
{
    if (!out) return fail(TG_EINVAL, "tg_server_create: out is NULL");
    if (budget_bytes == 0 || max_running < 1) return fail(TG_EINVAL, "tg_server_create: budget > 0, max_running >= 1");
    tg_server *s = new (std::nothrow) tg_server();
    if (!s) return fail(TG_ENOMEM, "tg_server_create: host allocation failed");
    s->budget = budget_bytes;
    s->max_running = max_running;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return TG_OK;
}

tg_status tg_server_destroy(tg_server *s)
{
    if (!s) return TG_OK;
    for (auto &kv : s->groups) free_group(kv.second);       // waits for the steps in flight
    for (auto &kv : s->jobs) {
        free_job(kv.second);
        delete kv.second;
    }
    delete s;
    return TG_OK;
}

double tg_server_time(const tg_server *s) { return s ? s->now() : 0.0; }

tg_status tg_server_set_policy(tg_server *s, int policy)
{
    if (!s || (policy != TG_ADMIT_FIFO && policy != TG_ADMIT_SMALLEST))
        return fail(TG_EINVAL, "tg_server_set_policy: bad argument");
    std::lock_guard<std::mutex> lock(s->mu);
    s->policy = policy;
    return TG_OK;
}

tg_status tg_fit_job(tg_server *s, const tg_fit_desc *d, tg_job_id *id)
{
    if (!s || !d || !id) return fail(TG_EINVAL, "tg_fit_job: NULL argument");
    if (d->res < 2 || d->order < 0 || d->order > 2 || d->points_per_step < 1 || d->eval_points < 1 ||
        d->eval_every < 1 || d->max_steps < 1 || d->n_spheres < 0 || d->n_boxes < 0 ||
        d->n_spheres + d->n_boxes < 1 || (d->n_spheres && !d->spheres) || (d->n_boxes && !d->boxes) || !d->area_cdf)
        return fail(TG_EINVAL, "tg_fit_job: bad job description");
    if (d->dtype != TG_F32 && d->dtype != TG_BF16 && d->dtype != TG_F16) return fail(TG_EINVAL, "tg_fit_job: bad dtype");
    if ((d->flags & ~(TG_FIT_DETERMINISTIC | TG_FIT_LAZY_ADAM)) != 0) return fail(TG_EINVAL, "tg_fit_job: bad flags");
    const size_t need = fit_bytes(*d);
    if (need > s->budget)
        return fail(TG_EBUDGET, "tg_fit_job: the job needs %zu bytes, over the budget of %zu", need, s->budget);
    Job *j = new (std::nothrow) Job();
    if (!j) return fail(TG_ENOMEM, "tg_fit_job: host allocation failed");
    j->kind = 0;
    j->desc = *d;
    j->batched = !runs_alone(*d);
    j->group = d->order * 8 + (int)d->dtype;
    j->sph.assign(d->spheres, d->spheres + 4 * d->n_spheres);
    j->box.assign(d->boxes, d->boxes + 6 * d->n_boxes);
    j->cdf.assign(d->area_cdf, d->area_cdf + d->n_spheres + d->n_boxes);
    j->desc.spheres = j->desc.boxes = j->desc.area_cdf = nullptr;
    j->bytes = need;
    std::lock_guard<std::mutex> lock(s->mu);
    j->id = s->next++;
    j->t_submit = s->now();
    s->jobs[j->id] = j;
    s->queue.push_back(j->id);
    *id = j->id;
    return TG_OK;
}

tg_status tg_query_job(tg_server *s, tg_job_id grid_job, const float *pts, int64_t N, float *out, tg_job_id *id)
{
    if (!s || !id || N < 0 || (N > 0 && (!pts || !out))) return fail(TG_EINVAL, "tg_query_job: bad argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(grid_job);
    if (it == s->jobs.end() || it->second->kind != 0 || it->second->state == TG_JOB_FAILED)
        return fail(TG_ENOTFOUND, "tg_query_job: no fit job %lld", (long long)grid_job);
    Job *j = new (std::nothrow) Job();
    if (!j) return fail(TG_ENOMEM, "tg_query_job: host allocation failed");
    j->kind = 1;
    j->grid_of = grid_job;
    j->qpts = pts; j->qout = out; j->qn = N;
    j->id = s->next++;
    j->t_submit = s->now();
    s->jobs[j->id] = j;
    s->queue.push_back(j->id);
    *id = j->id;
    return TG_OK;
}

// Group of a batched job (created on first use).
static tg_status group_of(tg_server *s, const Job *j, Group **out)
{
    auto it = s->groups.find(j->group);
    if (it != s->groups.end()) {
        *out = it->second;
        return TG_OK;
    }
    Group *g = new (std::nothrow) Group();
    if (!g) return fail(TG_ENOMEM, "server: host allocation failed");
    g->order = j->desc.order;
    g->dtype = j->desc.dtype;
    tg_status st = cuda_status(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking), "server: group stream");
    if (st == TG_OK) st = cuda_status(cudaEventCreateWithFlags(&g->event, cudaEventDisableTiming), "server: group event");
    if (st != TG_OK) {
        free_group(g);
        return st;
    }
    s->groups[j->group] = g;
    *out = g;
    return TG_OK;
}

static void finish(tg_server *s, Job *j, int state)
{
    j->state = state;
    j->t_done = s->now();
    free_fit_scratch(j);
}

tg_status tg_server_step(tg_server *s, int *pending)
{
    if (!s) return fail(TG_EINVAL, "tg_server_step: server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    int running = 0;
    // 1. retire finished steps: jobs that run alone and queries by their own
    //    event, batched jobs by their group's
    for (auto &kv : s->jobs) {
        Job *j = kv.second;
        if (j->state != TG_JOB_RUNNING || !j->in_flight || j->batched) continue;
        const cudaError_t q = cudaEventQuery(j->event);
        if (q == cudaErrorNotReady) continue;
        j->in_flight = false;
        if (q != cudaSuccess) {
            j->state = TG_JOB_FAILED;
            j->t_done = s->now();
            cudaGetLastError();
            continue;
        }
        if (j->kind == 1) {
            j->state = TG_JOB_DONE;
            j->t_done = s->now();
            continue;
        }
        j->steps = j->status_host->steps;
        if (j->status_host->error >= 0.f && j->steps >= j->desc.eval_every) j->error = j->status_host->error;
        if (j->status_host->done) finish(s, j, TG_JOB_DONE);
    }
    for (auto &kv : s->groups) {
        Group *g = kv.second;
        if (!g->in_flight) continue;
        const cudaError_t q = cudaEventQuery(g->event);
        if (q == cudaErrorNotReady) continue;
        g->in_flight = false;
        for (size_t k = 0; k < g->members.size(); ++k) {
            Job *j = g->members[k];
            j->in_flight = false;
            if (q != cudaSuccess) {
                finish(s, j, TG_JOB_FAILED);
                continue;
            }
            const DevStatus &ds = g->status_host[k];
            j->steps = ds.steps;
            if (ds.error >= 0.f && j->steps >= j->desc.eval_every) j->error = ds.error;
            if (ds.done) finish(s, j, TG_JOB_DONE);
        }
        if (q != cudaSuccess) cudaGetLastError();
        g->members.clear();
    }
    // cancelled fit jobs whose last step has retired stop here; their grid stays until tg_release
    for (auto &kv : s->jobs) {
        Job *j = kv.second;
        if (j->kind != 0 || j->state != TG_JOB_RUNNING || j->in_flight || !j->cancel) continue;
        finish(s, j, TG_JOB_CANCELLED);
    }
    for (auto &kv : s->jobs)
        if (kv.second->kind == 0 && kv.second->state == TG_JOB_RUNNING) ++running;
    // 2. admission scan over the queue: arrival order, or (TG_ADMIT_SMALLEST)
    //    fit jobs by increasing device bytes. A query runs as soon as its grid
    //    exists and otherwise stays queued without blocking anything; the first
    //    fit job that does not fit the budget or the running-job limit stops
    //    admission of every fit job behind it (no overtaking by larger jobs).
    if (s->policy == TG_ADMIT_SMALLEST && s->queue.size() > 1) {
        std::stable_sort(s->queue.begin(), s->queue.end(), [&](tg_job_id a, tg_job_id b) {
            const Job *ja = s->jobs[a], *jb = s->jobs[b];
            const size_t ka = ja->kind == 1 ? 0 : ja->bytes, kb = jb->kind == 1 ? 0 : jb->bytes;
            return ka < kb;
        });
    }
    std::deque<tg_job_id> keep;
    bool fit_blocked = false;
    for (tg_job_id id : s->queue) {
        Job *j = s->jobs[id];
        if (j->kind == 1) {
            auto it = s->jobs.find(j->grid_of);
            Job *g = it == s->jobs.end() ? nullptr : it->second;
            if (g && g->state == TG_JOB_QUEUED) {         // grid not created yet
                keep.push_back(id);
                continue;
            }
            if (!g || g->state == TG_JOB_FAILED || !g->grid) {     // also a fit job cancelled before it ran
                j->state = TG_JOB_FAILED;
                j->t_done = s->now();
                continue;
            }
            // behind the grid's step in flight, on the stream that updates it
            cudaStream_t qs = g->stream;
            if (g->batched) {
                Group *grp = nullptr;
                if (group_of(s, g, &grp) != TG_OK) {
                    j->state = TG_JOB_FAILED;
                    j->t_done = s->now();
                    continue;
                }
                qs = grp->stream;
            }
            j->event = nullptr;
            tg_status st = cuda_status(cudaEventCreateWithFlags(&j->event, cudaEventDisableTiming), "server: event");
            // point-parallel: no binning scratch outside the admission budget
            if (st == TG_OK) st = query_point_parallel(g->grid, j->qpts, j->qn, j->qout, nullptr, qs);
            if (st == TG_OK) st = cuda_status(cudaEventRecord(j->event, qs), "server: query event");
            j->t_start = s->now();
            j->state = st == TG_OK ? TG_JOB_RUNNING : TG_JOB_FAILED;
            j->in_flight = st == TG_OK;
            if (st != TG_OK) j->t_done = j->t_start;
            continue;
        }
        if (fit_blocked || running >= s->max_running || s->used + j->bytes > s->budget) {
            fit_blocked = true;
            keep.push_back(id);
            continue;
        }
        j->t_start = s->now();
        Group *grp = nullptr;
        tg_status st = j->batched ? group_of(s, j, &grp) : TG_OK;
        // a batched job is set up on its group's stream, behind the group's step in flight
        if (st == TG_OK) st = admit_fit(j, grp ? grp->stream : nullptr);
        if (st != TG_OK) {
            if (grp) cudaStreamSynchronize(grp->stream);     // the copies of the partial set-up
            j->state = TG_JOB_FAILED;
            j->t_done = s->now();
            free_job(j);
            continue;
        }
        s->used += j->bytes;
        j->state = TG_JOB_RUNNING;
        ++running;
    }
    s->queue.swap(keep);
    // 3a. one step of every running job that runs alone and whose previous step has retired
    for (auto &kv : s->jobs) {
        Job *j = kv.second;
        if (j->kind != 0 || j->batched || j->state != TG_JOB_RUNNING || j->in_flight || j->cancel) continue;
        tg_status st = TG_OK;
        if (j->graph) st = cuda_status(cudaGraphLaunch(j->graph, j->stream), "server: graph launch");
        else st = record_step(j);
        if (st == TG_OK)
            st = cuda_status(cudaMemcpyAsync(j->status_host, j->status(), sizeof(DevStatus), cudaMemcpyDeviceToHost,
                                             j->stream), "server: status copy");
        if (st == TG_OK) st = cuda_status(cudaEventRecord(j->event, j->stream), "server: step event");
        if (st != TG_OK) {
            j->state = TG_JOB_FAILED;
            j->t_done = s->now();
            continue;
        }
        j->in_flight = true;
    }
    // 3b. one step of every group whose previous step has retired: all its running jobs in one table
    for (auto &kv : s->groups) {
        Group *g = kv.second;
        if (g->in_flight) continue;
        std::vector<Job *> mem;
        for (auto &jk : s->jobs) {
            Job *j = jk.second;
            if (j->kind == 0 && j->batched && j->group == kv.first && j->state == TG_JOB_RUNNING && !j->cancel)
                mem.push_back(j);
        }
        if (mem.empty()) continue;
        tg_status st = group_capacity(g, (int)mem.size());
        int64_t pbase = 0, gbase = 0;
        for (size_t k = 0; st == TG_OK && k < mem.size(); ++k) {
            Job *j = mem[k];
            const tg_fit_desc &d = j->desc;
            BatchJob &b = g->table_host[k];
            b.store = j->grid->store;
            b.master = j->grid->master;
            b.grad = j->grad;
            b.m = j->grid->adam_m;
            b.v = j->grid->adam_v;
            b.shadow = j->grid->dtype == TG_F32 ? nullptr : j->grid->store;
            b.block = j->small;
            b.eval_pts = j->eval_pts;
            b.shape = j->sv;
            b.seed = d.seed;
            b.ncoef = j->grid->ncoef;
            b.pbase = pbase;
            b.npts = d.points_per_step;
            b.gbase = gbase;
            b.touched = j->touched;
            b.nv = j->grid->nv;
            b.K = j->grid->K;
            b.n_eval = d.eval_points;
            b.res = d.res;
            b.eval_every = d.eval_every;
            b.max_steps = d.max_steps;
            b.lazy = (d.flags & TG_FIT_LAZY_ADAM) ? 1 : 0;
            b.lambda_eik = d.lambda_eik;
            b.k_weight = d.k_weight;
            b.lr = d.lr;
            b.tol = d.tol;
            pbase += d.points_per_step;
            gbase += j->touched ? (j->grid->nv + 3) / 4 : (j->grid->ncoef + 3) / 4;
        }
        if (st == TG_OK) st = batch_step(g->table_host, g->table_dev, (int)mem.size(), g->order, g->dtype, g->status_dev,
                                         g->stream);
        if (st == TG_OK)
            st = cuda_status(cudaMemcpyAsync(g->status_host, g->status_dev, mem.size() * sizeof(DevStatus),
                                             cudaMemcpyDeviceToHost, g->stream), "server: status copy");
        if (st == TG_OK) st = cuda_status(cudaEventRecord(g->event, g->stream), "server: step event");
        if (st != TG_OK) {
            cudaStreamSynchronize(g->stream);     // whatever part of the step was launched
            cudaGetLastError();
            for (Job *j : mem) finish(s, j, TG_JOB_FAILED);
            continue;
        }
        for (Job *j : mem) j->in_flight = true;
        g->members.swap(mem);
        g->in_flight = true;
    }
    if (pending) {
        int p = 0;
        for (auto &kv : s->jobs) p += (kv.second->state == TG_JOB_QUEUED || kv.second->state == TG_JOB_RUNNING);
        *pending = p;
    }
    return TG_OK;
}

tg_status tg_poll(tg_server *s, tg_job_id id, tg_job_result *r)
{
    if (!s || !r) return fail(TG_EINVAL, "tg_poll: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return fail(TG_ENOTFOUND, "tg_poll: no job %lld", (long long)id);
    const Job *j = it->second;
    r->state = j->state;
    r->kind = j->kind;
    r->steps = j->steps;
    r->error = j->error;
    r->t_submit = j->t_submit;
    r->t_start = j->t_start;
    r->t_done = j->t_done;
    r->points = j->kind == 0 ? j->steps * j->desc.points_per_step : j->qn;
    r->bytes = j->bytes;
    return TG_OK;
}

tg_status tg_server_grid(tg_server *s, tg_job_id id, tg_grid **grid)
{
    if (!s || !grid) return fail(TG_EINVAL, "tg_server_grid: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end() || it->second->kind != 0 || !it->second->grid)
        return fail(TG_ENOTFOUND, "tg_server_grid: no resident grid for job %lld", (long long)id);
    *grid = it->second->grid;
    return TG_OK;
}

tg_status tg_cancel(tg_server *s, tg_job_id id)
{
    if (!s) return fail(TG_EINVAL, "tg_cancel: server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return fail(TG_ENOTFOUND, "tg_cancel: no job %lld", (long long)id);
    Job *j = it->second;
    if (j->state == TG_JOB_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), id), s->queue.end());
        j->state = TG_JOB_CANCELLED;
        j->t_done = s->now();
        return TG_OK;
    }
    if (j->state == TG_JOB_RUNNING) {
        if (j->kind == 1) return fail(TG_EBUSY, "tg_cancel: the query has been launched");
        j->cancel = true;
    }
    return TG_OK;
}

tg_status tg_release(tg_server *s, tg_job_id id)
{
    if (!s) return fail(TG_EINVAL, "tg_release: server is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return fail(TG_ENOTFOUND, "tg_release: no job %lld", (long long)id);
    Job *j = it->second;
    if (j->state == TG_JOB_RUNNING || j->state == TG_JOB_QUEUED) return fail(TG_EBUSY, "tg_release: job is not finished");
    if (j->kind == 0) {
        for (auto &kv : s->jobs)   // queries still pending on this grid keep it alive
            if (kv.second->kind == 1 && kv.second->grid_of == id &&
                (kv.second->state == TG_JOB_RUNNING || kv.second->state == TG_JOB_QUEUED))
                return fail(TG_EBUSY, "tg_release: queries on this grid are pending");
        if (j->grid && j->bytes <= s->used) s->used -= j->bytes;
    }
    free_job(j);
    delete j;
    s->jobs.erase(it);
    return TG_OK;
}

}  // extern "C"
