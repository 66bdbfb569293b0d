// server.cu -- continuous-batching detection server on top of the per-job
// contexts of runtime.cu (see mocd_server_* in include/mocd.h).
//
// Every running job owns a context (graph, population buffers, stream and
// per-generation CUDA graph). A scheduling round retires finished jobs,
// admits queued ones within the device-memory budget and enqueues more
// generation-graph launches for each running job on its own stream; the GPU
// runs the jobs' kernels concurrently, and jobs enter and leave between
// rounds without any re-capture. In background mode (mocd_server_start) a
// scheduler thread runs the rounds and admission workers do the host-side
// graph validation, upload and initialisation of the next jobs while the GPU
// is busy with the running ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mocd.h"
#include "mocd_internal.h"

namespace {

enum { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    int state = kQueued;
    int status = MOCD_OK;
    bool admitting = false;
    int64_t n = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col_idx;
    mocd_params params{};
    int32_t generations = 0;
    int32_t issued = 0;
    int issue_error = MOCD_OK;  // first failure while issuing generations
    bool cancel = false;        // cancellation requested while admitted
    bool cancel_marked = false; // a marker after its last issued generation is recorded
    Clock::time_point submitted, started;
    int64_t footprint = 0;
    double work = 0.0;  // (n + 2m) x (G + 1): the admission policy's size of the job
    mocd_ctx *ctx = nullptr;
    cudaEvent_t done = nullptr;
    // result
    int32_t count = 0, best = -1;
    std::vector<int32_t> labels;
    std::vector<double> f1, f2;
    std::vector<int64_t> intra, sumsq;
};

// Device bytes a job holds while it runs (mocd_job_footprint).
int64_t footprint(int64_t n, const int64_t *row_ptr, int32_t pop)
{
    int64_t b = 0;
    mocd_job_footprint(n, row_ptr, pop, &b);
    return b;
}

}  // namespace

struct mocd_server {
    int64_t budget = 0;
    int64_t used = 0;  // footprint of admitting and running jobs
    int32_t max_running = 1;
    int32_t depth = 1;
    int32_t policy = 0;  // 0: first come first served, 1: highest response ratio next
    double sec_per_work = 3e-10;  // measured run time per unit of work (moving average)
    int64_t next_id = 1;
    int32_t done_count = 0;
    int device = 0;
    std::deque<Job *> queue;
    std::vector<Job *> running;   // admitted (initialising or running)
    std::map<int64_t, Job *> jobs;
    std::mutex mu;
    std::condition_variable cv_admit;  // admission workers
    std::vector<std::thread> threads;
    std::atomic<bool> stop{false};
    bool background = false;
    std::deque<Job *> to_admit;
};

namespace {

// Frees a job's device state (its context and completion event).
void release(Job *j)
{
    if (j->done) cudaEventDestroy(j->done);
    j->done = nullptr;
    if (j->ctx) mocd_destroy(j->ctx);
    j->ctx = nullptr;
}

void finish(mocd_server *s, Job *j, int state, int status)
{
    release(j);
    s->used -= j->footprint;
    j->state = state;
    j->status = status;
    s->done_count += 1;
}

// Host-side admission work (validation, upload, initialisation); no lock held.
int admit_job(Job *j)
{
    int rc = mocd_graph_upload(&j->ctx, j->n, j->row_ptr.data(), j->col_idx.data(), nullptr);
    if (rc == MOCD_OK) rc = mocd_population_init(j->ctx, &j->params);
    if (rc == MOCD_OK && cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming) != cudaSuccess)
        rc = MOCD_ERR_CUDA;
    std::vector<int64_t>().swap(j->row_ptr);
    std::vector<int32_t>().swap(j->col_idx);
    return rc;
}

// Next queued job to admit under the policy: the front of the queue, or the
// highest response ratio (waiting time + estimated run time) / estimated run
// time, the run time estimated from the job's size and the measured time per
// unit of work of the jobs completed so far. Short jobs go first, and a
// waiting job's ratio grows until it is admitted, so no job starves.
std::deque<Job *>::iterator pick(mocd_server *s)
{
    auto it = s->queue.begin();
    if (s->policy == 1) {
        const Clock::time_point now = Clock::now();
        double best = -1.0;
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
            const double service = std::max((*q)->work * s->sec_per_work, 1e-6);
            const double wait = std::chrono::duration<double>(now - (*q)->submitted).count();
            const double ratio = (wait + service) / service;
            if (ratio > best) {
                best = ratio;
                it = q;
            }
        }
    }
    return it;
}

// One scheduling round; the lock is held by the caller. In background mode
// admitted jobs are handed to the workers instead of being initialised here.
void round_locked(mocd_server *s, std::unique_lock<std::mutex> &lock)
{
    // 1. Retire jobs whose last generation has completed, and cancelled jobs
    // once the generations already issued for them have completed.
    for (size_t k = 0; k < s->running.size();) {
        Job *j = s->running[k];
        if (!j->admitting && j->cancel && !j->cancel_marked) {
            // Nothing more is issued; the marker follows the work in flight.
            if (mocd::record_on_stream(j->ctx, j->done) != MOCD_OK) j->issue_error = MOCD_ERR_CUDA;
            j->cancel_marked = true;
            j->issued = j->generations;
        }
        if (j->admitting || j->issued < j->generations) {
            ++k;
            continue;
        }
        if (j->issue_error != MOCD_OK) {
            // A generation or the completion marker could not be issued: the
            // population did not reach its last generation, so the job fails
            // (its stream is drained before the context is released).
            finish(s, j, kFailed, j->issue_error);
            s->running.erase(s->running.begin() + k);
            continue;
        }
        const cudaError_t q = cudaEventQuery(j->done);
        if (q == cudaErrorNotReady) {
            ++k;
            continue;
        }
        if (q != cudaSuccess) {
            finish(s, j, kFailed, MOCD_ERR_CUDA);
        } else if (j->cancel) {
            finish(s, j, kCancelled, MOCD_ERR_CANCELLED);
        } else {
            const int64_t cap = j->params.pop_size;
            j->labels.resize((size_t)cap * (size_t)j->n);
            j->f1.resize(cap);
            j->f2.resize(cap);
            j->intra.resize(cap);
            j->sumsq.resize(cap);
            const int rc = mocd_pareto_front(j->ctx, (int32_t)cap, &j->count, j->labels.data(), j->f1.data(),
                                             j->f2.data(), j->intra.data(), j->sumsq.data(), &j->best);
            if (rc == MOCD_OK) j->labels.resize((size_t)j->count * (size_t)j->n);
            if (rc == MOCD_OK && j->work > 0.0) {
                const double took = std::chrono::duration<double>(Clock::now() - j->started).count();
                s->sec_per_work = 0.8 * s->sec_per_work + 0.2 * (took / j->work);
            }
            finish(s, j, rc == MOCD_OK ? kDone : kFailed, rc);
        }
        s->running.erase(s->running.begin() + k);
    }
    // 2. Admit queued jobs while they fit.
    while (!s->queue.empty() && (int32_t)s->running.size() < s->max_running) {
        auto it = pick(s);
        Job *j = *it;
        if (j->footprint > s->budget) {
            s->queue.erase(it);
            j->state = kFailed;
            j->status = MOCD_ERR_OUT_OF_MEMORY;
            s->done_count += 1;
            continue;
        }
        if (s->used + j->footprint > s->budget) break;
        s->queue.erase(it);
        s->used += j->footprint;
        j->admitting = true;
        j->started = Clock::now();
        s->running.push_back(j);
        if (s->background) {
            s->to_admit.push_back(j);
            s->cv_admit.notify_one();
        } else {
            lock.unlock();
            const int rc = admit_job(j);
            lock.lock();
            j->admitting = false;
            if (rc) {
                for (size_t k = 0; k < s->running.size(); ++k)
                    if (s->running[k] == j) s->running.erase(s->running.begin() + k);
                finish(s, j, kFailed, rc);
            } else {
                j->state = kRunning;
            }
        }
    }
    // 3. Enqueue more generations of every running job on its own stream.
    for (Job *j : s->running) {
        if (j->admitting || j->cancel) continue;
        const int32_t k = j->generations - j->issued < s->depth ? j->generations - j->issued : s->depth;
        if (k <= 0) continue;
        int rc = mocd_generation(j->ctx, k);
        j->issued += k;
        // Completion marker after the job's last generation, on its own stream.
        if (rc == MOCD_OK && j->issued == j->generations) rc = mocd::record_on_stream(j->ctx, j->done);
        if (rc) {
            // Nothing more is issued; retirement fails the job with this status.
            j->issue_error = rc;
            j->issued = j->generations;
        }
    }
}

void admission_worker(mocd_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        s->cv_admit.wait(lock, [&] { return s->stop || !s->to_admit.empty(); });
        if (s->stop) break;
        Job *j = s->to_admit.front();
        s->to_admit.pop_front();
        lock.unlock();
        const int rc = admit_job(j);
        lock.lock();
        j->admitting = false;
        if (rc) {
            for (size_t k = 0; k < s->running.size(); ++k)
                if (s->running[k] == j) s->running.erase(s->running.begin() + k);
            finish(s, j, kFailed, rc);
        } else {
            j->state = kRunning;
        }
    }
}

void scheduler(mocd_server *s)
{
    cudaSetDevice(s->device);
    while (!s->stop) {
        {
            std::unique_lock<std::mutex> lock(s->mu);
            round_locked(s, lock);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

}  // namespace

extern "C" {

int mocd_job_footprint(int64_t n, const int64_t *row_ptr, int32_t pop_size, int64_t *bytes)
{
    if (!bytes || !row_ptr || n < 1 || pop_size < 1 || pop_size > mocd::kMaxPop) return MOCD_ERR_INVALID_ARG;
    const int64_t nnz = row_ptr[n];
    int64_t deferred_nodes = 0;  // degree 33 .. kDeferMax and hubs: deferred mutation votes
    int64_t dmax = 0;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        deferred_nodes += ((d > 32 && d <= mocd::kDeferMax) || d > mocd::kSharedTableMax) ? 1 : 0;
        dmax = d > dmax ? d : dmax;
    }
    // The hub count tables: per warp of the hub kernel (at most four per SM),
    // 2 x the smallest power of two >= max(1024, 2 dmax) ints, 1 GiB at most.
    int64_t hub_tables = 0;
    if (dmax > mocd::kSharedTableMax) {
        int64_t hs = 1024;
        while (hs < 2 * dmax) hs <<= 1;
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
        }
        const int64_t per_warp = 2 * hs * 4;
        int64_t warps = ((int64_t)1 << 30) / per_warp;
        if (warps > 4 * (int64_t)sms) warps = 4 * (int64_t)sms;
        if (warps < 4) warps = 4;
        hub_tables = (warps & ~3ll) * per_warp;
    }
    const int64_t W = (pop_size + 3) & ~3;
    const int64_t labels = 4 * n * W * 4;         // P halves, Q, post-crossover children
    const int64_t hist = W * n * 4;               // degree histogram
    const int64_t mutation = n * 4 + deferred_nodes * pop_size * 8 + hub_tables;  // hints, deferred votes
    const int64_t graph = 2 * (n + 1) * 4 + (nnz + nnz / 2) * 4 + n * 4 + 4;  // CSR, oriented CSR, order, flag
    const int64_t front = (int64_t)pop_size * n * 4 + 2 * mocd::kMaxPop * 4;  // front download
    const int64_t fixed = (int64_t)1 << 20;       // small state, graph executable, events
    *bytes = labels + hist + mutation + graph + front + fixed;
    return MOCD_OK;
}

int mocd_server_create(mocd_server **out, int64_t hbm_budget_bytes, int32_t max_running, int32_t depth)
{
    if (!out) return MOCD_ERR_INVALID_ARG;
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_running < 1 || depth < 1) return MOCD_ERR_INVALID_ARG;
    mocd_server *s = new (std::nothrow) mocd_server();
    if (!s) return MOCD_ERR_OUT_OF_MEMORY;
    s->budget = hbm_budget_bytes;
    s->max_running = max_running;
    s->depth = depth;
    if (cudaGetDevice(&s->device) != cudaSuccess) s->device = 0;
    *out = s;
    return MOCD_OK;
}

int mocd_server_start(mocd_server *s, int32_t admission_threads, int32_t policy)
{
    if (!s || admission_threads < 1 || admission_threads > 16 || policy < 0 || policy > 1)
        return MOCD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->background) return MOCD_ERR_INVALID_ARG;
    s->background = true;
    s->policy = policy;
    lock.unlock();
    try {
        for (int32_t k = 0; k < admission_threads; ++k) s->threads.emplace_back(admission_worker, s);
        s->threads.emplace_back(scheduler, s);
    } catch (...) {
        return MOCD_ERR_OUT_OF_MEMORY;
    }
    return MOCD_OK;
}

int mocd_server_submit(mocd_server *s, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const mocd_params *params, int32_t generations, int64_t *job_id)
{
    if (!s || !row_ptr || !params || !job_id || n < 1 || generations < 0) return MOCD_ERR_INVALID_ARG;
    if (row_ptr[n] > 0 && !col_idx) return MOCD_ERR_INVALID_ARG;
    Job *j = new (std::nothrow) Job();
    if (!j) return MOCD_ERR_OUT_OF_MEMORY;
    j->n = n;
    j->row_ptr.assign(row_ptr, row_ptr + n + 1);
    if (row_ptr[n] > 0) j->col_idx.assign(col_idx, col_idx + row_ptr[n]);
    j->params = *params;
    j->generations = generations;
    j->footprint = footprint(n, row_ptr, params->pop_size);
    j->work = (double)(n + row_ptr[n]) * (double)(generations + 1);
    j->submitted = Clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    j->id = s->next_id++;
    s->queue.push_back(j);
    s->jobs[j->id] = j;
    *job_id = j->id;
    return MOCD_OK;
}

int mocd_server_step(mocd_server *s, int32_t *running, int32_t *queued, int32_t *done)
{
    if (!s) return MOCD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    if (!s->background) round_locked(s, lock);
    if (running) *running = (int32_t)s->running.size();
    if (queued) *queued = (int32_t)s->queue.size();
    if (done) *done = s->done_count;
    return MOCD_OK;
}

int mocd_server_cancel(mocd_server *s, int64_t job_id)
{
    if (!s) return MOCD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return MOCD_ERR_INVALID_ARG;
    Job *j = it->second;
    if (j->state == kCancelled) return MOCD_OK;
    if (j->state == kDone || j->state == kFailed) return MOCD_ERR_INVALID_ARG;
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
        if (*q == j) {
            s->queue.erase(q);
            j->state = kCancelled;
            j->status = MOCD_ERR_CANCELLED;
            std::vector<int64_t>().swap(j->row_ptr);
            std::vector<int32_t>().swap(j->col_idx);
            s->done_count += 1;
            return MOCD_OK;
        }
    }
    j->cancel = true;  // admitted: retired by a later round
    return MOCD_OK;
}

int mocd_server_job_state(mocd_server *s, int64_t job_id, int32_t *state, int32_t *status)
{
    if (!s || !state) return MOCD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return MOCD_ERR_INVALID_ARG;
    *state = it->second->state;
    if (status) *status = it->second->status;
    return MOCD_OK;
}

int mocd_server_result(mocd_server *s, int64_t job_id, int32_t cap, int32_t *count, int32_t *labels,
                       double *f1, double *f2, int64_t *intra, int64_t *sumsq, int32_t *best)
{
    if (!s || !count || cap < 0) return MOCD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return MOCD_ERR_INVALID_ARG;
    Job *j = it->second;
    if (j->state == kFailed || j->state == kCancelled) return j->status;
    if (j->state != kDone) return MOCD_ERR_NOT_READY;
    *count = j->count;
    if (j->count > cap) return MOCD_ERR_BUFFER_TOO_SMALL;
    for (int32_t k = 0; k < j->count; ++k) {
        if (f1) f1[k] = j->f1[k];
        if (f2) f2[k] = j->f2[k];
        if (intra) intra[k] = j->intra[k];
        if (sumsq) sumsq[k] = j->sumsq[k];
    }
    if (labels)
        for (size_t k = 0; k < j->labels.size(); ++k) labels[k] = j->labels[k];
    if (best) *best = j->best;
    return MOCD_OK;
}

void mocd_server_destroy(mocd_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_admit.notify_all();
    for (std::thread &t : s->threads) t.join();
    for (auto &kv : s->jobs) {
        release(kv.second);
        delete kv.second;
    }
    delete s;
}

}  // extern "C"
