// runtime.cu -- host side of the C ABI declared in include/mocd.h.
//
// A context owns the uploaded CSR, the population buffers (node-major label
// rows, see mocd_internal.h) and one CUDA graph that runs a whole generation
// of Alg. 1: crossover -> mutation (which also builds the degree histogram of
// the offspring) -> evaluate -> select.
// Every kernel reads the generation number from device memory, so the same
// graph is replayed for every generation with no host work in between.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <unistd.h>

#include "mocd.h"
#include "mocd_internal.h"

using namespace mocd;

namespace {

constexpr int kStages = 4;

}  // namespace

struct mocd_ctx {
    int device = 0;
    int sms = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    int64_t n = 0, m = 0;
    int dmax = 0;
    int64_t n_defer[3] = {0, 0, 0};  // nodes of degree 33..64, 65..128 and > 512 (deferred mutation votes)
    int32_t *d_row_ptr = nullptr;
    int32_t *d_col_idx = nullptr;
    int32_t *d_order = nullptr;   // nodes by degree, descending
    // The offspring evaluation's adjacency: each undirected edge once, listed
    // at its endpoint of lower (degree, id), so that the label rows it reads
    // are those of the higher-degree endpoints (fewer, each read more often:
    // more of them stay in L2). eptr [n + 1], eidx [m].
    int32_t *d_eptr = nullptr;
    int32_t *d_eidx = nullptr;

    // Population.
    bool ready = false;
    mocd_params params{};
    GenParams gp{};
    PopState ps{};
    int W = 0;
    size_t pop_cells = 0;   // n * W of the allocated label buffers
    size_t hist_cap = 0;    // entries of ps.hist
    size_t hint_cap = 0;    // entries of ps.hint
    size_t dlist_cap = 0;   // entries of ps.dlist
    size_t hub_cap = 0;     // entries of ps.hub_table
    void *d_small = nullptr;
    int grid_eval = 0, grid_cross = 0, grid_mut = 0;
    int grid_eval_intra = 0, grid_vote64 = 0, grid_vote128 = 0;
    int occ_eval = 0, occ_cross = 0, occ_mut = 0;  // occupancy-limited grids
    int occ_eval_intra = 0;
    int nodes_per_warp = 1;                         // launch shape (autotuned for batches)
    int32_t host_gen = 0;   // generations run since init
    int32_t version = 0;    // bumped whenever the population is (re)built
    uint32_t gen_host_value = 0;

    // Generation graphs: [0] plain, [1] with stage events (timing); each is
    // captured on first use and both stay valid until the population or the
    // launch shape changes.
    cudaGraph_t graph[2] = {};
    cudaGraphExec_t graph_exec[2] = {};
    bool timing = false;
    bool timing_valid = false;
    cudaEvent_t ev[kStages + 1] = {};

    // Scratch for downloads and for mocd_evaluate.
    int32_t *d_im = nullptr;   // individual-major [rows][n]
    size_t im_cap = 0;
    int32_t *d_nm = nullptr;   // node-major [n][128]
    size_t nm_cap = 0;
    unsigned long long *d_eval_acc = nullptr;
    uint32_t *d_eval_hist = nullptr;
    size_t eval_hist_cap = 0;
    int32_t *d_idx = nullptr;

    // Scratch for mocd_front_stats.
    unsigned long long *d_volsize = nullptr;  // [count][n]
    size_t volsize_cap = 0;
    uint32_t *d_cut = nullptr;                // [count][n]
    size_t cut_cap = 0;
    unsigned long long *d_stats = nullptr;    // acc words, then out [4][kMaxPop]
};

namespace {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return MOCD_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MOCD_ERR_OUT_OF_MEMORY;
    }
    return MOCD_ERR_CUDA;
}

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_status(e_);\
    } while (0)

// Device memory is stream-ordered (allocated and freed on the owner's
// stream): releasing one context never synchronises the device, so other
// contexts (batch members, server jobs) keep running. It comes from one
// memory pool per device owned by the library, which keeps freed memory
// for the next context instead of returning it to the driver at every
// synchronisation (mapping fresh memory costs a job hundreds of
// microseconds); mocd_pool_trim returns it.
constexpr int kMaxDevices = 64;

cudaError_t library_pool(int dev, cudaMemPool_t *out)
{
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

void dev_free(void *p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

template <class T>
int grow(cudaStream_t st, T **p, size_t *cap, size_t need)
{
    if (*p && *cap >= need) return MOCD_OK;
    dev_free(*p, st);
    *p = nullptr;
    *cap = 0;
    void *q = nullptr;
    cudaError_t e = dev_alloc(&q, std::max<size_t>(need, 1) * sizeof(T), st);
    if (e != cudaSuccess) return cuda_status(e);
    *p = static_cast<T *>(q);
    *cap = need;
    return MOCD_OK;
}

void drop_graphs(mocd_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph_exec[k]) cudaGraphExecDestroy(c->graph_exec[k]);
        if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
        c->graph_exec[k] = nullptr;
        c->graph[k] = nullptr;
    }
}

void free_population(mocd_ctx *c)
{
    drop_graphs(c);
    dev_free(c->ps.buf[0], c->stream);
    dev_free(c->ps.buf[1], c->stream);
    dev_free(c->ps.q, c->stream);
    dev_free(c->ps.c, c->stream);
    dev_free(c->ps.hist, c->stream);
    dev_free(c->ps.hint, c->stream);
    dev_free(c->ps.dlist, c->stream);
    dev_free(c->ps.hub_table, c->stream);
    dev_free(c->d_small, c->stream);
    c->ps = PopState{};
    c->d_small = nullptr;
    c->pop_cells = 0;
    c->hist_cap = 0;
    c->hint_cap = 0;
    c->dlist_cap = 0;
    c->hub_cap = 0;
    c->ready = false;
}

int label_bits_for(int64_t n)
{
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

int check_params(const mocd_ctx *c, const mocd_params *p)
{
    if (!p) return MOCD_ERR_INVALID_ARG;
    if (p->pop_size < 1 || p->pop_size > kMaxPop) return MOCD_ERR_INVALID_ARG;
    if (p->n_parents < 1 || p->n_parents > kMaxParents) return MOCD_ERR_INVALID_ARG;
    if (!(p->p_crossover >= 0.0 && p->p_crossover <= 1.0)) return MOCD_ERR_INVALID_ARG;
    if (!(p->p_mutation >= 0.0 && p->p_mutation <= 1.0)) return MOCD_ERR_INVALID_ARG;
    if (p->init_mode != 0 && p->init_mode != 1) return MOCD_ERR_INVALID_ARG;
    return MOCD_OK;
}

// Grids of the node-parallel kernels: enough warps for nodes_per_warp nodes
// each, never more than fit on the GPU at once (the kernels stride over the
// remaining nodes). Small graphs get small grids, which matters when several
// instances share the GPU.
void size_grids(mocd_ctx *c)
{
    const long long n = c->n;
    auto shape = [&](int occ, int warps_per_block) {
        const long long per_block = (long long)warps_per_block * c->nodes_per_warp;
        const long long want = (n + per_block - 1) / per_block;
        return (int)std::max<long long>(1, std::min<long long>(occ, want));
    };
    c->grid_eval = shape(c->occ_eval, kBlock / 32);
    c->grid_eval_intra = shape(c->occ_eval_intra, kBlock / 32);
    c->grid_cross = shape(c->occ_cross, kBlock / 32);
    c->grid_mut = shape(c->occ_mut, mutation_warps_per_block());
}

// Allocate (or reuse) the population buffers for params and fill gp / ps.
int prepare_population(mocd_ctx *c, const mocd_params *p)
{
    const int W = (p->pop_size + 3) & ~3;
    const size_t cells = (size_t)c->n * (size_t)W;
    drop_graphs(c);
    if (c->pop_cells != cells) {
        free_population(c);
        int32_t *b[4] = {};
        for (int k = 0; k < 4; ++k) {
            void *q = nullptr;
            cudaError_t e = dev_alloc(&q, cells * sizeof(int32_t), c->stream);
            if (e != cudaSuccess) {
                for (int j = 0; j < k; ++j) dev_free(b[j], c->stream);
                return cuda_status(e);
            }
            b[k] = static_cast<int32_t *>(q);
        }
        c->ps.buf[0] = b[0];
        c->ps.buf[1] = b[1];
        c->ps.q = b[2];
        c->ps.c = b[3];
        // Small per-generation state in one allocation.
        const size_t bytes = sizeof(unsigned long long) * 2 * kMaxPop   // acc
                             + sizeof(int64_t) * 2 * kMaxPop              // pk
                             + sizeof(int64_t) * 4 * kMaxPop              // rk
                             + sizeof(int32_t) * kMaxPop                  // prank
                             + sizeof(int32_t) * kMaxPop                  // keep
                             + sizeof(int32_t) * kMaxPop * kMaxParents    // par_r
                             + sizeof(int32_t) * kMaxPop                  // copy_r
                             + sizeof(int32_t) * (2 + kMaxPop)            // front
                             + sizeof(int64_t) * 2 * kMaxPop              // fint
                             + sizeof(double) * 2 * kMaxPop               // fval
                             + 64;                                        // gen, alignment
        void *s = nullptr;
        cudaError_t e = dev_alloc(&s, bytes, c->stream);
        if (e != cudaSuccess) {
            free_population(c);  // the label buffers too: pop_cells stays 0
            return cuda_status(e);
        }
        c->d_small = s;
        c->pop_cells = cells;  // every population buffer exists from here on
        char *q = static_cast<char *>(s);
        c->ps.acc = reinterpret_cast<unsigned long long *>(q); q += sizeof(unsigned long long) * 2 * kMaxPop;
        c->ps.pk = reinterpret_cast<int64_t *>(q); q += sizeof(int64_t) * 2 * kMaxPop;
        c->ps.rk = reinterpret_cast<int64_t *>(q); q += sizeof(int64_t) * 4 * kMaxPop;
        c->ps.prank = reinterpret_cast<int32_t *>(q); q += sizeof(int32_t) * kMaxPop;
        c->ps.keep = reinterpret_cast<int32_t *>(q); q += sizeof(int32_t) * kMaxPop;
        c->ps.par_r = reinterpret_cast<int32_t *>(q); q += sizeof(int32_t) * kMaxPop * kMaxParents;
        c->ps.copy_r = reinterpret_cast<int32_t *>(q); q += sizeof(int32_t) * kMaxPop;
        c->ps.front = reinterpret_cast<int32_t *>(q); q += sizeof(int32_t) * (2 + kMaxPop);
        q = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(q) + 15) & ~uintptr_t(15));
        c->ps.fint = reinterpret_cast<int64_t *>(q); q += sizeof(int64_t) * 2 * kMaxPop;
        c->ps.fval = reinterpret_cast<double *>(q); q += sizeof(double) * 2 * kMaxPop;
        c->ps.gen = reinterpret_cast<uint32_t *>(q);
        c->ps.dcount = reinterpret_cast<int *>(q + 16);  // [3], within the 64-byte tail
        CK(cudaMemsetAsync(s, 0, bytes, c->stream));
        CK(cudaMemsetAsync(c->ps.q, 0, cells * sizeof(int32_t), c->stream));
        CK(cudaMemsetAsync(c->ps.buf[0], 0, cells * sizeof(int32_t), c->stream));
    }
    const size_t hist_need = (size_t)W * (size_t)c->n;
    // The deferred-vote list holds every pair a generation can defer; its
    // per-class counts are 32-bit.
    if ((int64_t)p->pop_size * (c->n_defer[0] + c->n_defer[1] + c->n_defer[2]) > INT_MAX)
        return MOCD_ERR_INVALID_ARG;
    const size_t defer_need = (size_t)p->pop_size * (size_t)(c->n_defer[0] + c->n_defer[1] + c->n_defer[2]);
    // Hubs above the shared table's degree: one count table of hub_hs slots
    // (keys and counts) per warp of the hub kernel, at most 1 GiB in all.
    int hub_hs = 0, hub_warps = 0;
    if (c->dmax > kSharedTableMax) {
        hub_hs = 1024;
        while (hub_hs < 2 * c->dmax) hub_hs <<= 1;
        const int64_t per_warp = 2 * (int64_t)hub_hs * (int64_t)sizeof(int);
        const int64_t fit = ((int64_t)1 << 30) / per_warp;
        hub_warps = (int)std::max<int64_t>(4, std::min<int64_t>((int64_t)c->sms * 4, fit)) & ~3;
    }
    {
        int rc = grow(c->stream, &c->ps.hist, &c->hist_cap, hist_need);
        if (rc) return rc;
        if ((rc = grow(c->stream, &c->ps.hint, &c->hint_cap, (size_t)c->n))) return rc;
        if ((rc = grow(c->stream, &c->ps.dlist, &c->dlist_cap, defer_need))) return rc;
        if (hub_hs > 0 &&
            (rc = grow(c->stream, &c->ps.hub_table, &c->hub_cap, (size_t)hub_warps * 2 * (size_t)hub_hs)))
            return rc;
    }
    c->W = W;
    c->params = *p;
    c->version += 1;
    GenParams &gp = c->gp;
    gp.n = (int)c->n;
    gp.W = W;
    gp.np = p->pop_size;
    gp.es = p->n_parents;
    gp.label_bits = label_bits_for(c->n);
    int hs = 0;  // shared count table of degrees kDeferMax + 1 .. kSharedTableMax
    if (c->dmax > kDeferMax) {
        hs = 256;
        while (hs < 2 * std::min(c->dmax, kSharedTableMax)) hs <<= 1;
    }
    gp.hash_size = hs;
    gp.defer_cap[0] = (int)((int64_t)p->pop_size * c->n_defer[0]);
    gp.defer_cap[1] = (int)((int64_t)p->pop_size * c->n_defer[1]);
    gp.defer_cap[2] = (int)((int64_t)p->pop_size * c->n_defer[2]);
    gp.hub_hs = hub_hs;
    gp.hub_warps = hub_warps;
    {
        // The degree 33..64 vote's network holds the largest degree of that
        // class in the graph: 40, 48, 56 or 64 entries.
        const int64_t d0 = std::min<int64_t>(std::max<int64_t>(c->dmax, 33), 64);
        gp.vote_n0 = (int)((d0 + 7) / 8 * 8);
    }
    gp.m = c->m;
    gp.key0 = (uint32_t)p->seed;
    gp.key1 = (uint32_t)(p->seed >> 32);
    gp.thr_c = (unsigned long long)floor(p->p_crossover * 4294967296.0);
    gp.thr_m = (unsigned long long)floor(p->p_mutation * 4294967296.0);
    c->occ_eval = grid_for_eval(c->sms);
    c->occ_eval_intra = grid_for_eval_intra(c->sms);
    grid_for_votes(c->sms, gp.vote_n0, &c->grid_vote64, &c->grid_vote128);
    c->occ_cross = grid_for_crossover(c->sms, gp.es);
    int smem = 0;
    c->occ_mut = grid_for_mutation(c->sms, gp.hash_size, &smem);
    size_grids(c);
    return MOCD_OK;
}

int clear_eval_state(mocd_ctx *c, uint32_t *hist, size_t hist_entries, unsigned long long *acc)
{
    CK(cudaMemsetAsync(hist, 0, hist_entries * sizeof(uint32_t), c->stream));
    CK(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * kMaxPop, c->stream));
    return MOCD_OK;
}

// Timing events become event-record nodes of the captured graph.
cudaError_t mark(mocd_ctx *c, int k, cudaStream_t st)
{
    return cudaEventRecordWithFlags(c->ev[k], st, cudaEventRecordExternal);
}

// One generation of Alg. 1 on stream st. The mutation kernel also clears the
// accumulators and adds the offspring's degrees to the histogram that the
// evaluation then squares (and zeroes).
int issue_generation(mocd_ctx *c, cudaStream_t st, bool events, bool with_select = true)
{
    const GenParams &gp = c->gp;
    const PopState &ps = c->ps;
    if (events) CK(mark(c, 0, st));
    CK(launch_crossover(gp, ps, c->grid_cross, st));
    if (events) CK(mark(c, 1, st));
    CK(launch_mutation(gp, ps, c->d_row_ptr, c->d_col_idx, c->d_order, c->grid_mut, c->grid_vote64,
                       c->grid_vote128, st));
    if (events) CK(mark(c, 2, st));
    CK(launch_evaluate_offspring(gp.n, gp.W, gp.np, c->d_eptr, c->d_eidx, ps.q, ps.hist, ps.acc,
                                 c->grid_eval_intra, st, c->d_order));
    if (events) CK(mark(c, 3, st));
    if (!with_select) return MOCD_OK;  // a batch selects all its members in one launch
    CK(launch_select(gp, ps, 1, st));
    if (events) CK(mark(c, 4, st));
    return MOCD_OK;
}

// Capture the generation graph of the current timing mode (if missing).
int build_graph(mocd_ctx *c)
{
    const int k = c->timing ? 1 : 0;
    if (c->graph_exec[k]) return MOCD_OK;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = issue_generation(c, c->stream, c->timing);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CK(e);
    c->graph[k] = g;
    CK(cudaGraphInstantiate(&c->graph_exec[k], g, 0));
    return MOCD_OK;
}

// Evaluate, rank and draw the first tournament of a population whose labels
// are in the P half of generation base_gen (buf[(base_gen + 1) & 1]).
int start_population(mocd_ctx *c, uint32_t base_gen)
{
    const GenParams &gp = c->gp;
    PopState &ps = c->ps;
    int32_t *phalf = ps.buf[(base_gen + 1u) & 1u];
    int rc = clear_eval_state(c, ps.hist, (size_t)gp.W * (size_t)gp.n, ps.acc);
    if (rc) return rc;
    // No mutation history yet: every node starts with the Misra-Gries pass.
    CK(cudaMemsetAsync(ps.hint, 0, sizeof(uint32_t) * (size_t)gp.n, c->stream));
    CK(launch_evaluate(gp.n, gp.W, gp.np, c->d_row_ptr, c->d_col_idx, phalf, ps.hist, ps.acc,
                       c->grid_eval, c->stream));
    // Generations expect a zero histogram (the mutation kernel adds into it).
    CK(cudaMemsetAsync(ps.hist, 0, (size_t)gp.W * (size_t)gp.n * sizeof(uint32_t), c->stream));
    c->gen_host_value = base_gen;
    CK(cudaMemcpyAsync(ps.gen, &c->gen_host_value, sizeof(uint32_t), cudaMemcpyHostToDevice, c->stream));
    CK(launch_select(gp, ps, 0, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->host_gen = (int32_t)base_gen;
    drop_graphs(c);
    rc = build_graph(c);
    if (rc) return rc;
    c->ready = true;
    c->timing_valid = false;
    return MOCD_OK;
}

int validate_labels(const mocd_ctx *c, const int32_t *labels, size_t count)
{
    const int32_t n = (int32_t)c->n;
    for (size_t k = 0; k < count; ++k)
        if (labels[k] < 0 || labels[k] >= n) return MOCD_ERR_INVALID_ARG;
    return MOCD_OK;
}

// Host worker threads for the data-parallel host steps (graph validation,
// mapping download pages). Created once per process on first use and kept:
// a host step of a small job is shorter than creating and joining its
// threads. run(T, f) calls f(t) for t in [0, T), chunk 0 on the calling
// thread, and returns when all have finished. One step uses the workers at a
// time; a call that finds them busy (another host thread of the caller, e.g.
// a server admission thread) runs its chunks itself.
class WorkerPool {
  public:
    static WorkerPool &get()
    {
        static std::mutex init_mu;
        static WorkerPool *pool = nullptr;
        static pid_t owner = 0;
        std::lock_guard<std::mutex> lock(init_mu);
        // A forked child has none of the parent's threads: it makes its own
        // pool (the parent's object is left as it is).
        if (!pool || owner != getpid()) {
            const unsigned hw = std::thread::hardware_concurrency();
            pool = new WorkerPool((int)std::min<unsigned>(hw ? hw : 1, 16) - 1);
            owner = getpid();
        }
        return *pool;
    }

    int width() const { return (int)threads_.size() + 1; }

    void run(int T, const std::function<void(int)> &f)
    {
        std::unique_lock<std::mutex> busy(run_mu_, std::try_to_lock);
        if (T <= 1 || threads_.empty() || !busy.owns_lock()) {
            for (int t = 0; t < T; ++t) f(t);
            return;
        }
        {
            std::lock_guard<std::mutex> lock(mu_);
            job_ = &f;
            chunks_ = T;
            next_ = 1;
            pending_ = T - 1;
            ++epoch_;
        }
        cv_work_.notify_all();
        f(0);
        for (;;) {  // the caller takes chunks too
            int t;
            {
                std::lock_guard<std::mutex> lock(mu_);
                if (next_ >= chunks_) break;
                t = next_++;
            }
            f(t);
            std::lock_guard<std::mutex> lock(mu_);
            --pending_;
        }
        std::unique_lock<std::mutex> lock(mu_);
        cv_done_.wait(lock, [&] { return pending_ == 0; });
        job_ = nullptr;
    }

  private:
    explicit WorkerPool(int workers)
    {
        for (int k = 0; k < workers; ++k) {
            std::thread th([this] { loop(); });
            th.detach();  // the pool lives until the process ends
            threads_.push_back(std::move(th));
        }
    }

    void loop()
    {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lock(mu_);
        for (;;) {
            cv_work_.wait(lock, [&] { return epoch_ != seen && next_ < chunks_; });
            seen = epoch_;
            while (next_ < chunks_) {
                const int t = next_++;
                const std::function<void(int)> *f = job_;
                lock.unlock();
                (*f)(t);
                lock.lock();
                if (--pending_ == 0) cv_done_.notify_all();
            }
        }
    }

    std::mutex run_mu_;  // one host step at a time
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::vector<std::thread> threads_;
    const std::function<void(int)> *job_ = nullptr;
    int chunks_ = 0, next_ = 0, pending_ = 0;
    uint64_t epoch_ = 0;
};

// Runs f(v0, v1) on contiguous node ranges of about equal edge counts, on the
// worker pool (inline when the graph is small).
template <class F>
void parallel_rows(const int64_t *row_ptr, int64_t n, F f)
{
    const int64_t nnz = row_ptr[n];
    WorkerPool &pool = WorkerPool::get();
    const int64_t T = std::min<int64_t>(pool.width(), (nnz + n) / (1 << 15) + 1);
    if (T <= 1) {
        f(0, n);
        return;
    }
    std::vector<int64_t> cut((size_t)T + 1);
    cut[0] = 0;
    cut[(size_t)T] = n;
    for (int64_t t = 1; t < T; ++t)
        cut[(size_t)t] = std::lower_bound(row_ptr, row_ptr + n, nnz * t / T) - row_ptr;
    pool.run((int)T, [&](int t) { f(cut[(size_t)t], cut[(size_t)t + 1]); });
}

// Writes one zero per 4 KiB of [p, p + bytes) on the worker pool: maps every
// page of a buffer that is about to be overwritten, so that the copy into it
// does not fault page by page.
void prefault(void *p, size_t bytes)
{
    constexpr size_t kPage = 4096;
    const size_t pages = bytes / kPage;
    if (pages < 256) return;
    volatile char *base = static_cast<volatile char *>(p);
    WorkerPool &pool = WorkerPool::get();
    const size_t T = std::min<size_t>((size_t)pool.width(), pages / 256);
    pool.run((int)T, [&](int t) {
        for (size_t k = pages * (size_t)t / T; k < pages * ((size_t)t + 1) / T; ++k) base[k * kPage] = 0;
    });
}

// The status of the lowest-numbered failing row among concurrent checks.
struct FirstError {
    std::mutex mu;
    int64_t row = INT64_MAX;
    int code = MOCD_OK;
    void record(int64_t v, int rc)
    {
        std::lock_guard<std::mutex> lock(mu);
        if (v < row) {
            row = v;
            code = rc;
        }
    }
    int status() { return code; }
};

// Individual-major labels of `count` members of R = (P half, Q), given by
// their R indices on the host.
int download_r(mocd_ctx *c, const int32_t *ridx, int count, int32_t *labels)
{
    if (count <= 0 || !labels) return MOCD_OK;
    int rc = grow(c->stream, &c->d_im, &c->im_cap, (size_t)count * (size_t)c->n);
    if (rc) return rc;
    if (!c->d_idx) {
        void *q = nullptr;
        CK(dev_alloc(&q, sizeof(int32_t) * 2 * kMaxPop, c->stream));
        c->d_idx = static_cast<int32_t *>(q);
    }
    CK(cudaMemcpyAsync(c->d_idx, ridx, sizeof(int32_t) * count, cudaMemcpyHostToDevice, c->stream));
    const int32_t *phalf = c->ps.buf[(uint32_t)(c->host_gen + 1) & 1u];
    CK(launch_gather_individuals((int)c->n, c->W, c->gp.np, phalf, c->ps.q, c->d_idx, count, c->d_im,
                                 c->stream));
    // While the gather runs: map the caller's (possibly freshly allocated)
    // pages on several threads, so the copy does not fault page by page.
    prefault(labels, sizeof(int32_t) * (size_t)count * (size_t)c->n);
    CK(cudaMemcpyAsync(labels, c->d_im, sizeof(int32_t) * (size_t)count * (size_t)c->n,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MOCD_OK;
}

// Individual-major labels of `count` P positions (pos NULL: all of P).
int download_members(mocd_ctx *c, const int32_t *pos_host, int count, int32_t *labels)
{
    if (count <= 0 || !labels) return MOCD_OK;
    std::vector<int32_t> keep(c->gp.np);
    CK(cudaMemcpyAsync(keep.data(), c->ps.keep, sizeof(int32_t) * c->gp.np, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<int32_t> ridx(count);
    for (int k = 0; k < count; ++k) ridx[k] = keep[pos_host ? pos_host[k] : k];
    return download_r(c, ridx.data(), count, labels);
}

// F_1 as front_kernel lists it: fr = count, best, P positions; fint = intra
// [kMaxPop] then S [kMaxPop] of each member.
int read_front(mocd_ctx *c, std::vector<int32_t> &fr, std::vector<int64_t> &fint)
{
    const int np = c->gp.np;
    CK(launch_front(c->gp, c->ps, c->stream));
    fr.assign(2 + np, 0);
    fint.assign(2 * kMaxPop, 0);
    CK(cudaMemcpyAsync(fr.data(), c->ps.front, sizeof(int32_t) * (2 + np), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(fint.data(), c->ps.fint, sizeof(int64_t) * 2 * kMaxPop, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MOCD_OK;
}

// Community statistics of the `count` members of the front that front_kernel
// listed last; out = [4][kMaxPop] words (see launch_front_stats).
int front_stats(mocd_ctx *c, int count, std::vector<unsigned long long> &out)
{
    const size_t n = (size_t)c->n;
    const size_t Wf = (size_t)((count + 3) & ~3);
    int rc;
    if ((rc = grow(c->stream, &c->d_nm, &c->nm_cap, n * Wf))) return rc;
    if ((rc = grow(c->stream, &c->d_volsize, &c->volsize_cap, n * (size_t)count))) return rc;
    if ((rc = grow(c->stream, &c->d_cut, &c->cut_cap, n * (size_t)count))) return rc;
    const size_t acc_words = stats_acc_words();
    if (!c->d_stats) {
        void *p = nullptr;
        CK(dev_alloc(&p, sizeof(unsigned long long) * (acc_words + 4 * kMaxPop), c->stream));
        c->d_stats = static_cast<unsigned long long *>(p);
    }
    CK(cudaMemsetAsync(c->d_volsize, 0, sizeof(unsigned long long) * n * (size_t)count, c->stream));
    CK(cudaMemsetAsync(c->d_cut, 0, sizeof(uint32_t) * n * (size_t)count, c->stream));
    CK(cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * (acc_words + 4 * kMaxPop), c->stream));
    const int32_t *phalf = c->ps.buf[(uint32_t)(c->host_gen + 1) & 1u];
    CK(launch_front_stats(c->gp, c->ps, phalf, count, c->d_row_ptr, c->d_col_idx, c->d_order, c->d_nm,
                          c->d_volsize, c->d_cut, c->d_stats, c->d_stats + acc_words, c->sms, c->stream));
    out.assign(4 * kMaxPop, 0ull);
    CK(cudaMemcpyAsync(out.data(), c->d_stats + acc_words, sizeof(unsigned long long) * 4 * kMaxPop,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MOCD_OK;
}

struct FrontMember {
    int64_t K;            // 4 m (m - intra) + S: Alg. 3 order (smaller = larger Q)
    int64_t communities;  // k
    int64_t size_sumsq;   // sum_c n_c^2
    double mean_phi, max_phi;
};

// a * b as three 64-bit limbs, most significant first.
void mul_u128_u64(unsigned __int128 a, uint64_t b, uint64_t w[3])
{
    const unsigned __int128 lo = (unsigned __int128)(uint64_t)a * b;
    const unsigned __int128 hi = (unsigned __int128)(uint64_t)(a >> 64) * b + (uint64_t)(lo >> 64);
    w[2] = (uint64_t)lo;
    w[1] = (uint64_t)hi;
    w[0] = (uint64_t)(hi >> 64);
}

// Sign of var(a) - var(b), var = sum n_c^2 / k - (n / k)^2 = (k sumsq - n^2) / k^2,
// compared exactly: (k_a sumsq_a - n^2) k_b^2 against (k_b sumsq_b - n^2) k_a^2.
int compare_size_variance(const FrontMember &a, const FrontMember &b, int64_t n)
{
    const unsigned __int128 n2 = (unsigned __int128)n * (uint64_t)n;
    const unsigned __int128 na = (unsigned __int128)(uint64_t)a.communities * (uint64_t)a.size_sumsq - n2;
    const unsigned __int128 nb = (unsigned __int128)(uint64_t)b.communities * (uint64_t)b.size_sumsq - n2;
    uint64_t x[3], y[3];
    mul_u128_u64(na, (uint64_t)(b.communities * b.communities), x);
    mul_u128_u64(nb, (uint64_t)(a.communities * a.communities), y);
    for (int t = 0; t < 3; ++t)
        if (x[t] != y[t]) return x[t] < y[t] ? -1 : 1;
    return 0;
}

// Sign of (criterion of a) - (criterion of b); smaller is preferred.
int compare_criterion(const FrontMember &a, const FrontMember &b, int criterion, int64_t target, int64_t n)
{
    switch (criterion) {
    case MOCD_SELECT_COMMUNITIES: {
        const int64_t da = a.communities > target ? a.communities - target : target - a.communities;
        const int64_t db = b.communities > target ? b.communities - target : target - b.communities;
        return da < db ? -1 : da > db ? 1 : 0;
    }
    case MOCD_SELECT_SIZE_VARIANCE: return compare_size_variance(a, b, n);
    case MOCD_SELECT_MEAN_CONDUCTANCE: return a.mean_phi < b.mean_phi ? -1 : a.mean_phi > b.mean_phi ? 1 : 0;
    case MOCD_SELECT_MAX_CONDUCTANCE: return a.max_phi < b.max_phi ? -1 : a.max_phi > b.max_phi ? 1 : 0;
    default: return 0;
    }
}

// The preferred member: least criterion, then least K (Alg. 3's order), then
// the first in front order.
int select_member(const std::vector<FrontMember> &mem, int criterion, int64_t target, int64_t n)
{
    int best = -1;
    for (int k = 0; k < (int)mem.size(); ++k) {
        if (best < 0) {
            best = k;
            continue;
        }
        int d = compare_criterion(mem[k], mem[best], criterion, target, n);
        if (d == 0) d = mem[k].K < mem[best].K ? -1 : 0;
        if (d < 0) best = k;
    }
    return best;
}

}  // namespace

namespace {

// Host-side failure injection (mocd_debug_inject): per site, the number of
// calls still to pass, then the number to fail and the status to fail with.
struct InjectSite {
    int skip = 0, count = 0, status = 0;
};
std::mutex g_inject_mu;
InjectSite g_inject[2];
std::atomic<bool> g_inject_armed{false};  // some site has failures pending

}  // namespace

bool mocd::inject_failure(int site, int *status)
{
    if (!g_inject_armed.load(std::memory_order_relaxed)) return false;
    std::lock_guard<std::mutex> lock(g_inject_mu);
    InjectSite &q = g_inject[site];
    if (q.count <= 0) return false;
    if (q.skip > 0) {
        --q.skip;
        return false;
    }
    --q.count;
    if (status) *status = q.status;
    return true;
}

cudaError_t mocd::dev_alloc(void **p, size_t bytes, cudaStream_t st)
{
    if (inject_failure(kSiteDeviceAlloc, nullptr)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = library_pool(dev, &pool);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

int mocd::record_on_stream(mocd_ctx *c, cudaEvent_t ev)
{
    if (!c || !ev) return MOCD_ERR_INVALID_ARG;
    CK(cudaEventRecord(ev, c->stream));
    return MOCD_OK;
}

extern "C" {

const char *mocd_status_string(int status)
{
    switch (status) {
    case MOCD_OK: return "ok";
    case MOCD_ERR_INVALID_ARG: return "invalid argument";
    case MOCD_ERR_NOT_SYMMETRIC: return "adjacency is not symmetric";
    case MOCD_ERR_SELF_LOOP: return "self loop";
    case MOCD_ERR_DUPLICATE_EDGE: return "repeated edge";
    case MOCD_ERR_EMPTY_GRAPH: return "graph has no edges";
    case MOCD_ERR_OUT_OF_MEMORY: return "out of device memory";
    case MOCD_ERR_BUFFER_TOO_SMALL: return "output buffer too small";
    case MOCD_ERR_CUDA: return "CUDA error";
    case MOCD_ERR_NOT_READY: return "population not initialised";
    case MOCD_ERR_TOO_LARGE: return "count * n exceeds the fixed scratch of the no-allocation entry point";
    case MOCD_ERR_CANCELLED: return "job cancelled";
    default: return "unknown status";
    }
}

int mocd_graph_upload(mocd_ctx **out, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                      void *cuda_stream)
{
    if (!out) return MOCD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!row_ptr || n < 1 || n >= (int64_t(1) << 30)) return MOCD_ERR_INVALID_ARG;
    if (row_ptr[0] != 0) return MOCD_ERR_INVALID_ARG;
    int dmax = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (row_ptr[v + 1] < row_ptr[v]) return MOCD_ERR_INVALID_ARG;
        dmax = (int)std::min<int64_t>(std::max<int64_t>(dmax, row_ptr[v + 1] - row_ptr[v]), INT_MAX);
    }
    const int64_t nnz = row_ptr[n];
    if (nnz >= (int64_t(1) << 31)) return MOCD_ERR_INVALID_ARG;
    if (nnz > 0 && !col_idx) return MOCD_ERR_INVALID_ARG;
    // Per row, in sorted order: range, self loop, repeat; then symmetry. The
    // first failing row decides the status, as a sequential scan would. One
    // pass checks the rows as given and whether each is strictly increasing;
    // if one is not, a sorted copy of the adjacency is made and checked again
    // (the order of the entries decides which failure a row reports).
    auto check_rows = [&](const int32_t *adj_rows, std::atomic<bool> *increasing) {
        FirstError err;
        parallel_rows(row_ptr, n, [&](int64_t v0, int64_t v1) {
            for (int64_t v = v0; v < v1; ++v) {
                const int32_t *b = adj_rows + row_ptr[v], *e = adj_rows + row_ptr[v + 1];
                for (const int32_t *q = b; q < e; ++q) {
                    if (increasing && q > b && q[-1] > *q) increasing->store(false, std::memory_order_relaxed);
                    int rc = MOCD_OK;
                    if (*q < 0 || *q >= n) rc = MOCD_ERR_INVALID_ARG;
                    else if (*q == v) rc = MOCD_ERR_SELF_LOOP;
                    else if (q > b && q[-1] == *q) rc = MOCD_ERR_DUPLICATE_EDGE;
                    if (rc) {
                        // The row's failure is the one its sorted order shows
                        // first: if the row is not sorted, the sorted copy
                        // decides (the rows before it in this range were
                        // scanned in full).
                        for (const int32_t *r = q + 1; increasing && r < e; ++r)
                            if (r[-1] > *r) increasing->store(false, std::memory_order_relaxed);
                        err.record(v, rc);
                        return;
                    }
                }
            }
        });
        return err.status();
    };
    std::atomic<bool> all_increasing{true};
    std::vector<int32_t> adj;
    const int32_t *src = col_idx;
    int status = check_rows(col_idx, &all_increasing);
    if (!all_increasing.load()) {
        adj.assign(col_idx, col_idx + nnz);
        parallel_rows(row_ptr, n, [&](int64_t v0, int64_t v1) {
            for (int64_t v = v0; v < v1; ++v) std::sort(adj.data() + row_ptr[v], adj.data() + row_ptr[v + 1]);
        });
        src = adj.data();
        status = check_rows(src, nullptr);
    }
    if (status) return status;
    // Symmetry is checked on the device once the CSR is there (below): a
    // binary search per stored entry, which the host's scattered memory
    // accesses make slow for large graphs.
    if (nnz == 0) return MOCD_ERR_EMPTY_GRAPH;

    mocd_ctx *c = new (std::nothrow) mocd_ctx();
    if (!c) return MOCD_ERR_OUT_OF_MEMORY;
    auto fail = [&](int rc) {
        mocd_destroy(c);
        return rc;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return fail(MOCD_ERR_CUDA);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(MOCD_ERR_CUDA);
        c->own_stream = true;
    }
    for (int k = 0; k <= kStages; ++k)
        if (cudaEventCreate(&c->ev[k]) != cudaSuccess) return fail(MOCD_ERR_CUDA);
    c->n = n;
    c->m = nnz / 2;
    c->dmax = dmax;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d > 32 && d <= 64) c->n_defer[0] += 1;
        else if (d > 64 && d <= kDeferMax) c->n_defer[1] += 1;
        else if (d > kSharedTableMax) c->n_defer[2] += 1;
    }
    std::vector<int32_t> rp32(n + 1);
    for (int64_t v = 0; v <= n; ++v) rp32[v] = (int32_t)row_ptr[v];
    void *p = nullptr;
    cudaError_t e = dev_alloc(&p, sizeof(int32_t) * (n + 1), c->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    c->d_row_ptr = static_cast<int32_t *>(p);
    e = dev_alloc(&p, sizeof(int32_t) * nnz, c->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    c->d_col_idx = static_cast<int32_t *>(p);
    // Work order of the degree-proportional kernels: degree descending (ties
    // by node id), so that the costliest nodes are spread over all warps. A
    // counting sort on the degree.
    std::vector<int32_t> order(n);
    {
        std::vector<int64_t> at((size_t)dmax + 2, 0);
        for (int64_t v = 0; v < n; ++v) at[(size_t)(dmax - (row_ptr[v + 1] - row_ptr[v])) + 1] += 1;
        for (size_t d = 1; d < at.size(); ++d) at[d] += at[d - 1];
        for (int64_t v = 0; v < n; ++v) order[at[(size_t)(dmax - (row_ptr[v + 1] - row_ptr[v]))]++] = (int32_t)v;
    }
    e = dev_alloc(&p, sizeof(int32_t) * n, c->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    c->d_order = static_cast<int32_t *>(p);
    if (cudaMemcpyAsync(c->d_order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
        return fail(MOCD_ERR_CUDA);
    e = dev_alloc(&p, sizeof(int32_t) * (n + 1), c->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    c->d_eptr = static_cast<int32_t *>(p);
    e = dev_alloc(&p, sizeof(int32_t) * (size_t)(nnz / 2), c->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    c->d_eidx = static_cast<int32_t *>(p);
    int *d_bad = nullptr;
    int h_bad = 0;
    e = dev_alloc(reinterpret_cast<void **>(&d_bad), sizeof(int), c->stream);
    if (e != cudaSuccess) return fail(cuda_status(e));
    const bool copied =
        cudaMemcpyAsync(c->d_row_ptr, rp32.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice,
                        c->stream) == cudaSuccess &&
        cudaMemcpyAsync(c->d_col_idx, src, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, c->stream) ==
            cudaSuccess &&
        cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream) == cudaSuccess &&
        launch_symmetry_check((int)n, c->d_row_ptr, c->d_col_idx, d_bad, c->sms, c->stream) == cudaSuccess &&
        launch_orient((int)n, c->d_row_ptr, c->d_col_idx, c->d_eptr, c->d_eidx, (int)(nnz / 2), c->sms,
                      c->stream) == cudaSuccess &&
        cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) == cudaSuccess;
    cudaFreeAsync(d_bad, c->stream);
    if (!copied || cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(MOCD_ERR_CUDA);
    if (h_bad) return fail(MOCD_ERR_NOT_SYMMETRIC);
    *out = c;
    return MOCD_OK;
}

int mocd_population_init(mocd_ctx *c, const mocd_params *params)
{
    if (!c) return MOCD_ERR_INVALID_ARG;
    int rc = check_params(c, params);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    // Until the new population is complete, nothing may run on the old one.
    c->ready = false;
    rc = prepare_population(c, params);
    if (rc) return rc;
    CK(launch_init_population(c->gp, params->init_mode, c->d_row_ptr, c->d_col_idx, c->ps.buf[1], c->stream));
    return start_population(c, 0);
}

int mocd_set_population(mocd_ctx *c, const mocd_params *params, const int32_t *labels, int32_t generation)
{
    if (!c || !labels || generation < 0) return MOCD_ERR_INVALID_ARG;
    int rc = check_params(c, params);
    if (rc) return rc;
    rc = validate_labels(c, labels, (size_t)params->pop_size * (size_t)c->n);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    c->ready = false;
    rc = prepare_population(c, params);
    if (rc) return rc;
    rc = grow(c->stream, &c->d_im, &c->im_cap, (size_t)params->pop_size * (size_t)c->n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->d_im, labels, sizeof(int32_t) * (size_t)params->pop_size * (size_t)c->n,
                       cudaMemcpyHostToDevice, c->stream));
    int32_t *phalf = c->ps.buf[((uint32_t)generation + 1u) & 1u];
    CK(launch_to_node_major((int)c->n, c->W, params->pop_size, c->d_im, phalf, c->stream));
    return start_population(c, (uint32_t)generation);
}

int mocd_generation(mocd_ctx *c, int32_t n_generations)
{
    if (!c || n_generations < 0) return MOCD_ERR_INVALID_ARG;
    if (!c->ready) return MOCD_ERR_NOT_READY;
    int injected = 0;
    if (n_generations > 0 && inject_failure(kSiteGeneration, &injected)) return injected;
    const int g = c->timing ? 1 : 0;
    if (!c->graph_exec[g]) {
        const int rc = build_graph(c);
        if (rc) return rc;
    }
    for (int32_t k = 0; k < n_generations; ++k) CK(cudaGraphLaunch(c->graph_exec[g], c->stream));
    c->host_gen += n_generations;
    if (n_generations > 0 && c->timing) c->timing_valid = true;
    return MOCD_OK;
}

int mocd_generation_kernels(mocd_ctx *c, int32_t *kernels)
{
    if (!c || !kernels) return MOCD_ERR_INVALID_ARG;
    if (!c->ready) return MOCD_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    const bool timing = c->timing;
    c->timing = false;
    const int rc = build_graph(c);
    c->timing = timing;
    if (rc) return rc;
    size_t count = 0;
    CK(cudaGraphGetNodes(c->graph[0], nullptr, &count));
    std::vector<cudaGraphNode_t> nodes(count);
    CK(cudaGraphGetNodes(c->graph[0], nodes.data(), &count));
    int32_t k = 0;
    for (size_t t = 0; t < count; ++t) {
        cudaGraphNodeType type;
        CK(cudaGraphNodeGetType(nodes[t], &type));
        if (type == cudaGraphNodeTypeKernel) ++k;
    }
    *kernels = k;
    return MOCD_OK;
}

int mocd_front_stats(mocd_ctx *c, int32_t cap, int32_t *count, int64_t *communities, int64_t *size_sumsq,
                     double *mean_conductance, double *max_conductance)
{
    if (!c || !count || cap < 0) return MOCD_ERR_INVALID_ARG;
    if (!c->ready) return MOCD_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    std::vector<int32_t> fr;
    std::vector<int64_t> fint;
    int rc = read_front(c, fr, fint);
    if (rc) return rc;
    const int cnt = fr[0];
    *count = cnt;
    if (cnt > cap) return MOCD_ERR_BUFFER_TOO_SMALL;
    std::vector<unsigned long long> out;
    rc = front_stats(c, cnt, out);
    if (rc) return rc;
    for (int k = 0; k < cnt; ++k) {
        if (communities) communities[k] = (int64_t)out[k];
        if (size_sumsq) size_sumsq[k] = (int64_t)out[kMaxPop + k];
        if (mean_conductance) std::memcpy(mean_conductance + k, &out[2 * kMaxPop + k], sizeof(double));
        if (max_conductance) std::memcpy(max_conductance + k, &out[3 * kMaxPop + k], sizeof(double));
    }
    return MOCD_OK;
}

int mocd_select_solution(mocd_ctx *c, int32_t criterion, int64_t target, int32_t *index)
{
    if (!c || !index) return MOCD_ERR_INVALID_ARG;
    if (criterion < MOCD_SELECT_MODULARITY || criterion > MOCD_SELECT_MAX_CONDUCTANCE) return MOCD_ERR_INVALID_ARG;
    if (criterion == MOCD_SELECT_COMMUNITIES && target < 1) return MOCD_ERR_INVALID_ARG;
    if (!c->ready) return MOCD_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    std::vector<int32_t> fr;
    std::vector<int64_t> fint;
    int rc = read_front(c, fr, fint);
    if (rc) return rc;
    const int cnt = fr[0];
    std::vector<unsigned long long> out(4 * kMaxPop, 0ull);
    if (criterion != MOCD_SELECT_MODULARITY) {
        rc = front_stats(c, cnt, out);
        if (rc) return rc;
    }
    std::vector<FrontMember> mem(cnt);
    for (int k = 0; k < cnt; ++k) {
        FrontMember &f = mem[k];
        f.K = 4 * c->m * (c->m - fint[k]) + fint[kMaxPop + k];
        f.communities = (int64_t)out[k];
        f.size_sumsq = (int64_t)out[kMaxPop + k];
        std::memcpy(&f.mean_phi, &out[2 * kMaxPop + k], sizeof(double));
        std::memcpy(&f.max_phi, &out[3 * kMaxPop + k], sizeof(double));
    }
    *index = select_member(mem, criterion, target, c->n);
    return MOCD_OK;
}

int mocd_pareto_front(mocd_ctx *c, int32_t cap, int32_t *count, int32_t *labels, double *f1, double *f2,
                      int64_t *intra, int64_t *sumsq, int32_t *best)
{
    if (!c || !count || cap < 0) return MOCD_ERR_INVALID_ARG;
    if (!c->ready) return MOCD_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    const int np = c->gp.np;
    CK(launch_front(c->gp, c->ps, c->stream));
    std::vector<int32_t> fr(2 + np);
    std::vector<int64_t> fint(2 * kMaxPop);
    std::vector<double> fval(2 * kMaxPop);
    CK(cudaMemcpyAsync(fr.data(), c->ps.front, sizeof(int32_t) * (2 + np), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(fint.data(), c->ps.fint, sizeof(int64_t) * 2 * kMaxPop, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(fval.data(), c->ps.fval, sizeof(double) * 2 * kMaxPop, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int cnt = fr[0];
    *count = cnt;
    if (cnt > cap) return MOCD_ERR_BUFFER_TOO_SMALL;
    if (best) *best = fr[1];
    const int32_t *members = fr.data() + 2;
    for (int k = 0; k < cnt; ++k) {
        if (intra) intra[k] = fint[k];
        if (sumsq) sumsq[k] = fint[kMaxPop + k];
        if (f1) f1[k] = fval[k];
        if (f2) f2[k] = fval[kMaxPop + k];
    }
    return download_members(c, members, cnt, labels);
}

int mocd_get_population(mocd_ctx *c, int32_t *labels, int64_t *k1, int64_t *k2, int32_t *generation)
{
    if (!c) return MOCD_ERR_INVALID_ARG;
    if (!c->ready) return MOCD_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    const int np = c->gp.np;
    std::vector<int64_t> pk(2 * kMaxPop);
    CK(cudaMemcpyAsync(pk.data(), c->ps.pk, sizeof(int64_t) * 2 * kMaxPop, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < np; ++k) {
        if (k1) k1[k] = pk[k];
        if (k2) k2[k] = pk[kMaxPop + k];
    }
    if (generation) *generation = c->host_gen;
    return download_members(c, nullptr, np, labels);
}

int mocd_get_offspring(mocd_ctx *c, int32_t *labels, int64_t *k1, int64_t *k2)
{
    if (!c) return MOCD_ERR_INVALID_ARG;
    if (!c->ready || c->host_gen < 1) return MOCD_ERR_NOT_READY;
    CK(cudaSetDevice(c->device));
    const int np = c->gp.np;
    std::vector<int64_t> rk(4 * kMaxPop);
    CK(cudaMemcpyAsync(rk.data(), c->ps.rk, sizeof(int64_t) * 4 * kMaxPop, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < np; ++i) {
        if (k1) k1[i] = rk[np + i];
        if (k2) k2[i] = rk[2 * kMaxPop + np + i];
    }
    std::vector<int32_t> ridx(np);
    for (int i = 0; i < np; ++i) ridx[i] = np + i;
    return download_r(c, ridx.data(), np, labels);
}

int mocd_evaluate(mocd_ctx *c, int32_t count, const int32_t *labels, int64_t *intra, int64_t *sumsq)
{
    if (!c || count < 0) return MOCD_ERR_INVALID_ARG;
    if (count == 0) return MOCD_OK;
    if (!labels || !intra || !sumsq) return MOCD_ERR_INVALID_ARG;
    int rc = validate_labels(c, labels, (size_t)count * (size_t)c->n);
    if (rc) return rc;
    CK(cudaSetDevice(c->device));
    const int batch = std::min<int>(count, kMaxPop);
    const size_t n = (size_t)c->n;
    if ((rc = grow(c->stream, &c->d_im, &c->im_cap, (size_t)batch * n))) return rc;
    if ((rc = grow(c->stream, &c->d_nm, &c->nm_cap, (size_t)kMaxPop * n))) return rc;
    if ((rc = grow(c->stream, &c->d_eval_hist, &c->eval_hist_cap, (size_t)((batch + 3) & ~3) * n))) return rc;
    if (!c->d_eval_acc) {
        void *q = nullptr;
        CK(dev_alloc(&q, sizeof(unsigned long long) * 2 * kMaxPop, c->stream));
        c->d_eval_acc = static_cast<unsigned long long *>(q);
    }
    const int grid = grid_for_eval(c->sms);
    std::vector<unsigned long long> acc(2 * kMaxPop);
    for (int b0 = 0; b0 < count; b0 += batch) {
        const int b = std::min(batch, count - b0);
        const int W = (b + 3) & ~3;
        CK(cudaMemcpyAsync(c->d_im, labels + (size_t)b0 * n, sizeof(int32_t) * (size_t)b * n,
                           cudaMemcpyHostToDevice, c->stream));
        CK(launch_to_node_major((int)n, W, b, c->d_im, c->d_nm, c->stream));
        if ((rc = clear_eval_state(c, c->d_eval_hist, (size_t)W * n, c->d_eval_acc))) return rc;
        CK(launch_evaluate((int)n, W, b, c->d_row_ptr, c->d_col_idx, c->d_nm, c->d_eval_hist, c->d_eval_acc,
                           grid, c->stream));
        CK(cudaMemcpyAsync(acc.data(), c->d_eval_acc, sizeof(unsigned long long) * 2 * kMaxPop,
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < b; ++k) {
            intra[b0 + k] = (int64_t)acc[k];
            sumsq[b0 + k] = (int64_t)acc[kMaxPop + k];
        }
    }
    return MOCD_OK;
}

int mocd_synchronize(mocd_ctx *c)
{
    if (!c) return MOCD_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->stream));
    return MOCD_OK;
}

int mocd_set_timing(mocd_ctx *c, int32_t enable)
{
    if (!c) return MOCD_ERR_INVALID_ARG;
    const bool want = enable != 0;
    if (want == c->timing) return MOCD_OK;
    c->timing = want;
    c->timing_valid = false;
    // Switching between the two graphs costs nothing once both exist.
    if (c->ready && !c->graph_exec[want ? 1 : 0]) return build_graph(c);
    return MOCD_OK;
}

int mocd_kernel_times(mocd_ctx *c, float *ms, int32_t cap)
{
    if (!c || !ms || cap < kStages) return MOCD_ERR_INVALID_ARG;
    if (!c->timing || !c->timing_valid) return MOCD_ERR_NOT_READY;
    CK(cudaEventSynchronize(c->ev[kStages]));
    for (int k = 0; k < kStages; ++k) CK(cudaEventElapsedTime(ms + k, c->ev[k], c->ev[k + 1]));
    return kStages;
}

int mocd_info(mocd_ctx *c, int64_t *n, int64_t *m, int32_t *pop_size, int32_t *generation)
{
    if (!c) return MOCD_ERR_INVALID_ARG;
    if (n) *n = c->n;
    if (m) *m = c->m;
    if (pop_size) *pop_size = c->ready ? c->gp.np : 0;
    if (generation) *generation = c->host_gen;
    return MOCD_OK;
}

struct mocd_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // Form 0: each member's kernel chain, selection included, on its own
    // graph branch. Form 1: the selections of all members in one
    // multi-population launch after the chains. Form 2: also crossover, the
    // deferred mutation votes and the evaluation of all members in one
    // multi-member launch each; only the mutation kernels stay per member.
    int form = 0;
    GenParams *d_gp = nullptr;  // [count], for the merged selection
    PopState *d_ps = nullptr;
    BatchMember *d_members = nullptr;  // [count], for the multi-member launches
    int *d_starts = nullptr;           // [4][count + 1] block ranges: crossover, votes 33..64, 65..128, evaluation
    int blocks[4] = {0, 0, 0, 0};      // blocks of each multi-member launch
    int es_max = 0;
    std::vector<mocd_ctx *> ctx;
    std::vector<int32_t> version;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static int batch_build(mocd_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    const int count = (int)b->ctx.size();
    if (b->form >= 1) {
        // The members' current parameters and states, for the merged launches.
        std::vector<GenParams> gps;
        std::vector<PopState> pss;
        std::vector<BatchMember> mbs;
        std::vector<int> starts(4 * (size_t)(count + 1), 0);
        b->es_max = 0;
        for (int i = 0; i < count; ++i) {
            mocd_ctx *c = b->ctx[(size_t)i];
            gps.push_back(c->gp);
            pss.push_back(c->ps);
            mbs.push_back(BatchMember{c->gp, c->ps, c->d_row_ptr, c->d_col_idx, c->d_order, c->d_eptr, c->d_eidx});
            b->es_max = std::max(b->es_max, c->gp.es);
            // Per member and stage: its own grid (a deferred class's votes get
            // about one thread per four listed pairs at full capacity, at most
            // its single-member grid).
            const int g[4] = {
                c->grid_cross,
                c->gp.defer_cap[0] > 0 ? std::min(c->grid_vote64, (c->gp.defer_cap[0] + 4 * 128 - 1) / (4 * 128)) : 0,
                c->gp.defer_cap[1] > 0 ? std::min(c->grid_vote128, (c->gp.defer_cap[1] + 4 * 128 - 1) / (4 * 128)) : 0,
                c->grid_eval_intra};
            for (int st = 0; st < 4; ++st)
                starts[(size_t)st * (count + 1) + i + 1] = starts[(size_t)st * (count + 1) + i] + g[st];
        }
        for (int st = 0; st < 4; ++st) b->blocks[st] = starts[(size_t)st * (count + 1) + count];
        CK(cudaMemcpyAsync(b->d_gp, gps.data(), sizeof(GenParams) * gps.size(), cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(b->d_ps, pss.data(), sizeof(PopState) * pss.size(), cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(b->d_members, mbs.data(), sizeof(BatchMember) * mbs.size(), cudaMemcpyHostToDevice,
                           b->stream));
        CK(cudaMemcpyAsync(b->d_starts, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice,
                           b->stream));
        CK(cudaStreamSynchronize(b->stream));
    }
    const int *st_cross = b->d_starts, *st_v64 = b->d_starts + (count + 1), *st_v128 = b->d_starts + 2 * (count + 1),
              *st_eval = b->d_starts + 3 * (count + 1);
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = MOCD_OK;
    cudaError_t e = cudaSuccess;
    if (b->form == 2) e = launch_crossover_multi(b->d_members, st_cross, count, b->blocks[0], b->es_max, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    for (int i = 0; i < count && rc == MOCD_OK && e == cudaSuccess; ++i) {
        mocd_ctx *c = b->ctx[(size_t)i];
        e = cudaStreamWaitEvent(b->branch[(size_t)i], b->fork, 0);
        if (e != cudaSuccess) break;
        if (b->form == 2)
            e = launch_mutation(c->gp, c->ps, c->d_row_ptr, c->d_col_idx, c->d_order, c->grid_mut, c->grid_vote64,
                                c->grid_vote128, b->branch[(size_t)i], false);
        else
            rc = issue_generation(c, b->branch[(size_t)i], false, b->form == 0);
        if (rc == MOCD_OK && e == cudaSuccess) e = cudaEventRecord(b->join[(size_t)i], b->branch[(size_t)i]);
        if (rc == MOCD_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[(size_t)i], 0);
    }
    if (rc == MOCD_OK && e == cudaSuccess && b->form == 2) {
        e = launch_vote_multi(b->d_members, st_v64, count, b->blocks[1], 0, b->stream);
        if (e == cudaSuccess) e = launch_vote_multi(b->d_members, st_v128, count, b->blocks[2], 1, b->stream);
        if (e == cudaSuccess) e = launch_evaluate_multi(b->d_members, st_eval, count, b->blocks[3], b->stream);
    }
    if (rc == MOCD_OK && e == cudaSuccess && b->form >= 1)
        e = launch_select_multi(b->d_gp, b->d_ps, count, 1, b->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (rc || e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : cuda_status(e != cudaSuccess ? e : e2);
    }
    b->graph = g;
    CK(cudaGraphInstantiate(&b->exec, g, 0));
    return MOCD_OK;
}

int mocd_batch_create(mocd_batch **out, int32_t count, mocd_ctx *const *ctxs, void *cuda_stream)
{
    if (!out) return MOCD_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !ctxs) return MOCD_ERR_INVALID_ARG;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    for (int32_t i = 0; i < count; ++i) {
        if (!ctxs[i]) return MOCD_ERR_INVALID_ARG;
        if (ctxs[i]->device != dev) return MOCD_ERR_INVALID_ARG;
        if (!ctxs[i]->ready) return MOCD_ERR_NOT_READY;
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return MOCD_ERR_INVALID_ARG;
    }
    mocd_batch *b = new (std::nothrow) mocd_batch();
    if (!b) return MOCD_ERR_OUT_OF_MEMORY;
    b->device = dev;
    auto fail = [&](int rc) {
        mocd_batch_destroy(b);
        return rc;
    };
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(MOCD_ERR_CUDA);
        b->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return fail(MOCD_ERR_CUDA);
    {
        void *p = nullptr;
        if (dev_alloc(&p, sizeof(GenParams) * (size_t)count, b->stream) != cudaSuccess) return fail(MOCD_ERR_OUT_OF_MEMORY);
        b->d_gp = static_cast<GenParams *>(p);
        if (dev_alloc(&p, sizeof(PopState) * (size_t)count, b->stream) != cudaSuccess) return fail(MOCD_ERR_OUT_OF_MEMORY);
        b->d_ps = static_cast<PopState *>(p);
        if (dev_alloc(&p, sizeof(BatchMember) * (size_t)count, b->stream) != cudaSuccess)
            return fail(MOCD_ERR_OUT_OF_MEMORY);
        b->d_members = static_cast<BatchMember *>(p);
        if (dev_alloc(&p, sizeof(int) * 4 * (size_t)(count + 1), b->stream) != cudaSuccess)
            return fail(MOCD_ERR_OUT_OF_MEMORY);
        b->d_starts = static_cast<int *>(p);
    }
    for (int32_t i = 0; i < count; ++i) {
        // Work already issued on a member's own stream finishes first.
        if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) return fail(MOCD_ERR_CUDA);
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(MOCD_ERR_CUDA);
        b->branch.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(MOCD_ERR_CUDA);
        b->join.push_back(ev);
        b->ctx.push_back(ctxs[i]);
        b->version.push_back(ctxs[i]->version);
    }
    const int rc = batch_build(b);
    if (rc) return fail(rc);
    *out = b;
    return MOCD_OK;
}

int mocd_batch_generation(mocd_batch *b, int32_t n_generations)
{
    if (!b || n_generations < 0) return MOCD_ERR_INVALID_ARG;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (!b->ctx[i]->ready || b->ctx[i]->version != b->version[i]) return MOCD_ERR_NOT_READY;
    for (int32_t k = 0; k < n_generations; ++k) CK(cudaGraphLaunch(b->exec, b->stream));
    for (mocd_ctx *c : b->ctx) {
        c->host_gen += n_generations;
        c->timing_valid = false;
    }
    return MOCD_OK;
}

int mocd_batch_synchronize(mocd_batch *b)
{
    if (!b) return MOCD_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(b->stream));
    return MOCD_OK;
}

int mocd_batch_autotune(mocd_batch *b, int32_t generations_per_trial, int32_t *nodes_per_warp)
{
    if (!b || generations_per_trial < 1) return MOCD_ERR_INVALID_ARG;
    static const int kShapes[] = {1, 2, 4, 8, 16};
    b->form = 0;  // the shapes are compared in the per-member form
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    float best_ms = 0.0f;
    int best = 1;
    int rc = MOCD_OK;
    for (int shape : kShapes) {
        for (mocd_ctx *c : b->ctx) {
            c->nodes_per_warp = shape;
            size_grids(c);
        }
        if ((rc = batch_build(b))) break;
        if ((rc = mocd_batch_generation(b, 1))) break;  // warm-up
        if (cudaEventRecord(t0, b->stream) != cudaSuccess) { rc = MOCD_ERR_CUDA; break; }
        if ((rc = mocd_batch_generation(b, generations_per_trial))) break;
        if (cudaEventRecord(t1, b->stream) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess) {
            rc = MOCD_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (shape == kShapes[0] || ms < best_ms) {
            best_ms = ms;
            best = shape;
        }
    }
    // Then the form at that shape: per member, merged selection, or
    // multi-member launches for every stage but the mutation kernel.
    int best_form = 0;
    if (rc == MOCD_OK) {
        for (mocd_ctx *c : b->ctx) {
            c->nodes_per_warp = best;
            size_grids(c);
        }
        for (int form = 1; form <= 2 && rc == MOCD_OK; ++form) {
            b->form = form;
            float ms = 0.0f;
            if ((rc = batch_build(b)) != MOCD_OK || (rc = mocd_batch_generation(b, 1)) != MOCD_OK) break;
            if (cudaEventRecord(t0, b->stream) != cudaSuccess) rc = MOCD_ERR_CUDA;
            if (rc == MOCD_OK) rc = mocd_batch_generation(b, generations_per_trial);
            if (rc == MOCD_OK &&
                (cudaEventRecord(t1, b->stream) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess))
                rc = MOCD_ERR_CUDA;
            if (rc == MOCD_OK) cudaEventElapsedTime(&ms, t0, t1);
            if (rc == MOCD_OK && ms < best_ms) {
                best_ms = ms;
                best_form = form;
            }
        }
        b->form = best_form;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) return rc;
    if ((rc = mocd_batch_configure(b, best, best_form))) return rc;
    if (nodes_per_warp) *nodes_per_warp = best;
    return MOCD_OK;
}

int mocd_batch_configure(mocd_batch *b, int32_t nodes_per_warp, int32_t form)
{
    if (!b || (nodes_per_warp != 1 && nodes_per_warp != 2 && nodes_per_warp != 4 && nodes_per_warp != 8 &&
               nodes_per_warp != 16) ||
        form < 0 || form > 2)
        return MOCD_ERR_INVALID_ARG;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (!b->ctx[i]->ready || b->ctx[i]->version != b->version[i]) return MOCD_ERR_NOT_READY;
    int rc;
    for (mocd_ctx *c : b->ctx) {
        c->nodes_per_warp = nodes_per_warp;
        size_grids(c);
        // Keep each member's own generation graph in the same launch shape.
        drop_graphs(c);
        if ((rc = build_graph(c))) return rc;
    }
    b->form = form;
    return batch_build(b);
}

int mocd_batch_form(mocd_batch *b, int32_t *nodes_per_warp, int32_t *form)
{
    if (!b || b->ctx.empty()) return MOCD_ERR_INVALID_ARG;
    if (nodes_per_warp) *nodes_per_warp = b->ctx[0]->nodes_per_warp;
    if (form) *form = b->form;
    return MOCD_OK;
}

void mocd_batch_destroy(mocd_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    dev_free(b->d_gp, b->stream);
    dev_free(b->d_ps, b->stream);
    dev_free(b->d_members, b->stream);
    dev_free(b->d_starts, b->stream);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int mocd_debug_inject(int32_t site, int32_t skip, int32_t count, int32_t status)
{
    if (site != MOCD_SITE_DEVICE_ALLOC && site != MOCD_SITE_GENERATION) return MOCD_ERR_INVALID_ARG;
    if (skip < 0 || count < 0 || (count > 0 && site == MOCD_SITE_GENERATION && status >= 0))
        return MOCD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_inject_mu);
    g_inject[site] = InjectSite{skip, count, status};
    g_inject_armed.store(g_inject[0].count > 0 || g_inject[1].count > 0, std::memory_order_relaxed);
    return MOCD_OK;
}

int mocd_debug_checks(uint64_t *out, int32_t reset)
{
    if (!out) return MOCD_ERR_INVALID_ARG;
    unsigned long long a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    CK(check_record_eval(a, reset != 0));
    CK(check_record_variation(b, reset != 0));
    out[0] = a[0] + b[0];
    out[1] = a[0] ? a[1] : b[1];
    out[2] = a[0] ? a[2] : b[2];
#ifdef MOCD_DEBUG_CHECKS
    return 1;
#else
    return 0;
#endif
}

int mocd_pool_trim(int64_t keep_bytes)
{
    if (keep_bytes < 0) return MOCD_ERR_INVALID_ARG;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    CK(library_pool(dev, &pool));
    CK(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
    return MOCD_OK;
}

int mocd_debug_pool_usage(int32_t reset_peak, int64_t *current, int64_t *peak)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    CK(library_pool(dev, &pool));
    if (reset_peak) {
        unsigned long long zero = 0;
        CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    unsigned long long cur = 0, hi = 0;
    CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur));
    CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &hi));
    if (current) *current = (int64_t)cur;
    if (peak) *peak = (int64_t)hi;
    return MOCD_OK;
}

void mocd_destroy(mocd_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_population(c);
    dev_free(c->d_row_ptr, c->stream);
    dev_free(c->d_col_idx, c->stream);
    dev_free(c->d_order, c->stream);
    dev_free(c->d_eptr, c->stream);
    dev_free(c->d_eidx, c->stream);
    dev_free(c->d_im, c->stream);
    dev_free(c->d_nm, c->stream);
    dev_free(c->d_eval_acc, c->stream);
    dev_free(c->d_idx, c->stream);
    dev_free(c->d_eval_hist, c->stream);
    dev_free(c->d_volsize, c->stream);
    dev_free(c->d_cut, c->stream);
    dev_free(c->d_stats, c->stream);
    for (int k = 0; k <= kStages; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
