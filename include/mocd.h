/*
 * mocd.h -- C ABI of the GB300 (sm_103a) HP-MOCD generation engine.
 *
 * HP-MOCD (arXiv 2506.01752) evolves a population of N_p partitions of an
 * undirected, unweighted graph G = (V, E) with NSGA-II (Alg. 1), minimising
 *   f1(C) = 1 - sum_c |E(c)| / m   and   f2(C) = sum_c (sum_{v in c} deg v / 2m)^2
 * (Eq. objectives, Sec. 4.1). One generation (Alg. 1, loop body) is:
 * rank and crowding of P, tournament selection of E_S parents per child,
 * topology-aware crossover (Sec. 4.3.1, Alg. 2), topology-aware mutation
 * (Sec. 4.3.2), evaluation of both objectives for every child, and
 * environmental selection of the next P from P u Q.
 *
 * Conventions for every call:
 *   - Return value: MOCD_OK (0) or a negative MOCD_ERR_* status; a call that
 *     fails leaves the context usable unless it returns MOCD_ERR_CUDA.
 *   - Host pointers are read or written only during the call and stay owned
 *     by the caller. The context owns all device memory it allocates.
 *   - Work is issued on the context's CUDA stream; calls that return host data
 *     synchronise that stream first. Calls on one context are not re-entrant;
 *     separate contexts are independent.
 *   - Labels are int32 community ids in [0, n); a label vector of an
 *     individual is n consecutive int32 (individual-major on the host).
 *   - Integer objective keys: k1 = m - intra, where intra = sum_c |E(c)|, and
 *     k2 = S = sum_c D_c^2 with D_c = sum_{v in c} deg v. Then f1 = k1 / m and
 *     f2 = S / (4 m^2), each computed as one IEEE double division. Dominance
 *     (Sec. 2.2) compares (k1, k2) exactly.
 *
 * Limits: 1 <= N_p <= 128, 1 <= E_S <= 16, n < 2^30, 2m < 2^31, and
 * N_p x (number of nodes of degree 33..128 or above 512) < 2^31. There is no
 * degree limit: the mutation's count tables of hubs above degree 512 live in
 * a global scratch of at most 1 GiB per context (one table per warp of the
 * hub kernel, each 2 x the smallest power of two >= 2 d_max ints).
 */
#ifndef MOCD_H
#define MOCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MOCD_OK = 0,
    MOCD_ERR_INVALID_ARG = -1,     /* null pointer, bad size or parameter, label out of range */
    MOCD_ERR_NOT_SYMMETRIC = -2,   /* edge (u, v) present without (v, u) */
    MOCD_ERR_SELF_LOOP = -3,       /* edge (v, v): Sec. 2.1 requires u != v */
    MOCD_ERR_DUPLICATE_EDGE = -4,  /* repeated neighbour: E is a set */
    MOCD_ERR_EMPTY_GRAPH = -5,     /* m = 0: f1 and f2 are undefined */
    MOCD_ERR_OUT_OF_MEMORY = -6,   /* device allocation failed */
    MOCD_ERR_BUFFER_TOO_SMALL = -7,/* caller's capacity below the result size (count set) */
    MOCD_ERR_CUDA = -8,            /* a CUDA call failed */
    MOCD_ERR_NOT_READY = -9,       /* population not initialised yet */
    MOCD_ERR_TOO_LARGE = -10,      /* count * n exceeds MOCD_NOALLOC_MAX_CELLS */
    MOCD_ERR_CANCELLED = -11       /* the server job was cancelled */
};

/* Histogram cells (count * n) the fixed scratch of mocd_evaluate_noalloc holds. */
#define MOCD_NOALLOC_MAX_CELLS 4194304

typedef struct mocd_ctx mocd_ctx;  /* opaque; owns device memory and a stream */

/* Alg. 1 parameters (Table of parameter settings: N_p = 100, C_P = 0.8,
 * M_P = 0.2, E_S = 4). */
typedef struct {
    int32_t pop_size;     /* N_p, 1..128 */
    int32_t n_parents;    /* E_S, parents per crossover, 1..16 */
    double p_crossover;   /* C_P in [0, 1]: crossover iff u <= floor(C_P 2^32) */
    double p_mutation;    /* M_P in [0, 1]: node mutates iff u < floor(M_P 2^32) */
    uint64_t seed;        /* Philox4x32-10 key */
    int32_t init_mode;    /* 0: labels uniform in [0, n) (Alg. 1 InitializePopulation);
                             1: hybrid seeding: every node its own community,
                             then one synchronous full-rate neighbour-majority
                             step (the mutation rule of Sec. 4.3.2), ties broken
                             by the INIT word of (node, individual) */
} mocd_params;

/*
 * Upload a graph (Alg. 1 phase 1: graph storage and PrecomputeDegrees;
 * Sec. 4.2 graph representation).
 *   out      receives a new context (set to NULL on failure)
 *   n        number of nodes, 1 <= n < 2^30
 *   row_ptr  host int64[n + 1], non-decreasing, row_ptr[0] = 0
 *   col_idx  host int32[row_ptr[n]]: symmetric adjacency (each undirected
 *            edge in both rows), no self loops, no repeated neighbours
 *   cuda_stream  cudaStream_t to issue work on, or NULL for a stream the
 *            context creates and owns
 * Rows may come in any order (a sorted copy is made when needed). The host
 * checks every row first (ids in range, self loops, repeats; the first
 * failing row decides the status), then symmetry is checked on the device.
 * The context keeps on the device the CSR (4(n + 1) + 8m bytes), the nodes
 * in degree order (4n) and, for the offspring evaluation, the adjacency with
 * each undirected edge listed once (4(n + 1) + 4m); mocd_job_footprint
 * counts them.
 * Errors: INVALID_ARG, NOT_SYMMETRIC, SELF_LOOP, DUPLICATE_EDGE, EMPTY_GRAPH,
 * OUT_OF_MEMORY, CUDA.
 */
int mocd_graph_upload(mocd_ctx **out, int64_t n, const int64_t *row_ptr,
                      const int32_t *col_idx, void *cuda_stream);

/*
 * Create and evaluate the initial population P^(0) (Alg. 1 phases 1-2:
 * InitializePopulation, then EvaluateIndividual for each member), rank it and
 * draw the tournament of generation 1. Resets the generation counter to 0.
 * Errors: INVALID_ARG (params out of the limits above), OUT_OF_MEMORY, CUDA.
 */
int mocd_population_init(mocd_ctx *ctx, const mocd_params *params);

/*
 * Run n_generations generations of Alg. 1 (the "for gen" loop body), issued
 * asynchronously on the context stream as one CUDA graph launch each.
 * Errors: INVALID_ARG (n_generations < 0), NOT_READY, CUDA.
 */
int mocd_generation(mocd_ctx *ctx, int32_t n_generations);

/*
 * Pareto front of the current population (Alg. 1 phase 4):
 * F_1 = {p in P : rank(p) = 1}, members in P order, and the recommended
 * solution of SelectSolution (Alg. 3, Q = 1 - f1 - f2, Eq. selection; the
 * first member with the largest Q wins).
 *   cap      capacity (members) of the output arrays
 *   count    receives |F_1|; if |F_1| > cap, MOCD_ERR_BUFFER_TOO_SMALL is
 *            returned with count set and nothing else written
 *   labels   host int32[cap * n] or NULL: labels of member k at [k * n]
 *   f1, f2   host double[cap] or NULL
 *   intra, sumsq  host int64[cap] or NULL: exact intra = sum_c |E(c)| and S
 *   best     host int32 or NULL: index into the front of the recommended one
 */
int mocd_pareto_front(mocd_ctx *ctx, int32_t cap, int32_t *count, int32_t *labels,
                      double *f1, double *f2, int64_t *intra, int64_t *sumsq,
                      int32_t *best);

/*
 * Community statistics of every member of the current Pareto front, in the
 * order mocd_pareto_front lists them: the structural properties that Sec. 4.4
 * names as alternative selection criteria and Alg. 3 leaves to the user.
 * For a member with communities c (node sets V_c):
 *   communities       host int64[cap] or NULL: number of non-empty communities k
 *   size_sumsq        host int64[cap] or NULL: sum_c |V_c|^2 (mean size n / k,
 *                     size variance size_sumsq / k - (n / k)^2)
 *   mean_conductance  host double[cap] or NULL: (sum_c phi_c) / k with
 *                     phi_c = cut_c / min(vol_c, 2m - vol_c) rounded once
 *                     (one IEEE division; phi_c = 0 when cut_c = 0), cut_c the
 *                     edges leaving V_c, vol_c the degree total of V_c; the sum
 *                     is exact and rounded once to nearest, then divided by k
 *   max_conductance   host double[cap] or NULL: max_c phi_c
 * The results are exact functions of the labels (no dependence on launch
 * order). Temporary device memory: 12 bytes per (member, node).
 * Errors: INVALID_ARG, NOT_READY, BUFFER_TOO_SMALL (count set, nothing else
 * written), OUT_OF_MEMORY, CUDA.
 */
int mocd_front_stats(mocd_ctx *ctx, int32_t cap, int32_t *count, int64_t *communities,
                     int64_t *size_sumsq, double *mean_conductance,
                     double *max_conductance);

/* Selection criteria over the front (Alg. 3 and the alternatives of Sec. 4.4). */
enum {
    MOCD_SELECT_MODULARITY = 0,       /* largest Q = 1 - f1 - f2 (Alg. 3; Q is
                                         Newman's modularity of the partition) */
    MOCD_SELECT_COMMUNITIES = 1,      /* number of communities nearest `target` */
    MOCD_SELECT_SIZE_VARIANCE = 2,    /* least variance of community sizes (exact) */
    MOCD_SELECT_MEAN_CONDUCTANCE = 3, /* least mean conductance */
    MOCD_SELECT_MAX_CONDUCTANCE = 4   /* least conductance of the worst community */
};

/*
 * Index into the current front (mocd_pareto_front order) of the member that
 * `criterion` prefers; ties go to the larger Q, then to the first in front
 * order, so MOCD_SELECT_MODULARITY returns mocd_pareto_front's `best`.
 *   target  the wanted number of communities (>= 1) for
 *           MOCD_SELECT_COMMUNITIES, ignored otherwise
 * Errors: INVALID_ARG (unknown criterion, target < 1 where it is used),
 * NOT_READY, OUT_OF_MEMORY, CUDA.
 */
int mocd_select_solution(mocd_ctx *ctx, int32_t criterion, int64_t target, int32_t *index);

/*
 * Copy out the whole current population P in P order (checkpoint; also the
 * state that environmental selection of Alg. 1 produced).
 *   labels   host int32[N_p * n] or NULL;  k1, k2 host int64[N_p] or NULL
 *   generation  host int32 or NULL: generations run since initialisation
 */
int mocd_get_population(mocd_ctx *ctx, int32_t *labels, int64_t *k1, int64_t *k2,
                        int32_t *generation);

/*
 * Copy out the offspring Q of the most recent generation, in child order
 * (Alg. 1, the parallel map's output Q^(gen) before environmental selection).
 *   labels   host int32[N_p * n] or NULL;  k1, k2 host int64[N_p] or NULL
 * Errors: NOT_READY (no generation has run since initialisation), CUDA.
 */
int mocd_get_offspring(mocd_ctx *ctx, int32_t *labels, int64_t *k1, int64_t *k2);

/*
 * Replace the population with caller labels (resume from a checkpoint): the
 * labels are evaluated on the device (Eq. objectives), ranked, and the
 * tournament of generation `generation + 1` is drawn, so a run resumed from
 * mocd_get_population continues exactly as the uninterrupted run would.
 *   params   as in mocd_population_init
 *   labels   host int32[N_p * n], values in [0, n)
 *   generation  number of generations already run, >= 0
 * Errors: INVALID_ARG (labels out of range, params as in
 * mocd_population_init, generation < 0), OUT_OF_MEMORY, CUDA.
 */
int mocd_set_population(mocd_ctx *ctx, const mocd_params *params, const int32_t *labels,
                        int32_t generation);

/*
 * Evaluate arbitrary labellings (Eq. objectives; Alg. 1 EvaluateIndividual):
 *   count    number of labellings, >= 0
 *   labels   host int32[count * n], values in [0, n)
 *   intra, sumsq  host int64[count]: exact intra and S of each labelling
 * Uses context-owned scratch; does not touch the population.
 * Errors: INVALID_ARG (labels out of range), OUT_OF_MEMORY, CUDA.
 */
int mocd_evaluate(mocd_ctx *ctx, int32_t count, const int32_t *labels, int64_t *intra,
                  int64_t *sumsq);

/*
 * Objective evaluation that allocates nothing (the paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- e.g. a
 * plug-in whose process gives all free device memory to another allocator, a
 * component under a fixed device-memory budget, or a latency-critical loop
 * that cannot take cudaMalloc's implicit synchronisation). It computes the
 * same exact intra and S as mocd_evaluate, with the evaluation kernel's
 * per-individual histogram kept in a fixed 16 MiB array compiled into the
 * library, which every GPU that loads the library holds until exit.
 *   row_ptr  device int32[n + 1], col_idx device int32[row_ptr[n]]: the
 *            symmetric CSR (no self loops, no repeats; not validated here)
 *   n        nodes, 1 <= n < 2^30
 *   labels   device int32, node-major [n][W], W = count rounded up to a
 *            multiple of 4, 16-byte aligned: labels[v * W + i] is individual
 *            i's label of node v, in [0, n) (not validated here)
 *   count    individuals, 1 <= count <= 128, with count * n <= MOCD_NOALLOC_MAX_CELLS
 *   intra, sumsq  device int64[count], written by the call
 *   cuda_stream   stream to issue on (NULL: the legacy default stream)
 * The call is asynchronous on the stream and calls no cudaMalloc/cudaFree.
 * The first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress) on the current device and keeps it for the rest of
 * the process; make that first call before any stream capture, and do not
 * call the entry point again after a cudaDeviceReset of that device (the kept
 * address would be stale). All calls share the one scratch array, which keeps the
 * previous call's contents (the call clears what it needs), so calls that
 * overlap on the GPU -- e.g. on two streams at once -- race and give wrong
 * results; serialise them.
 * Errors: INVALID_ARG (null pointer, bad n or count), TOO_LARGE
 * (count * n > MOCD_NOALLOC_MAX_CELLS), CUDA.
 */
int mocd_evaluate_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int64_t n,
                          const int32_t *labels, int32_t count, int64_t *intra, int64_t *sumsq,
                          void *cuda_stream);

/*
 * Batched generations of several independent instances -- a deployment form,
 * not a step of the paper (whose Alg. 1 evolves one population). A batch
 * groups initialised contexts on one device; each generation of all of them
 * is ONE CUDA-graph launch in which the per-instance kernel chains
 * (crossover, mutation, evaluation, selection) run concurrently, so small
 * instances and the one-block selection steps of different instances share
 * the GPU. Every instance's results are bit-identical to running it alone.
 *   mocd_batch_create   ctxs: `count` contexts, each initialised
 *                       (mocd_population_init or mocd_set_population), all on
 *                       the current device; the batch does not own them and
 *                       must be destroyed before them. cuda_stream: stream for
 *                       the batch launches, or NULL for one the batch owns.
 *                       Errors: INVALID_ARG, NOT_READY, CUDA.
 *   mocd_batch_generation  n_generations generations of every instance,
 *                       asynchronous on the batch stream. Call
 *                       mocd_batch_synchronize before using a member context
 *                       (its own calls run on its own stream). Re-initialising
 *                       a member invalidates the batch (NOT_READY).
 *   mocd_batch_autotune picks the launch shape (nodes per warp of the node
 *                       kernels, one of 1, 2, 4, 8, 16) with the shortest
 *                       measured batch generation, then the form at that
 *                       shape (below); each trial runs
 *                       `generations_per_trial` generations, so the
 *                       populations advance (re-initialise afterwards for a
 *                       run from generation 0). Results never depend on the
 *                       launch shape or form. Writes the shape to
 *                       *nodes_per_warp.
 *   mocd_batch_configure sets the form explicitly: the nodes per warp (1, 2,
 *                       4, 8 or 16) and form: 0 runs each member's whole
 *                       kernel chain, environmental selection included, on
 *                       its own graph branch (the chains proceed
 *                       independently); 1 runs the selections of all members
 *                       in one launch (a block per member) after every chain
 *                       has evaluated; 2 also runs the crossover, the
 *                       deferred per-pair mutation votes and the evaluation
 *                       of all members in one launch each (each member owns a
 *                       range of the launch's blocks), only the mutation
 *                       kernels staying per member.
 *                       Errors: INVALID_ARG, NOT_READY, CUDA.
 *   mocd_batch_form     reports the current nodes per warp and form.
 */
typedef struct mocd_batch mocd_batch;
int mocd_batch_create(mocd_batch **out, int32_t count, mocd_ctx *const *ctxs, void *cuda_stream);
int mocd_batch_generation(mocd_batch *b, int32_t n_generations);
int mocd_batch_autotune(mocd_batch *b, int32_t generations_per_trial, int32_t *nodes_per_warp);
int mocd_batch_synchronize(mocd_batch *b);
int mocd_batch_configure(mocd_batch *b, int32_t nodes_per_warp, int32_t form);
int mocd_batch_form(mocd_batch *b, int32_t *nodes_per_warp, int32_t *form);
void mocd_batch_destroy(mocd_batch *b);

/*
 * Continuous-batching detection server -- a deployment form, not a step of the
 * paper. Jobs (a graph, parameters and a generation count) are queued by
 * mocd_server_submit; each mocd_server_step call (a scheduling round):
 *   1. retires running jobs whose last generation has completed: their Pareto
 *      front (as mocd_pareto_front returns it) is kept for mocd_server_result
 *      and their device memory is released;
 *   2. admits queued jobs in submission order while the estimated device
 *      footprint of the running jobs stays within hbm_budget_bytes and fewer
 *      than max_running jobs run (a job larger than the whole budget fails
 *      with OUT_OF_MEMORY); admission uploads the graph and initialises the
 *      population (host work, blocking);
 *   3. issues up to `depth` further generations of every running job, each job
 *      on its own CUDA stream, so running jobs share the GPU concurrently.
 * A job's result depends only on its own inputs: it is identical alone and in
 * any mix. mocd_server_step never blocks on the GPU except to copy finished
 * fronts; call it in a loop.
 *   mocd_server_submit  copies the host CSR (validated at admission); the
 *                       job id is written to *job_id (ids start at 1).
 *   mocd_server_job_state  *state: 0 queued, 1 running, 2 done, 3 failed
 *                       (*status then holds the MOCD_ERR_* code), 4 cancelled.
 *   mocd_server_cancel  cancels a job: a queued job at once; an admitted job
 *                       gets no further generations and is retired (its
 *                       device memory released, its state cancelled) by a
 *                       later round, once the generations already issued for
 *                       it have completed. OK for a job already cancelled;
 *                       INVALID_ARG for an unknown or finished job.
 *   mocd_server_result  as mocd_pareto_front, for a done job; the job's
 *                       status for a failed or cancelled one, NOT_READY
 *                       while it is queued or running.
 *   mocd_server_start   switches to background mode: a scheduler thread runs
 *                       the rounds (mocd_server_step then only reports counts)
 *                       and `admission_threads` workers (1..16) validate,
 *                       upload and initialise admitted jobs while the GPU runs
 *                       the others. policy 0 admits in submission order;
 *                       policy 1 admits the queued job with the highest
 *                       response ratio (waiting time + estimated run time) /
 *                       estimated run time, the run time estimated from its
 *                       size (n + 2m) x (G + 1) and the measured time per
 *                       unit of size of the jobs completed so far: short jobs
 *                       first, and a waiting job's priority grows until it is
 *                       admitted.
 * Calls on one server may come from any host thread.
 *   mocd_job_footprint  the device bytes the server accounts for a job on the
 *                       graph with host row pointers row_ptr[n + 1] while it
 *                       runs (admission compares their sum with the budget):
 *                       the four label buffers and the degree histogram
 *                       (5 x 4 n W bytes, W = N_p rounded up to a multiple of
 *                       4), the CSR and node order, the mutation's per-node
 *                       hints (4 n), deferred-vote list (8 N_p per node of
 *                       degree 33..128 or above 512) and hub count tables
 *                       (graphs with a degree above 512), the individual-major
 *                       buffer of the
 *                       front download (4 n N_p) and 1 MiB of small state.
 *                       Errors: INVALID_ARG.
 */
typedef struct mocd_server mocd_server;
int mocd_server_create(mocd_server **out, int64_t hbm_budget_bytes, int32_t max_running, int32_t depth);
int mocd_server_start(mocd_server *s, int32_t admission_threads, int32_t policy);
int mocd_server_submit(mocd_server *s, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const mocd_params *params, int32_t generations, int64_t *job_id);
int mocd_server_step(mocd_server *s, int32_t *running, int32_t *queued, int32_t *done);
int mocd_server_job_state(mocd_server *s, int64_t job_id, int32_t *state, int32_t *status);
int mocd_server_cancel(mocd_server *s, int64_t job_id);
int mocd_server_result(mocd_server *s, int64_t job_id, int32_t cap, int32_t *count, int32_t *labels,
                       double *f1, double *f2, int64_t *intra, int64_t *sumsq, int32_t *best);
void mocd_server_destroy(mocd_server *s);
int mocd_job_footprint(int64_t n, const int64_t *row_ptr, int32_t pop_size, int64_t *bytes);

/*
 * Test support (not a step of the method): host-side failure injection, so
 * that error paths can be exercised without any GPU fault. After `skip`
 * further calls at `site` succeed, the next `count` calls there fail; the
 * setting is process-wide and count = 0 disarms the site.
 *   MOCD_SITE_DEVICE_ALLOC  every device allocation of the library fails as
 *                           if the device were out of memory (the calling
 *                           entry point returns OUT_OF_MEMORY; `status` is
 *                           ignored)
 *   MOCD_SITE_GENERATION    mocd_generation returns `status` (a negative
 *                           MOCD_ERR_* code) without launching anything
 * Errors: INVALID_ARG (unknown site, negative skip or count, non-negative
 * status for the generation site).
 */
enum { MOCD_SITE_DEVICE_ALLOC = 0, MOCD_SITE_GENERATION = 1 };
int mocd_debug_inject(int32_t site, int32_t skip, int32_t count, int32_t status);

/*
 * Test support: the bounds checks of the debug build (the library built with
 * -DMOCD_DEBUG_CHECKS, see paper_2506_01752_gb300.build.build(debug=True)).
 * There the kernels check the invariants their memory accesses rely on (CSR
 * row pointers non-decreasing, neighbour ids and labels in [0, n), indices
 * into P u Q below 2 N_p); a failed check never traps: the access is skipped
 * (or redirected in bounds) and the failure recorded. out[0] receives the
 * number of failures since the last reset, out[1] the first failure's code
 * (1 row pointers, 2 node id, 3 label, 4 index into P u Q) and out[2] its
 * node or slot; reset != 0 then clears the record. Returns 1 in the debug
 * build, 0 in the normal one (whose kernels check nothing: out is zero), or
 * a negative status (INVALID_ARG, CUDA).
 */
int mocd_debug_checks(uint64_t *out, int32_t reset);

/*
 * Device memory: every device allocation of the library comes from one
 * stream-ordered memory pool per device that the library creates. Memory a
 * destroyed context (or finished server job) freed stays reserved in the
 * pool for the next one, which then allocates without mapping fresh memory.
 * mocd_pool_trim releases reserved memory of the current device's pool that
 * is not in use, down to keep_bytes (0: all of it), e.g. before another part
 * of the process needs the device memory. Errors: INVALID_ARG
 * (keep_bytes < 0), CUDA.
 */
int mocd_pool_trim(int64_t keep_bytes);

/*
 * Test support: bytes in use now and the high-water mark since the last
 * reset in the current device's memory pool of the library (see
 * mocd_pool_trim; reset_peak != 0 first resets the mark to the current use).
 * Either pointer may be NULL. Errors: CUDA.
 */
int mocd_debug_pool_usage(int32_t reset_peak, int64_t *current, int64_t *peak);

/* Block until all work issued on the context stream is done. */
int mocd_synchronize(mocd_ctx *ctx);

/*
 * Per-kernel timing of the generation step (measurement support, not part
 * of the method): when enabled, the generation graph records CUDA events
 * between its kernels. mocd_kernel_times writes, for the most recent
 * generation, the duration in milliseconds of each stage, in this order:
 * crossover, mutation (its main kernel plus the per-pair vote kernels of
 * the graph's degree classes; it also builds the degree histogram of the
 * children), evaluation (which squares and clears that histogram),
 * selection; returns the number of stages (4) or a negative status.
 * NOT_READY if timing is off or no generation ran since it was enabled.
 */
int mocd_set_timing(mocd_ctx *ctx, int32_t enable);
int mocd_kernel_times(mocd_ctx *ctx, float *ms, int32_t cap);

/*
 * Number of kernel launches in one generation (measurement support): the
 * kernel nodes of the captured generation graph without timing events.
 * It depends on the graph: crossover, mutation, evaluation and selection,
 * plus one per-pair vote kernel for each degree class the graph has
 * (33..64, 65..128, above 512). Captures the graph if it does not exist
 * yet. NOT_READY before initialisation.
 */
int mocd_generation_kernels(mocd_ctx *ctx, int32_t *kernels);

/* Graph size and population shape: any pointer may be NULL. */
int mocd_info(mocd_ctx *ctx, int64_t *n, int64_t *m, int32_t *pop_size, int32_t *generation);

/* Release the context and all device memory it owns. NULL is ignored. */
void mocd_destroy(mocd_ctx *ctx);

/* Static description of a status code. */
const char *mocd_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* MOCD_H */
