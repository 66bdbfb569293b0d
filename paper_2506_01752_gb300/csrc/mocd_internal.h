// mocd_internal.h -- declarations shared by the CUDA translation units of the
// HP-MOCD generation engine (kernels + host runtime). Not part of the C ABI.
//
// Device data layout (node-major, "row per node"):
//   labels   int32 [n][W]   W = pop_size rounded up to a multiple of 4; column i
//                            of row v is individual i's label of node v, so a
//                            warp reads a node's labels for every individual
//                            as one contiguous 16-byte-per-lane row.
//   hist     uint32 [Np][n] per-individual community degree totals D_c
//                            (scratch, cleared before every evaluation)
//   CSR      int32 row_ptr[n + 1], int32 col_idx[2m] (symmetric)
//   order    int32[n] nodes by degree, descending (work order of the
//            degree-proportional kernels; results do not depend on it)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct mocd_ctx;

namespace mocd {

// Record `ev` on the context's stream (after all work issued so far).
int record_on_stream(mocd_ctx *c, cudaEvent_t ev);

// Every device allocation of the library (stream-ordered cudaMallocAsync);
// fails with cudaErrorMemoryAllocation when a test injects a failure there.
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);

// Host-side failure injection (mocd_debug_inject): true if the next call at
// `site` is to fail; *status (if given) receives the status to return.
constexpr int kSiteDeviceAlloc = 0;
constexpr int kSiteGeneration = 1;
bool inject_failure(int site, int *status);

constexpr int kMaxPop = 128;      // N_p limit: one int4 of labels per lane per row
constexpr int kMaxParents = 16;   // E_S limit
constexpr int kBlock = 256;       // threads per block of the node-parallel kernels
// Mutation votes of nodes with degree 33..kDeferMax that the Misra-Gries
// pass leaves open run one pair per thread in a second kernel (degree
// classes 33..64 and 65..128); higher degrees use a per-warp count table.
constexpr int kDeferMax = 128;
// Above this degree a node's count table no longer fits in shared memory:
// its open pairs are listed for mutation_hub_kernel, which keeps the table of
// each pair in a per-warp slice of global scratch.
constexpr int kSharedTableMax = 512;

// Random stream stages (third word of the Philox counter is the generation).
constexpr uint32_t kStageInit = 1;
constexpr uint32_t kStageSelect = 2;
constexpr uint32_t kStageCrossTie = 3;
constexpr uint32_t kStageMutCoin = 4;
constexpr uint32_t kStageMutTie = 5;

// Per-generation device state of one population.
struct PopState {
    int32_t *buf[2];          // P halves [n][W]: the P of R is buf[(g + 1) & 1]
    int32_t *q;               // Q [n][W]
    int32_t *c;               // post-crossover children [n][W]
    uint32_t *hist;           // [n][W] label-major D of (individual, label); zero between evaluations
    unsigned long long *acc;  // [2][kMaxPop]: intra (undirected edges), S
    int64_t *pk;              // [2][kMaxPop]: P keys k1 (m - intra), k2 (S), P order
    int64_t *rk;              // [2][2 kMaxPop]: R keys (P then Q) of the last selection
    int32_t *prank;           // [kMaxPop] rank of P on its own keys (1-based)
    int32_t *keep;            // [kMaxPop] R index of each P position
    int32_t *par_r;           // [kMaxPop][kMaxParents] parent R indices per child
    int32_t *copy_r;          // [kMaxPop] R index copied when crossover is skipped, else -1
    uint32_t *gen;            // next generation number to run (device counter)
    int32_t *front;           // [2 + kMaxPop]: count, best, members (P positions)
    int64_t *fint;            // [2][kMaxPop]: intra, S of each front member
    double *fval;             // [2][kMaxPop]: f1, f2 of each front member
    uint32_t *hint;           // [n]: (mutating pairs << 16) | pairs the Misra-Gries pass settles (a label above
                              // deg / (K + 1), K its counters), last generation; nodes of degree > 32
    int2 *dlist;              // deferred mutation votes (node, child): class 0 then class 1
    int *dcount;              // [3]: deferred votes appended this generation: degree 33..64, 65..128, hubs
    int *hub_table;           // hub_warps x 2 hub_hs: per-warp count tables of the hub votes
};

struct GenParams {
    int n;                    // nodes
    int W;                    // row width (ints)
    int np;                   // N_p
    int es;                   // E_S
    int label_bits;           // bits needed for a label in [0, n)
    int hash_size;            // per-warp hash entries for degree > kDeferMax (0: none)
    int defer_cap[3];         // deferred-vote capacity per class: N_p x nodes of the class
    int hub_hs;               // slots of a hub count table (power of two >= 2 dmax; 0: no hubs)
    int hub_warps;            // warps of mutation_hub_kernel (one table slice each)
    int vote_n0;              // entries of the degree 33..64 vote's sorting network: the smallest multiple
                              // of 8 that holds the graph's largest degree in that class (40, 48, 56 or 64)
    int64_t m;                // edges
    uint32_t key0, key1;      // Philox key (seed)
    unsigned long long thr_c; // crossover iff u <= thr_c
    unsigned long long thr_m; // mutate iff u < thr_m
};

// One member of a multi-member launch (a batch of contexts): its parameters,
// state and graph.
struct BatchMember {
    GenParams gp;
    PopState ps;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *order;
    const int32_t *eptr;  // the offspring evaluation's oriented adjacency (mocd_ctx::d_eptr / d_eidx)
    const int32_t *eidx;
};

// Launch wrappers (stream-ordered, return cudaGetLastError()).
// init_mode 0: labels uniform in [0, n); 1: singletons then one full-rate
// neighbour-majority step (needs the sorted, repeat-free adjacency).
cudaError_t launch_init_population(const GenParams &gp, int init_mode, const int32_t *row_ptr,
                                   const int32_t *col_idx, int32_t *dst, cudaStream_t s);
cudaError_t launch_crossover(const GenParams &gp, const PopState &ps, int grid, cudaStream_t s);
// order: the nodes in the sequence the grid-stride loop visits them
// (degree descending), or NULL for 0..n-1 (evaluation only).
// with_votes false: the per-pair votes of the deferred classes are left to
// launch_vote_multi (a batch launches them for all members at once).
cudaError_t launch_mutation(const GenParams &gp, const PopState &ps, const int32_t *row_ptr,
                            const int32_t *col_idx, const int32_t *order, int grid, int grid64, int grid128,
                            cudaStream_t s, bool with_votes = true);
// Multi-member launches of a batch: member k owns blocks starts[k] ..
// starts[k + 1] - 1 of the launch's `blocks` (each member's own grid for
// the stage; zero for a member with nothing to do).
cudaError_t launch_crossover_multi(const BatchMember *members, const int *starts, int count, int blocks, int es_max,
                                   cudaStream_t s);
cudaError_t launch_vote_multi(const BatchMember *members, const int *starts, int count, int blocks, int cls,
                              cudaStream_t s);
cudaError_t launch_evaluate_multi(const BatchMember *members, const int *starts, int count, int blocks,
                                  cudaStream_t s);
// Resident-block grids of the two per-pair vote kernels (degree classes
// 33..64 and 65..128).
void grid_for_votes(int sms, int vote_n0, int *grid64, int *grid128);
// hist: label-major [n][W] (label_major) or individual-major [count][n],
// zeroed by the caller.
cudaError_t launch_evaluate(int n, int W, int count, const int32_t *row_ptr, const int32_t *col_idx,
                            const int32_t *labels, uint32_t *hist, unsigned long long *acc,
                            int grid, cudaStream_t s, const int32_t *order = nullptr,
                            bool label_major = true);
// mode 0: keys of a fresh P from acc, keep = identity; mode 1: R = P u Q,
// environmental selection. Both then rank P and draw the next tournament.
cudaError_t launch_select(const GenParams &gp, const PopState &ps, int mode, cudaStream_t s);
// The selections of `count` populations (device arrays of their parameters
// and states) in one launch, a block each.
cudaError_t launch_select_multi(const GenParams *gps, const PopState *pss, int count, int mode, cudaStream_t s);
cudaError_t launch_front(const GenParams &gp, const PopState &ps, cudaStream_t s);
// Community statistics of the `count` front members (front_kernel's list):
// rows [n][round4(count)] ints, volsize [count][n] u64 and cut [count][n] u32
// zeroed, acc stats_acc_words() u64 zeroed; out [4][kMaxPop] u64 receives
// communities, size_sumsq, mean conductance and max conductance (double bits).
size_t stats_acc_words();
cudaError_t launch_front_stats(const GenParams &gp, const PopState &ps, const int32_t *phalf, int count,
                               const int32_t *row_ptr, const int32_t *col_idx, const int32_t *order,
                               int32_t *rows, unsigned long long *volsize, uint32_t *cut,
                               unsigned long long *acc, unsigned long long *out, int sms, cudaStream_t s);
// out[k][v] = R_v[idx[k]] for k < count, R_v = (phalf row v | q row v); idx NULL: identity on phalf.
cudaError_t launch_gather_individuals(int n, int W, int np, const int32_t *phalf, const int32_t *q,
                                      const int32_t *idx, int count, int32_t *out, cudaStream_t s);
// dst[v][k] = src[k][v] for k < count, zero for count <= k < W.
cudaError_t launch_to_node_major(int n, int W, int count, const int32_t *src, int32_t *dst,
                                 cudaStream_t s);
// The offspring evaluation's oriented adjacency of a host-checked CSR: eptr
// [n + 1] row pointers, eidx [cap] entries (cap = m for a symmetric graph),
// each undirected edge listed once, at its endpoint of lower (degree, id).
cudaError_t launch_orient(int n, const int32_t *row_ptr, const int32_t *col_idx, int32_t *eptr, int32_t *eidx,
                          int cap, int sms, cudaStream_t s);
// *bad = 1 if some stored entry (v, u) has no mirror (u, v); rows must be
// sorted, in range and free of self loops (checked on the host first).
cudaError_t launch_symmetry_check(int n, const int32_t *row_ptr, const int32_t *col_idx, int *bad, int sms,
                                  cudaStream_t s);
// Debug-build bounds-check records of the kernel translation units
// (mocd_check.cuh): out[3] = failures, first code, first index.
cudaError_t check_record_eval(unsigned long long *out, bool reset);
cudaError_t check_record_variation(unsigned long long *out, bool reset);

// Occupancy-derived grid sizes.
// Resident blocks of the evaluation kernel in the given histogram layout.
int grid_for_eval(int sms, bool label_major = true);
int grid_for_eval_intra(int sms);
// Objectives of the offspring inside a generation: the mutation kernel has
// already added every child's degrees to the label-major histogram (and
// cleared acc); one launch counts intra, then forms S from the histogram and
// zeroes it. eptr / eidx: the oriented adjacency, each undirected edge once
// (mocd_ctx::d_eptr / d_eidx).
cudaError_t launch_evaluate_offspring(int n, int W, int count, const int32_t *eptr, const int32_t *eidx,
                                      const int32_t *labels, uint32_t *hist, unsigned long long *acc,
                                      int grid, cudaStream_t s, const int32_t *order);
int grid_for_crossover(int sms, int es);
int grid_for_mutation(int sms, int hash_size, int *smem_bytes);
int mutation_warps_per_block();

}  // namespace mocd
