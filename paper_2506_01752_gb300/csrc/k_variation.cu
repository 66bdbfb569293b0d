// k_variation.cu -- InitializePopulation and the offspring map of Alg. 1:
// topology-aware crossover (Sec. 4.3.1, Alg. 2) and topology-aware mutation
// (Sec. 4.3.2), for all N_p children of a generation at once.
//
// Both kernels work on node-major rows: a warp owns node v; lane q owns the
// four children 4q..4q+3, which share one Philox call per stage because the
// stream counter of (child i, node v) is (v, i / 4, g, stage), word i % 4.
#include <limits.h>

#include <utility>

#include "mocd_check.cuh"
#include "mocd_internal.h"
#include "philox.cuh"

namespace mocd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// InitializePopulation: label of (individual i, node v) = pick(u, n), u the
// INIT word of (v, i) at generation 0.
// ---------------------------------------------------------------------------
__global__ void init_population_kernel(int n, int W, int np, uint32_t k0, uint32_t k1,
                                       int32_t *__restrict__ dst)
{
    const int nq = W >> 2;
    const long long total = (long long)n * nq;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / nq);
        const int q = (int)(t % nq);
        const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)q, 0u, kStageInit), k0, k1);
        int4 o;
        o.x = 4 * q + 0 < np ? (int)pick_index(r.x, (uint32_t)n) : 0;
        o.y = 4 * q + 1 < np ? (int)pick_index(r.y, (uint32_t)n) : 0;
        o.z = 4 * q + 2 < np ? (int)pick_index(r.z, (uint32_t)n) : 0;
        o.w = 4 * q + 3 < np ? (int)pick_index(r.w, (uint32_t)n) : 0;
        reinterpret_cast<int4 *>(dst)[t] = o;
    }
}

// ---------------------------------------------------------------------------
// Hybrid initialisation (init_mode 1): every node starts as its own community
// and then takes one synchronous neighbour-majority step at full rate, the tie
// broken by the INIT word of (v, i). In a singleton partition the labels of
// v's neighbours are their ids, all distinct because the uploaded adjacency
// has no repeats, so every neighbour ties at count 1 and the tied labels in
// ascending order are the adjacency row itself (it is stored sorted). The
// step therefore reads entry pick(u, deg v) of the row; a node of degree 0
// keeps label v.
// ---------------------------------------------------------------------------
__global__ void init_sweep_kernel(int n, int W, int np, uint32_t k0, uint32_t k1,
                                  const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col_idx, int32_t *__restrict__ dst)
{
    const int nq = W >> 2;
    const long long total = (long long)n * nq;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / nq);
        const int q = (int)(t % nq);
        const int beg = __ldg(row_ptr + v);
        const uint32_t d = (uint32_t)(__ldg(row_ptr + v + 1) - beg);
        int4 o = make_int4(v, v, v, v);
        if (d > 0) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)q, 0u, kStageInit), k0, k1);
            o.x = __ldg(col_idx + beg + pick_index(r.x, d));
            o.y = __ldg(col_idx + beg + pick_index(r.y, d));
            o.z = __ldg(col_idx + beg + pick_index(r.z, d));
            o.w = __ldg(col_idx + beg + pick_index(r.w, d));
        }
        if (4 * q + 0 >= np) o.x = 0;
        if (4 * q + 1 >= np) o.y = 0;
        if (4 * q + 2 >= np) o.z = 0;
        if (4 * q + 3 >= np) o.w = 0;
        reinterpret_cast<int4 *>(dst)[t] = o;
    }
}

// ---------------------------------------------------------------------------
// Crossover. Row v of R = (P half | Q) is staged in shared memory; the next P
// (environmental selection's keep list) is compacted into the other P half,
// and child i of the generation gets
//   copy_r[i] >= 0 : R_v[copy_r[i]]                    (x > C_P: random parent)
//   otherwise      : majority of R_v[par_r[i][j]], j < E_S, the tie among the t
//                    most frequent labels broken by the XTIE word: the
//                    pick(u, t)-th smallest of them (Eq. arg_max).
// ---------------------------------------------------------------------------

// Count of the maximal label and number t of distinct labels reaching it.
template <int EMAX>
__device__ __forceinline__ int mode_ties(const int (&x)[EMAX], int E, int &best)
{
    int cnt[EMAX];
#pragma unroll
    for (int a = 0; a < EMAX; ++a) {
        cnt[a] = 0;
#pragma unroll
        for (int b = 0; b < EMAX; ++b)
            if (a < E && b < E && x[b] == x[a]) cnt[a] += 1;
    }
    best = 0;
#pragma unroll
    for (int a = 0; a < EMAX; ++a)
        if (a < E && cnt[a] > best) best = cnt[a];
    int t = 0;
#pragma unroll
    for (int a = 0; a < EMAX; ++a) {
        bool first = a < E && cnt[a] == best;
#pragma unroll
        for (int b = 0; b < EMAX; ++b)
            if (b < a && x[b] == x[a]) first = false;
        t += first ? 1 : 0;
    }
    // Distinct maximal labels: a label's first occurrence is counted once.
    return t;
}

// The k-th smallest distinct label among those of count `best`.
template <int EMAX>
__device__ __forceinline__ int kth_tied(const int (&x)[EMAX], int E, int best, int k)
{
    int res = x[0];
#pragma unroll
    for (int a = 0; a < EMAX; ++a) {
        if (a >= E) continue;
        int c = 0;
        bool first = true;
#pragma unroll
        for (int b = 0; b < EMAX; ++b) {
            if (b >= E) continue;
            c += x[b] == x[a];
            if (b < a && x[b] == x[a]) first = false;
        }
        if (!first || c != best) continue;
        // rank of x[a] among the distinct tied labels
        int rank = 0;
#pragma unroll
        for (int b = 0; b < EMAX; ++b) {
            if (b >= E) continue;
            int cb = 0;
            bool fb = true;
#pragma unroll
            for (int e = 0; e < EMAX; ++e) {
                if (e >= E) continue;
                cb += x[e] == x[b];
                if (e < b && x[e] == x[b]) fb = false;
            }
            if (fb && cb == best && x[b] < x[a]) rank += 1;
        }
        if (rank == k) res = x[a];
    }
    return res;
}

template <int EMAX>
__device__ __forceinline__ void crossover_body(const GenParams gp, const int32_t *buf0, const int32_t *buf1,
                                               int32_t *out0, int32_t *out1, const int32_t *__restrict__ q,
                                               int32_t *__restrict__ child, const int32_t *__restrict__ keep,
                                               const int32_t *__restrict__ par_r, const int32_t *__restrict__ copy_r,
                                               const uint32_t *__restrict__ gen_ptr, int *__restrict__ dcount,
                                               int vblock, int vgrid)
{
    // The mutation kernel that follows appends deferred pairs from zero.
    if (vblock == 0 && threadIdx.x < 3) dcount[threadIdx.x] = 0;
    extern __shared__ int smem[];
    const int W = gp.W, np = gp.np, E = gp.es;
    const int nq = W >> 2;
    // Per-child tables, stored so that lane q reading child 4q + k hits bank q:
    // entry (k, q) of a table lives at [k * 32 + q] (and [(j * 4 + k) * 32 + q]
    // for parent j).
    int *s_keep = smem;                    // row position of P position i
    int *s_copy = s_keep + kMaxPop;        // row position copied, or -1
    int *s_par = s_copy + kMaxPop;         // row positions of parents
    int *s_rows = s_par + kMaxPop * EMAX;  // per warp: [2W] staged row of R

    const uint32_t g = *gen_ptr;
    // R index r -> position in the staged row (P half at [0, W), Q at [W, 2W)).
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int slot = (t & 3) * 32 + (t >> 2);
        int r = keep[t];
        if (!MOCD_CHECK(r >= 0 && r < 2 * np, kCheckRIndex, t)) r = 0;
        s_keep[slot] = r < np ? r : W + (r - np);
        int c = copy_r[t];
        if (!MOCD_CHECK(c >= -1 && c < 2 * np, kCheckRIndex, t)) c = 0;
        s_copy[slot] = c < 0 ? -1 : (c < np ? c : W + (c - np));
        for (int j = 0; j < E; ++j) {
            int p = par_r[t * kMaxParents + j];
            if (!MOCD_CHECK(p >= 0 && p < 2 * np, kCheckRIndex, t)) p = 0;
            s_par[(j * 4 + (t & 3)) * 32 + (t >> 2)] = p < np ? p : W + (p - np);
        }
    }
    __syncthreads();

    // Generation g reads the P half buf[g & 1] and writes the compacted P
    // into the other half (the two never alias within one launch).
    const int4 *P4 = reinterpret_cast<const int4 *>((g & 1u) ? buf1 : buf0);
    int4 *D4 = reinterpret_cast<int4 *>((g & 1u) ? out0 : out1);
    const int4 *__restrict__ Q4 = reinterpret_cast<const int4 *>(q);
    int4 *__restrict__ C4 = reinterpret_cast<int4 *>(child);

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int *row = s_rows + wib * 2 * W;
    const int warp = (vblock * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (vgrid * blockDim.x) >> 5;
    const bool active = lane < nq;

    // Software pipeline: the next node's rows are requested before the
    // current node is processed.
    int4 cur_p = make_int4(0, 0, 0, 0), cur_q = make_int4(0, 0, 0, 0);
    if (active && warp < gp.n) {
        cur_p = P4[(size_t)warp * nq + lane];
        cur_q = Q4[(size_t)warp * nq + lane];
    }
    for (int v = warp; v < gp.n; v += nwarps) {
        const int vn = v + nwarps;
        int4 nxt_p = make_int4(0, 0, 0, 0), nxt_q = make_int4(0, 0, 0, 0);
        if (active && vn < gp.n) {
            nxt_p = P4[(size_t)vn * nq + lane];
            nxt_q = Q4[(size_t)vn * nq + lane];
        }
        if (active) {
            reinterpret_cast<int4 *>(row)[lane] = cur_p;
            reinterpret_cast<int4 *>(row + W)[lane] = cur_q;
        }
        cur_p = nxt_p;
        cur_q = nxt_q;
        __syncwarp();
        if (active && EMAX == 4 && E == 4) {
            // Sort each child's four votes (5 comparators); the run pattern of
            // the sorted values gives the maximal labels in ascending order:
            // t = 4 (all distinct), t = 2 (two pairs) or a unique maximum. All
            // four children are classified first so that the lane's tie word
            // (one Philox call for its four children) is computed at most once.
            int o[4], srt[4][4], tk[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * lane + k;
                o[k] = i < np ? row[s_keep[k * 32 + lane]] : 0;
                const int cp = i < np ? s_copy[k * 32 + lane] : 0;
                // Children past N_p (padding of the last quad) have no parent table.
                const bool real = i < np;
                int s0 = row[real ? s_par[(0 * 4 + k) * 32 + lane] : 0];
                int s1 = row[real ? s_par[(1 * 4 + k) * 32 + lane] : 0];
                int s2 = row[real ? s_par[(2 * 4 + k) * 32 + lane] : 0];
                int s3 = row[real ? s_par[(3 * 4 + k) * 32 + lane] : 0];
                int lo, hi;
                lo = min(s0, s1); hi = max(s0, s1); s0 = lo; s1 = hi;
                lo = min(s2, s3); hi = max(s2, s3); s2 = lo; s3 = hi;
                lo = min(s0, s2); hi = max(s0, s2); s0 = lo; s2 = hi;
                lo = min(s1, s3); hi = max(s1, s3); s1 = lo; s3 = hi;
                lo = min(s1, s2); hi = max(s1, s2); s1 = lo; s2 = hi;
                const bool e01 = s0 == s1, e12 = s1 == s2, e23 = s2 == s3;
                int t = (!e01 && !e12 && !e23) ? 4 : ((e01 && e23 && !e12) ? 2 : 1);
                int uniq = e01 ? s0 : (e12 ? s1 : s2);
                if (i >= np) {
                    t = 1;
                    uniq = 0;
                } else if (cp >= 0) {
                    t = 1;
                    uniq = row[cp];
                }
                srt[k][0] = t == 1 ? uniq : s0;
                srt[k][1] = s1;
                srt[k][2] = s2;
                srt[k][3] = s3;
                tk[k] = t;
            }
            uint4 u = make_uint4(0, 0, 0, 0);
            if (tk[0] > 1 || tk[1] > 1 || tk[2] > 1 || tk[3] > 1)
                u = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)lane, g, kStageCrossTie), gp.key0, gp.key1);
            int r[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t w = word_of(u, k);
                if (tk[k] == 4) {
                    const uint32_t kk = pick_index(w, 4u);
                    r[k] = kk == 0 ? srt[k][0] : kk == 1 ? srt[k][1] : kk == 2 ? srt[k][2] : srt[k][3];
                } else if (tk[k] == 2) {
                    r[k] = pick_index(w, 2u) == 0 ? srt[k][0] : srt[k][2];
                } else {
                    r[k] = srt[k][0];
                }
            }
            D4[(size_t)v * nq + lane] = make_int4(o[0], o[1], o[2], o[3]);
            C4[(size_t)v * nq + lane] = make_int4(r[0], r[1], r[2], r[3]);
        } else if (active) {
            int o[4];
            int r[4];
            bool have_u = false;
            uint4 u = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * lane + k;
                o[k] = i < np ? row[s_keep[k * 32 + lane]] : 0;
                r[k] = 0;
                if (i >= np) continue;
                const int cp = s_copy[k * 32 + lane];
                if (cp >= 0) {
                    r[k] = row[cp];
                    continue;
                }
                int x[EMAX];
#pragma unroll
                for (int j = 0; j < EMAX; ++j) x[j] = j < E ? row[s_par[(j * 4 + k) * 32 + lane]] : 0;
                int best;
                const int t = mode_ties<EMAX>(x, E, best);
                int kk = 0;
                if (t > 1) {
                    if (!have_u) {
                        u = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)lane, g, kStageCrossTie),
                                          gp.key0, gp.key1);
                        have_u = true;
                    }
                    kk = (int)pick_index(word_of(u, k), (uint32_t)t);
                }
                r[k] = kth_tied<EMAX>(x, E, best, kk);
            }
            D4[(size_t)v * nq + lane] = make_int4(o[0], o[1], o[2], o[3]);
            C4[(size_t)v * nq + lane] = make_int4(r[0], r[1], r[2], r[3]);
        }
        __syncwarp();
    }
}

template <int EMAX>
__global__ void __launch_bounds__(kBlock)
crossover_kernel(GenParams gp, const int32_t *buf0, const int32_t *buf1, int32_t *out0, int32_t *out1,
                 const int32_t *__restrict__ q, int32_t *__restrict__ child,
                 const int32_t *__restrict__ keep, const int32_t *__restrict__ par_r,
                 const int32_t *__restrict__ copy_r, const uint32_t *__restrict__ gen_ptr,
                 int *__restrict__ dcount)
{
    crossover_body<EMAX>(gp, buf0, buf1, out0, out1, q, child, keep, par_r, copy_r, gen_ptr, dcount, blockIdx.x,
                         gridDim.x);
}

// The member of a multi-member launch that block blockIdx.x belongs to:
// members own consecutive block ranges, starts[k] .. starts[k + 1] - 1
// (empty for a member with nothing to do).
__device__ __forceinline__ int member_of_block(const int *__restrict__ starts, int count)
{
    const int b = (int)blockIdx.x;
    int lo = 0, hi = count;  // starts[lo] <= b < starts[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(starts + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Crossover of every member of a batch in one launch.
template <int EMAX>
__global__ void __launch_bounds__(kBlock)
crossover_multi_kernel(const BatchMember *__restrict__ members, const int *__restrict__ starts, int count)
{
    const int k = member_of_block(starts, count);
    const BatchMember &mb = members[k];
    const PopState &ps = mb.ps;
    const int b0 = __ldg(starts + k);
    crossover_body<EMAX>(mb.gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r,
                         ps.copy_r, ps.gen, ps.dcount, (int)blockIdx.x - b0, __ldg(starts + k + 1) - b0);
}

// ---------------------------------------------------------------------------
// Mutation (Sec. 4.3.2). Node v of child i mutates iff its MCOIN word is
// below thr_m and deg(v) > 0; it then takes the most frequent label among its
// neighbours in the post-crossover child (synchronous: all reads come from
// `child`), the tie among the t most frequent labels broken by the MTIE word
// (the pick(u, t)-th smallest). A warp takes a node; its lanes take the
// node's selected children, whose neighbour labels are staged into a
// per-warp tile (a column per pair). Degree <= 32: when many pairs are
// selected, each lane sorts its own pair's labels in registers with a
// merge-exchange network of 8, 12, .., 28 or 32 entries (the smallest that
// holds the degree) and reads the tied labels off the runs, all pairs at
// once; when few are, the whole warp votes on two pairs at a time (one
// neighbour per lane grouped by __match_any_sync, the pick(u, t)-th tied
// label by removing minima or, for deep ranks, by sorting the tied labels
// across the warp). Degree > 32: when the node's history says it pays, a
// Misra-Gries summary with K counters (K = 1 up to degree 64, 3 above) and an
// exact recount of its survivors settle every pair whose best count c has
// (K + 1) c > deg (every label reaching c is then a candidate); the other
// pairs of degree 33..kDeferMax are listed for mutation_vote_kernel (one pair
// per thread, labels sorted in registers), those of degree kDeferMax + 1 ..
// kSharedTableMax take a count table in shared memory, one pair at a time,
// and those above are listed for mutation_hub_kernel (a warp per pair, its
// count table in global scratch).
// ---------------------------------------------------------------------------

// The ka-th and kb-th smallest of the distinct labels held by the lanes of
// two candidate sets ca and cb, by removing the minimum k times; the two
// chains run side by side so that their reductions overlap. la / lb receive
// the lanes (-1 for an empty set). Labels are non-negative.
__device__ __forceinline__ void select_kth_lane2(unsigned ca, int xa, unsigned ka, unsigned cb, int xb, unsigned kb,
                                                 int &la, int &lb)
{
    const int lane = threadIdx.x & 31;
    unsigned acta = ca, actb = cb;
    const unsigned kmax = ka > kb ? ka : kb;
    for (unsigned s = 0; s < kmax; ++s) {
        const unsigned mna = __reduce_min_sync(kFull, ((acta >> lane) & 1u) ? (unsigned)xa : 0xffffffffu);
        const unsigned mnb = __reduce_min_sync(kFull, ((actb >> lane) & 1u) ? (unsigned)xb : 0xffffffffu);
        const unsigned ra = __ballot_sync(kFull, ((acta >> lane) & 1u) && (unsigned)xa == mna);
        const unsigned rb = __ballot_sync(kFull, ((actb >> lane) & 1u) && (unsigned)xb == mnb);
        if (s < ka) acta &= ~ra;
        if (s < kb) actb &= ~rb;
    }
    const unsigned mna = __reduce_min_sync(kFull, ((acta >> lane) & 1u) ? (unsigned)xa : 0xffffffffu);
    const unsigned mnb = __reduce_min_sync(kFull, ((actb >> lane) & 1u) ? (unsigned)xb : 0xffffffffu);
    la = __ffs(__ballot_sync(kFull, ((acta >> lane) & 1u) && (unsigned)xa == mna)) - 1;
    lb = __ffs(__ballot_sync(kFull, ((actb >> lane) & 1u) && (unsigned)xb == mnb)) - 1;
}

// Two ascending bitonic sorts across the warp (one value per lane each),
// run as independent chains.
__device__ __forceinline__ void warp_sort32x2(unsigned &a, unsigned &b)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned pa = __shfl_xor_sync(kFull, a, j);
            const unsigned pb = __shfl_xor_sync(kFull, b, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            a = keep_min ? min(a, pa) : max(a, pa);
            b = keep_min ? min(b, pb) : max(b, pb);
        }
    }
}

// Above this tie rank the k-th tied label comes from sorting the tied labels
// rather than from removing the minimum k times.
constexpr unsigned kRemovalMax = 4;

// MTIE words of the lane's four children at node v (computed by every lane
// together, the first time a tie occurs at v).
__device__ __forceinline__ uint4 tie_words(const GenParams &gp, int v, int lane, uint32_t g)
{
    return philox4x32_10(make_uint4((uint32_t)v, (uint32_t)lane, g, kStageMutTie), gp.key0, gp.key1);
}

// A neighbour id read from the CSR; in the debug build an id outside [0, n)
// is recorded and replaced by 0, so that the access it feeds stays in bounds.
__device__ __forceinline__ int checked_node(int u, int n)
{
    return MOCD_CHECK(u >= 0 && u < n, kCheckNode, u) ? u : 0;
}

__device__ __forceinline__ uint32_t hash_slot(int x, int hbits)
{
    return ((uint32_t)x * 2654435761u) >> (32 - hbits);
}

// Asynchronous 4-byte global -> shared copy (no register staging) and the
// wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

constexpr int kTileStride = 33;  // padded row of the per-warp label tile
constexpr int kTileRows = 32;    // neighbours whose labels the tile keeps
static_assert(kDeferMax == 4 * kTileRows, "deferred classes: degrees 33..64 and 65..128");

// Start of deferred-vote class c in the list: the classes are stored one
// after the other (written with selects: indexing the kernel parameter array
// at run time would copy it to local memory).
__device__ __forceinline__ int defer_offset(const GenParams &gp, int c)
{
    return c == 0 ? 0 : c == 1 ? gp.defer_cap[0] : gp.defer_cap[0] + gp.defer_cap[1];
}
__device__ __forceinline__ int defer_capacity(const GenParams &gp, int c)
{
    return c == 0 ? gp.defer_cap[0] : c == 1 ? gp.defer_cap[1] : gp.defer_cap[2];
}
constexpr int kMutBlock = 128;   // mutation threads per block (shared memory bound)

// Sorting networks for any N: Batcher's merge exchange in the form of
// Knuth, TAOCP vol. 3, Sec. 5.2.2, Algorithm M (for a power of two it is
// Batcher's odd-even merge sort: 19, 63, 191, 543 comparators for 8, 16, 32,
// 64 entries; 41, 97, 127, 161 for 12, 20, 24, 28). The comparator list is
// generated at compile time and unrolled, so every index is a constant and
// the array stays in registers.
template <int A, int B>
__device__ __forceinline__ void cmp_exchange(int *x)
{
    const int lo = min(x[A], x[B]);
    const int hi = max(x[A], x[B]);
    x[A] = lo;
    x[B] = hi;
}

template <int N>
struct MergeExchange {
    // Calls f(i, i + d) for every comparator in order (Algorithm M, steps
    // M1..M5: p = 2^(t-1), 2^(t-2), ..., 1; for each p the passes d = p,
    // q - p, ... with r = 0 then p).
    template <class F>
    static constexpr void each(F f)
    {
        int t = 0;
        while ((1 << t) < N) ++t;
        for (int p = t > 0 ? 1 << (t - 1) : 0; p > 0; p >>= 1) {
            int q = 1 << (t - 1), r = 0, d = p;
            while (d > 0) {
                for (int i = 0; i < N - d; ++i)
                    if ((i & p) == r) f(i, i + d);
                d = q - p;
                q >>= 1;
                r = p;
            }
        }
    }
    static constexpr int count()
    {
        int c = 0;
        each([&](int, int) { ++c; });
        return c;
    }
    static constexpr int C = count();
    struct List {
        int a[C > 0 ? C : 1];
        int b[C > 0 ? C : 1];
    };
    static constexpr List make()
    {
        List l{};
        int k = 0;
        each([&](int i, int j) {
            l.a[k] = i;
            l.b[k] = j;
            ++k;
        });
        return l;
    }
    static constexpr List P = make();
};

template <int N, std::size_t... K>
__device__ __forceinline__ void apply_network(int (&x)[N], std::index_sequence<K...>)
{
    (cmp_exchange<MergeExchange<N>::P.a[K], MergeExchange<N>::P.b[K]>(x), ...);
}

template <int N>
__device__ __forceinline__ void sort_network(int (&x)[N])
{
    apply_network<N>(x, std::make_index_sequence<MergeExchange<N>::C>{});
}

// x[pos] for a run-time pos < N without indexing the register array: a
// tree of selects on the bits of pos, one level per bit (LEN live entries).
template <int N, int LEN, int B>
__device__ __forceinline__ void select_level(int (&y)[N], int pos)
{
    if constexpr (LEN > 1) {
        const bool hi = (pos >> B) & 1;
#pragma unroll
        for (int k = 0; k < (LEN + 1) / 2; ++k) y[k] = (2 * k + 1 < LEN && hi) ? y[2 * k + 1] : y[2 * k];
        select_level<N, (LEN + 1) / 2, B + 1>(y, pos);
    }
}

template <int N>
__device__ __forceinline__ int select_at(const int (&x)[N], int pos)
{
    int y[N];
#pragma unroll
    for (int j = 0; j < N; ++j) y[j] = x[j];
    select_level<N, N, 0>(y, pos);
    return y[0];
}

// Exact neighbour-majority of one pair by its own lane: the pair's deg <= N
// labels (1 <= deg <= N <= 32) are sorted in registers; equal labels then
// form runs, the longest runs are the tied labels in ascending order, and the
// pick(u, t)-th of them is the result. Bit j of e is set when entries j and
// j + 1 are equal, so a run of L labels is L - 1 consecutive set bits; each
// step m &= m >> 1 shortens every run of set bits by one, and the last
// non-zero m has one bit per longest run, at its first entry (all entries
// when no two labels are equal).
template <int N>
__device__ __forceinline__ int lane_pick(int (&x)[N], int deg, uint32_t u)
{
    sort_network<N>(x);
    unsigned e = 0;
#pragma unroll
    for (int j = 0; j + 1 < N; ++j) e |= (x[j] == x[j + 1] ? 1u : 0u) << j;
    e &= deg >= 2 ? 0xffffffffu >> (33 - deg) : 0u;  // pairs (j, j + 1) with j + 1 < deg
    unsigned starts = deg >= 32 ? 0xffffffffu : (1u << deg) - 1u;
    for (unsigned m = e; m != 0u; m &= m >> 1) starts = m;
    const int t = __popc(starts);
    const unsigned kk = t > 1 ? pick_index(u, (uint32_t)t) : 0u;
    // Position of the kk-th set bit of `starts`, halving the window each step.
    unsigned m = starts, k = kk;
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const unsigned low = m & ((1u << w) - 1u);
        const unsigned c = (unsigned)__popc(low);
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return select_at<N>(x, pos);
}

// Lane-parallel exact vote of every selected pair of a node with
// deg <= kTileRows (N >= deg): each lane sorts its pair's deg labels (its
// column of the staged tile) in registers and writes its result.
template <int N>
__device__ __forceinline__ void lane_votes(const int *tile, int deg, bool mine, int i, uint4 tw, int *s_res)
{
    const int src = i >> 2;
    const uint32_t w0 = __shfl_sync(0xffffffffu, tw.x, src);
    const uint32_t w1 = __shfl_sync(0xffffffffu, tw.y, src);
    const uint32_t w2 = __shfl_sync(0xffffffffu, tw.z, src);
    const uint32_t w3 = __shfl_sync(0xffffffffu, tw.w, src);
    const int k = i & 3;
    const uint32_t u = k == 0 ? w0 : (k == 1 ? w1 : (k == 2 ? w2 : w3));
    const int *col = tile + (threadIdx.x & 31);
    int x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = j < deg ? col[j * kTileStride] : INT_MAX;
    const int res = lane_pick<N>(x, deg, u);
    if (mine) s_res[i] = res;
}

// The smallest network size of the per-lane vote that holds deg labels, and
// the fewest pairs (lanes) for which the per-lane vote beats the warp vote.
__device__ __forceinline__ int lane_vote_min_pairs(int deg)
{
    return deg <= 8 ? 2 : deg <= 16 ? 5 : 10;
}

// Exact neighbour-majority of one pair of a node with degree > kDeferMax by
// the whole warp: a per-warp open-addressing count table (in shared memory,
// or for the hubs above kSharedTableMax in global scratch), sized to the
// node (the
// smallest power of two with at least 2 deg slots), filled with one insert
// per distinct label of each 32-neighbour chunk (__match_any_sync gives the
// multiplicity). The labels reaching the largest count are then compacted
// (one slot per distinct label) and the pick(u, t)-th smallest of them is
// found either by stepping up through the minima (shallow ranks) or bit by
// bit from the top (deep ranks).
__device__ __forceinline__ int warp_mode_table(const GenParams &gp, const int32_t *__restrict__ child,
                                            const int32_t *__restrict__ col_idx, int beg, int deg,
                                            const int *tile_col, int i, int *hkey, int *hcnt, uint32_t tie_u,
                                            unsigned &best_count)
{
    // tile_col: the staged labels of the first kTileRows neighbours, or NULL
    // (all are gathered from `child`).
    const int lane = threadIdx.x & 31;
    const int W = gp.W;
    // 2 deg <= 2 dmax <= the per-warp capacity, so the table fits.
    int hbits = 7;
    while ((1 << hbits) < 2 * deg) ++hbits;
    const int HS = 1 << hbits;
    const int per_lane = HS >> 5;
    for (int e = lane; e < HS; e += 32) {
        hkey[e] = -1;
        hcnt[e] = 0;
    }
    __syncwarp();
    for (int e0 = 0; e0 < deg; e0 += 32) {
        const bool in = e0 + lane < deg;
        int x = (int)(0x80000000u | lane);
        if (in)
            x = (tile_col && e0 + lane < kTileRows) ? tile_col[(e0 + lane) * kTileStride]
                                                    : child[(size_t)checked_node(__ldg(col_idx + beg + e0 + lane), gp.n) * W + i];
        // One insert per distinct label of the chunk, with its multiplicity.
        const unsigned peers = __match_any_sync(kFull, x);
        if (in && (peers & ((1u << lane) - 1u)) == 0) {
            uint32_t h = hash_slot(x, hbits);
            // The table holds at most deg <= HS / 2 distinct labels, so an empty
            // or matching slot is always found.
            for (int probe = 0; probe < HS; ++probe) {
                const int prev = atomicCAS(hkey + h, -1, x);
                if (prev == -1 || prev == x) {
                    atomicAdd(hcnt + h, __popc(peers));
                    break;
                }
                h = (h + 1) & (uint32_t)(HS - 1);
            }
        }
    }
    __syncwarp();
    unsigned mx_l = 0;
    for (int s = 0; s < per_lane; ++s) mx_l = max(mx_l, (unsigned)hcnt[lane + 32 * s]);
    const unsigned mx = __reduce_max_sync(kFull, mx_l);
    best_count = mx;
    // The tied labels: compacted into hcnt[0, t) when each lane has at most
    // 32 slots (a bit mask per lane); in larger (hub) tables the keys of the
    // slots below the top count are cleared instead, and the tied labels are
    // the keys still set, scanned over the whole table.
    int t;
    const int *tied;
    int span;
    if (per_lane <= 32) {
        unsigned act = 0;
        for (int s = 0; s < per_lane; ++s)
            if ((unsigned)hcnt[lane + 32 * s] == mx) act |= 1u << s;
        // Compact the tied labels into hcnt[0, t) (the counts are no longer needed).
        const unsigned mine = (unsigned)__popc(act);
        unsigned incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        t = (int)__shfl_sync(kFull, incl, 31);
        int at = (int)(incl - mine);
        __syncwarp();
        for (int s = 0; s < per_lane; ++s)
            if ((act >> s) & 1u) hcnt[at++] = hkey[lane + 32 * s];
        tied = hcnt;
        span = t;
    } else {
        unsigned mine = 0;
        for (int s = 0; s < per_lane; ++s) {
            const int e = lane + 32 * s;
            if ((unsigned)hcnt[e] == mx) ++mine;
            else hkey[e] = -1;
        }
        t = (int)__reduce_add_sync(kFull, mine);
        tied = hkey;
        span = HS;
    }
    __syncwarp();
    const unsigned kk = t > 1 ? pick_index(tie_u, (uint32_t)t) : 0u;
    int res;
    if (kk > (unsigned)gp.label_bits) {
        // Deep rank: at bit b (from the top), count the tied labels that agree
        // with the bits chosen so far and have a 0 there; the rank falls among
        // them or, past them, among those with a 1. Labels are below
        // 2^label_bits.
        unsigned prefix = 0, rank = kk;
        for (int b = gp.label_bits - 1; b >= 0; --b) {
            const unsigned above = ~((2u << b) - 1u);  // the bits above b
            unsigned c = 0;
            for (int e = lane; e < span; e += 32) {
                const int key = tied[e];
                if (key < 0) continue;  // a cleared slot of a hub table
                c += (((unsigned)key & above) == prefix && (((unsigned)key >> b) & 1u) == 0u) ? 1u : 0u;
            }
            const unsigned cnt = __reduce_add_sync(kFull, c);
            if (rank >= cnt) {
                rank -= cnt;
                prefix |= 1u << b;
            }
        }
        res = (int)prefix;
    } else {
        // Shallow rank: the smallest tied label, then kk times the smallest
        // one above the previous (the tied labels are distinct, >= 0).
        int last = -1;
        for (unsigned s = 0; s <= kk; ++s) {
            unsigned my = 0xffffffffu;
            for (int e = lane; e < span; e += 32) {
                const int key = tied[e];
                if (key > last) my = min(my, (unsigned)key);
            }
            last = (int)__reduce_min_sync(kFull, my);
        }
        res = last;
    }
    __syncwarp();
    return res;
}

__global__ void __launch_bounds__(kMutBlock, 6)
mutation_kernel(GenParams gp, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                const int32_t *__restrict__ order, const int32_t *__restrict__ child, int32_t *__restrict__ q,
                const uint32_t *__restrict__ gen_ptr, uint32_t *__restrict__ hist,
                unsigned long long *__restrict__ acc, uint32_t *__restrict__ hint, int2 *__restrict__ dlist,
                int *__restrict__ dcount)
{
    extern __shared__ int smem[];
    const int W = gp.W, np = gp.np;
    const int nq = W >> 2;
    const uint32_t g = *gen_ptr;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int HS = gp.hash_size;
    int *s_list = smem + wib * (2 * kMaxPop + kTileRows * kTileStride + 2 * HS);  // selected children
    int *s_res = s_list + kMaxPop;              // by child index: v's own label, then the result
    int *tile = s_res + kMaxPop;                // [kTileRows][kTileStride]: label of neighbour j, pair lane
    int *hkey = tile + kTileRows * kTileStride;
    int *hcnt = hkey + HS;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool active = lane < nq;
    const int4 *__restrict__ C4 = reinterpret_cast<const int4 *>(child);
    int4 *__restrict__ Q4 = reinterpret_cast<int4 *>(q);

    // The evaluation that follows accumulates into acc: clear it here. The
    // histogram is zero on entry (the previous evaluation's square sweep
    // cleared it) and receives D below.
    if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < 2 * kMaxPop; t += blockDim.x) acc[t] = 0;

    // Nodes in degree-descending order: every warp starts with one of the
    // costliest nodes, which balances the grid-stride loop.
    for (int idx = warp; idx < gp.n; idx += nwarps) {
        const int v = __ldg(order + idx);
        const int beg = __ldg(row_ptr + v);
        const int end = __ldg(row_ptr + v + 1);
        const int deg = MOCD_CHECK(end >= beg, kCheckRowPtr, v) ? end - beg : 0;
        int4 out = active ? C4[(size_t)v * nq + lane] : make_int4(0, 0, 0, 0);
        unsigned sel = 0;  // bit k: child 4 * lane + k mutates
        if (active && deg > 0) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)lane, g, kStageMutCoin),
                                          gp.key0, gp.key1);
            const int i0 = 4 * lane;
            sel = ((i0 + 0 < np && (unsigned long long)r.x < gp.thr_m) ? 1u : 0u) |
                  ((i0 + 1 < np && (unsigned long long)r.y < gp.thr_m) ? 2u : 0u) |
                  ((i0 + 2 < np && (unsigned long long)r.z < gp.thr_m) ? 4u : 0u) |
                  ((i0 + 3 < np && (unsigned long long)r.w < gp.thr_m) ? 8u : 0u);
        }
        // Compact the selected children of v into s_list (warp prefix sum).
        const int mine = __popc(sel);
        int incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        const int nsel = __shfl_sync(kFull, incl, 31);
        if (nsel > 0) {
            int at = incl - mine;
            for (int k = 0; k < 4; ++k)
                if ((sel >> k) & 1u) s_list[at++] = 4 * lane + k;
            if (active) reinterpret_cast<int4 *>(s_res)[lane] = out;
            __syncwarp();
            const int my_u0 = lane < deg ? checked_node(__ldg(col_idx + beg + lane), gp.n) : 0;
            // Degree <= kTileRows: the exact per-lane votes below settle all
            // pairs at once and cost less than the Misra-Gries pass, even once
            // the population has settled. Above: the pass runs when the last
            // generation's exact results (whichever path produced them) say
            // that most of v's pairs had a label above deg / (K + 1), the pairs
            // the pass settles. hint = (pairs << 16) | such pairs; 0: no
            // history.
            const uint32_t h = deg > kTileRows ? hint[v] : 0u;
            const bool use_mg = deg > kTileRows && (h == 0u || 2u * (h & 0xffffu) >= (h >> 16));
            const bool deferred_class = (deg > kTileRows && deg <= kDeferMax) || deg > kSharedTableMax;
            int nsettle = 0;  // pairs of v with 4 (best count) > deg, settled here
            bool have_tw = false;
            uint4 tw = make_uint4(0, 0, 0, 0);
            for (int base = 0; base < nsel; base += 32) {
                // Lane = pair (selected child i of node v).
                const bool has = base + lane < nsel;
                const int i = has ? s_list[base + lane] : 0;
                // The tile is read by the pass and by the votes of degree <= 32
                // and > kDeferMax; pairs of the deferred degrees need it only
                // for the pass. Degree <= kTileRows with enough selected pairs
                // takes the per-lane vote, else the warp vote.
                const bool lane_path =
                    deg <= kTileRows && __popc(__ballot_sync(kFull, has)) >= lane_vote_min_pairs(deg);
                const int dt = (use_mg || !deferred_class) ? min(deg, kTileRows) : 0;
                for (int j = 0; j < dt; ++j) {
                    const int u = __shfl_sync(kFull, my_u0, j);
                    if (has) cp_async4(tile + j * kTileStride + lane, child + (size_t)u * W + i);
                }
                cp_async_wait_all();
                __syncwarp();
                // Pass 1: a Misra-Gries summary with K counters keeps every
                // label occurring more than deg / (K + 1) times; pass 2 counts
                // the survivors exactly. K = 1 (Boyer-Moore) up to degree
                // 2 kTileRows, whose unsettled pairs take the cheap deferred
                // vote; K = 3 above, where the fallback costs more and settling
                // more pairs pays. The labels of the first kTileRows
                // neighbours are read from the tile, the rest from global
                // memory (eight loads in flight). Empty counters keep distinct
                // negative labels until first filled; an empty counter that
                // still holds x takes it back (the same summary as filling a
                // free one, since no label is ever held by two counters).
                const int kc = deg <= 2 * kTileRows ? 1 : 3;
                int s0 = -2, s1 = -3, s2 = -4;  // candidates (labels no neighbour has when empty)
                int h0 = 0, h1 = 0, h2 = 0;     // their exact counts
                auto pass = [&](auto kconst) {
                    constexpr int K = decltype(kconst)::value;
                    int c0 = -1, c1 = -2, c2 = -3, n0 = 0, n1 = 0, n2 = 0;
                    auto mg = [&](int x, bool ok) {
                        if (K == 1) {
                            const bool e0 = n0 == 0;
                            n0 = !ok ? n0 : (x == c0 || e0) ? n0 + 1 : n0 - 1;
                            c0 = ok && e0 ? x : c0;
                            return;
                        }
                        const bool m0 = x == c0, m1 = x == c1, m2 = x == c2;
                        const bool hit = m0 || m1 || m2;
                        const bool e0 = n0 == 0, e1 = n1 == 0, e2 = n2 == 0;
                        const bool f0 = !hit && e0, f1 = !hit && !e0 && e1, f2 = !hit && !e0 && !e1 && e2;
                        const int dec = (ok && !hit && !e0 && !e1 && !e2) ? 1 : 0;
                        n0 = ok && (m0 || f0) ? n0 + 1 : n0 - dec;
                        n1 = ok && (m1 || f1) ? n1 + 1 : n1 - dec;
                        n2 = ok && (m2 || f2) ? n2 + 1 : n2 - dec;
                        c0 = ok && f0 ? x : c0;
                        c1 = ok && f1 ? x : c1;
                        c2 = ok && f2 ? x : c2;
                    };
                    if (has) {
#pragma unroll 4
                        for (int j = 0; j < dt; ++j) mg(tile[j * kTileStride + lane], true);
                    }
                    for (int e0 = kTileRows; e0 < deg; e0 += 32) {
                        const int my_u = e0 + lane < deg ? checked_node(__ldg(col_idx + beg + e0 + lane), gp.n) : 0;
                        const int cnt = min(32, deg - e0);
                        for (int j0 = 0; j0 < cnt; j0 += 8) {
                            int xs[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int u = __shfl_sync(kFull, my_u, min(j0 + t, cnt - 1));
                                xs[t] = (has && j0 + t < cnt) ? child[(size_t)u * W + i] : 0;
                            }
#pragma unroll
                            for (int t = 0; t < 8; ++t) mg(xs[t], has && j0 + t < cnt);
                        }
                    }
                    s0 = n0 > 0 ? c0 : -2;
                    if (K > 1) {
                        s1 = n1 > 0 ? c1 : -3;
                        s2 = n2 > 0 ? c2 : -4;
                    }
                    auto tally = [&](int x) {
                        h0 += x == s0;
                        if (K > 1) {
                            h1 += x == s1;
                            h2 += x == s2;
                        }
                    };
                    // The first kTileRows labels are still in the tile.
                    if (has) {
#pragma unroll 4
                        for (int j = 0; j < kTileRows; ++j) tally(tile[j * kTileStride + lane]);
                    }
                    for (int e0 = kTileRows; e0 < deg; e0 += 32) {
                        const int my_u = e0 + lane < deg ? checked_node(__ldg(col_idx + beg + e0 + lane), gp.n) : 0;
                        const int cnt = min(32, deg - e0);
                        for (int j0 = 0; j0 < cnt; j0 += 8) {
                            int xs[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int u = __shfl_sync(kFull, my_u, min(j0 + t, cnt - 1));
                                xs[t] = (has && j0 + t < cnt) ? child[(size_t)u * W + i] : -1;
                            }
#pragma unroll
                            for (int t = 0; t < 8; ++t) tally(xs[t]);
                        }
                    }
                };
                if (use_mg) {
                    if (kc == 1)
                        pass(std::integral_constant<int, 1>{});
                    else
                        pass(std::integral_constant<int, 3>{});
                }
                // If the best candidate count c satisfies (K + 1) c > deg, every
                // label reaching c is a candidate: the tied set is complete and
                // exact.
                const int best = max(h0, max(h1, h2));
                const bool done = has && use_mg && (kc + 1) * best > deg;
                if (done) {
                    // Tied candidates in ascending order, then the MTIE pick.
                    int a = h0 == best ? s0 : INT_MAX;
                    int b = h1 == best ? s1 : INT_MAX;
                    int c = h2 == best ? s2 : INT_MAX;
                    int lo = min(a, b), hi = max(a, b);
                    a = lo; b = hi;
                    lo = min(b, c); hi = max(b, c);
                    b = lo; c = hi;
                    lo = min(a, b); hi = max(a, b);
                    a = lo; b = hi;
                    const int t = 1 + (b != INT_MAX) + (c != INT_MAX);
                    int lab = a;
                    if (t > 1) {
                        const uint4 r = tie_words(gp, v, i >> 2, g);
                        const uint32_t kk = pick_index(word_of(r, i & 3), (uint32_t)t);
                        lab = kk == 0 ? a : (kk == 1 ? b : c);
                    }
                    s_res[i] = lab;
                }
                __syncwarp();
                unsigned rest = __ballot_sync(kFull, has && !done);
                nsettle += __popc(__ballot_sync(kFull, done));
                if (rest && deferred_class) {
                    // Degrees kTileRows + 1 .. kDeferMax: the exact vote of every
                    // remaining pair runs in mutation_vote_kernel, one pair per
                    // thread with its labels sorted in registers; hubs above
                    // kSharedTableMax: in mutation_hub_kernel, a warp per pair.
                    // The pair's slot of the row holds -1 until then.
                    const int cls = deg > kDeferMax ? 2 : deg <= 2 * kTileRows ? 0 : 1;
                    int first = 0;
                    if (lane == 0) first = atomicAdd(dcount + cls, __popc(rest));
                    first = __shfl_sync(kFull, first, 0);
                    if ((rest >> lane) & 1u) {
                        const int at_list = first + __popc(rest & ((1u << lane) - 1u));
                        // The capacity is the class's nodes x N_p, every pair
                        // a generation can defer: the check only keeps a
                        // corrupted count in bounds.
                        if (at_list < defer_capacity(gp, cls)) dlist[defer_offset(gp, cls) + at_list] = make_int2(v, i);
                        s_res[i] = -1;
                    }
                    rest = 0;
                }
                if (rest && !have_tw) {
                    tw = tie_words(gp, v, lane, g);
                    have_tw = true;
                }
                if (lane_path) {
                    // Many selected pairs: every lane settles its own pair with
                    // a sorting network of the smallest size that holds deg
                    // labels (all pairs at once).
                    const bool mine = (rest >> lane) & 1u;
                    if (deg <= 8) lane_votes<8>(tile, deg, mine, i, tw, s_res);
                    else if (deg <= 12) lane_votes<12>(tile, deg, mine, i, tw, s_res);
                    else if (deg <= 16) lane_votes<16>(tile, deg, mine, i, tw, s_res);
                    else if (deg <= 20) lane_votes<20>(tile, deg, mine, i, tw, s_res);
                    else if (deg <= 24) lane_votes<24>(tile, deg, mine, i, tw, s_res);
                    else if (deg <= 28) lane_votes<28>(tile, deg, mine, i, tw, s_res);
                    else lane_votes<32>(tile, deg, mine, i, tw, s_res);
                    rest = 0;
                }
                if (deg <= kTileRows) {
                    // Exact vote by the whole warp (lane = neighbour), two
                    // unresolved pairs at a time as independent chains.
                    const unsigned lt = (1u << lane) - 1u;
                    const bool nb = lane < deg;
                    const int pad = (int)(0x80000000u | (unsigned)lane);  // distinct, never a label
                    while (rest) {
                        const int la = __ffs(rest) - 1;
                        rest &= rest - 1;
                        const bool two = rest != 0u;
                        const int lb = two ? __ffs(rest) - 1 : la;
                        if (two) rest &= rest - 1;
                        const int ia = __shfl_sync(kFull, i, la);
                        const int ib = __shfl_sync(kFull, i, lb);
                        const int xa = nb ? tile[lane * kTileStride + la] : pad;
                        const int xb = (nb && two) ? tile[lane * kTileStride + lb] : pad;
                        const unsigned pa = __match_any_sync(kFull, xa);
                        const unsigned pb = __match_any_sync(kFull, xb);
                        const unsigned ca = nb ? (unsigned)__popc(pa) : 0u;
                        const unsigned cb = nb ? (unsigned)__popc(pb) : 0u;
                        const unsigned ma = __reduce_max_sync(kFull, ca);
                        const unsigned mb = __reduce_max_sync(kFull, cb);
                        const unsigned da = __ballot_sync(kFull, ca == ma && (pa & lt) == 0u);
                        const unsigned db = __ballot_sync(kFull, cb == mb && (pb & lt) == 0u);
                        const uint32_t ua = __shfl_sync(kFull, word_of(tw, ia & 3), ia >> 2);
                        const uint32_t ub = __shfl_sync(kFull, word_of(tw, ib & 3), ib >> 2);
                        const int ta = __popc(da), tb = __popc(db);
                        const unsigned ka = ta > 1 ? pick_index(ua, (uint32_t)ta) : 0u;
                        const unsigned kb = (two && tb > 1) ? pick_index(ub, (uint32_t)tb) : 0u;
                        int ra, rb;
                        if (ka > kRemovalMax || kb > kRemovalMax) {
                            // The tied labels are distinct (one leader per label):
                            // sorted ascending, with the other lanes last, the
                            // k-th tied label sits in lane k.
                            unsigned va = ((da >> lane) & 1u) ? (unsigned)xa : 0xffffffffu;
                            unsigned vb = (two && ((db >> lane) & 1u)) ? (unsigned)xb : 0xffffffffu;
                            warp_sort32x2(va, vb);
                            ra = (int)__shfl_sync(kFull, va, (int)ka);
                            rb = (int)__shfl_sync(kFull, vb, (int)kb);
                        } else {
                            int sa = __ffs(da) - 1, sb = __ffs(db) - 1;
                            if (ta > 1 || (two && tb > 1)) select_kth_lane2(da, xa, ka, two ? db : 0u, xb, kb, sa, sb);
                            if (!two) sb = 0;
                            ra = __shfl_sync(kFull, xa, sa);
                            rb = __shfl_sync(kFull, xb, sb);
                        }
                        if (lane == 0) {
                            s_res[ia] = ra;
                            if (two) s_res[ib] = rb;
                        }
                    }
                }
                // Degree > kDeferMax: a shared count table, one pair at a time.
                while (rest) {
                    const int l = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const int ic = __shfl_sync(kFull, i, l);
                    const uint32_t u = __shfl_sync(kFull, word_of(tw, ic & 3), ic >> 2);
                    unsigned mx = 0;
                    const int lab = warp_mode_table(gp, child, col_idx, beg, deg, tile + l, ic, hkey, hcnt, u, mx);
                    if (lane == 0) s_res[ic] = lab;
                    nsettle += 4 * (int)mx > deg ? 1 : 0;
                }
                __syncwarp();
            }
            __syncwarp();
            // The deferred pairs add theirs in mutation_vote_kernel.
            if (lane == 0 && deg > kTileRows) hint[v] = ((uint32_t)nsel << 16) | (uint32_t)nsettle;
            // s_res holds the unselected children's labels and the results.
            if (active) out = reinterpret_cast<const int4 *>(s_res)[lane];
            __syncwarp();
        }
        if (active) {
            Q4[(size_t)v * nq + lane] = out;
            // D of the evaluation's degree histogram: every child's final label
            // of v gets deg(v) (label-major cell label * W + child). The old
            // value is not needed, so these are reductions that do not stall.
            // A deferred pair (-1) gets its label and its addition from
            // mutation_vote_kernel.
            if (deg > 0) {
                const int i0 = 4 * lane;
                const unsigned d = (unsigned)deg;
                if (i0 + 0 < np && out.x >= 0 && MOCD_CHECK(out.x < gp.n, kCheckLabel, v))
                    atomicAdd(hist + (size_t)out.x * W + i0 + 0, d);
                if (i0 + 1 < np && out.y >= 0 && MOCD_CHECK(out.y < gp.n, kCheckLabel, v))
                    atomicAdd(hist + (size_t)out.y * W + i0 + 1, d);
                if (i0 + 2 < np && out.z >= 0 && MOCD_CHECK(out.z < gp.n, kCheckLabel, v))
                    atomicAdd(hist + (size_t)out.z * W + i0 + 2, d);
                if (i0 + 3 < np && out.w >= 0 && MOCD_CHECK(out.w < gp.n, kCheckLabel, v))
                    atomicAdd(hist + (size_t)out.w * W + i0 + 3, d);
            }
        }
    }
}

// The exact neighbour-majority of one deferred pair (node of degree
// kTileRows + 1 .. N) per thread: the pair's labels are gathered into
// registers (INT_MAX beyond the degree), sorted by the odd-even merge
// network, and the pick(u, t)-th of the t longest runs is the result, u the
// MTIE word. The thread writes the label into Q, adds deg(v) to the degree
// histogram (as the mutation kernel does for the other pairs) and, when the
// best count c has (K + 1) c > deg (K the counters of the node's Misra-Gries
// pass: 1 for degree <= 64, else 3), counts the pair in v's hint.
template <int N>
__device__ __forceinline__ void mutation_vote_body(const GenParams gp, int cls, const int32_t *__restrict__ row_ptr,
                                                   const int32_t *__restrict__ col_idx,
                                                   const int32_t *__restrict__ child, int32_t *__restrict__ q,
                                                   const uint32_t *__restrict__ gen_ptr, uint32_t *__restrict__ hist,
                                                   uint32_t *__restrict__ hint, const int2 *__restrict__ dlist,
                                                   const int *__restrict__ dcount, int vblock, int vgrid)
{
    constexpr int NW = (N + 63) / 64;
    const uint32_t g = *gen_ptr;
    const int W = gp.W;
    const int total = min(dcount[cls], defer_capacity(gp, cls));
    const int2 *list = dlist + defer_offset(gp, cls);
    for (int t = vblock * blockDim.x + threadIdx.x; t < total; t += vgrid * blockDim.x) {
        const int2 e = list[t];
        const int v = e.x, i = e.y;
        if (!MOCD_CHECK(v >= 0 && v < gp.n && i >= 0 && i < gp.np, kCheckNode, t)) continue;
        const int beg = __ldg(row_ptr + v);
        const int deg = min(__ldg(row_ptr + v + 1) - beg, N);
        int x[N];
#pragma unroll
        for (int j = 0; j < N; ++j)
            x[j] = j < deg ? child[(size_t)checked_node(__ldg(col_idx + beg + j), gp.n) * W + i] : INT_MAX;
        sort_network<N>(x);
        // Runs of equal labels as in lane_pick, over NW 64-bit words: bit j
        // of eq is set when entries j and j + 1 (< deg) are equal; each step
        // m &= m >> 1 (across words) shortens every run of set bits by one,
        // and the last non-zero m marks the first entry of each longest run.
        unsigned long long eq[NW], starts[NW], m[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) eq[w] = 0ull;
#pragma unroll
        for (int j = 0; j + 1 < N; ++j) eq[j >> 6] |= (x[j] == x[j + 1] ? 1ull : 0ull) << (j & 63);
        bool any = false;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int pairs = deg - 1 - 64 * w;  // valid bits of word w
            const int ents = deg - 64 * w;
            eq[w] &= pairs >= 64 ? ~0ull : pairs <= 0 ? 0ull : (1ull << pairs) - 1ull;
            starts[w] = ents >= 64 ? ~0ull : ents <= 0 ? 0ull : (1ull << ents) - 1ull;
            m[w] = eq[w];
            any |= eq[w] != 0ull;
        }
        int best = 1;
        while (any) {
            any = false;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                starts[w] = m[w];
                const unsigned long long carry = w + 1 < NW ? m[w + 1 < NW ? w + 1 : w] << 63 : 0ull;
                m[w] &= (m[w] >> 1) | carry;
                any |= m[w] != 0ull;
            }
            ++best;
        }
        int tcount = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) tcount += __popcll(starts[w]);
        unsigned kk = 0;
        if (tcount > 1) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)(i >> 2), g, kStageMutTie), gp.key0,
                                          gp.key1);
            kk = pick_index(word_of(r, i & 3), (uint32_t)tcount);
        }
        // Position of the kk-th set bit of the starts mask.
        int pos = 0;
        unsigned k = kk;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const unsigned c = (unsigned)__popcll(starts[w]);
            if (k >= c) {
                k -= c;
                continue;
            }
            unsigned long long mm = starts[w];
            int p = 64 * w;
#pragma unroll
            for (int width = 32; width >= 1; width >>= 1) {
                const unsigned long long low = mm & ((1ull << width) - 1ull);
                const unsigned lc = (unsigned)__popcll(low);
                if (k >= lc) {
                    k -= lc;
                    mm >>= width;
                    p += width;
                } else {
                    mm = low;
                }
            }
            pos = p;
            break;
        }
        const int res = select_at<N>(x, pos);
        q[(size_t)v * W + i] = res;
        if (MOCD_CHECK(res >= 0 && res < gp.n, kCheckLabel, v)) atomicAdd(hist + (size_t)res * W + i, (unsigned)deg);
        if ((N <= 2 * kTileRows ? 2 : 4) * best > deg) atomicAdd(hint + v, 1u);
    }
}

template <int N>
__global__ void __launch_bounds__(kMutBlock)
mutation_vote_kernel(GenParams gp, int cls, const int32_t *__restrict__ row_ptr,
                     const int32_t *__restrict__ col_idx, const int32_t *__restrict__ child,
                     int32_t *__restrict__ q, const uint32_t *__restrict__ gen_ptr, uint32_t *__restrict__ hist,
                     uint32_t *__restrict__ hint, const int2 *__restrict__ dlist, const int *__restrict__ dcount)
{
    mutation_vote_body<N>(gp, cls, row_ptr, col_idx, child, q, gen_ptr, hist, hint, dlist, dcount, blockIdx.x,
                          gridDim.x);
}

// The deferred votes of one degree class of every member of a batch.
// (Register cap: the single-member kernel's occupancy, 5 blocks of 128
// threads for 64 entries; 2 for 128, whose registers do not fit 3 here.)
template <int N>
__global__ void __launch_bounds__(kMutBlock, N <= 64 ? 5 : 2)
mutation_vote_multi_kernel(const BatchMember *__restrict__ members, const int *__restrict__ starts, int count,
                           int cls)
{
    const int k = member_of_block(starts, count);
    const BatchMember &mb = members[k];
    const PopState &ps = mb.ps;
    const int b0 = __ldg(starts + k);
    mutation_vote_body<N>(mb.gp, cls, mb.row_ptr, mb.col_idx, ps.c, ps.q, ps.gen, ps.hist, ps.hint, ps.dlist,
                          ps.dcount, (int)blockIdx.x - b0, __ldg(starts + k + 1) - b0);
}

// The listed votes of hubs above kSharedTableMax: a warp per pair, its count
// table in the warp's slice of the global scratch (2 gp.hub_hs ints). Writes
// the label into Q, adds deg(v) to the histogram and counts the pair in v's
// hint when its best count c has 4 c > deg.
__global__ void __launch_bounds__(kMutBlock)
mutation_hub_kernel(GenParams gp, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                    const int32_t *__restrict__ child, int32_t *__restrict__ q, const uint32_t *__restrict__ gen_ptr,
                    uint32_t *__restrict__ hist, uint32_t *__restrict__ hint, const int2 *__restrict__ dlist,
                    const int *__restrict__ dcount, int *__restrict__ hub_table)
{
    const uint32_t g = *gen_ptr;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int *hkey = hub_table + (size_t)warp * 2 * gp.hub_hs;
    int *hcnt = hkey + gp.hub_hs;
    const int total = min(dcount[2], defer_capacity(gp, 2));
    const int2 *list = dlist + defer_offset(gp, 2);
    for (int t = warp; t < total; t += nwarps) {
        const int2 e = list[t];
        const int v = e.x, i = e.y;
        if (!MOCD_CHECK(v >= 0 && v < gp.n && i >= 0 && i < gp.np, kCheckNode, t)) continue;  // (warp-uniform)
        const int beg = __ldg(row_ptr + v);
        const int deg = min(__ldg(row_ptr + v + 1) - beg, gp.hub_hs / 2);
        const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)(i >> 2), g, kStageMutTie), gp.key0, gp.key1);
        unsigned mx = 0;
        const int lab = warp_mode_table(gp, child, col_idx, beg, deg, nullptr, i, hkey, hcnt, word_of(r, i & 3), mx);
        if (lane == 0) {
            q[(size_t)v * gp.W + i] = lab;
            if (MOCD_CHECK(lab >= 0 && lab < gp.n, kCheckLabel, v)) atomicAdd(hist + (size_t)lab * gp.W + i, (unsigned)deg);
            if (4 * (int)mx > deg) atomicAdd(hint + v, 1u);
        }
    }
}

template <int EMAX>
size_t crossover_smem()
{
    return sizeof(int) * (2 * kMaxPop + kMaxPop * EMAX + (kBlock / 32) * 2 * kMaxPop);
}

}  // namespace

cudaError_t launch_init_population(const GenParams &gp, int init_mode, const int32_t *row_ptr,
                                   const int32_t *col_idx, int32_t *dst, cudaStream_t s)
{
    const long long total = (long long)gp.n * (gp.W >> 2);
    long long blocks = (total + kBlock - 1) / kBlock;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    if (init_mode == 1)
        init_sweep_kernel<<<(int)blocks, kBlock, 0, s>>>(gp.n, gp.W, gp.np, gp.key0, gp.key1, row_ptr,
                                                         col_idx, dst);
    else
        init_population_kernel<<<(int)blocks, kBlock, 0, s>>>(gp.n, gp.W, gp.np, gp.key0, gp.key1, dst);
    return cudaGetLastError();
}

int grid_for_crossover(int sms, int es)
{
    int per_sm = 0;
    if (es <= 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crossover_kernel<4>, kBlock, crossover_smem<4>());
    else if (es <= 8)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crossover_kernel<8>, kBlock, crossover_smem<8>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crossover_kernel<16>, kBlock, crossover_smem<16>());
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_crossover(const GenParams &gp, const PopState &ps, int grid, cudaStream_t s)
{
    if (gp.es <= 4)
        crossover_kernel<4><<<grid, kBlock, crossover_smem<4>(), s>>>(
            gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r, ps.copy_r, ps.gen,
            ps.dcount);
    else if (gp.es <= 8)
        crossover_kernel<8><<<grid, kBlock, crossover_smem<8>(), s>>>(
            gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r, ps.copy_r, ps.gen,
            ps.dcount);
    else
        crossover_kernel<16><<<grid, kBlock, crossover_smem<16>(), s>>>(
            gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r, ps.copy_r, ps.gen,
            ps.dcount);
    return cudaGetLastError();
}

cudaError_t launch_crossover_multi(const BatchMember *members, const int *starts, int count, int blocks, int es_max,
                                   cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    if (es_max <= 4)
        crossover_multi_kernel<4><<<blocks, kBlock, crossover_smem<4>(), s>>>(members, starts, count);
    else if (es_max <= 8)
        crossover_multi_kernel<8><<<blocks, kBlock, crossover_smem<8>(), s>>>(members, starts, count);
    else
        crossover_multi_kernel<16><<<blocks, kBlock, crossover_smem<16>(), s>>>(members, starts, count);
    return cudaGetLastError();
}

cudaError_t launch_vote_multi(const BatchMember *members, const int *starts, int count, int blocks, int cls,
                              cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    if (cls == 0)
        mutation_vote_multi_kernel<2 * kTileRows><<<blocks, kMutBlock, 0, s>>>(members, starts, count, 0);
    else
        mutation_vote_multi_kernel<kDeferMax><<<blocks, kMutBlock, 0, s>>>(members, starts, count, 1);
    return cudaGetLastError();
}

int mutation_smem(int hash_size)
{
    return (kMutBlock / 32) * (2 * kMaxPop + kTileRows * kTileStride + 2 * hash_size) * (int)sizeof(int);
}

int mutation_warps_per_block()
{
    return kMutBlock / 32;
}

int grid_for_mutation(int sms, int hash_size, int *smem_bytes)
{
    const int smem = mutation_smem(hash_size);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(mutation_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mutation_kernel, kMutBlock, smem);
    if (per_sm < 1) per_sm = 1;
    *smem_bytes = smem;
    return sms * per_sm;
}

void grid_for_votes(int sms, int vote_n0, int *grid64, int *grid128)
{
    int a = 0, b = 0;
    switch (vote_n0) {
    case 40: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, mutation_vote_kernel<40>, kMutBlock, 0); break;
    case 48: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, mutation_vote_kernel<48>, kMutBlock, 0); break;
    case 56: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, mutation_vote_kernel<56>, kMutBlock, 0); break;
    default:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, mutation_vote_kernel<2 * kTileRows>, kMutBlock, 0);
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, mutation_vote_kernel<kDeferMax>, kMutBlock, 0);
    *grid64 = sms * (a < 1 ? 1 : a);
    *grid128 = sms * (b < 1 ? 1 : b);
}

cudaError_t launch_mutation(const GenParams &gp, const PopState &ps, const int32_t *row_ptr,
                            const int32_t *col_idx, const int32_t *order, int grid, int grid64, int grid128,
                            cudaStream_t s, bool with_votes)
{
    mutation_kernel<<<grid, kMutBlock, mutation_smem(gp.hash_size), s>>>(gp, row_ptr, col_idx, order, ps.c, ps.q,
                                                                       ps.gen, ps.hist, ps.acc, ps.hint, ps.dlist,
                                                                       ps.dcount);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (with_votes && gp.defer_cap[0] > 0) {
        // The class's network holds the graph's largest degree in it.
        switch (gp.vote_n0) {
        case 40:
            mutation_vote_kernel<40><<<grid64, kMutBlock, 0, s>>>(gp, 0, row_ptr, col_idx, ps.c, ps.q, ps.gen,
                                                                  ps.hist, ps.hint, ps.dlist, ps.dcount);
            break;
        case 48:
            mutation_vote_kernel<48><<<grid64, kMutBlock, 0, s>>>(gp, 0, row_ptr, col_idx, ps.c, ps.q, ps.gen,
                                                                  ps.hist, ps.hint, ps.dlist, ps.dcount);
            break;
        case 56:
            mutation_vote_kernel<56><<<grid64, kMutBlock, 0, s>>>(gp, 0, row_ptr, col_idx, ps.c, ps.q, ps.gen,
                                                                  ps.hist, ps.hint, ps.dlist, ps.dcount);
            break;
        default:
            mutation_vote_kernel<2 * kTileRows><<<grid64, kMutBlock, 0, s>>>(gp, 0, row_ptr, col_idx, ps.c, ps.q,
                                                                               ps.gen, ps.hist, ps.hint, ps.dlist,
                                                                               ps.dcount);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (with_votes && gp.defer_cap[1] > 0) {
        mutation_vote_kernel<kDeferMax><<<grid128, kMutBlock, 0, s>>>(gp, 1, row_ptr, col_idx, ps.c, ps.q, ps.gen,
                                                                        ps.hist, ps.hint, ps.dlist, ps.dcount);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (gp.defer_cap[2] > 0) {
        mutation_hub_kernel<<<gp.hub_warps / (kMutBlock / 32), kMutBlock, 0, s>>>(
            gp, row_ptr, col_idx, ps.c, ps.q, ps.gen, ps.hist, ps.hint, ps.dlist, ps.dcount, ps.hub_table);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace mocd

namespace mocd {
cudaError_t check_record_variation(unsigned long long *out, bool reset)
{
    return check_record(out, reset);
}
}  // namespace mocd
