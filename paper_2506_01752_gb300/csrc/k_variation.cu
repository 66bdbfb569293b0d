// k_variation.cu -- InitializePopulation and the offspring map of Alg. 1:
// topology-aware crossover (Sec. 4.3.1, Alg. 2) and topology-aware mutation
// (Sec. 4.3.2), for all N_p children of a generation at once.
//
// Both kernels work on node-major rows: a warp owns node v; lane q owns the
// four children 4q..4q+3, which share one Philox call per stage because the
// stream counter of (child i, node v) is (v, i / 4, g, stage), word i % 4.
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
__global__ void __launch_bounds__(kBlock)
crossover_kernel(GenParams gp, const int32_t *buf0, const int32_t *buf1, int32_t *out0, int32_t *out1,
                 const int32_t *__restrict__ q, int32_t *__restrict__ child,
                 const int32_t *__restrict__ keep, const int32_t *__restrict__ par_r,
                 const int32_t *__restrict__ copy_r, const uint32_t *__restrict__ gen_ptr)
{
    extern __shared__ int smem[];
    const int W = gp.W, np = gp.np, E = gp.es;
    const int nq = W >> 2;
    int *s_keep = smem;                  // [W]   row position of P position k
    int *s_copy = s_keep + kMaxPop;      // [W]   row position copied, or -1
    int *s_par = s_copy + kMaxPop;       // [np * E] row positions of parents
    int *s_rows = s_par + kMaxPop * EMAX;  // per warp: [2W] staged row of R

    const uint32_t g = *gen_ptr;
    // R index r -> position in the staged row (P half at [0, W), Q at [W, 2W)).
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        const int r = keep[t];
        s_keep[t] = r < np ? r : W + (r - np);
        const int c = copy_r[t];
        s_copy[t] = c < 0 ? -1 : (c < np ? c : W + (c - np));
        for (int j = 0; j < E; ++j) {
            const int p = par_r[t * kMaxParents + j];
            s_par[t * EMAX + j] = p < np ? p : W + (p - np);
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
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool active = lane < nq;

    for (int v = warp; v < gp.n; v += nwarps) {
        if (active) {
            reinterpret_cast<int4 *>(row)[lane] = P4[(size_t)v * nq + lane];
            reinterpret_cast<int4 *>(row + W)[lane] = Q4[(size_t)v * nq + lane];
        }
        __syncwarp();
        if (active) {
            int o[4];
            int r[4];
            bool have_u = false;
            uint4 u = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * lane + k;
                o[k] = i < np ? row[s_keep[i]] : 0;
                r[k] = 0;
                if (i >= np) continue;
                const int cp = s_copy[i];
                if (cp >= 0) {
                    r[k] = row[cp];
                    continue;
                }
                int x[EMAX];
#pragma unroll
                for (int j = 0; j < EMAX; ++j) x[j] = j < E ? row[s_par[i * EMAX + j]] : 0;
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

// ---------------------------------------------------------------------------
// Mutation. Node v of child i mutates iff its MCOIN word is below thr_m and
// deg(v) > 0; it then takes the most frequent label among its neighbours in
// the post-crossover child (synchronous: all reads come from `child`), the
// tie among the t most frequent labels broken by the MTIE word (the
// pick(u, t)-th smallest). Degree <= 32: one neighbour per lane and
// __match_any_sync groups equal labels. Degree > 32: a per-warp open-addressing
// count table in shared memory.
// ---------------------------------------------------------------------------

// k-th smallest label held by the lanes of `cand` (distinct labels), by
// binary radix selection over the label bits.
__device__ __forceinline__ int select_kth_lane(unsigned cand, int x, unsigned k, int bits)
{
    unsigned act = cand;
    for (int b = bits - 1; b >= 0; --b) {
        const unsigned zero = __ballot_sync(kFull, ((x >> b) & 1) == 0) & act;
        const unsigned c = __popc(zero);
        if (k < c) {
            act = zero;
        } else {
            k -= c;
            act &= ~zero;
        }
    }
    return __ffs(act) - 1;
}

__device__ __forceinline__ uint32_t tie_word(const GenParams &gp, int v, int i, uint32_t g)
{
    const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)(i >> 2), g, kStageMutTie),
                                  gp.key0, gp.key1);
    return word_of(r, i & 3);
}

__device__ __forceinline__ uint32_t hash_slot(int x, int hbits)
{
    return ((uint32_t)x * 2654435761u) >> (32 - hbits);
}

__global__ void __launch_bounds__(kBlock)
mutation_kernel(GenParams gp, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                const int32_t *__restrict__ child, int32_t *__restrict__ q,
                const uint32_t *__restrict__ gen_ptr)
{
    extern __shared__ int smem[];
    const int W = gp.W, np = gp.np;
    const int nq = W >> 2;
    const uint32_t g = *gen_ptr;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int HS = gp.hash_size;
    const int hbits = HS > 0 ? __ffs(HS) - 1 : 0;
    int *hkey = smem + wib * 2 * HS;
    int *hcnt = hkey + HS;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool active = lane < nq;
    const int4 *__restrict__ C4 = reinterpret_cast<const int4 *>(child);
    int4 *__restrict__ Q4 = reinterpret_cast<int4 *>(q);

    for (int v = warp; v < gp.n; v += nwarps) {
        const int beg = __ldg(row_ptr + v);
        const int end = __ldg(row_ptr + v + 1);
        const int deg = end - beg;
        int4 out = active ? C4[(size_t)v * nq + lane] : make_int4(0, 0, 0, 0);
        bool s0 = false, s1 = false, s2 = false, s3 = false;
        if (active && deg > 0) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)v, (uint32_t)lane, g, kStageMutCoin),
                                          gp.key0, gp.key1);
            const int i0 = 4 * lane;
            s0 = i0 + 0 < np && (unsigned long long)r.x < gp.thr_m;
            s1 = i0 + 1 < np && (unsigned long long)r.y < gp.thr_m;
            s2 = i0 + 2 < np && (unsigned long long)r.z < gp.thr_m;
            s3 = i0 + 3 < np && (unsigned long long)r.w < gp.thr_m;
        }
        const unsigned b[4] = {__ballot_sync(kFull, s0), __ballot_sync(kFull, s1),
                               __ballot_sync(kFull, s2), __ballot_sync(kFull, s3)};
        if ((b[0] | b[1] | b[2] | b[3]) != 0) {
            if (deg <= 32) {
                const int my_u = lane < deg ? __ldg(col_idx + beg + lane) : 0;
                const unsigned lt = (1u << lane) - 1u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    unsigned msk = b[k];
                    while (msk) {
                        const int ql = __ffs(msk) - 1;
                        msk &= msk - 1;
                        const int i = 4 * ql + k;
                        const int x = lane < deg ? child[(size_t)my_u * W + i] : (int)(0x80000000u | lane);
                        const unsigned peers = __match_any_sync(kFull, x);
                        const unsigned cnt = lane < deg ? __popc(peers) : 0u;
                        const unsigned mx = __reduce_max_sync(kFull, cnt);
                        const unsigned cand = __ballot_sync(kFull, lane < deg && cnt == mx && (peers & lt) == 0);
                        const int t = __popc(cand);
                        int src;
                        if (t == 1) {
                            src = __ffs(cand) - 1;
                        } else {
                            const uint32_t u = tie_word(gp, v, i, g);
                            src = select_kth_lane(cand, x, pick_index(u, (uint32_t)t), gp.label_bits);
                        }
                        const int lab = __shfl_sync(kFull, x, src);
                        if (lane == ql) {
                            if (k == 0) out.x = lab;
                            else if (k == 1) out.y = lab;
                            else if (k == 2) out.z = lab;
                            else out.w = lab;
                        }
                    }
                }
            } else {
                const int per_lane = HS >> 5;  // table entries owned by each lane when scanning
#pragma unroll 1
                for (int k = 0; k < 4; ++k) {
                    unsigned msk = b[k];
                    while (msk) {
                        const int ql = __ffs(msk) - 1;
                        msk &= msk - 1;
                        const int i = 4 * ql + k;
                        for (int e = lane; e < HS; e += 32) {
                            hkey[e] = -1;
                            hcnt[e] = 0;
                        }
                        __syncwarp();
                        for (int e0 = beg; e0 < end; e0 += 32) {
                            if (e0 + lane < end) {
                                const int x = child[(size_t)__ldg(col_idx + e0 + lane) * W + i];
                                uint32_t h = hash_slot(x, hbits);
                                // The table holds at most deg < HS / 2 distinct labels,
                                // so an empty or matching slot is always found.
                                for (int probe = 0; probe < HS; ++probe) {
                                    const int prev = atomicCAS(hkey + h, -1, x);
                                    if (prev == -1 || prev == x) {
                                        atomicAdd(hcnt + h, 1);
                                        break;
                                    }
                                    h = (h + 1) & (uint32_t)(HS - 1);
                                }
                            }
                        }
                        __syncwarp();
                        unsigned mx_l = 0;
                        for (int s = 0; s < per_lane; ++s) {
                            const unsigned c = (unsigned)hcnt[lane + 32 * s];
                            mx_l = c > mx_l ? c : mx_l;
                        }
                        const unsigned mx = __reduce_max_sync(kFull, mx_l);
                        unsigned act = 0;
                        for (int s = 0; s < per_lane; ++s)
                            if ((unsigned)hcnt[lane + 32 * s] == mx) act |= 1u << s;
                        const unsigned t = __reduce_add_sync(kFull, (unsigned)__popc(act));
                        unsigned kk = 0;
                        if (t > 1) kk = pick_index(tie_word(gp, v, i, g), t);
                        for (int bit = gp.label_bits - 1; bit >= 0 && t > 1; --bit) {
                            unsigned zero = 0;
                            for (int s = 0; s < per_lane; ++s)
                                if (((act >> s) & 1u) && ((hkey[lane + 32 * s] >> bit) & 1) == 0) zero |= 1u << s;
                            const unsigned c = __reduce_add_sync(kFull, (unsigned)__popc(zero));
                            if (kk < c) {
                                act = zero;
                            } else {
                                kk -= c;
                                act &= ~zero;
                            }
                        }
                        const unsigned holder = __ballot_sync(kFull, act != 0);
                        const int src = __ffs(holder) - 1;
                        const int mine = act ? hkey[lane + 32 * (__ffs(act) - 1)] : 0;
                        const int lab = __shfl_sync(kFull, mine, src);
                        if (lane == ql) {
                            if (k == 0) out.x = lab;
                            else if (k == 1) out.y = lab;
                            else if (k == 2) out.z = lab;
                            else out.w = lab;
                        }
                        __syncwarp();
                    }
                }
            }
        }
        if (active) Q4[(size_t)v * nq + lane] = out;
    }
}

template <int EMAX>
size_t crossover_smem()
{
    return sizeof(int) * (2 * kMaxPop + kMaxPop * EMAX + (kBlock / 32) * 2 * kMaxPop);
}

}  // namespace

cudaError_t launch_init_population(const GenParams &gp, int32_t *dst, cudaStream_t s)
{
    const long long total = (long long)gp.n * (gp.W >> 2);
    long long blocks = (total + kBlock - 1) / kBlock;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
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
            gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r, ps.copy_r, ps.gen);
    else if (gp.es <= 8)
        crossover_kernel<8><<<grid, kBlock, crossover_smem<8>(), s>>>(
            gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r, ps.copy_r, ps.gen);
    else
        crossover_kernel<16><<<grid, kBlock, crossover_smem<16>(), s>>>(
            gp, ps.buf[0], ps.buf[1], ps.buf[0], ps.buf[1], ps.q, ps.c, ps.keep, ps.par_r, ps.copy_r, ps.gen);
    return cudaGetLastError();
}

int grid_for_mutation(int sms, int hash_size, int *smem_bytes)
{
    const int smem = (kBlock / 32) * 2 * hash_size * (int)sizeof(int);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(mutation_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mutation_kernel, kBlock, smem);
    if (per_sm < 1) per_sm = 1;
    *smem_bytes = smem;
    return sms * per_sm;
}

cudaError_t launch_mutation(const GenParams &gp, const PopState &ps, const int32_t *row_ptr,
                            const int32_t *col_idx, int grid, cudaStream_t s)
{
    const int smem = (kBlock / 32) * 2 * gp.hash_size * (int)sizeof(int);
    mutation_kernel<<<grid, kBlock, smem, s>>>(gp, row_ptr, col_idx, ps.c, ps.q, ps.gen);
    return cudaGetLastError();
}

}  // namespace mocd
