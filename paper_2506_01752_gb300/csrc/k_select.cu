// k_select.cu -- the NSGA-II bookkeeping of Alg. 1 on one thread block:
// FastNonDominatedSort, CrowdingDistanceAssignment, SortByRankAndDistance,
// TournamentSelection(P, E_S, k = 2) and EnvironmentalSelection(P u Q, N_p),
// plus Pareto-front extraction with SelectSolution (Alg. 3) and the layout
// conversions used by the host API.
//
// All ranking works on the exact integer keys (k1 = m - intra, k2 = S), so
// dominance (Sec. 2.2) is exact. Crowding distance follows Deb et al. 2002 on
// the integer keys: per front and objective, members ordered by (key,
// position); both ends +inf; an interior member adds
// (double)(k[next] - k[prev]) / (double)(k_max - k_min), objective 1 first,
// then objective 2; a zero range adds nothing; fronts of one or two members
// are all +inf. This file is built with -fmad=false; each floating-point
// operation is one correctly rounded IEEE operation.
#include <limits.h>
#include <math.h>

#include "mocd_internal.h"
#include "philox.cuh"

namespace mocd {

namespace {

constexpr int kMaxPoints = 2 * kMaxPop;   // members of R = P u Q
constexpr int kSelThreads = kMaxPoints;     // one thread per point
constexpr int kSelWarps = kSelThreads / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kInf64 = 0xffffffffffffffffull;

// Sort key: the pair (a, b) in lexicographic order of unsigned words. Every
// key a sort sees is distinct (the point index is packed into b).
struct Key {
    unsigned long long a, b;
};

__device__ __forceinline__ bool key_less(const Key &x, const Key &y)
{
    return x.a < y.a || (x.a == y.a && x.b < y.b);
}

struct SelShared {
    long long k1[kMaxPoints];
    long long k2[kMaxPoints];
    int rank[kMaxPoints];        // by point
    double crowd[kMaxPoints];    // by point
    int order[kMaxPoints];       // (rank, crowding desc, index) order
    // scratch by sorted position
    unsigned long long sa[kMaxPoints], sb[kMaxPoints];
    int ib[kMaxPoints];
    unsigned long long wscan[kSelWarps];
    int wscan2[kSelWarps];
    int fsize[kMaxPoints + 1];
    int keep[kMaxPop];
    unsigned long long xa[2][kMaxPoints], xb[2][kMaxPoints];  // sort exchange, double-buffered
};

// Bitonic sort, ascending, of one key per thread over the first SIZE threads
// (a power of two, 32..kSelThreads); the other threads only join the
// barriers. Fully unrolled: distances below 32 exchange by shuffles, larger
// ones through shared memory. The compare-exchange is branch-free.
template <int SIZE>
__device__ __forceinline__ Key block_sort_fixed(SelShared &S, Key key)
{
    const int t = threadIdx.x;
    const bool in = t < SIZE;
    int buf = 0;  // exchange buffer of the next shared-memory stage
#pragma unroll
    for (int k = 2; k <= SIZE; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            Key other;
            if (j >= 32) {
                // Consecutive shared-memory stages alternate buffers, so the
                // barrier of one stage also orders the previous stage's reads
                // before the next write of the same buffer.
                if (in) {
                    S.xa[buf][t] = key.a;
                    S.xb[buf][t] = key.b;
                }
                __syncthreads();
                if (in) {
                    other.a = S.xa[buf][t ^ j];
                    other.b = S.xb[buf][t ^ j];
                }
                buf ^= 1;
            } else if (in) {
                other.a = __shfl_xor_sync(kFull, key.a, j);
                other.b = __shfl_xor_sync(kFull, key.b, j);
            }
            if (in) {
                // Keep the smaller key where (t is the lower index) == (ascending run).
                const bool want_min = ((t & j) == 0) == ((t & k) == 0);
                const bool take = key_less(other, key) == want_min;
                key.a = take ? other.a : key.a;
                key.b = take ? other.b : key.b;
            }
        }
    }
    __syncthreads();  // the last exchange's reads precede any later use of the buffers
    return key;
}

// The sort above for size = 32, 64, 128 or 256 (the power of two covering
// the points).
__device__ __noinline__ Key block_sort(SelShared &S, Key key, int size)
{
    switch (size) {
    case 32: return block_sort_fixed<32>(S, key);
    case 64: return block_sort_fixed<64>(S, key);
    case 128: return block_sort_fixed<128>(S, key);
    default: return block_sort_fixed<kSelThreads>(S, key);
    }
}

// Inclusive block-wide scans over thread order (min of u64, max of int).
__device__ unsigned long long block_min_scan(SelShared &S, unsigned long long v)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v = min(v, y);
    }
    if (lane == 31) S.wscan[w] = v;
    __syncthreads();
    unsigned long long pre = kInf64;
#pragma unroll
    for (int q = 0; q < kSelWarps; ++q) pre = q < w ? min(pre, S.wscan[q]) : pre;
    __syncthreads();
    return min(v, pre);
}

__device__ int block_max_scan(SelShared &S, int v)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v = max(v, y);
    }
    if (lane == 31) S.wscan[w] = (unsigned long long)(unsigned)v;
    __syncthreads();
    int pre = 0;
#pragma unroll
    for (int q = 0; q < kSelWarps; ++q) pre = q < w ? max(pre, (int)(unsigned)S.wscan[q]) : pre;
    __syncthreads();
    return max(v, pre);
}

// In one pass over the block: a forward inclusive max-scan of two 16-bit
// values packed in a (per half-word) and a backward inclusive min-scan of b
// (over threads t .. kSelThreads - 1).
__device__ void block_scan_pair(SelShared &S, unsigned &a, int &b)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned ya = __shfl_up_sync(kFull, a, d);
        const int yb = __shfl_down_sync(kFull, b, d);
        if (lane >= d) a = __vmaxu2(a, ya);
        if (lane + d < 32) b = min(b, yb);
    }
    if (lane == 31) S.wscan[w] = a;
    if (lane == 0) S.wscan2[w] = b;
    __syncthreads();
    unsigned pa = 0;
    int pb = INT_MAX;
#pragma unroll
    for (int q = 0; q < kSelWarps; ++q) {
        pa = q < w ? __vmaxu2(pa, (unsigned)S.wscan[q]) : pa;
        pb = q > w ? min(pb, S.wscan2[q]) : pb;
    }
    __syncthreads();
    a = __vmaxu2(a, pa);
    b = min(b, pb);
}

// rank[], crowd[] and order[] of the first N points of S.k1 / S.k2 (N <= 256),
// all indexed by point; ranks are 1-based. Same definitions as the textbook
// O(N^2) procedure, computed with block sorts and scans. With known_rank,
// S.rank already holds every point's front (P's fronts are those R gave its
// members) and only crowding and the order are computed.
__device__ void rank_crowd_order(SelShared &S, int N, bool known_rank)
{
    const int t = threadIdx.x;
    const bool valid = t < N;
    int size = 32;
    while (size < N) size <<= 1;
    const bool in = t < size;

    int e;  // point at position t of the fronts-contiguous (rank, k1, k2, index) order
    if (!known_rank) {
        // (1) Sort by (k1, k2, index); invalid points go last. k1 < 2^31, so
        // (k1 : hi32(k2), lo32(k2) : index) orders like the triple.
        Key k;
        {
            const unsigned long long k1 = valid ? (unsigned long long)S.k1[t] : 0xffffffffull;
            const unsigned long long k2 = valid ? (unsigned long long)S.k2[t] : kInf64;
            k.a = (k1 << 32) | (k2 >> 32);
            k.b = (k2 << 32) | (unsigned long long)t;
        }
        k = block_sort(S, k, size);
        // Thread t now holds sorted position t.
        const int id = (int)(k.b & 0xffffffffull);
        const bool real = in && id < N;
        const unsigned long long my1 = k.a >> 32;
        const unsigned long long my2 = ((k.a & 0xffffffffull) << 32) | (k.b >> 32);
        S.sa[t] = my1;
        S.sb[t] = my2;
        __syncthreads();
        // Start of t's group of identical keys (identical points never
        // dominate each other and share a front).
        const bool head = t == 0 || S.sa[t - 1] != my1 || S.sb[t - 1] != my2;
        const int gstart = block_max_scan(S, head ? t : 0);

        // (2) Fronts. A remaining point is dominated iff some remaining point
        // sorted before its group has k2 <= its k2. (3) Each front, once
        // found, is laid out contiguously after the earlier ones, its members
        // in sorted (k1, k2, index) order: position = points placed so far +
        // members of the front at earlier sorted positions.
        const int lane = t & 31, w = t >> 5;
        const unsigned lt = (1u << lane) - 1u;
        bool rem = real;
        int myrank = 0;
        int placed = 0;  // points of the fronts found so far (block-uniform)
        for (int r = 1;; ++r) {
            const unsigned long long pm = block_min_scan(S, rem ? my2 : kInf64);
            S.sa[t] = pm;
            __syncthreads();
            const unsigned long long before = gstart > 0 ? S.sa[gstart - 1] : kInf64;
            const bool inf = rem && before > my2;
            const unsigned bal = __ballot_sync(kFull, inf);
            if (lane == 0) S.wscan[w] = (unsigned long long)__popc(bal);
            __syncthreads();
            int off = placed, tot = 0;
#pragma unroll
            for (int q = 0; q < kSelWarps; ++q) {
                const int c = (int)S.wscan[q];
                off += q < w ? c : 0;
                tot += c;
            }
            if (inf) {
                S.ib[off + __popc(bal & lt)] = id;
                myrank = r;
                rem = false;
            }
            placed += tot;
            if (!__syncthreads_or(rem)) break;
        }
        if (real) S.rank[id] = myrank;
        __syncthreads();
        e = t < N ? S.ib[t] : N;
    } else {
        // Ranks known: one sort by (rank, k1, k2, index), packed as
        // rank:9 | k1:31 | hi24(k2) and lo40(k2) | index:24.
        Key f;
        if (valid) {
            const unsigned long long r = (unsigned long long)S.rank[t];
            const unsigned long long k1 = (unsigned long long)S.k1[t];
            const unsigned long long k2 = (unsigned long long)S.k2[t];
            f.a = (r << 55) | (k1 << 24) | (k2 >> 40);
            f.b = ((k2 & 0xffffffffffull) << 24) | (unsigned long long)t;
        } else {
            f.a = kInf64;
            f.b = kInf64 - (unsigned long long)(kSelThreads - t);
        }
        f = block_sort(S, f, size);
        e = (int)(f.b & 0xffffffull);
    }
    for (int q = t; q <= kSelThreads; q += blockDim.x) S.fsize[q] = 0;
    __syncthreads();
    const bool ereal = in && e < N;
    if (ereal) atomicAdd(&S.fsize[S.rank[e]], 1);
    const int er = ereal ? S.rank[e] : 0;
    const long long e1 = ereal ? S.k1[e] : 0, e2 = ereal ? S.k2[e] : 0;
    S.sa[t] = (unsigned long long)e1;
    S.sb[t] = (unsigned long long)e2;
    S.ib[t] = er;
    __syncthreads();
    // Start of t's front and of its group of identical points (forward max
    // scans of the head positions), and the end of its group (the next group
    // head after t: a backward min scan), all in one pass.
    const bool fhead = t == 0 || S.ib[t - 1] != er;
    const bool ghead = fhead || S.sa[t - 1] != (unsigned long long)e1 || S.sb[t - 1] != (unsigned long long)e2;
    const bool gnext = t == kSelThreads - 1 || S.ib[t + 1] != er || S.sa[t + 1] != (unsigned long long)e1 ||
                       S.sb[t + 1] != (unsigned long long)e2;
    unsigned heads = ((fhead ? (unsigned)t : 0u) << 16) | (ghead ? (unsigned)t : 0u);
    int ge = gnext ? t + 1 : INT_MAX;
    block_scan_pair(S, heads, ge);
    const int fstart = (int)(heads >> 16), gs = (int)(heads & 0xffffu);
    if (ereal) {
        const int F = S.fsize[er];
        const int fpos = t - fstart, gsl = gs - fstart, gel = ge - fstart;
        double c;
        if (F <= 2) {
            c = INFINITY;
        } else {
            c = 0.0;
            if (fpos == 0 || fpos == F - 1) {
                c = INFINITY;
            } else {
                const long long range = (long long)S.sa[fstart + F - 1] - (long long)S.sa[fstart];
                if (range > 0) {
                    const long long gap = (long long)S.sa[t + 1] - (long long)S.sa[t - 1];
                    c = __dadd_rn(c, __ddiv_rn((double)gap, (double)range));
                }
            }
            // Objective 2: groups in reverse order, index order inside a group.
            const int pos2 = (F - gel) + (fpos - gsl);
            if (pos2 == 0 || pos2 == F - 1) {
                c = INFINITY;
            } else {
                const long long range = (long long)S.sb[fstart] - (long long)S.sb[fstart + F - 1];
                if (range > 0) {
                    const long long lo2 = fpos > gsl ? e2 : (long long)S.sb[ge];
                    const long long hi2 = fpos < gel - 1 ? e2 : (long long)S.sb[gs - 1];
                    c = __dadd_rn(c, __ddiv_rn((double)(hi2 - lo2), (double)range));
                }
            }
        }
        S.crowd[e] = c;
    }
    __syncthreads();

    // (4) Final order by (rank, crowding desc, index). Crowding values are
    // non-negative or +inf, so their bit patterns order like the values.
    Key o;
    {
        const unsigned long long r = valid ? (unsigned long long)S.rank[t] : 0xffffffffull;
        const unsigned long long cb = valid ? ~(unsigned long long)__double_as_longlong(S.crowd[t]) : kInf64;
        o.a = (r << 32) | (cb >> 32);
        o.b = (cb << 32) | (unsigned long long)t;
    }
    o = block_sort(S, o, size);
    S.order[t] = (int)(o.b & 0xffffffffull);
    __syncthreads();
}

// One block: selection of one population (mode 0: keys of a fresh P from
// acc; mode 1: R = P u Q), then rank, crowding and order of P and the next
// tournament.
__device__ __forceinline__ void select_body(const GenParams &gp, const PopState &ps, int mode, SelShared &S)
{
    const int p = threadIdx.x;  // loads, stores and the tournament: one thread per item
    const int np = gp.np;
    const long long m = gp.m;
    const uint32_t g = *ps.gen;
    const unsigned long long *acc = ps.acc;

    if (mode == 0) {
        if (p < np) {
            S.k1[p] = m - (long long)acc[p];
            S.k2[p] = (long long)acc[kMaxPop + p];
            S.keep[p] = p;
        }
        __syncthreads();
    } else {
        if (p < np) {
            S.k1[p] = ps.pk[p];
            S.k2[p] = ps.pk[kMaxPop + p];
        } else if (p < 2 * np) {
            const int i = p - np;
            S.k1[p] = m - (long long)acc[i];
            S.k2[p] = (long long)acc[kMaxPop + i];
        }
        __syncthreads();
        if (p < 2 * np) {
            ps.rk[p] = S.k1[p];
            ps.rk[2 * kMaxPop + p] = S.k2[p];
        }
        rank_crowd_order(S, 2 * np, false);
        // The kept members keep their fronts: P is R's first fronts plus part
        // of the next one, so every dominator of a member is kept too.
        long long n1 = 0, n2 = 0;
        int nr = 0;
        if (p < np) {
            const int r = S.order[p];
            S.keep[p] = r;
            n1 = S.k1[r];
            n2 = S.k2[r];
            nr = S.rank[r];
        }
        __syncthreads();
        if (p < np) {
            S.k1[p] = n1;
            S.k2[p] = n2;
            S.rank[p] = nr;
        }
        __syncthreads();
    }
    if (p < np) {
        ps.pk[p] = S.k1[p];
        ps.pk[kMaxPop + p] = S.k2[p];
        ps.keep[p] = S.keep[p];
    }

    // Rank and crowding recomputed on P (Alg. 1, start of the generation).
    rank_crowd_order(S, np, mode == 1);
    if (p < np) ps.prank[p] = S.rank[p];

    // TournamentSelection for generation gn = g + 1: parent j of child i is
    // the better of sorted positions a, b, i.e. position min(a, b).
    const uint32_t gn = g + 1u;
    if (p < np) {
        const int E = gp.es;
        uint4 blk = make_uint4(0, 0, 0, 0);
        int have = -1;
        auto word = [&](int w) -> uint32_t {
            if ((w >> 2) != have) {
                blk = philox4x32_10(make_uint4((uint32_t)(w >> 2), (uint32_t)p, gn, kStageSelect),
                                    gp.key0, gp.key1);
                have = w >> 2;
            }
            return word_of(blk, w & 3);
        };
        int par[kMaxParents];
        for (int j = 0; j < E; ++j) {
            const uint32_t a = pick_index(word(2 * j), (uint32_t)np);
            const uint32_t b = pick_index(word(2 * j + 1), (uint32_t)np);
            const int pos = S.order[a < b ? a : b];
            par[j] = S.keep[pos];
            ps.par_r[p * kMaxParents + j] = par[j];
        }
        const uint32_t x = word(2 * E);
        const uint32_t sk = pick_index(word(2 * E + 1), (uint32_t)E);
        ps.copy_r[p] = ((unsigned long long)x <= gp.thr_c) ? -1 : par[sk];
    }
    __syncthreads();
    if (p == 0) *ps.gen = gn;
}

__global__ void __launch_bounds__(kSelThreads)
select_kernel(GenParams gp, PopState ps, int mode)
{
    __shared__ SelShared S;
    select_body(gp, ps, mode, S);
}

// The selections of several populations in one launch (a batch of
// instances): block b selects population b.
__global__ void __launch_bounds__(kSelThreads)
select_multi_kernel(const GenParams *__restrict__ gps, const PopState *__restrict__ pss, int mode)
{
    __shared__ SelShared S;
    const GenParams gp = gps[blockIdx.x];
    const PopState ps = pss[blockIdx.x];
    select_body(gp, ps, mode, S);
}

// F_1 of P in P order and SelectSolution: argmin of 4 m k1 + k2 (= argmax of
// Q = 1 - f1 - f2), first member on ties. Also each member's exact intra and
// S, and f1 = k1 / m, f2 = S / (4 m^2) as single IEEE divisions.
__global__ void front_kernel(GenParams gp, PopState ps)
{
    if (threadIdx.x != 0) return;
    int count = 0, best = -1;
    long long bestK = 0;
    const long long m = gp.m;
    for (int p = 0; p < gp.np; ++p) {
        if (ps.prank[p] != 1) continue;
        const long long k1 = ps.pk[p], k2 = ps.pk[kMaxPop + p];
        const long long K = 4ll * m * k1 + k2;
        if (best < 0 || K < bestK) {
            best = count;
            bestK = K;
        }
        ps.front[2 + count] = p;
        ps.fint[count] = m - k1;
        ps.fint[kMaxPop + count] = k2;
        ps.fval[count] = __ddiv_rn((double)k1, (double)m);
        ps.fval[kMaxPop + count] = __ddiv_rn((double)k2, (double)(4ll * m * m));
        ++count;
    }
    ps.front[0] = count;
    ps.front[1] = best;
}

__global__ void gather_individuals_kernel(int n, int W, int np, const int32_t *__restrict__ phalf,
                                          const int32_t *__restrict__ q, const int32_t *__restrict__ idx,
                                          int count, int32_t *__restrict__ out)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        for (int k = 0; k < count; ++k) {
            const int r = idx ? idx[k] : k;
            const int32_t val = r < np ? phalf[(size_t)v * W + r] : q[(size_t)v * W + (r - np)];
            out[(size_t)k * n + v] = val;
        }
    }
}

__global__ void to_node_major_kernel(int n, int W, int count, const int32_t *__restrict__ src,
                                     int32_t *__restrict__ dst)
{
    const int nq = W >> 2;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        for (int qd = 0; qd < nq; ++qd) {
            int4 o;
            const int k = 4 * qd;
            o.x = k + 0 < count ? src[(size_t)(k + 0) * n + v] : 0;
            o.y = k + 1 < count ? src[(size_t)(k + 1) * n + v] : 0;
            o.z = k + 2 < count ? src[(size_t)(k + 2) * n + v] : 0;
            o.w = k + 3 < count ? src[(size_t)(k + 3) * n + v] : 0;
            reinterpret_cast<int4 *>(dst)[(size_t)v * nq + qd] = o;
        }
    }
}

int blocks_for(int n)
{
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

}  // namespace

cudaError_t launch_select(const GenParams &gp, const PopState &ps, int mode, cudaStream_t s)
{
    select_kernel<<<1, kSelThreads, 0, s>>>(gp, ps, mode);
    return cudaGetLastError();
}

cudaError_t launch_select_multi(const GenParams *gps, const PopState *pss, int count, int mode, cudaStream_t s)
{
    select_multi_kernel<<<count, kSelThreads, 0, s>>>(gps, pss, mode);
    return cudaGetLastError();
}

cudaError_t launch_front(const GenParams &gp, const PopState &ps, cudaStream_t s)
{
    front_kernel<<<1, 32, 0, s>>>(gp, ps);
    return cudaGetLastError();
}

cudaError_t launch_gather_individuals(int n, int W, int np, const int32_t *phalf, const int32_t *q,
                                      const int32_t *idx, int count, int32_t *out, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    gather_individuals_kernel<<<blocks_for(n), 256, 0, s>>>(n, W, np, phalf, q, idx, count, out);
    return cudaGetLastError();
}

cudaError_t launch_to_node_major(int n, int W, int count, const int32_t *src, int32_t *dst,
                                 cudaStream_t s)
{
    to_node_major_kernel<<<blocks_for(n), 256, 0, s>>>(n, W, count, src, dst);
    return cudaGetLastError();
}

}  // namespace mocd
