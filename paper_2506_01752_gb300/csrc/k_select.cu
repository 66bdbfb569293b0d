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

constexpr int kMaxPoints = 2 * kMaxPop;      // members of R = P u Q
constexpr int kTpp = 4;                         // threads per point
constexpr int kSelThreads = kMaxPoints * kTpp;  // 1024
constexpr int kWords = kMaxPoints / 32;
constexpr unsigned kFull = 0xffffffffu;

struct SelShared {
    long long k1[kMaxPoints];
    long long k2[kMaxPoints];
    double crowd[kMaxPoints];
    int rank[kMaxPoints];
    int order[kMaxPoints];
    int ord1[kMaxPoints];
    int ord2[kMaxPoints];
    unsigned dom[kMaxPoints][kWords];  // dom[p] bit q: q dominates p
    unsigned unassigned[kWords];
    int keep[kMaxPop];
};

// Sum over the kTpp threads of one point (consecutive lanes of one warp).
__device__ __forceinline__ int point_sum(int v)
{
    v += __shfl_xor_sync(kFull, v, 1);
    v += __shfl_xor_sync(kFull, v, 2);
    return v;
}

// rank[], crowd[] and order[] of the first N points of S.k1 / S.k2. Point p
// is handled by threads 4p..4p+3, each taking every 4th comparison partner.
// Ranks are 1-based.
__device__ void rank_crowd_order(SelShared &S, int N)
{
    const int p = threadIdx.x >> 2;
    const int sub = threadIdx.x & 3;
    const bool mine = p < N;
    const int nw = (N + 31) >> 5;
    const int Npad = nw * 32;
    // Padding points beyond N never dominate and never share a rank.
    for (int q = N + (int)threadIdx.x; q < Npad; q += blockDim.x) {
        S.k1[q] = LLONG_MAX;
        S.k2[q] = LLONG_MAX;
        S.rank[q] = INT_MAX;
    }
    __syncthreads();
    if (mine) {
        const long long a1 = S.k1[p], a2 = S.k2[p];
        for (int w = sub; w < nw; w += kTpp) {
            unsigned bits = 0;
#pragma unroll 8
            for (int b = 0; b < 32; ++b) {
                const long long b1 = S.k1[w * 32 + b], b2 = S.k2[w * 32 + b];
                if (b1 <= a1 && b2 <= a2 && (b1 < a1 || b2 < a2)) bits |= 1u << b;
            }
            S.dom[p][w] = bits;
        }
    }
    if (threadIdx.x < kWords) {
        unsigned m = 0;
        if ((int)threadIdx.x < nw) {
            const int cnt = min(32, N - (int)threadIdx.x * 32);
            m = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
        }
        S.unassigned[threadIdx.x] = m;
    }
    __syncthreads();

    // Peel fronts: a point joins front r when none of its dominators is still
    // unassigned (Deb's domination count reaching zero).
    int myrank = 0;
    for (int r = 1;; ++r) {
        int blocked = 0;
        if (mine && myrank == 0)
            for (int w = sub; w < nw; w += kTpp) blocked |= (S.dom[p][w] & S.unassigned[w]) != 0;
        else
            blocked = 1;
        const bool front = point_sum(blocked) == 0;
        __syncthreads();
        if (front) {
            myrank = r;
            if (sub == 0) atomicAnd(&S.unassigned[p >> 5], ~(1u << (p & 31)));
        }
        if (!__syncthreads_or(front)) break;
    }
    if (mine && sub == 0) S.rank[p] = myrank;
    __syncthreads();
    const int per = Npad / kTpp;  // comparison partners per thread (a multiple of 8)

    // Front offset and size, and the position of p in its front ordered by
    // (k1, position) and by (k2, position): counting sorts.
    int below = 0, same = 0, pos1 = 0, pos2 = 0;
    if (mine) {
        const long long a1 = S.k1[p], a2 = S.k2[p];
#pragma unroll 8
        for (int t = 0; t < per; ++t) {
            const int q = sub + kTpp * t;
            const int rq = S.rank[q];
            const long long b1 = S.k1[q], b2 = S.k2[q];
            const bool sr = rq == myrank;
            below += rq < myrank;
            same += sr;
            pos1 += sr && ((b1 < a1) || (b1 == a1 && q < p));
            pos2 += sr && ((b2 < a2) || (b2 == a2 && q < p));
        }
    }
    below = point_sum(below);
    same = point_sum(same);
    pos1 = point_sum(pos1);
    pos2 = point_sum(pos2);
    if (mine && sub == 0) {
        S.ord1[below + pos1] = p;
        S.ord2[below + pos2] = p;
    }
    __syncthreads();
    if (mine && sub == 0) {
        const int F = same, off = below;
        double c;
        if (F <= 2) {
            c = INFINITY;
        } else {
            c = 0.0;
            if (pos1 == 0 || pos1 == F - 1) {
                c = INFINITY;
            } else {
                const long long range = S.k1[S.ord1[off + F - 1]] - S.k1[S.ord1[off]];
                if (range > 0) {
                    const long long gap = S.k1[S.ord1[off + pos1 + 1]] - S.k1[S.ord1[off + pos1 - 1]];
                    c = __dadd_rn(c, __ddiv_rn((double)gap, (double)range));
                }
            }
            if (pos2 == 0 || pos2 == F - 1) {
                c = INFINITY;
            } else {
                const long long range = S.k2[S.ord2[off + F - 1]] - S.k2[S.ord2[off]];
                if (range > 0) {
                    const long long gap = S.k2[S.ord2[off + pos2 + 1]] - S.k2[S.ord2[off + pos2 - 1]];
                    c = __dadd_rn(c, __ddiv_rn((double)gap, (double)range));
                }
            }
        }
        S.crowd[p] = c;
    }
    __syncthreads();
    // Crowding values are non-negative or +inf (never NaN or -0), so their
    // IEEE-754 bit patterns order exactly like the values: compare them as
    // integers rather than on the FP64 pipe.
    int pos = 0;
    if (mine) {
        const unsigned long long c = (unsigned long long)__double_as_longlong(S.crowd[p]);
#pragma unroll 8
        for (int t = 0; t < per; ++t) {
            const int q = sub + kTpp * t;
            const int rq = S.rank[q];
            const unsigned long long cq = (unsigned long long)__double_as_longlong(S.crowd[q]);
            pos += (rq < myrank) || (rq == myrank && (cq > c || (cq == c && q < p)));
        }
    }
    pos = point_sum(pos);
    if (mine && sub == 0) S.order[pos] = p;
    __syncthreads();
}

__global__ void __launch_bounds__(kSelThreads)
select_kernel(GenParams gp, PopState ps, int mode)
{
    __shared__ SelShared S;
    const int p = threadIdx.x;  // loads, stores and the tournament: one thread per item
    const int np = gp.np;
    const long long m = gp.m;
    const uint32_t g = *ps.gen;
    const unsigned long long *acc = ps.acc;

    if (mode == 0) {
        if (p < np) {
            S.k1[p] = m - (long long)(acc[p] / 2ull);
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
            S.k1[p] = m - (long long)(acc[i] / 2ull);
            S.k2[p] = (long long)acc[kMaxPop + i];
        }
        __syncthreads();
        if (p < 2 * np) {
            ps.rk[p] = S.k1[p];
            ps.rk[2 * kMaxPop + p] = S.k2[p];
        }
        rank_crowd_order(S, 2 * np);
        long long n1 = 0, n2 = 0;
        if (p < np) {
            const int r = S.order[p];
            S.keep[p] = r;
            n1 = S.k1[r];
            n2 = S.k2[r];
        }
        __syncthreads();
        if (p < np) {
            S.k1[p] = n1;
            S.k2[p] = n2;
        }
        __syncthreads();
    }
    if (p < np) {
        ps.pk[p] = S.k1[p];
        ps.pk[kMaxPop + p] = S.k2[p];
        ps.keep[p] = S.keep[p];
    }

    // Rank and crowding recomputed on P (Alg. 1, start of the generation).
    rank_crowd_order(S, np);
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
