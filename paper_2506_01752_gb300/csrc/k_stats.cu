// k_stats.cu -- community statistics of every member of the Pareto front:
// the "domain-specific selection criteria" that Alg. 3 leaves open and Sec.
// 4.4 lists (number of communities, spread of community sizes, conductance).
//
// For member i and community c (its nodes V_c):
//   n_c   = |V_c|
//   vol_c = sum_{v in V_c} deg v
//   cut_c = #edges with exactly one endpoint in V_c
//   phi_c = cut_c / min(vol_c, 2m - vol_c)   (conductance; 0 when cut_c = 0)
// and per member
//   k          = #non-empty communities
//   size_sumsq = sum_c n_c^2            (the size variance is sumsq/k - (n/k)^2)
//   mean_phi   = (sum_c phi_c) / k      the sum exact, rounded once to double
//   max_phi    = max_c phi_c
//
// Exactness. Each phi_c is one IEEE division of two exactly converted
// integers. Their sum is accumulated exactly as a 128-bit fixed-point integer
// in units of 2^-88: phi_c is 0 or lies in [2^-30, 1] (the denominator is at
// most m < 2^30 and cut_c <= min(vol_c, 2m - vol_c)), so its lowest mantissa
// bit is at least 2^-82 and phi_c * 2^88 is an integer below 2^89; fewer than
// 2^30 communities keep the total below 2^119. Integer addition is
// associative, so the atomics' order cannot change the result, and the total
// is rounded to the nearest double (ties to even) once.
#include "mocd_internal.h"

namespace mocd {

namespace {

constexpr int kStatWords = 6;  // per member: k, sumsq, sum lo, sum hi, max bits, pad

// Labels of the front members, node-major [n][Wf]: slot k is the member at P
// position front[2 + k], read from R (P half, then Q) through keep.
__global__ void front_rows_kernel(int n, int W, int np, const int32_t *__restrict__ phalf,
                                  const int32_t *__restrict__ q, const int32_t *__restrict__ keep,
                                  const int32_t *__restrict__ front, int Wf, int32_t *__restrict__ dst)
{
    const int count = front[0];
    const long long total = (long long)n * Wf;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / Wf);
        const int k = (int)(t % Wf);
        int32_t lab = 0;
        if (k < count) {
            const int r = keep[front[2 + k]];
            lab = r < np ? phalf[(size_t)v * W + r] : q[(size_t)v * W + (r - np)];
        }
        dst[t] = lab;
    }
}

// Warp per node v, lane q holds slots 4q..4q+3. For every member: n_c and
// vol_c of v's community grow by 1 and deg v (packed as vol << 32 | size:
// sizes stay below 2^30, so the low half never carries), and cut_c by the
// number of v's neighbours outside it.
__global__ void __launch_bounds__(kBlock)
community_tally_kernel(int n, int Wf, int count, const int32_t *__restrict__ row_ptr,
                       const int32_t *__restrict__ col_idx, const int32_t *__restrict__ order,
                       const int32_t *__restrict__ labels, unsigned long long *__restrict__ volsize,
                       uint32_t *__restrict__ cut)
{
    const int lane = threadIdx.x & 31;
    const int nq = Wf >> 2;
    const bool active = lane < nq;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int4 *__restrict__ L4 = reinterpret_cast<const int4 *>(labels);
    const int i0 = 4 * lane;

    for (int idx = warp; idx < n; idx += nwarps) {
        const int v = __ldg(order + idx);
        const int beg = __ldg(row_ptr + v);
        const int end = __ldg(row_ptr + v + 1);
        const int4 own = active ? L4[(size_t)v * nq + lane] : make_int4(0, 0, 0, 0);
        int s0 = 0, s1 = 0, s2 = 0, s3 = 0;  // neighbours sharing the label
        for (int e0 = beg; e0 < end; e0 += 32) {
            const int cnt = min(32, end - e0);
            const int my_u = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
            for (int j0 = 0; j0 < cnt; j0 += 4) {
                int4 a[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int u = __shfl_sync(0xffffffffu, my_u, min(j0 + t, cnt - 1));
                    a[t] = (active && j0 + t < cnt) ? L4[(size_t)u * nq + lane] : make_int4(-1, -1, -1, -1);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    s0 += a[t].x == own.x;
                    s1 += a[t].y == own.y;
                    s2 += a[t].z == own.z;
                    s3 += a[t].w == own.w;
                }
            }
        }
        if (!active) continue;
        const int d = end - beg;
        const unsigned long long add = ((unsigned long long)d << 32) | 1ull;
        const int lab[4] = {own.x, own.y, own.z, own.w};
        const int same[4] = {s0, s1, s2, s3};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int i = i0 + s;
            if (i >= count) break;
            const size_t cell = (size_t)i * n + lab[s];
            atomicAdd(volsize + cell, add);
            if (d - same[s] > 0) atomicAdd(cut + cell, (uint32_t)(d - same[s]));
        }
    }
}

// phi * 2^88 as a 128-bit integer (hi, lo); phi in [2^-30, 1] (see above).
__device__ __forceinline__ void fixed88(double phi, unsigned long long &lo, unsigned long long &hi)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(phi);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;         // phi = mant * 2^(e - 52)
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int s = e + 36;                                       // in [6, 36]
    lo = mant << s;
    hi = mant >> (64 - s);
}

__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long blo,
                                       unsigned long long bhi)
{
    const unsigned long long r = lo + blo;
    hi += bhi + (r < lo ? 1ull : 0ull);
    lo = r;
}

// Block (member slot blockIdx.y, a range of community labels): k, sumsq,
// the fixed-point sum and the maximum of phi, then atomics into acc.
__global__ void __launch_bounds__(kBlock)
community_reduce_kernel(int n, long long two_m, const unsigned long long *__restrict__ volsize,
                        const uint32_t *__restrict__ cut, unsigned long long *__restrict__ acc)
{
    __shared__ unsigned long long s_red[kBlock / 32][5];
    const int i = blockIdx.y;
    unsigned long long k = 0, sq = 0, lo = 0, hi = 0, mx = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const size_t cell = (size_t)i * n + c;
        const unsigned long long a = volsize[cell];
        const unsigned long long sz = a & 0xffffffffull;
        if (!sz) continue;
        k += 1;
        sq += sz * sz;
        const uint32_t ct = cut[cell];
        if (ct) {
            const long long vol = (long long)(a >> 32);
            const long long den = vol < two_m - vol ? vol : two_m - vol;
            const double phi = __ddiv_rn((double)ct, (double)den);
            const unsigned long long pb = (unsigned long long)__double_as_longlong(phi);
            mx = pb > mx ? pb : mx;
            unsigned long long flo, fhi;
            fixed88(phi, flo, fhi);
            add128(lo, hi, flo, fhi);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        k += __shfl_down_sync(0xffffffffu, k, o);
        sq += __shfl_down_sync(0xffffffffu, sq, o);
        const unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, o);
        const unsigned long long ohi = __shfl_down_sync(0xffffffffu, hi, o);
        add128(lo, hi, olo, ohi);
        const unsigned long long om = __shfl_down_sync(0xffffffffu, mx, o);
        mx = om > mx ? om : mx;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_red[w][0] = k;
        s_red[w][1] = sq;
        s_red[w][2] = lo;
        s_red[w][3] = hi;
        s_red[w][4] = mx;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int t = 1; t < kBlock / 32; ++t) {
        k += s_red[t][0];
        sq += s_red[t][1];
        add128(lo, hi, s_red[t][2], s_red[t][3]);
        mx = s_red[t][4] > mx ? s_red[t][4] : mx;
    }
    unsigned long long *a = acc + (size_t)i * kStatWords;
    if (k) atomicAdd(a + 0, k);
    if (sq) atomicAdd(a + 1, sq);
    if (lo | hi) {
        const unsigned long long old = atomicAdd(a + 2, lo);
        const unsigned long long carry = old + lo < old ? 1ull : 0ull;
        if (hi + carry) atomicAdd(a + 3, hi + carry);
    }
    if (mx) atomicMax(a + 4, mx);
}

// (hi, lo) * 2^-88 rounded to the nearest double, ties to even.
__device__ double fixed88_to_double(unsigned long long hi, unsigned long long lo)
{
    if (!hi && !lo) return 0.0;
    const unsigned __int128 x = ((unsigned __int128)hi << 64) | lo;
    const int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading bit
    int e = p - 88;
    unsigned long long mant;
    if (p <= 52) {
        mant = (unsigned long long)(x << (52 - p));
    } else {
        const int r = p - 52;
        mant = (unsigned long long)(x >> r);
        const unsigned __int128 rem = x & ((((unsigned __int128)1) << r) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (r - 1);
        if (rem > half || (rem == half && (mant & 1ull))) {
            ++mant;
            if (mant >> 53) {
                mant >>= 1;
                ++e;
            }
        }
    }
    const unsigned long long bits = ((unsigned long long)(e + 1023) << 52) | (mant & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// out [4][kMaxPop]: k, size_sumsq (int64), mean_phi, max_phi (double bits).
__global__ void stats_finish_kernel(int count, const unsigned long long *__restrict__ acc,
                                    unsigned long long *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const unsigned long long *a = acc + (size_t)i * kStatWords;
    const unsigned long long k = a[0];
    const double sum = fixed88_to_double(a[3], a[2]);
    out[i] = k;
    out[kMaxPop + i] = a[1];
    out[2 * kMaxPop + i] = (unsigned long long)__double_as_longlong(__ddiv_rn(sum, (double)k));
    out[3 * kMaxPop + i] = a[4];
}

}  // namespace

size_t stats_acc_words() { return (size_t)kMaxPop * kStatWords; }

cudaError_t launch_front_stats(const GenParams &gp, const PopState &ps, const int32_t *phalf, int count,
                               const int32_t *row_ptr, const int32_t *col_idx, const int32_t *order,
                               int32_t *rows, unsigned long long *volsize, uint32_t *cut,
                               unsigned long long *acc, unsigned long long *out, int sms, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int n = gp.n;
    const int Wf = (count + 3) & ~3;
    const long long cells = (long long)n * Wf;
    long long blocks = (cells + kBlock - 1) / kBlock;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    front_rows_kernel<<<(int)blocks, kBlock, 0, s>>>(n, gp.W, gp.np, phalf, ps.q, ps.keep, ps.front, Wf, rows);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, community_tally_kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    long long tally_blocks = ((long long)n + kBlock / 32 - 1) / (kBlock / 32);
    if (tally_blocks > (long long)sms * per_sm) tally_blocks = (long long)sms * per_sm;
    community_tally_kernel<<<(int)tally_blocks, kBlock, 0, s>>>(n, Wf, count, row_ptr, col_idx, order, rows,
                                                                volsize, cut);
    long long bx = ((long long)n + kBlock - 1) / kBlock;
    const long long want = ((long long)sms * 8 + count - 1) / count;
    if (bx > want) bx = want;
    if (bx < 1) bx = 1;
    community_reduce_kernel<<<dim3((unsigned)bx, (unsigned)count), kBlock, 0, s>>>(n, 2 * gp.m, volsize, cut, acc);
    stats_finish_kernel<<<1, kMaxPop, 0, s>>>(count, acc, out);
    return cudaGetLastError();
}

}  // namespace mocd
