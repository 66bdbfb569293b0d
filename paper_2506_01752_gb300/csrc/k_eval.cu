// k_eval.cu -- objective evaluation of a whole population (Eq. objectives,
// Sec. 4.1; Alg. 1 EvaluateIndividual, run for every individual at once).
//
// For each individual i the kernel accumulates
//   intra_i = #{{v, u} in E : L_i(v) = L_i(u)}   (= sum_c |E(c)|)
//   S_i     = sum_c D_c^2,  D_c = sum_{v : L_i(v) = c} deg v
// exactly in integers. Each undirected edge is counted once, from one
// endpoint: with the full adjacency (the initial population, mocd_evaluate)
// a warp reads the label rows of the neighbours u > v only; the offspring
// evaluation inside a generation walks an oriented adjacency that lists
// every edge once, at its endpoint of lower (degree, id), so the rows it
// reads are the higher-degree endpoints' -- fewer distinct rows, each read
// more often, which keeps more of them in L2.
//
// Layout is node-major: a warp owns node v and lane q holds the int4 of
// labels of individuals 4q..4q+3, so each neighbour u costs one coalesced
// row read of all individuals' labels instead of N_p scattered 4-byte
// gathers, and the CSR is streamed once per population, not once per
// individual.
//
// S without a sweep over the histogram: when node v adds deg(v) to D_c, the
// atomic returns the old total o, and (o + d)^2 - o^2 = 2 o d + d^2. Summed
// over every addition these increments telescope to D_c^2 whatever the order
// of the atomics, so S is exact and deterministic.
//
// Histogram layout: label-major, D of (individual i, label c) at c * W + i,
// so that one atomic instruction of a warp (25 individuals of node v) lands
// in few cache lines whenever individuals share v's label; or
// individual-major, i * n + c (count * n cells, for fixed-size scratch).
//
// Inside a generation the D histogram is not built here: the mutation kernel,
// which writes every child's final label of node v, adds deg(v) to the
// label-major cell of that label as it goes (fire-and-forget reductions that
// overlap its own latency-bound work). The evaluation of the offspring then
// counts intra (COUNT_D = false) and, in the same launch once a warp's nodes
// are done, forms S = sum_c D_c^2 in a coalesced sweep of the histogram rows,
// zeroing them for the next generation. While the labels are still nearly all distinct, the N_p n
// histogram additions land on different sectors, which at n = 10^6 (a 400 MB
// histogram) cost a DRAM read and write-back each; done by the mutation
// kernel, that traffic overlaps with its own work instead of stalling the
// evaluation's row stream.
#include "mocd_check.cuh"
#include "mocd_internal.h"

namespace mocd {

namespace {

template <bool LABEL_MAJOR, bool COUNT_D>
__device__ __forceinline__ void evaluate_body(int n, int W, int count, const int32_t *__restrict__ row_ptr,
                                              const int32_t *__restrict__ col_idx,
                                              const int32_t *__restrict__ labels, uint32_t *__restrict__ hist,
                                              unsigned long long *__restrict__ acc,
                                              const int32_t *__restrict__ order, int vblock, int vgrid)
{
    __shared__ unsigned long long s_intra[kMaxPop];
    __shared__ unsigned long long s_sq[kMaxPop];
    __shared__ int s_nb[kBlock];  // per warp: the chunk's neighbours u > v
    for (int t = threadIdx.x; t < kMaxPop; t += blockDim.x) {
        s_intra[t] = 0;
        s_sq[t] = 0;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int nq = W >> 2;
    const bool active = lane < nq;
    const int warp = (vblock * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (vgrid * blockDim.x) >> 5;
    const int4 *__restrict__ L4 = reinterpret_cast<const int4 *>(labels);
    const int i0 = 4 * lane;
    int *nb = s_nb + (threadIdx.x & ~31);
    const unsigned lt = (1u << lane) - 1u;

    auto cell = [&](int i, int c) -> size_t {
        return LABEL_MAJOR ? (size_t)c * W + i : (size_t)i * n + c;
    };
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    unsigned long long q0 = 0, q1 = 0, q2 = 0, q3 = 0;

    for (int idx = warp; idx < n; idx += nwarps) {
        const int v = order ? __ldg(order + idx) : idx;
        const int beg = __ldg(row_ptr + v);
        const int end = __ldg(row_ptr + v + 1);
        if (!MOCD_CHECK(end >= beg, kCheckRowPtr, v)) continue;  // (warp-uniform)
        const int4 own = active ? L4[(size_t)v * nq + lane] : make_int4(0, 0, 0, 0);
        for (int e0 = beg; e0 < end; e0 += 32) {
            const int cnt = min(32, end - e0);
            const int my_u = lane < cnt ? __ldg(col_idx + e0 + lane) : 0;
            // Keep the neighbours whose rows v reads, compacted: u > v of the
            // full adjacency, or every entry of the oriented one.
            const bool up = lane < cnt && (!COUNT_D || my_u > v) && MOCD_CHECK(my_u < n, kCheckNode, v);
            const unsigned upm = __ballot_sync(0xffffffffu, up);
            const int cu = __popc(upm);
            if (up) nb[__popc(upm & lt)] = my_u;
            __syncwarp();
            // Four independent row loads in flight per lane.
            for (int j0 = 0; j0 < cu; j0 += 4) {
                int4 a[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int u = nb[min(j0 + t, cu - 1)];
                    a[t] = (active && j0 + t < cu) ? L4[(size_t)u * nq + lane] : make_int4(-1, -1, -1, -1);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    c0 += a[t].x == own.x;
                    c1 += a[t].y == own.y;
                    c2 += a[t].z == own.z;
                    c3 += a[t].w == own.w;
                }
            }
            __syncwarp();
        }
        const unsigned long long d = (unsigned long long)(end - beg);
        if (COUNT_D && active && d > 0) {
            const unsigned dd = (unsigned)d;
            if (i0 + 0 < count && MOCD_CHECK((unsigned)own.x < (unsigned)n, kCheckLabel, v)) {
                const unsigned long long o = atomicAdd(hist + cell(i0 + 0, own.x), dd);
                q0 += 2ull * o * d + d * d;
            }
            if (i0 + 1 < count && MOCD_CHECK((unsigned)own.y < (unsigned)n, kCheckLabel, v)) {
                const unsigned long long o = atomicAdd(hist + cell(i0 + 1, own.y), dd);
                q1 += 2ull * o * d + d * d;
            }
            if (i0 + 2 < count && MOCD_CHECK((unsigned)own.z < (unsigned)n, kCheckLabel, v)) {
                const unsigned long long o = atomicAdd(hist + cell(i0 + 2, own.z), dd);
                q2 += 2ull * o * d + d * d;
            }
            if (i0 + 3 < count && MOCD_CHECK((unsigned)own.w < (unsigned)n, kCheckLabel, v)) {
                const unsigned long long o = atomicAdd(hist + cell(i0 + 3, own.w), dd);
                q3 += 2ull * o * d + d * d;
            }
        }
    }

    if (!COUNT_D && LABEL_MAJOR && active) {
        // S from the histogram [n][W] that the mutation kernel built: a warp
        // per row, lane q the int4 of individuals 4q..4q+3; every non-zero
        // cell is squared and cleared. D_c^2 < 2^62 and S <= (2m)^2, so the
        // 64-bit sums are exact.
        uint4 *__restrict__ H4 = reinterpret_cast<uint4 *>(hist);
        // Four rows in flight per lane.
        for (int c0 = warp; c0 < n; c0 += 4 * nwarps) {
            uint4 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c0 + k * nwarps;
                x[k] = c < n ? H4[(size_t)c * nq + lane] : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c0 + k * nwarps;
                if (x[k].x | x[k].y | x[k].z | x[k].w) {
                    q0 += (unsigned long long)x[k].x * x[k].x;
                    q1 += (unsigned long long)x[k].y * x[k].y;
                    q2 += (unsigned long long)x[k].z * x[k].z;
                    q3 += (unsigned long long)x[k].w * x[k].w;
                    H4[(size_t)c * nq + lane] = make_uint4(0, 0, 0, 0);
                }
            }
        }
    }
    if (active) {
        if (i0 + 0 < count) { atomicAdd(&s_intra[i0 + 0], (unsigned long long)c0); atomicAdd(&s_sq[i0 + 0], q0); }
        if (i0 + 1 < count) { atomicAdd(&s_intra[i0 + 1], (unsigned long long)c1); atomicAdd(&s_sq[i0 + 1], q1); }
        if (i0 + 2 < count) { atomicAdd(&s_intra[i0 + 2], (unsigned long long)c2); atomicAdd(&s_sq[i0 + 2], q2); }
        if (i0 + 3 < count) { atomicAdd(&s_intra[i0 + 3], (unsigned long long)c3); atomicAdd(&s_sq[i0 + 3], q3); }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        if (s_intra[t]) atomicAdd(acc + t, s_intra[t]);
        if (s_sq[t]) atomicAdd(acc + kMaxPop + t, s_sq[t]);
    }
}

template <bool LABEL_MAJOR, bool COUNT_D>
__global__ void __launch_bounds__(kBlock)
evaluate_kernel(int n, int W, int count, const int32_t *__restrict__ row_ptr,
                const int32_t *__restrict__ col_idx, const int32_t *__restrict__ labels,
                uint32_t *__restrict__ hist, unsigned long long *__restrict__ acc,
                const int32_t *__restrict__ order)
{
    evaluate_body<LABEL_MAJOR, COUNT_D>(n, W, count, row_ptr, col_idx, labels, hist, acc, order, blockIdx.x,
                                        gridDim.x);
}

// The offspring evaluation of every member of a batch in one launch: members
// own consecutive block ranges (starts[k] .. starts[k + 1] - 1).
__global__ void __launch_bounds__(kBlock, 4)
evaluate_multi_kernel(const BatchMember *__restrict__ members, const int *__restrict__ starts, int count)
{
    const int bk = (int)blockIdx.x;
    int lo = 0, hi = count;  // starts[lo] <= bk < starts[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(starts + mid) <= bk) lo = mid;
        else hi = mid;
    }
    const BatchMember &mb = members[lo];
    const int b0 = __ldg(starts + lo);
    evaluate_body<true, false>(mb.gp.n, mb.gp.W, mb.gp.np, mb.eptr, mb.eidx, mb.ps.q, mb.ps.hist, mb.ps.acc,
                               mb.order, bk - b0, __ldg(starts + lo + 1) - b0);
}

}  // namespace

int grid_for_eval(int sms, bool label_major)
{
    int per_sm = 0;
    if (label_major)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_kernel<true, true>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_kernel<false, true>, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

int grid_for_eval_intra(int sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_kernel<true, false>, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_evaluate(int n, int W, int count, const int32_t *row_ptr, const int32_t *col_idx,
                            const int32_t *labels, uint32_t *hist, unsigned long long *acc,
                            int grid, cudaStream_t s, const int32_t *order, bool label_major)
{
    if (label_major)
        evaluate_kernel<true, true><<<grid, kBlock, 0, s>>>(n, W, count, row_ptr, col_idx, labels, hist, acc,
                                                            order);
    else
        evaluate_kernel<false, true><<<grid, kBlock, 0, s>>>(n, W, count, row_ptr, col_idx, labels, hist, acc,
                                                             order);
    return cudaGetLastError();
}

cudaError_t launch_evaluate_multi(const BatchMember *members, const int *starts, int count, int blocks,
                                  cudaStream_t s)
{
    if (blocks > 0) evaluate_multi_kernel<<<blocks, kBlock, 0, s>>>(members, starts, count);
    return cudaGetLastError();
}

cudaError_t launch_evaluate_offspring(int n, int W, int count, const int32_t *eptr, const int32_t *eidx,
                                      const int32_t *labels, uint32_t *hist, unsigned long long *acc,
                                      int grid, cudaStream_t s, const int32_t *order)
{
    evaluate_kernel<true, false><<<grid, kBlock, 0, s>>>(n, W, count, eptr, eidx, labels, hist, acc, order);
    return cudaGetLastError();
}

}  // namespace mocd

namespace mocd {
cudaError_t check_record_eval(unsigned long long *out, bool reset)
{
    return check_record(out, reset);
}
}  // namespace mocd
