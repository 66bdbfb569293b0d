// k_graph.cu -- device work on an uploaded graph, after the host has checked
// every row (ids in range, no self loop, strictly increasing, so no repeat):
//
// * the symmetry check (an undirected graph, Sec. 2.1: u ~ v iff v ~ u). A
//   warp takes a row v; each lane takes one of its neighbours u and binary
//   searches v in the (sorted) row of u. A missing mirror sets *bad.
// * the oriented adjacency of the offspring evaluation: every undirected
//   edge listed once, at its endpoint of lower (degree, id). A warp per node
//   counts the neighbours above it, one block scans the counts into row
//   pointers, and a warp per node writes the entries in row order.
//
// Every index these kernels form is in range because the host checks ran
// first; the oriented entries are also bounded by their buffer, so a graph
// that the symmetry check is about to reject cannot write past it.
#include "mocd_internal.h"

namespace mocd {

namespace {

__global__ void __launch_bounds__(kBlock)
symmetry_check_kernel(int n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                      int *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    bool ok = true;
    for (int v = warp; v < n; v += nwarps) {
        const int beg = __ldg(row_ptr + v), end = __ldg(row_ptr + v + 1);
        for (int k = beg + lane; k < end; k += 32) {
            const int u = __ldg(col_idx + k);
            int lo = __ldg(row_ptr + u), hi = __ldg(row_ptr + u + 1);  // search [lo, hi)
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if (__ldg(col_idx + mid) < v)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            ok = ok && lo < __ldg(row_ptr + u + 1) && __ldg(col_idx + lo) == v;
        }
    }
    if (!ok) atomicExch(bad, 1);
}

// (deg u, u) > (deg v, v): the edge {u, v} is listed at v.
__device__ __forceinline__ bool above(const int32_t *__restrict__ row_ptr, int v, int dv, int u)
{
    const int du = __ldg(row_ptr + u + 1) - __ldg(row_ptr + u);
    return du > dv || (du == dv && u > v);
}

// eptr[v + 1] = neighbours of v above v; eptr[0] = 0.
__global__ void __launch_bounds__(kBlock)
orient_count_kernel(int n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                    int32_t *__restrict__ eptr)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    if (warp == 0 && lane == 0) eptr[0] = 0;
    for (int v = warp; v < n; v += nwarps) {
        const int beg = __ldg(row_ptr + v), end = __ldg(row_ptr + v + 1);
        int cnt = 0;
        for (int k0 = beg; k0 < end; k0 += 32) {
            const bool up = k0 + lane < end && above(row_ptr, v, end - beg, __ldg(col_idx + k0 + lane));
            cnt += __popc(__ballot_sync(0xffffffffu, up));
        }
        if (lane == 0) eptr[v + 1] = cnt;
    }
}

// In-place inclusive scan of a[0, len) by one block: each warp takes one
// contiguous segment, sums it, then scans it 32 entries at a time from the
// total of the segments before it.
__global__ void scan_kernel(int32_t *__restrict__ a, int len)
{
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int seg = (len + nw - 1) / nw;
    const int b = (int)min((long long)len, (long long)w * seg), e = min(len, b + seg);
    int s = 0;
    for (int i = b + lane; i < e; i += 32) s += a[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) wsum[w] = s;
    __syncthreads();
    int off = 0;
    for (int q = 0; q < w; ++q) off += wsum[q];
    for (int i0 = b; i0 < e; i0 += 32) {
        int x = i0 + lane < e ? a[i0 + lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (i0 + lane < e) a[i0 + lane] = off + x;
        off += __shfl_sync(0xffffffffu, x, 31);
    }
}

// eidx[eptr[v] ..] = the neighbours of v above v, in row order; positions at
// or past cap (possible only for an asymmetric graph) are skipped.
__global__ void __launch_bounds__(kBlock)
orient_fill_kernel(int n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                   const int32_t *__restrict__ eptr, int32_t *__restrict__ eidx, int cap)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int v = warp; v < n; v += nwarps) {
        const int beg = __ldg(row_ptr + v), end = __ldg(row_ptr + v + 1);
        int at = eptr[v];
        for (int k0 = beg; k0 < end; k0 += 32) {
            const int u = k0 + lane < end ? __ldg(col_idx + k0 + lane) : 0;
            const bool up = k0 + lane < end && above(row_ptr, v, end - beg, u);
            const unsigned m = __ballot_sync(0xffffffffu, up);
            const int pos = at + __popc(m & lt);
            if (up && pos >= 0 && pos < cap) eidx[pos] = u;
            at += __popc(m);
        }
    }
}

int warp_grid(const void *kernel, int n, int sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    long long blocks = ((long long)n + kBlock / 32 - 1) / (kBlock / 32);
    if (blocks > (long long)sms * per_sm) blocks = (long long)sms * per_sm;
    return (int)blocks;
}

}  // namespace

cudaError_t launch_orient(int n, const int32_t *row_ptr, const int32_t *col_idx, int32_t *eptr, int32_t *eidx,
                          int cap, int sms, cudaStream_t s)
{
    orient_count_kernel<<<warp_grid((const void *)orient_count_kernel, n, sms), kBlock, 0, s>>>(n, row_ptr,
                                                                                                col_idx, eptr);
    scan_kernel<<<1, 1024, 0, s>>>(eptr, n + 1);
    orient_fill_kernel<<<warp_grid((const void *)orient_fill_kernel, n, sms), kBlock, 0, s>>>(n, row_ptr, col_idx,
                                                                                              eptr, eidx, cap);
    return cudaGetLastError();
}

cudaError_t launch_symmetry_check(int n, const int32_t *row_ptr, const int32_t *col_idx, int *bad, int sms,
                                  cudaStream_t s)
{
    symmetry_check_kernel<<<warp_grid((const void *)symmetry_check_kernel, n, sms), kBlock, 0, s>>>(
        n, row_ptr, col_idx, bad);
    return cudaGetLastError();
}

}  // namespace mocd
