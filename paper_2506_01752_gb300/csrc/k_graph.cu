// k_graph.cu -- the symmetry check of an uploaded graph (an undirected graph,
// Sec. 2.1: u ~ v iff v ~ u), run on the device after the host has checked
// every row (ids in range, no self loop, strictly increasing, so no repeat).
//
// A warp takes a row v; each lane takes one of its neighbours u and binary
// searches v in the (sorted) row of u. A missing mirror sets *bad. Every
// index the kernel forms is in range because the host checks ran first.
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

}  // namespace

cudaError_t launch_symmetry_check(int n, const int32_t *row_ptr, const int32_t *col_idx, int *bad, int sms,
                                  cudaStream_t s)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, symmetry_check_kernel, kBlock, 0);
    if (per_sm < 1) per_sm = 1;
    long long blocks = ((long long)n + kBlock / 32 - 1) / (kBlock / 32);
    if (blocks > (long long)sms * per_sm) blocks = (long long)sms * per_sm;
    symmetry_check_kernel<<<(int)blocks, kBlock, 0, s>>>(n, row_ptr, col_idx, bad);
    return cudaGetLastError();
}

}  // namespace mocd
