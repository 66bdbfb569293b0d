// mocd_check.cuh -- bounds checks of the debug build (-DMOCD_DEBUG_CHECKS).
//
// In the debug build the kernels check the invariants their memory accesses
// rely on (CSR row pointers non-decreasing, node ids and labels in [0, n),
// indices into R = P u Q below 2 N_p). A failed check never traps: the kernel
// skips the access it guards and records the failure in this translation
// unit's record (failures counted; the first failure's code and index kept),
// which the host reads with mocd_debug_checks. In the normal build every
// check is the constant `true` and compiles away.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mocd {

enum CheckCode : unsigned long long {
    kCheckRowPtr = 1,      // row_ptr[v + 1] < row_ptr[v]
    kCheckNode = 2,        // a neighbour id outside [0, n)
    kCheckLabel = 3,       // a label outside [0, n)
    kCheckRIndex = 4,      // an index into R = P u Q outside [0, 2 N_p)
};

namespace {

#ifdef MOCD_DEBUG_CHECKS
// [0] failures, [1] first failure's code, [2] its index (node or slot).
__device__ unsigned long long g_check[3];

__device__ __forceinline__ bool check_ok(bool ok, unsigned long long code, long long index)
{
    if (!ok) {
        if (atomicAdd(&g_check[0], 1ull) == 0ull) {
            g_check[1] = code;
            g_check[2] = (unsigned long long)index;
        }
    }
    return ok;
}

// Copies this translation unit's record to out[3] (and zeroes it if asked).
inline cudaError_t check_record(unsigned long long *out, bool reset)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_check, sizeof(unsigned long long) * 3);
    if (e == cudaSuccess && reset) {
        const unsigned long long z[3] = {0, 0, 0};
        e = cudaMemcpyToSymbol(g_check, z, sizeof(z));
    }
    return e;
}
#define MOCD_CHECK(cond, code, index) (::mocd::check_ok((cond), (code), (long long)(index)))
#else
inline cudaError_t check_record(unsigned long long *out, bool)
{
    out[0] = out[1] = out[2] = 0;
    return cudaSuccess;
}
#define MOCD_CHECK(cond, code, index) (true)
#endif

}  // namespace

}  // namespace mocd
