// noalloc.cu -- objective evaluation for callers that cannot allocate device
// memory.
//
// mocd_evaluate and the generation engine keep their per-individual degree
// histograms in memory that the context allocates with cudaMalloc. Some
// callers cannot do that: a plug-in whose process hands all free device
// memory to another allocator (a framework's caching pool), code under a fixed
// device-memory budget that must not grow after start-up, or a latency-critical
// loop that cannot afford cudaMalloc's implicit synchronisation. For them,
// mocd_evaluate_noalloc runs the same evaluation kernel with its scratch in a
// fixed array compiled into this library. The caller passes only its inputs
// and outputs.
//
// The scratch below is a device symbol: every GPU that loads this library
// holds it (16 MiB + 2 KiB) until the process exits. On the host its name is
// only a stand-in, never a device address, so the address is fetched once per
// device with cudaGetSymbolAddress (the first call on each device does that)
// and then passed to the kernels. The cached address belongs to the device's
// primary context of that moment: after a cudaDeviceReset the entry point
// must not be used again in the same process.
#include <mutex>

#include "mocd.h"
#include "mocd_internal.h"

using namespace mocd;

namespace {

constexpr size_t kAccWords = 4 * kMaxPop;  // 2 x kMaxPop unsigned long long
constexpr size_t kScratchWords = kAccWords + (size_t)MOCD_NOALLOC_MAX_CELLS;
constexpr int kMaxDevices = 64;

// [0, kAccWords): intra / S accumulators; then the histogram [count][n].
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

uint32_t *g_scratch_addr[kMaxDevices];
std::mutex g_setup_mutex;

__global__ void finish_keys_kernel(int count, const unsigned long long *__restrict__ acc,
                                   int64_t *__restrict__ intra, int64_t *__restrict__ sumsq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        intra[i] = (int64_t)acc[i];
        sumsq[i] = (int64_t)acc[kMaxPop + i];
    }
}

// Address of the scratch on the current device, set up on first use.
int scratch_on_current_device(uint32_t **out, int *device)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MOCD_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return MOCD_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MOCD_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_addr[dev];
    *device = dev;
    return MOCD_OK;
}

}  // namespace

extern "C" int mocd_evaluate_noalloc(const int32_t *row_ptr, const int32_t *col_idx, int64_t n,
                                     const int32_t *labels, int32_t count, int64_t *intra,
                                     int64_t *sumsq, void *cuda_stream)
{
    if (!row_ptr || !col_idx || !labels || !intra || !sumsq) return MOCD_ERR_INVALID_ARG;
    if (n < 1 || n >= (int64_t(1) << 30) || count < 1 || count > kMaxPop) return MOCD_ERR_INVALID_ARG;
    if ((int64_t)count * n > (int64_t)MOCD_NOALLOC_MAX_CELLS) return MOCD_ERR_TOO_LARGE;
    uint32_t *scratch = nullptr;
    int dev = 0;
    int rc = scratch_on_current_device(&scratch, &dev);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(scratch);
    uint32_t *hist = scratch + kAccWords;
    const int W = (count + 3) & ~3;
    // The scratch keeps the previous call's contents: clear what must start at 0.
    if (cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * (kAccWords + (size_t)count * (size_t)n), s) != cudaSuccess)
        return MOCD_ERR_CUDA;
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MOCD_ERR_CUDA;
    if (launch_evaluate((int)n, W, count, row_ptr, col_idx, labels, hist, acc, grid_for_eval(sms, false), s,
                        nullptr, false) != cudaSuccess)
        return MOCD_ERR_CUDA;
    finish_keys_kernel<<<1, kMaxPop, 0, s>>>(count, acc, intra, sumsq);
    if (cudaGetLastError() != cudaSuccess) return MOCD_ERR_CUDA;
    return MOCD_OK;
}
