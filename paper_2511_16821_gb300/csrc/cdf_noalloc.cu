// cdf_noalloc.cu -- the integer 2-D CDF build for callers that cannot allocate device memory.
//
// Its scratch (block partial sums and per-row totals) lives in one file-scope __device__ array of
// fixed size, held by every GPU that loads this library until the process exits. Host code may not
// hand the array's name to a kernel (on the host it is only a stand-in symbol), so the device
// address is looked up once per device with cudaGetSymbolAddress and cached for the life of the
// process. A cudaDeviceReset ends the context that address belongs to (with every other device
// object of this library: problems, batches), so the library is not called on that device again
// after a reset.
#include <cuda_runtime.h>

#include <mutex>

#include "hyb_device.cuh"

namespace {

// Rows served without allocation: up to 4096 (the library's mesh limit), i.e. 34,816 bytes.
constexpr int kNoAllocMaxRows = 4096;

__device__ __align__(256) double g_cdf_scratch[hyb::kCdfParts + kNoAllocMaxRows];

std::mutex g_scratch_mu;
void* g_scratch_addr[256] = {};

}  // namespace

extern "C" HYB_API hyb_status hyb_build_cdf_noalloc(const double* w_dev, int32_t nx, int32_t ny, int64_t* q_dev,
                                                    int64_t* row_pre_dev, int64_t* col_pre_dev, double* W_qmax_dev,
                                                    void* cuda_stream) {
    if (nx < 1 || ny < 1 || nx > 4096) return HYB_EINVAL;
    if (ny > kNoAllocMaxRows) return HYB_EINVAL;   // beyond the fixed scratch
    if (!w_dev || !q_dev || !row_pre_dev || !col_pre_dev || !W_qmax_dev) return HYB_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return HYB_ECUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_cdf_scratch) != cudaSuccess || !ptr) return HYB_ECUDA;
            g_scratch_addr[dev] = ptr;
        }
        scratch = g_scratch_addr[dev];
    }
    // every scratch word the build reads is written earlier in the same call; the max accumulator
    // (an output) is cleared by the build itself
    hyb::Cdf2DView cdf{(long long*)q_dev, (long long*)row_pre_dev, (long long*)col_pre_dev};
    const cudaError_t e = hyb::launch_cdf_build_raw(w_dev, nx, ny, cdf, W_qmax_dev, W_qmax_dev + 1, (double*)scratch,
                                                    (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? HYB_OK : HYB_ECUDA;
}
