// probe.cu -- throughput of the fixed-point tally additions (global 64-bit integer atomics), the
// denominator of the MC leg's atomic roofline. No counterpart in the paper: the method only fixes
// what is added (track-length contributions), and this measures how fast this GPU can add them.
#include <cuda_runtime.h>

#include <algorithm>

#include "hyb_device.cuh"

namespace {

// each thread adds 1 to `per_thread` addresses drawn uniformly from [0, n_addr) by a 64-bit LCG
// (Knuth's MMIX constants); the result is unused, so each addition is a fire-and-forget reduction
__global__ void atomic_rate_kernel(unsigned long long* a, unsigned long long n_addr, int per_thread, uint64_t seed) {
    uint64_t h = hyb::dmix64(seed ^ ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x));
    for (int i = 0; i < per_thread; ++i) {
        h = h * 6364136223846793005ull + 1442695040888963407ull;
        const unsigned long long k = __umul64hi(h, n_addr);
        atomicAdd(a + k, 1ull);
    }
}

}  // namespace

extern "C" HYB_API hyb_status hyb_atomic_rate(int64_t n_addr, int64_t n_ops, void* stream, double* ops_per_s) {
    if (n_addr < 1 || n_ops < 1 || !ops_per_s) return HYB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HYB_ECUDA;
    const int block = 256, grid = sms * 8;
    const long long threads = (long long)grid * block;
    const int per = (int)std::max<long long>(1, std::min<long long>(n_ops / threads, 1 << 20));
    unsigned long long* a = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hyb_status rc = HYB_OK;
    float best = 0.f;
    if (cudaMalloc(&a, (size_t)n_addr * 8) != cudaSuccess) return HYB_ENOMEM;
    if (cudaMemsetAsync(a, 0, (size_t)n_addr * 8, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = HYB_ECUDA;
    } else {
        atomic_rate_kernel<<<grid, block, 0, s>>>(a, (unsigned long long)n_addr, per, 99);   // warm-up
        for (int r = 0; r < 3 && rc == HYB_OK; ++r) {
            cudaEventRecord(e0, s);
            atomic_rate_kernel<<<grid, block, 0, s>>>(a, (unsigned long long)n_addr, per, 100 + r);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = HYB_ECUDA;
            else if (best == 0.f || ms < best) best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(a);
    if (rc == HYB_OK) *ops_per_s = best > 0.f ? (double)threads * per / (best * 1e-3) : 0.0;
    return rc;
}
