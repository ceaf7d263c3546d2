// census_sort.cu -- stable sort of the remap's survivors by cell (census in cell order).
//
// LSD radix sort of (key, slot) pairs, 8-bit digits, over the remap slots: key = the survivor's
// cell, or ncells for a slot whose particle did not survive (those sort last). Each pass:
//   1. per tile of kSortTile slots, the digit counts (shared-memory counters)
//   2. one block scans the counts in (digit, tile) order: the start of every (digit, tile) run
//   3. per tile, each warp ranks its 256 slots in slot order (warp match on the digit, ranks from
//      lane order), the warps of the tile take consecutive runs, and every pair is written to
//      its run start + rank.
// Equal digits keep their input order, so after all passes the slots are ordered by cell and,
// within a cell, by slot: the order a stable sort gives, whatever the launch configuration.
#include <cuda_runtime.h>

#include "hyb_device.cuh"

namespace hyb {

constexpr int kSortTile = 2048;            // slots per tile: 8 warps x 8 rounds x 32 lanes
constexpr int kSortThreads = 256;
constexpr int kSortRounds = kSortTile / kSortThreads;

__device__ __forceinline__ uint32_t sort_key(const int32_t* cells, const uint32_t* keys, long long e, uint32_t sentinel) {
    if (keys) return keys[e];
    const int32_t c = cells[e];
    return c < 0 ? sentinel : (uint32_t)c;
}

__global__ void __launch_bounds__(kSortThreads)
radix_count_kernel(const int32_t* cells, const uint32_t* keys, long long n, uint32_t sentinel, int shift,
                   uint32_t* counts, int ntiles) {
    __shared__ uint32_t c[256];
    c[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const long long e = base + r * kSortThreads + threadIdx.x;
        if (e < n) atomicAdd(&c[(sort_key(cells, keys, e, sentinel) >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

// exclusive scan of m counts in place (one block; contiguous chunks per thread)
__global__ void radix_scan_kernel(uint32_t* counts, long long m) {
    __shared__ uint32_t sw[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long per = (m + blockDim.x - 1) / blockDim.x;
    const long long i0 = (long long)threadIdx.x * per;
    uint32_t local = 0;
    for (long long i = i0; i < i0 + per && i < m; ++i) local += counts[i];
    uint32_t inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) sw[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t v = lane < nw ? sw[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) sw[lane] = v;
    }
    __syncthreads();
    uint32_t run = (wid > 0 ? sw[wid - 1] : 0u) + inc - local;
    for (long long i = i0; i < i0 + per && i < m; ++i) {
        const uint32_t c = counts[i];
        counts[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const int32_t* cells, const uint32_t* keys_in, const uint32_t* vals_in, long long n,
                     uint32_t sentinel, int shift, const uint32_t* starts, int ntiles, uint32_t* keys_out,
                     uint32_t* vals_out) {
    __shared__ uint32_t wrun[kSortThreads / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int d = lane; d < 256; d += 32) wrun[w][d] = 0;
    __syncwarp();
    const long long base = (long long)blockIdx.x * kSortTile + (long long)w * (kSortTile / (kSortThreads / 32));
    // this warp's digit counts, in slot order
    for (int r = 0; r < kSortRounds; ++r) {
        const long long e = base + r * 32 + lane;
        const bool ok = e < n;
        const uint32_t d = ok ? (sort_key(cells, keys_in, e, sentinel) >> shift) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & lt) == 0u) wrun[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // run starts of this tile's warps: the tile's run start, then the earlier warps' counts
    {
        const int d = threadIdx.x;
        uint32_t run = starts[(size_t)d * ntiles + blockIdx.x];
        for (int q = 0; q < kSortThreads / 32; ++q) {
            const uint32_t c = wrun[q][d];
            wrun[q][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < kSortRounds; ++r) {
        const long long e = base + r * 32 + lane;
        const bool ok = e < n;
        const uint32_t key = ok ? sort_key(cells, keys_in, e, sentinel) : 0u;
        const uint32_t d = ok ? (key >> shift) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok) {
            const uint32_t pos = wrun[w][d] + (uint32_t)__popc(peers & lt);
            keys_out[pos] = key;
            vals_out[pos] = vals_in ? vals_in[e] : (uint32_t)e;
        }
        __syncwarp();
        if (ok && (peers & lt) == 0u) wrun[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

// Sorts the n remap slots by the staged cells (dead slots last). keys, vals: two buffers of n
// uint32 each (ping-pong); counts: 256 x ceil(n / kSortTile) uint32. Returns the permutation
// (slot of every sorted position) and the sorted keys.
cudaError_t launch_census_sort(const int32_t* cells, long long n, uint32_t ncells, uint32_t* const keys[2],
                               uint32_t* const vals[2], uint32_t* counts, cudaStream_t s, const uint32_t** perm,
                               const uint32_t** sorted_keys) {
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)ncells) ++bits;   // keys in [0, ncells]
    const int passes = (bits + 7) / 8;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    for (int ps = 0; ps < passes && n > 0; ++ps) {
        const uint32_t* kin = ps == 0 ? nullptr : keys[(ps - 1) & 1];
        const uint32_t* vin = ps == 0 ? nullptr : vals[(ps - 1) & 1];
        radix_count_kernel<<<ntiles, kSortThreads, 0, s>>>(cells, kin, n, ncells, 8 * ps, counts, ntiles);
        radix_scan_kernel<<<1, 1024, 0, s>>>(counts, 256LL * ntiles);
        radix_scatter_kernel<<<ntiles, kSortThreads, 0, s>>>(cells, kin, vin, n, ncells, 8 * ps, counts, ntiles,
                                                             keys[ps & 1], vals[ps & 1]);
    }
    *perm = vals[(passes - 1) & 1];
    *sorted_keys = keys[(passes - 1) & 1];
    return cudaGetLastError();
}

}  // namespace hyb
