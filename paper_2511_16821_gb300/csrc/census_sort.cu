// census_sort.cu -- stable sort of the remap's survivors by cell (census in cell order).
//
// LSD radix sort of (key, slot) pairs packed in 64-bit words (key in the high half), 8-bit digits,
// over the remap slots: key = the survivor's cell, or ncells for a slot whose particle did not
// survive (those sort last). Each pass:
//   1. per tile of kSortTile slots, the digit counts (shared-memory counters)
//   2. the counts are scanned in (digit, tile) order: per digit over its tiles (one block per
//      digit), then over the 256 digit totals: the start of every (digit, tile) run
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

// the pair of element e: from the staged cells (first pass: slot = e) or the previous pass
__device__ __forceinline__ unsigned long long sort_pair(const int32_t* cells, const unsigned long long* pairs,
                                                        long long e, uint32_t sentinel) {
    if (pairs) return pairs[e];
    const int32_t c = cells[e];
    return ((unsigned long long)(c < 0 ? sentinel : (uint32_t)c) << 32) | (unsigned long long)(uint32_t)e;
}

__global__ void __launch_bounds__(kSortThreads)
radix_count_kernel(const int32_t* cells, const unsigned long long* pairs, long long n, uint32_t sentinel, int shift,
                   uint32_t* counts, int ntiles) {
    __shared__ uint32_t c[256];
    c[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const long long e = base + r * kSortThreads + threadIdx.x;
        if (e < n) atomicAdd(&c[(uint32_t)(sort_pair(cells, pairs, e, sentinel) >> (32 + shift)) & 255u], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

// per digit (one block each): exclusive scan of the digit's tile counts in place, digit total
__global__ void __launch_bounds__(kSortThreads) radix_digit_scan_kernel(uint32_t* counts, int ntiles, uint32_t* dtot) {
    __shared__ uint32_t sw[kSortThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* c = counts + (size_t)blockIdx.x * ntiles;
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    uint32_t local = 0;
    for (int i = i0; i < i0 + per && i < ntiles; ++i) local += c[i];
    uint32_t inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) sw[wid] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int q = 0; q < kSortThreads / 32; ++q) {
        if (q < wid) before += sw[q];
        total += sw[q];
    }
    uint32_t run = before + inc - local;
    for (int i = i0; i < i0 + per && i < ntiles; ++i) {
        const uint32_t v = c[i];
        c[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = total;
}

// exclusive scan of the 256 digit totals (one block of 256 threads)
__global__ void radix_base_kernel(uint32_t* dtot) {
    __shared__ uint32_t sw[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t v = dtot[threadIdx.x];
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) sw[wid] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int q = 0; q < wid; ++q) before += sw[q];
    dtot[threadIdx.x] = before + inc - v;
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const int32_t* cells, const unsigned long long* pairs_in, long long n, uint32_t sentinel,
                     int shift, const uint32_t* starts, const uint32_t* dbase, int ntiles,
                     unsigned long long* pairs_out) {
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
        const uint32_t d = ok ? (uint32_t)(sort_pair(cells, pairs_in, e, sentinel) >> (32 + shift)) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & lt) == 0u) wrun[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // run starts of this tile's warps: the tile's run start, then the earlier warps' counts
    {
        const int d = threadIdx.x;
        uint32_t run = dbase[d] + starts[(size_t)d * ntiles + blockIdx.x];
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
        const unsigned long long pr = ok ? sort_pair(cells, pairs_in, e, sentinel) : 0ull;
        const uint32_t d = ok ? (uint32_t)(pr >> (32 + shift)) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok) pairs_out[wrun[w][d] + (uint32_t)__popc(peers & lt)] = pr;
        __syncwarp();
        if (ok && (peers & lt) == 0u) wrun[w][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

// Sorts the n remap slots by the staged cells (dead slots last). pairs: two buffers of n uint64
// (ping-pong); counts: 256 x (ceil(n / kSortTile) + 1) uint32 (the tile counts, then the digit
// bases). Returns the sorted (cell << 32 | slot) pairs: the low half of entry p is the slot at
// sorted position p.
cudaError_t launch_census_sort(const int32_t* cells, long long n, uint32_t ncells, unsigned long long* const pairs[2],
                               uint32_t* counts, cudaStream_t s, const unsigned long long** sorted) {
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)ncells) ++bits;   // keys in [0, ncells]
    const int passes = (bits + 7) / 8;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    for (int ps = 0; ps < passes && n > 0; ++ps) {
        const unsigned long long* pin = ps == 0 ? nullptr : pairs[(ps - 1) & 1];
        uint32_t* dtot = counts + 256 * (size_t)ntiles;
        radix_count_kernel<<<ntiles, kSortThreads, 0, s>>>(cells, pin, n, ncells, 8 * ps, counts, ntiles);
        radix_digit_scan_kernel<<<256, kSortThreads, 0, s>>>(counts, ntiles, dtot);
        radix_base_kernel<<<1, 256, 0, s>>>(dtot);
        radix_scatter_kernel<<<ntiles, kSortThreads, 0, s>>>(cells, pin, n, ncells, 8 * ps, counts, dtot, ntiles,
                                                             pairs[ps & 1]);
    }
    *sorted = pairs[(passes - 1) & 1];
    return cudaGetLastError();
}

}  // namespace hyb
