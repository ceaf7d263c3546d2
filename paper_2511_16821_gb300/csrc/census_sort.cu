// census_sort.cu -- stable sort of the remap's survivors by cell (census in cell order), or by the
// 32-bit phase-space key.
//
// LSD radix sort of (key, slot) pairs packed in 64-bit words (key in the high half), 8-bit digits,
// over the remap slots: key = the survivor's cell (or phase-space key), or a sentinel above every
// key for a slot whose particle did not survive (those sort last).
//   * One launch counts the digits of every pass at once (every pass sorts the same keys), so each
//     pass knows where the run of each digit begins.
//   * One launch per pass. A tile of kSortTile consecutive elements takes its place in the pass
//     from a counter, so a tile only ever waits for tiles that started before it. It ranks its
//     elements by digit in element order (warp match on the digit), publishes its digit counts,
//     and finds the counts of all earlier tiles by walking back over their published records.
//     A record holds the count of d in a run of consecutive tiles that ends at its own tile, and
//     the first tile of that run; a tile that reads the record of the tile just before its run
//     adds that count and extends its run to that record's first tile, then republishes its own
//     record, so the runs grow by doubling (pointer jumping) and a walk ends in about log2 of the
//     number of tiles steps, even when every tile of the pass starts at once. (Decoupled look-back
//     for a single-pass scan: Merrill and Garland, 2016; single-pass radix sorting with it:
//     Adinets and Merrill, "Onesweep", 2022.) The tile then writes its elements through shared
//     memory in digit order, so that consecutive threads write consecutive addresses of each
//     digit's run.
// Equal digits keep their order within a tile (ranks in element order) and across tiles (tile
// order), so after all passes the slots are ordered by key and, within a key, by slot: the order
// a stable sort gives, whatever the launch configuration.
// Each pass has its own records, cleared (not yet published) with the digit counts by one
// memset per sort, so a sort recorded in a CUDA graph replays as it runs eagerly. A walk that
// waits longer than its bound sets the status bit kStSegments and stops (the sort is then invalid
// and the step reports HYB_ETIMEOUT); the positions it writes stay inside the output either way.
#include <cuda_runtime.h>

#include "hyb_device.cuh"
#include "hyb_internal.h"

namespace hyb {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 8;                                  // elements per lane
constexpr int kSortTile = kSortThreads * kSortRounds;           // 2048
constexpr int kSortMaxPasses = 4;
constexpr int kHistBatch = 8;                                   // keys in flight per thread when counting
// record: published (bit 63) | first tile of the run it covers (bits 32-62) | count (bits 0-31)
constexpr unsigned long long kPublished = 1ull << 63;

__device__ __forceinline__ unsigned long long run_record(long long first, uint32_t count) {
    return kPublished | ((unsigned long long)first << 32) | (unsigned long long)count;
}

// the pair of element e: from the staged keys (first pass: slot = e) or the previous pass
__device__ __forceinline__ unsigned long long sort_pair(const int32_t* keys, const unsigned long long* pairs,
                                                        long long e, uint32_t sentinel) {
    if (pairs) return pairs[e];
    const int32_t c = keys[e];
    return ((unsigned long long)(c < 0 ? sentinel : (uint32_t)c) << 32) | (unsigned long long)(uint32_t)e;
}

__device__ __forceinline__ unsigned long long ld_record(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_record(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// digit counts of every pass: hist[pass * 256 + digit] (zeroed by the caller)
__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const int32_t* keys, long long n, uint32_t sentinel, int passes, uint32_t* hist) {
    __shared__ uint32_t c[kSortMaxPasses * 256];
    for (int i = threadIdx.x; i < kSortMaxPasses * 256; i += blockDim.x) c[i] = 0;
    __syncthreads();
    // kHistBatch keys per thread loaded at once; dead slots (the sentinel, often most of the slots)
    // counted per thread and added once per warp
    const long long stride = (long long)gridDim.x * blockDim.x;
    uint32_t dead = 0;
    for (long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; e0 < n; e0 += kHistBatch * stride) {
        int32_t v[kHistBatch];
#pragma unroll
        for (int q = 0; q < kHistBatch; ++q) {
            const long long e = e0 + q * stride;
            v[q] = e < n ? keys[e] : INT32_MIN;
        }
#pragma unroll
        for (int q = 0; q < kHistBatch; ++q) {
            if (v[q] == INT32_MIN) continue;   // past the end
            if (v[q] < 0) { ++dead; continue; }
            for (int ps = 0; ps < passes; ++ps) atomicAdd(&c[ps * 256 + (((uint32_t)v[q] >> (8 * ps)) & 255u)], 1u);
        }
    }
    for (int o = 16; o > 0; o >>= 1) dead += __shfl_down_sync(0xffffffffu, dead, o);
    if ((threadIdx.x & 31) == 0 && dead)
        for (int ps = 0; ps < passes; ++ps) atomicAdd(&c[ps * 256 + ((sentinel >> (8 * ps)) & 255u)], dead);
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
        if (c[i]) atomicAdd(hist + i, c[i]);
}

// exclusive scans over the 256 threads of a block of two values at once (one digit per thread)
__device__ __forceinline__ void block_scan2(uint32_t a, uint32_t b, uint32_t* ea, uint32_t* eb, uint32_t* sa,
                                            uint32_t* sb) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t ia = a, ib = b;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t va = __shfl_up_sync(0xffffffffu, ia, o), vb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += va; ib += vb; }
    }
    if (lane == 31) { sa[w] = ia; sb[w] = ib; }
    __syncthreads();
    uint32_t pa = 0, pb = 0;
    for (int q = 0; q < w; ++q) { pa += sa[q]; pb += sb[q]; }
    *ea = pa + ia - a;
    *eb = pb + ib - b;
}

// One pass: the digit at bit `shift` of the key. hist: this pass's 256 digit counts; tile_ctr:
// this pass's tile counter; rec: this pass's ntiles x 256 records (both zeroed by the caller).
__global__ void __launch_bounds__(kSortThreads, 4)
radix_onesweep_kernel(const int32_t* keys, const unsigned long long* pairs_in, long long n, uint32_t sentinel,
                      int shift, const uint32_t* hist, uint32_t* tile_ctr, unsigned long long* rec, int wait_limit,
                      int* status, unsigned long long* pairs_out) {
    __shared__ uint32_t wrun[kSortWarps][256];        // per warp: digit counts, then its start in the tile's run
    __shared__ uint32_t s_lstart[256];                // start of each digit's run in the tile
    __shared__ long long s_gofs[256];                 // global start of the tile's run of d, minus s_lstart[d]
    __shared__ unsigned long long s_buf[kSortTile];   // the tile in digit order
    __shared__ uint32_t s_sa[kSortWarps], s_sb[kSortWarps];
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int d = lane; d < 256; d += 32) wrun[w][d] = 0;
    __syncthreads();
    const long long tile = s_tile;
    const long long base = tile * kSortTile + (long long)w * (kSortTile / kSortWarps);
    // this warp's 256 elements, ranked within their digit in element order
    unsigned long long pr[kSortRounds];
    uint32_t rk[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const long long e = base + r * 32 + lane;
        const bool ok = e < n;
        pr[r] = ok ? sort_pair(keys, pairs_in, e, sentinel) : 0ull;
        const uint32_t d = ok ? (uint32_t)(pr[r] >> (32 + shift)) & 255u : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = ok ? wrun[w][d] : 0u;
        rk[r] = before + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0u) wrun[w][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread d: the warps' starts within the tile's run of digit d, and the tile's count of d
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < kSortWarps; ++q) {
        const uint32_t c = wrun[q][d];
        wrun[q][d] = cnt;
        cnt += c;
    }
    unsigned long long* const my = rec + (size_t)tile * 256 + d;
    st_record(my, run_record(tile, cnt));
    uint32_t lstart, dbase;
    block_scan2(cnt, hist[d], &lstart, &dbase, s_sa, s_sb);
    s_lstart[d] = lstart;
    // the counts of d in every earlier tile: extend this tile's run back to tile 0
    uint32_t acc = cnt;
    long long first = tile;
    int polls = 0;
    while (first > 0) {
        const unsigned long long v = ld_record(rec + (size_t)(first - 1) * 256 + d);
        if (!(v & kPublished)) {   // the tile before the run has not published yet
            if (++polls > wait_limit) { atomicOr(status, kStSegments); break; }
            __nanosleep(20);
            continue;
        }
        acc += (uint32_t)v;
        first = (long long)((v >> 32) & 0x7fffffffull);
        st_record(my, run_record(first, acc));
    }
    const uint32_t earlier = acc - cnt;
    s_gofs[d] = (long long)dbase + (long long)earlier - (long long)lstart;
    __syncthreads();
    // the tile in digit order, then out: consecutive threads write consecutive slots of a run
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const long long e = base + r * 32 + lane;
        if (e < n) {
            const uint32_t dd = (uint32_t)(pr[r] >> (32 + shift)) & 255u;
            s_buf[s_lstart[dd] + wrun[w][dd] + rk[r]] = pr[r];
        }
    }
    __syncthreads();
    const long long rest = n - tile * kSortTile;
    const int nt = rest < kSortTile ? (int)rest : kSortTile;
    for (int i = threadIdx.x; i < nt; i += kSortThreads) {
        const unsigned long long v = s_buf[i];
        const uint32_t dd = (uint32_t)(v >> (32 + shift)) & 255u;
        pairs_out[s_gofs[dd] + i] = v;
    }
}

static int sort_passes(uint32_t sentinel) {
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) <= (uint64_t)sentinel) ++bits;   // keys in [0, sentinel]
    return (bits + 7) / 8;
}

size_t census_sort_scratch_bytes(long long n, uint32_t sentinel) {
    return kSortScratchHead +
           (size_t)sort_passes(sentinel) * (size_t)((n + kSortTile - 1) / kSortTile) * 256 * sizeof(unsigned long long);
}

// Sorts the n remap slots by their keys (negative: dead, sorted last under `sentinel`, which must
// exceed every key). pairs: two buffers of n uint64 (ping-pong); scratch:
// census_sort_scratch_bytes(n, sentinel) bytes (the digit counts and tile counters, then every
// pass's records; cleared here). Returns the sorted (key << 32 | slot) pairs: the low half of
// entry p is the slot at sorted position p.
cudaError_t launch_census_sort(const int32_t* keys, long long n, uint32_t sentinel, unsigned long long* const pairs[2],
                               void* scratch, int wait_limit, int* status, cudaStream_t s,
                               const unsigned long long** sorted) {
    const int passes = sort_passes(sentinel);
    *sorted = pairs[(passes - 1) & 1];
    if (n <= 0) return cudaSuccess;
    const long long ntiles = (n + kSortTile - 1) / kSortTile;
    uint32_t* hist = static_cast<uint32_t*>(scratch);
    uint32_t* ctr = hist + kSortMaxPasses * 256;
    unsigned long long* rec = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + kSortScratchHead);
    const size_t per_pass = (size_t)ntiles * 256;
    cudaError_t e = cudaMemsetAsync(scratch, 0, kSortScratchHead + passes * per_pass * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const long long hg = (n + kSortThreads - 1) / kSortThreads;
    radix_hist_kernel<<<(unsigned)(hg < 152 * 2 ? hg : 152 * 2), kSortThreads, 0, s>>>(keys, n, sentinel, passes, hist);
    for (int ps = 0; ps < passes; ++ps) {
        const unsigned long long* pin = ps == 0 ? nullptr : pairs[(ps - 1) & 1];
        radix_onesweep_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(keys, pin, n, sentinel, 8 * ps, hist + 256 * ps,
                                                                      ctr + ps, rec + ps * per_pass, wait_limit,
                                                                      status, pairs[ps & 1]);
    }
    return cudaGetLastError();
}

}  // namespace hyb
