// remap.cu -- scatter-free census remap (Sec. 2.2 steps 3-4, Eq. (R)) and the integer 2-D CDF.
//
// CDF build (shared by the static source and the remap source): per cell |q| -> max and sum
// (deterministic block order) -> q_int = rint(|q| / max |q| 2^B), B = min(40, 62 - ceil(log2 ncells))
// -> per-row exclusive scans
// (column conditional) and column guides -> row-total scan (row marginal) and row guide in the
// last row block. Exact integer arithmetic, so cells are picked identically on the FP32 and FP64
// paths.
//
// Remap: slot j in [bank slots | births] is re-streamed straight with sigma_t attenuation from its
// step-start state (bank particles are copied, births come from the remap source density
// Q + sigma_s (phi_pre + phi_post + phi_c), bilinear within a cell). Three launches:
//   pass A  re-stream every slot, stage its end state (24 B/slot FP32), count survivors, sum
//           quantised |w| and |w| per block
//   scan    one block: block offsets, totals, comb decision and tooth offset
//   pass B  read the staged states, block scan, write survivors (or their comb copies) into the
//           other bank in slot order.
// Staging costs ~48 B of HBM traffic per slot, far less than redoing a birth (two CDF searches,
// the point draws, sincos) and its stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "hyb_device.cuh"
#include "pdl.cuh"

namespace hyb {

constexpr int kRounds = 8;                       // slot rounds per pass-B block (2048 census positions)
constexpr int kSlotsPerBlock = kTile * kRounds;
constexpr int kPartSlots = kSlotsPerBlock;      // census piece: the unit of the partials (one pass B block)
constexpr int kPartsPerBlock = kSlotsPerBlock / kPartSlots;

// ---------------------------------------------------------------------------------------------
// CDF build
// ---------------------------------------------------------------------------------------------
__global__ void cdf_reduce_kernel(const double* __restrict__ w, int ncells, double* part_sum, double* qmax) {
    pdl_wait();
    pdl_trigger();
    double s = 0, m = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncells; k += gridDim.x * blockDim.x) {
        const double a = fabs(w[k]);
        s += a;
        m = fmax(m, a);
    }
    s = warp_sum(s);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double ss[32];
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        if (m > 0) atomicMax((unsigned long long*)qmax, (unsigned long long)__double_as_longlong(m));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ss[q];
        part_sum[blockIdx.x] = t;
    }
}

// one warp: strided partial sums, then a fixed-order shuffle tree (deterministic); afterwards the
// first partial's word is the row kernel's arrival counter, so it is zeroed here
__global__ void cdf_total_kernel(double* part_sum, int nparts, double* W) {
    pdl_wait();
    pdl_trigger();
    double t = 0;
    for (int i = threadIdx.x; i < nparts; i += 32) t += part_sum[i];
    t = warp_sum(t);
    if (threadIdx.x == 0) {
        *W = t;
        *reinterpret_cast<unsigned*>(part_sum) = 0u;
    }
}

// the bin of point x in pre[0..n] searched in [lo, hi]: the decisions of pick_bin, for the guide
// tables (pre may have been written earlier in the same launch, so it is read without __restrict__)
__device__ __forceinline__ int guide_bin(const long long* pre, int n, uint32_t x, int lo, int hi) {
    const unsigned long long total = (unsigned long long)pre[n];
    const unsigned long long m = 2ull * (unsigned long long)x + 1ull;
    const unsigned long long Plo = m * total, Phi = __umul64hi(m, total);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const unsigned long long v = (unsigned long long)pre[mid];
        const unsigned long long vhi = v >> 31, vlo = v << 33;
        if (vhi < Phi || (vhi == Phi && vlo <= Plo)) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* total);

// one block per row: q_int, the exclusive column scan of the row and the row's column guide; the
// last block to finish (arrival counter *done, zeroed beforehand) forms the row marginal from the
// row totals and the row guide, so the whole table is one launch
// the remap's per-step scalars (the comb's quantisation base, RemapScal); defined below
__device__ void remap_prep_body(DevState* st, long long n_hist, long long lead, double w_lead);

// prep: the remap's CDF (non-null) -- its last row block also forms the remap's per-step scalars
// (n_hist, lead, w_lead as for remap_prep_body), so that no launch of its own is needed
__global__ void cdf_rows_kernel(const double* __restrict__ w, const double* qmax, int nx, int ny, Cdf2DView C,
                                long long* row_tot, unsigned* done, DevState* prep, long long n_hist,
                                long long lead, double w_lead) {
    pdl_wait();
    pdl_trigger();
    const int iy = blockIdx.x;
    const double qm = *qmax;
    // 2^B with B = min(40, 62 - ceil(log2 ncells)): the table's total stays below 2^62
    int lg = 0;
    while ((1ll << lg) < (long long)nx * ny) ++lg;
    const double qsc = ldexp(1.0, min(40, 62 - lg));
    const int per = (nx + blockDim.x - 1) / blockDim.x;
    const int c0 = threadIdx.x * per;
    long long local = 0;
    for (int c = c0; c < c0 + per && c < nx; ++c) {
        const size_t k = (size_t)iy * nx + c;
        const long long q = qm > 0 ? __double2ll_rn((fabs(w[k]) / qm) * qsc) : 0;
        C.q[k] = q;
        local += q;
    }
    // block exclusive scan of the per-thread totals
    __shared__ long long sw[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) sw[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        long long v = lane < nw ? sw[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) sw[lane] = v;
    }
    __syncthreads();
    long long run = (wid > 0 ? sw[wid - 1] : 0) + inc - local;
    long long* pre = C.col_pre + (size_t)iy * (nx + 1);
    for (int c = c0; c < c0 + per && c < nx; ++c) {
        pre[c] = run;
        run += C.q[(size_t)iy * nx + c];
    }
    if (threadIdx.x == blockDim.x - 1) {
        const long long tot = sw[(blockDim.x >> 5) - 1];
        pre[nx] = tot;
        row_tot[iy] = tot;
    }
    __syncthreads();
    // column guide of this row: entry g is the bin of the bucket's smallest point g 2^(32-gc)
    const bool guides = C.row_g != nullptr && C.col_g != nullptr;
    if (guides) {
        const int Gc = 1 << C.gc;
        int* cg = C.col_g + (size_t)iy * (Gc + 1);
        for (int g = threadIdx.x; g <= Gc; g += blockDim.x)
            cg[g] = g == Gc ? nx - 1 : guide_bin(pre, nx, (uint32_t)((unsigned long long)g << (32 - C.gc)), 0, nx - 1);
    }
    // the last row block: row marginal and row guide
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == (unsigned)ny - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int rper = (ny + blockDim.x - 1) / blockDim.x;
    const int r0 = threadIdx.x * rper;
    long long rl = 0;
    for (int r = r0; r < r0 + rper && r < ny; ++r) rl += __ldcg(row_tot + r);
    long long total;
    long long rrun = block_exclusive_scan(rl, &total);
    for (int r = r0; r < r0 + rper && r < ny; ++r) { C.row_pre[r] = rrun; rrun += __ldcg(row_tot + r); }
    if (threadIdx.x == 0) C.row_pre[ny] = total;
    __syncthreads();
    if (guides) {
        const int Gr = 1 << C.gr;
        for (int g = threadIdx.x; g <= Gr; g += blockDim.x)
            C.row_g[g] = g == Gr ? ny - 1 : guide_bin(C.row_pre, ny, (uint32_t)((unsigned long long)g << (32 - C.gr)), 0, ny - 1);
    }
    if (threadIdx.x == 0) {
        *done = 0u;   // ready for the next build
        if (prep) remap_prep_body(prep, n_hist, lead, w_lead);
    }
}

// block inclusive scan of a per-thread total (int64, exact); returns the exclusive prefix
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* total) {
    __shared__ long long sw[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) sw[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long x = lane < nw ? sw[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < nw) sw[lane] = x;
    }
    __syncthreads();
    const long long ex = (wid > 0 ? sw[wid - 1] : 0) + inc - v;
    *total = sw[nw - 1];
    __syncthreads();
    return ex;
}

// scratch: kCdfParts doubles of block partial sums (the first word then the rows' arrival
// counter), then ny int64 row totals
cudaError_t launch_cdf_build_raw(const double* cell_w, int nx, int ny, Cdf2DView cdf, double* W_out,
                                 double* qmax_out, double* scratch, cudaStream_t stream, bool pdl) {
    cudaError_t e = cudaMemsetAsync(qmax_out, 0, sizeof(double), stream);
    if (e != cudaSuccess) return e;
    double* part = scratch;
    long long* row_tot = (long long*)(scratch + kCdfParts);
    cdf_reduce_kernel<<<kCdfParts, 256, 0, stream>>>(cell_w, nx * ny, part, qmax_out);
    e = launch_pdl(pdl, cdf_total_kernel, dim3(1), dim3(32), 0, stream, part, (int)kCdfParts, W_out);
    if (e != cudaSuccess) return e;
    e = launch_pdl(pdl, cdf_rows_kernel, dim3(ny), dim3(256), 0, stream, cell_w, (const double*)qmax_out, nx, ny, cdf,
                   row_tot, reinterpret_cast<unsigned*>(part), (DevState*)nullptr, 0ll, 0ll, 0.0);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_cdf_build(hyb_problem* p, const double* cell_w, Cdf2DView cdf, double* W_out, double* qmax_out) {
    return launch_cdf_build_raw(cell_w, p->nx, p->ny, cdf, W_out, qmax_out, p->cell_scratch, p->stream, p->pdl);
}

// ---------------------------------------------------------------------------------------------
// remap density: f = (Q + sigma_s (phi_pre + phi_post) + sigma_s phi_c0, sigma_s phi_c1..3) for
// Eq. (R); (sigma_s phi_post + sigma_s phi_c0, sigma_s phi_c1..3) for Eq. (R') (relabel = 0)
// ---------------------------------------------------------------------------------------------
// pre_raw, post_raw: the leg's raw track-length sums (the step-average flux times A dt); the
// density is formed in separately rounded operations in the order of its definition, so the FP64
// remap follows the reference arithmetic bit for bit
// The remap density, its cells' weights q and the reduction the CDF build needs, in one launch of
// kCdfParts blocks: thread (b, t) takes cells b 256 + t + i kCdfParts 256 (cdf_reduce_kernel's
// partition, so sum |q| comes out in the same order, bit for bit), the blocks leave their
// partials (sum |q|, max |q|, max weight-factor bound) in scratch, and the last block to arrive
// forms remap_W, remap_qmax and remap_rmax (cdf_total_kernel's order for the sum) and zeroes the
// row kernel's arrival counter. The same launch zeroes the census pieces of pass A and, without a
// bank pre-pass, the remap counters.
__global__ void remap_density_cdf_kernel(int ncells, double adt, const double* __restrict__ Q,
                                         const double* __restrict__ ss, const double* __restrict__ pre_raw,
                                         const double* __restrict__ post_raw, const double* __restrict__ phi,
                                         double* f, float* f32, int* fpos, double* q, DevState* st, int relabel,
                                         double area, double dt, double* part, double* part_max, double* part_r,
                                         long long* blk, long long blk_words, int zero_counters) {
    pdl_wait();
    pdl_trigger();
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
    for (long long i = gt; i < blk_words; i += gs) blk[i] = 0;
    if (zero_counters) {
        unsigned long long* rc = reinterpret_cast<unsigned long long*>(&st->r_histories);
        const long long nw = (long long)(offsetof(DevState, n_bank) - offsetof(DevState, r_histories)) / 8;
        for (long long i = gt; i < nw; i += gs) rc[i] = 0ull;
    }
    double sq = 0, mq = 0, r = 0;
    for (long long kk = gt; kk < ncells; kk += gs) {
        const int k = (int)kk;
        const double s = ss[k];
        // Eq. (R): Q + sigma_s (T_pre + T_post) / (A dt) + sigma_s phi_c; Eq. (R'): sigma_s T_post / (A dt)
        // + sigma_s phi_c
        const double sphi = __dmul_rn(s, phi[4 * k]);
        const double f0 = relabel ? __dadd_rn(__dadd_rn(Q[k], __ddiv_rn(__dmul_rn(s, __dadd_rn(pre_raw[k], post_raw[k])), adt)), sphi)
                                  : __dadd_rn(__ddiv_rn(__dmul_rn(s, post_raw[k]), adt), sphi);
        const double f1 = s * phi[4 * k + 1], f2 = s * phi[4 * k + 2], f3 = s * phi[4 * k + 3];
        f[4 * k] = f0; f[4 * k + 1] = f1; f[4 * k + 2] = f2; f[4 * k + 3] = f3;
        reinterpret_cast<float4*>(f32)[k] = make_float4((float)f0, (float)f1, (float)f2, (float)f3);
        const double qc = __dmul_rn(__dmul_rn(f0, area), dt);   // (f0 A) dt
        q[k] = qc;
        // all four nodal values >= 0: births sampled from the bilinear density itself
        const bool pos = f0 - f1 - f2 + f3 >= 0 && f0 + f1 - f2 - f3 >= 0 && f0 - f1 + f2 - f3 >= 0 &&
                         f0 + f1 + f2 + f3 >= 0;
        fpos[k] = pos ? 1 : 0;
        if (qc != 0.0) r = fmax(r, pos ? 1.0 : (fabs(f0) + fabs(f1) + fabs(f2) + fabs(f3)) / fabs(f0));
        const double a = fabs(qc);
        sq += a;
        mq = fmax(mq, a);
    }
    sq = warp_sum(sq);
    for (int o = 16; o > 0; o >>= 1) {
        mq = fmax(mq, __shfl_down_sync(0xffffffffu, mq, o));
        r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    __shared__ double s_s[32], s_m[32], s_r[32];
    __shared__ bool s_last;
    if ((threadIdx.x & 31) == 0) { s_s[threadIdx.x >> 5] = sq; s_m[threadIdx.x >> 5] = mq; s_r[threadIdx.x >> 5] = r; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0, m = 0, rr = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += s_s[w]; m = fmax(m, s_m[w]); rr = fmax(rr, s_r[w]); }
        part[blockIdx.x] = t;
        part_max[blockIdx.x] = m;
        part_r[blockIdx.x] = rr;
        __threadfence();
        s_last = atomicAdd(&st->dens_done, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return;
    __threadfence();
    double t = 0, m = 0, rr = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) {
        t += __ldcg(part + i);
        m = fmax(m, __ldcg(part_max + i));
        rr = fmax(rr, __ldcg(part_r + i));
    }
    t = warp_sum(t);
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        rr = fmax(rr, __shfl_down_sync(0xffffffffu, rr, o));
    }
    if (threadIdx.x == 0) {
        st->remap_W = t;
        st->remap_qmax = m;
        st->remap_rmax = rr;
        *reinterpret_cast<unsigned*>(part) = 0u;   // the row kernel's arrival counter
        st->dens_done = 0u;
    }
}

__host__ __device__ inline double pow2_ceil(double w) {
    int e = 0;
    const double m = frexp(w, &e);
    return m == 0.5 ? w : ldexp(1.0, e);
}

// comb base w_ref and birth weight; runs after the CDF build. lead: the leg-census slots ahead of
// the births (steps 3'/4'), whose weights are bounded by the step-start bank's and by the leg's
// birth weight w_lead
// ---------------------------------------------------------------------------------------------
// remap streaming
// ---------------------------------------------------------------------------------------------
// shared-memory words of pass A's point tables (Sobol byte tables for its nbt birth dimensions, or
// nibble / Halton tables of ntab dimensions), ahead of the ntab digital shifts
__host__ __device__ __forceinline__ int remap_table_words(int ntab, int nbt) {
    return nbt ? nbt * kByteWords : ntab * kNibbleWords;
}

template <typename T>
struct RemapArgs {
    int nx, ny;
    T dx, dy, cdt, w_min;
    const T* sig;
    BankView<T> in, out, stg;   // stg: staged end states, one per slot (cell -1 = not alive)
    Cdf2DView cdf;
    const double* f;           // remap density, 4 Legendre coefficients per cell (FP64)
    const float* f32;          // the same in FP32 (FP32 path)
    const int* fpos;           // per cell: 1 if all four nodal values of f are >= 0
    long long n_hist, cap;
    const uint32_t* V;
    const uint32_t* bt;        // Sobol byte tables of the births' dimensions, or null
    int ntab, nbt, sampler;    // point-table dimensions; of them, dimensions with byte tables
    uint64_t seed;             // keys of the birth and comb point sets come from (seed, step)
    DevState* st;
    long long* blk;            // per block: alive count, sum q, sum|w| lo, sum|w| hi
    const unsigned long long* perm;   // census in cell order: (cell << 32 | slot) of every sorted position (else null)
    long long nslots;          // staging slots (bank capacity + n_hist); the sort covers all of them
    int perm_slots;            // 1: the census is sorted by cell after the count pass
    int lead_staged;           // 1 (steps 3'/4'): slots ahead of the births hold the MC leg's staged census
    int mode;                  // pass A: 0 every slot; 1 bank pre-pass (bank slots only, statistics at the
                               // bank's scale, no census partials); 2 after a bank pre-pass (bank slots staged)
    CellSplit split;           // cell index -> (ix, iy)
};

template <typename T>
struct Particle { int cell; T fx, fy, ox, oy, w; bool alive; };

// inverse CDF on [-1,1] of the density proportional to a + b s (a > 0, |b| <= a)
template <typename T>
__device__ __forceinline__ T inv_linear(T a, T b, T u) {
    using P = Prec<T>;
    if (!(a > T(0))) return T(2) * u - T(1);
    const T amb = a - b;
    // (a - b)^2 + 4 a b u with the products rounded apart on the FP64 path (a fused form on FP32)
    const T disc = P::madd(amb, amb, T(4) * a * b * u);
    const T t = T(4) * a * u / (amb + P::sqrt_(disc > T(0) ? disc : T(0)));
    return clamp_(t - T(1), T(-1), T(1));
}

// 2^k as a float for k in [-126, 126] (exact: the exponent field only)
__device__ __forceinline__ float pow2f(int k) {
    k = k < -126 ? -126 : (k > 126 ? 126 : k);
    return __int_as_float((k + 127) << 23);
}

// Per-thread weight sums of the remap statistics (start, absorbed, leaked, killed). FP64 path:
// doubles, scaled to 128-bit fixed point per block. FP32 path: int64 fixed point of scale 2^kf
// built from exact float products (kf = the block scale - 64, capped at 126), so the per-slot
// bookkeeping needs no FP64 arithmetic; a block sum v stands for v 2^(k - kf) at the block scale.
template <typename T> struct RemapSums;
template <> struct RemapSums<double> {
    double v[4] = {0, 0, 0, 0};
    __device__ void init(int) {}
    __device__ void add(int i, double x) { v[i] += x; }
};
template <> struct RemapSums<float> {
    long long v[4] = {0, 0, 0, 0};
    float sc = 1.f;
    __device__ void init(int kf) { sc = pow2f(kf); }
    __device__ void add(int i, float x) { v[i] += f2ll_rn(x * sc); }
};
enum { kRsSrc = 0, kRsAbs = 1, kRsLeak = 2, kRsKill = 3 };

// start state of slot j and its straight-line stream to t_{n+1} with sigma_t attenuation. Without
// scattering the weight removed along the stream telescopes, sum_s w_s (1 - e_s) = w_0 - w_end, so
// the absorbed-weight statistic is added once per slot (its fixed-point conversion is ~15 integer
// instructions on the FP32 path) rather than once per segment.
template <typename T, typename Pts>
__device__ Particle<T> remap_slot(const RemapArgs<T>& a, const Pts& pts, long long j, long long nb, T wbar,
                                  RemapSums<T>& sums, int* leaked, int* killed, int* segs, int* err) {
    using P = Prec<T>;
    int ix, iy;
    T fx, fy, ox, oy, w, srem;
    if (j < nb) {
        const int k = a.in.cell[j];
        a.split(k, &ix, &iy);
        fx = a.in.fx[j]; fy = a.in.fy[j]; ox = a.in.ox[j]; oy = a.in.oy[j]; w = a.in.w[j];
        srem = a.cdt;
    } else {
        const uint32_t i = (uint32_t)(j - nb);
        T frx, fry;
        const int k = sample_cell<T>(a.cdf, a.nx, a.ny, pts(i, 0), pts(i, 1), &frx, &fry);
        a.split(k, &ix, &iy);
        T f0, f1, f2, f3;
        if constexpr (sizeof(T) == 4) {
            const float4 fk = __ldg(reinterpret_cast<const float4*>(a.f32) + k);
            f0 = fk.x; f1 = fk.y; f2 = fk.z; f3 = fk.w;
        } else {
            const double* fk = a.f + 4 * (size_t)k;
            f0 = fk[0]; f1 = fk[1]; f2 = fk[2]; f3 = fk[3];
        }
        T xi, eta;
        if (a.fpos[k]) {
            xi = inv_linear<T>(f0, f1, frx);
            eta = inv_linear<T>(P::madd(f1, xi, f0), P::madd(f3, xi, f2), fry);
            w = wbar;
        } else {
            xi = T(2) * frx - T(1);
            eta = T(2) * fry - T(1);
            // f(xi, eta) = ((f0 + f1 xi) + f2 eta) + (f3 xi) eta, products rounded apart on FP64
            w = wbar * P::madd(f3 * xi, eta, P::madd(f2, eta, P::madd(f1, xi, f0))) / (f0 < T(0) ? -f0 : f0);
        }
        fx = T(0.5) * (xi + T(1)) * a.dx;
        fy = T(0.5) * (eta + T(1)) * a.dy;
        iso_dir<T>(pts(i, 3), pts(i, 4), &ox, &oy);
        srem = a.cdt * P::unit_c(pts(i, 2));
    }
    sums.add(kRsSrc, w);
    const T w0 = w;
    const T INF = (T)INFINITY;
    constexpr bool kF32 = sizeof(T) == 4;
    // FP32: face distances from the flight's reciprocals (FP64: divisions, as the oracle)
    const T rox = kF32 ? P::rcp(ox) : T(0), roy = kF32 ? P::rcp(oy) : T(0);
    Particle<T> r;
    r.alive = false;
    r.cell = iy * a.nx + ix;
    int s = 0;
    while (s < (int)kMaxSegments) {
        ++s;
        const int k = iy * a.nx + ix;
        const T st = a.sig[2 * k] + a.sig[2 * k + 1];
        T dxf, dyf;
        if constexpr (kF32) {
            dxf = ox > T(0) ? (a.dx - fx) * rox : (ox < T(0) ? fx * (-rox) : INF);
            dyf = oy > T(0) ? (a.dy - fy) * roy : (oy < T(0) ? fy * (-roy) : INF);
        } else {
            dxf = ox > T(0) ? (a.dx - fx) / ox : (ox < T(0) ? fx / (-ox) : INF);
            dyf = oy > T(0) ? (a.dy - fy) / oy : (oy < T(0) ? fy / (-oy) : INF);
        }
        T l;
        bool face = false, xc = false, yc = false;
        if (dxf <= srem || dyf <= srem) { l = dxf < dyf ? dxf : dyf; face = true; xc = dxf == l; yc = dyf == l; }
        else l = srem;
        T att, e;
        P::att_e(st * l, &att, &e);
        w = w * e;
        fx = P::madd(ox, l, fx);
        fy = P::madd(oy, l, fy);
        srem = srem - l;
        if (!face) {
            r.cell = k;
            r.fx = clamp_(fx, T(0), a.dx); r.fy = clamp_(fy, T(0), a.dy);
            r.ox = ox; r.oy = oy; r.w = w; r.alive = true;
            sums.add(kRsAbs, w0 - w);
            *segs += s;
            return r;
        }
        if (xc) { ix += ox > T(0) ? 1 : -1; fx = ox > T(0) ? T(0) : a.dx; } else fx = clamp_(fx, T(0), a.dx);
        if (yc) { iy += oy > T(0) ? 1 : -1; fy = oy > T(0) ? T(0) : a.dy; } else fy = clamp_(fy, T(0), a.dy);
        if (ix < 0 || ix >= a.nx || iy < 0 || iy >= a.ny) {
            sums.add(kRsAbs, w0 - w); sums.add(kRsLeak, w); ++*leaked; *segs += s; return r;
        }
        const T aw = w < T(0) ? -w : w, aw0 = w0 < T(0) ? -w0 : w0;
        if (a.w_min > T(0) && aw < a.w_min * aw0) {
            sums.add(kRsAbs, w0 - w); sums.add(kRsKill, w); ++*killed; *segs += s; return r;
        }
    }
    ++*err;
    sums.add(kRsAbs, w0 - w);
    *segs += s;
    return r;
}

// comb quantisation rint(|w| / w_ref 2^32) with w_ref a power of two: the FP32 path multiplies by
// the exact float 2^(32 - log2 w_ref) (same integer as the FP64 quotient), the FP64 path divides
__device__ __forceinline__ long long quant_w(float w, double, float qsc) { return f2ll_rn(fabsf(w) * qsc); }
__device__ __forceinline__ long long quant_w(double w, double w_ref, float) {
    return __double2ll_rn((fabs(w) / w_ref) * 0x1p32);
}

// float 2^(32 - log2 w_ref), or 0 when it is not a normal float (the FP32 path then divides)
__device__ __forceinline__ float quant_scale(double w_ref) {
    const int e = ilogb(w_ref);
    return (32 - e) <= 126 && (32 - e) >= -126 ? pow2f(32 - e) : 0.f;
}

template <typename T>
__device__ __forceinline__ long long quant(T w, double w_ref, float qsc) {
    if (sizeof(T) == 4 && qsc == 0.f) return quant_w((double)w, w_ref, 0.f);
    return quant_w(w, w_ref, qsc);
}

// The per-step scalars of the remap passes (RemapScal), formed once per step (remap_prep_body, in
// the last block of the remap CDF's row kernel).
__device__ __forceinline__ RemapScal remap_scalars(const DevState* st, long long n_hist) {
    RemapScal r;
    const long long nb = st->n_bank + st->r_lead;
    const long long nbirth = st->remap_W > 0 ? n_hist : 0;
    r.N = nb + nbirth;
    r.wbar = nbirth ? st->remap_W / (double)n_hist : 0.0;
    r.w_ref = st->w_ref;
    r.qsc = quant_scale(r.w_ref);
    r.krw = scale_exponent((double)(r.N > 0 ? r.N : 1) * r.w_ref, 125);
    r.kw = scale_exponent((double)(r.N > 0 ? r.N : 1) * fmax(r.w_ref, 1e-300) * 4.0, 125);
    r.kfa = min(r.krw - 64, 126);
    r.kf = min(r.kw - 64, 126);
    r.sca = pow2f(r.kfa);
    return r;
}

// one thread: the comb's quantisation base and the remap passes' scalars of this step
__device__ void remap_prep_body(DevState* st, long long n_hist, long long lead, double w_lead) {
    const double W = st->remap_W;
    const double wbar = W > 0 ? W / (double)n_hist : 0.0;
    st->r_lead = lead;
    double wmax = fmax(fmax(st->bank_wmax, w_lead), wbar * st->remap_rmax);
    st->w_ref = wmax > 0 ? pow2_ceil(wmax) : 1.0;
    st->rs = remap_scalars(st, n_hist);
}

// one thread: the scalars of the bank pre-pass, from the step-start bank alone (n_bank slots, the
// power of two at or above its max |w| as the statistics' base)
__global__ void remap_bank_prep_kernel(DevState* st) {
    RemapScal r;
    const long long nb = st->n_bank;
    r.N = nb;
    r.wbar = 0.0;
    r.w_ref = st->bank_wmax > 0 ? pow2_ceil(st->bank_wmax) : 1.0;
    r.qsc = quant_scale(r.w_ref);
    r.krw = scale_exponent((double)(nb > 0 ? nb : 1) * r.w_ref, 125);
    r.kw = scale_exponent((double)(nb > 0 ? nb : 1) * r.w_ref * 4.0, 125);
    r.kfa = min(r.krw - 64, 126);
    r.kf = min(r.kw - 64, 126);
    r.sca = pow2f(r.kfa);
    st->rsb = r;
}

// Block sum of v (one value per thread) in a fixed order (warp trees, then the warps in order);
// the result is valid in thread 0. Ends with the block synchronised (s may be reused after it).
template <typename V>
__device__ __forceinline__ V block_sum_fixed(V v, V* s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    V t = V(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < kTile / 32; ++w) t += s[w];
    __syncthreads();
    return t;
}

// 128-bit fixed point of a block's FP64 |w| sum (scale 2^k) or of an FP32 int64 sum at per-thread
// scale 2^kt (k - kt >= 64: the value shifted left by k - kt - 64 in the high word)
__device__ __forceinline__ void fixed128(double d, long long f, bool f32, int k, int kt, unsigned long long* lo,
                                         unsigned long long* hi) {
    if (f32) {
        const int sh = k - kt - 64;
        *lo = 0ull;
        *hi = sh < 63 ? (unsigned long long)f << sh : 0ull;   // two's complement: signed sums too
    } else {
        to_i128(d * ldexp(1.0, k), lo, hi);
    }
}

// Pass A. Slots are taken in rounds of 32 (one slot per lane of a warp), dealt to the warps of
// a persistent grid in a fixed interleave: warp g takes rounds g, g + W, g + 2W, ... of the order
// births first, then the slots ahead of them (a birth costs several times a staged or re-streamed
// bank slot). Every warp so ends within one round of the others, where a block per 2048 slots
// left a second, nearly empty wave of latency-bound birth blocks behind the first. Each round adds
// its census partials (alive count, quantised |w|, fixed-point |w|) to the piece of kPartSlots
// slots it belongs to (blk zeroed beforehand; integer additions, so the order does not matter).
// The bank pre-pass (mode 1) takes the bank slots' rounds and adds no partials. The rounds of a
// thread are fixed, so its weight sums (FP32 int64, FP64 doubles, summed per block in a fixed
// order at the end) are reproducible run to run.
template <typename T>
__global__ void __launch_bounds__(kTile, sizeof(T) == 4 ? 3 : 2) remap_count_kernel(RemapArgs<T> a) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* sV = sm;
    uint32_t* sSh = sm + remap_table_words(a.ntab, a.nbt);
    const bool prepass = a.mode == 1;
    // the bank pre-pass runs before the remap density exists: bank slots only (no step-start
    // r_lead slots there), scales from the bank alone
    const long long nb = prepass ? a.st->n_bank : a.st->n_bank + a.st->r_lead;   // slots ahead of the births
    const long long nrounds = prepass ? (nb + 31) / 32 : (a.nslots + 31) / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long gwarp = (long long)blockIdx.x * (kTile / 32) + wid, nwarps = (long long)gridDim.x * (kTile / 32);
    const uint64_t key = dstream_key(a.seed, (uint64_t)a.st->step, HYB_STREAM_REMAP_SOURCE);
    if (!prepass) {
        if (a.nbt) copy_byte_tables(a.bt, a.nbt, sV);
        else build_point_tables(a.V, a.ntab, sV, a.sampler);
        for (int d = threadIdx.x; d < a.ntab; d += blockDim.x) sSh[d] = dshift(key, (uint64_t)d);
    }
    __shared__ RemapScal s_rs;
    __shared__ long long s_red[kTile / 32];
    __shared__ double s_redd[kTile / 32];
    if (threadIdx.x == 0) s_rs = prepass ? a.st->rsb : a.st->rs;
    __syncthreads();
    const PointsB pts{sV, a.nbt, Points{sV, sSh, key, a.sampler, a.ntab}};
    const bool staged = a.lead_staged != 0 || a.mode == 2;   // slots below nb hold end states already
    const long long N = prepass ? nb : s_rs.N;
    const T wbar_t = (T)s_rs.wbar;
    const double w_ref = s_rs.w_ref;
    const float qsc = s_rs.qsc;
    // scales (128-bit): krw for the survivors' sum |w|, kw for the statistics
    const int krw = s_rs.krw, kw = s_rs.kw;
    constexpr bool kF32 = sizeof(T) == 4;
    const int kfa = s_rs.kfa, kf = s_rs.kf;   // FP32 per-thread scales
    const float sca = s_rs.sca;
    Acc128* wd[4] = {&a.st->r_w_source, &a.st->r_w_absorbed, &a.st->r_w_leaked, &a.st->r_w_killed};
    if (prepass) { wd[0] = &a.st->r_wb[0]; wd[1] = &a.st->r_wb[1]; wd[2] = &a.st->r_wb[2]; wd[3] = &a.st->r_wb[3]; }
    RemapSums<T> sums;
    sums.init(kf);
    int leaked = 0, killed = 0, segs = 0, err = 0;
    const long long first_birth = prepass ? 0 : nb / 32;   // births-first order of the rounds
    for (long long rr = gwarp; rr < nrounds; rr += nwarps) {
        const long long round = prepass ? rr : (rr + first_birth < nrounds ? rr + first_birth : rr + first_birth - nrounds);
        const long long j = round * 32 + lane;
        long long cnt = 0, qs = 0, wsf = 0;
        double ws = 0;
        if (j < N) {
            Particle<T> pr;
            if (staged && j < nb) {
                // steps 3'/4': the MC leg staged its census here; it enters the census as it is. After
                // a bank pre-pass: the bank particle's end state, staged (and counted) by the pre-pass
                pr.cell = a.stg.cell[j];
                pr.alive = pr.cell >= 0;
                pr.w = pr.alive ? a.stg.w[j] : T(0);
            } else {
                pr = remap_slot<T, PointsB>(a, pts, j, nb, wbar_t, sums, &leaked, &killed, &segs, &err);
                a.stg.cell[j] = pr.alive ? pr.cell : -1;
                a.stg.fx[j] = pr.fx; a.stg.fy[j] = pr.fy; a.stg.ox[j] = pr.ox; a.stg.oy[j] = pr.oy; a.stg.w[j] = pr.w;
            }
            if (pr.alive) {
                cnt = 1;
                qs = quant<T>(pr.w, w_ref, qsc);
                if constexpr (kF32) wsf = f2ll_rn(fabsf(pr.w) * sca);
                else ws = fabs((double)pr.w);
            }
        } else if (!prepass && a.perm_slots && j < a.nslots) {
            a.stg.cell[j] = -1;   // unused slots sort last, as dead
        }
        if (!prepass) {
            // the round's census partials into its piece (warp trees: a fixed order per round)
            cnt = (long long)__popc(__ballot_sync(0xffffffffu, cnt != 0));
            if (cnt) {
                qs = (long long)warp_sum_u64((unsigned long long)qs);
                if constexpr (kF32) wsf = (long long)warp_sum_u64((unsigned long long)wsf);
                else ws = warp_sum(ws);
                if (lane == 0) {
                    unsigned long long lo, hi;
                    fixed128(ws, wsf, kF32, krw, kfa, &lo, &hi);
                    long long* b = a.blk + 4 * (size_t)(round / (kPartSlots / 32));
                    atomicAdd((unsigned long long*)b, (unsigned long long)cnt);
                    if (qs) atomicAdd((unsigned long long*)(b + 1), (unsigned long long)qs);
                    atomic_add128(reinterpret_cast<Acc128*>(b + 2), lo, hi);
                }
            }
        }
    }
    if constexpr (!kF32) {
        // FP64 weight statistics: a fixed-order block sum, then 128-bit fixed point
        for (int t = 0; t < 4; ++t) {
            const double v = block_sum_fixed(sums.v[t], s_redd);
            if (threadIdx.x == 0) {
                unsigned long long lo, hi;
                to_i128(v * ldexp(1.0, kw), &lo, &hi);
                if (lo | hi) atomic_add128(wd[t], lo, hi);
            }
        }
    }
    // counters and the FP32 weight statistics, once per block
    const long long il = block_sum_fixed((long long)leaked, s_red);
    const long long ik = block_sum_fixed((long long)killed, s_red);
    const long long is = block_sum_fixed((long long)segs, s_red);
    const long long ie = block_sum_fixed((long long)err, s_red);
    long long fv[4] = {0, 0, 0, 0};
    if constexpr (kF32)
        for (int t = 0; t < 4; ++t) fv[t] = block_sum_fixed((long long)sums.v[t], s_red);
    if (threadIdx.x == 0) {
        if constexpr (kF32) {
            for (int t = 0; t < 4; ++t) {
                unsigned long long lo, hi;
                fixed128(0.0, fv[t], true, kw, kf, &lo, &hi);
                if (lo | hi) atomic_add128(wd[t], lo, hi);
            }
        }
        if (il) atomicAdd(&a.st->r_leaked, (unsigned long long)il);
        if (ik) atomicAdd(&a.st->r_killed, (unsigned long long)ik);
        if (is) atomicAdd(&a.st->r_segments, (unsigned long long)is);
        if (ie) { atomicAdd(&a.st->r_errors, (unsigned long long)ie); atomicOr(&a.st->status, kStSegments); }
        if (blockIdx.x == 0) {
            if (prepass) a.st->k_rwb = kw;
            else { a.st->k_rw = kw; a.st->r_histories = (unsigned long long)(N - a.st->r_lead); }
            // a pre-pass error flag may have been cleared with the status word since
            if (a.mode == 2 && a.st->r_errors) atomicOr(&a.st->status, kStSegments);
        }
    }
}

// The per-piece partials (alive count, quantised |w| sum, fixed-point |w| sum) of the staged end
// states in census order (sorted positions, or slots when perm is null), one block per piece. For a cell-ordered
// remap census they replace the slot-order partials of the count pass (the totals are the same
// integers in any order); for N_s = infinity they are the only partials.
template <typename T>
__global__ void __launch_bounds__(kTile) remap_partials_kernel(RemapArgs<T> a) {
    __shared__ RemapScal s_rs;
    if (threadIdx.x == 0) s_rs = a.st->rs;
    __syncthreads();
    const long long N = s_rs.N;
    const double w_ref = s_rs.w_ref;
    const float qsc = s_rs.qsc;
    const int krw = s_rs.krw;
    const int kfa = s_rs.kfa;
    const float sca = s_rs.sca;
    constexpr bool kF32 = sizeof(T) == 4;
    long long cnt = 0, qs = 0, wsf = 0;
    double ws = 0;
    const long long base = (long long)blockIdx.x * kPartSlots;
    for (int r = 0; r < kPartSlots / kTile; ++r) {
        const long long j = base + r * kTile + threadIdx.x;
        if (j >= N) break;
        const long long js = a.perm ? (long long)(uint32_t)a.perm[j] : j;
        if (a.stg.cell[js] < 0) continue;
        const T w = a.stg.w[js];
        ++cnt;
        qs += quant<T>(w, w_ref, qsc);
        if constexpr (kF32) wsf += f2ll_rn(fabsf(w) * sca);
        else ws += fabs((double)w);
    }
    __shared__ long long s_l[kTile / 32][3];
    __shared__ double s_d[kTile / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        qs += __shfl_down_sync(0xffffffffu, qs, o);
        wsf += __shfl_down_sync(0xffffffffu, wsf, o);
    }
    if constexpr (!kF32) ws = warp_sum(ws);
    if (lane == 0) { s_l[wid][0] = cnt; s_l[wid][1] = qs; s_l[wid][2] = wsf; s_d[wid] = ws; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long c = 0, q = 0, af = 0;
        double d = 0;
        for (int ww = 0; ww < kTile / 32; ++ww) { c += s_l[ww][0]; q += s_l[ww][1]; af += s_l[ww][2]; d += s_d[ww]; }
        unsigned long long lo, hi;
        if constexpr (kF32) {
            const int sh = krw - kfa - 64;
            lo = 0ull;
            hi = sh < 63 ? (unsigned long long)af << sh : 0ull;
        } else {
            to_i128(d * ldexp(1.0, krw), &lo, &hi);
        }
        long long* b = a.blk + 4 * (size_t)blockIdx.x;
        b[0] = c; b[1] = q; b[2] = (long long)lo; b[3] = (long long)hi;
    }
}

// ---------------------------------------------------------------------------------------------
// census in phase-space order (census_order 2): key = cell above a Morton interleave of b bits
// each of the in-cell x, y and the direction's diamond angle d in [0, 4) (monotone in the polar
// angle: one division, no arctangent); dead slots get -1 (sorted last). The FP64 path forms the
// key with the same operations, in the same order, as the oracle.
// ---------------------------------------------------------------------------------------------
int phase_key_bits(int ncells, int* cell_bits) {
    int cb = 0;
    while (((long long)1 << cb) < ncells) ++cb;
    *cell_bits = cb;
    const int b = (31 - cb) / 3;
    return b < 0 ? 0 : (b > 5 ? 5 : b);
}

// keys below 2^(cell bits + 3b) <= 2^31 (phase space) or below the cell count: that bound is the
// sentinel of dead slots
uint32_t census_sort_sentinel(int census_order, int ncells) {
    if (census_order != 2) return (uint32_t)ncells;
    int cb = 0;
    const int b = phase_key_bits(ncells, &cb);
    return (uint32_t)1u << (cb + 3 * b);
}

template <typename T>
__device__ __forceinline__ uint32_t phase_quant(T v, T s) {
    T t = floor(v * s);
    t = t < T(0) ? T(0) : (t > s - T(1) ? s - T(1) : t);
    return (uint32_t)t;
}

template <typename T>
__global__ void phase_key_kernel(BankView<T> stg, long long nslots, T dx, T dy, int b, int32_t* key) {
    const T s = (T)(1u << b);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nslots; j += (long long)gridDim.x * blockDim.x) {
        const int c = stg.cell[j];
        if (c < 0) { key[j] = -1; continue; }
        const T ox = stg.ox[j], oy = stg.oy[j];
        T d;
        if (ox == T(0) && oy == T(0)) d = T(0);
        else if (oy >= T(0)) d = ox >= T(0) ? oy / (ox + oy) : T(1) + (-ox) / (oy - ox);
        else d = ox < T(0) ? T(2) + (-oy) / (-ox - oy) : T(3) + ox / (ox - oy);
        const uint32_t qx = phase_quant<T>(stg.fx[j] / dx, s), qy = phase_quant<T>(stg.fy[j] / dy, s);
        const uint32_t qa = phase_quant<T>(d * T(0.25), s);
        uint32_t sub = 0;
        for (int i = 0; i < b; ++i)
            sub |= (((qx >> i) & 1u) << (3 * i)) | (((qy >> i) & 1u) << (3 * i + 1)) | (((qa >> i) & 1u) << (3 * i + 2));
        key[j] = (int32_t)(((uint32_t)c << (3 * b)) | sub);
    }
}

// The sort of the census (cell order, or phase-space order with its keys formed first) over the n
// staging slots; *perm: the sorted (key << 32 | slot) pairs.
// polls of one look-back wait of the census sort (the problem's device wait bound)
static int sort_wait_limit(const hyb_problem* p) { return p->d.wait_limit > 0 ? p->d.wait_limit : (1 << 22); }

template <typename T>
static cudaError_t sort_census(hyb_problem* p, const BankView<T>& stg, long long n, cudaStream_t s,
                               const unsigned long long** perm) {
    unsigned long long* const pairs[2] = {p->sort_pairs[0], p->sort_pairs[1]};
    if (p->d.census_order == 2) {
        int cb = 0;
        const int b = phase_key_bits(p->ncells, &cb);
        const long long g = (n + 255) / 256;
        phase_key_kernel<T><<<(unsigned)(g < 152 * 8 ? g : 152 * 8), 256, 0, s>>>(stg, n, (T)p->dx, (T)p->dy, b,
                                                                                 p->sort_keys);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_census_sort(p->d.census_order == 2 ? p->sort_keys : stg.cell, n,
                              census_sort_sentinel(p->d.census_order, p->ncells), pairs, p->sort_scratch,
                              sort_wait_limit(p), &p->st->status, s, perm);
}

// One block: exclusive scan of the pieces' alive counts and quantised sums in place (tiles of
// blockDim.x consecutive pieces, one per thread, so that every load and store is coalesced; the
// running totals carry from tile to tile), the 128-bit |w| total, and the comb decision.
__global__ void remap_scan_kernel(long long* blk, int nblk, DevState* st, long long cap, uint64_t seed, int sampler,
                                  long long n_hist) {
    pdl_wait();
    pdl_trigger();
    const uint32_t x_off = first_point(dstream_key(seed, (uint64_t)st->step, HYB_STREAM_REMAP_COMB), sampler);
    __shared__ unsigned long long slo[32], shi[32];
    const int t = threadIdx.x, nt = blockDim.x;
    long long run_c = 0, run_q = 0;          // totals of the tiles before (the same in every thread)
    unsigned long long lo = 0, hi = 0;       // this thread's share of the 128-bit |w| total
    for (int t0 = 0; t0 < nblk; t0 += nt) {
        const int b = t0 + t;
        long long c = 0, q = 0;
        if (b < nblk) {
            const longlong4_32a v = *reinterpret_cast<const longlong4_32a*>(blk + 4 * (size_t)b);
            c = v.x; q = v.y;
            const unsigned long long l = (unsigned long long)v.z, h = (unsigned long long)v.w;
            const unsigned long long nl = lo + l;
            hi += h + (nl < lo ? 1ull : 0ull);
            lo = nl;
        }
        long long tc, tq;
        const long long exc = block_exclusive_scan(c, &tc);
        const long long exq = block_exclusive_scan(q, &tq);
        if (b < nblk) { blk[4 * (size_t)b] = run_c + exc; blk[4 * (size_t)b + 1] = run_q + exq; }
        run_c += tc;
        run_q += tq;
    }
    // the 128-bit sum of |w|: a shuffle tree per warp, then the warp sums (exact modular integer
    // additions, so the order does not matter)
    {
        unsigned long long wl = lo, wh = hi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long l2 = __shfl_down_sync(0xffffffffu, wl, o), h2 = __shfl_down_sync(0xffffffffu, wh, o);
            const unsigned long long nl = wl + l2;
            wh += h2 + (nl < wl ? 1ull : 0ull);
            wl = nl;
        }
        if ((t & 31) == 0) { slo[t >> 5] = wl; shi[t >> 5] = wh; }
    }
    __syncthreads();
    if (t == 0) {
        unsigned long long al = 0, ah = 0;
        for (int u = 0; u < (nt + 31) / 32; ++u) {
            const unsigned long long nl = al + slo[u];
            ah += shi[u] + (nl < al ? 1ull : 0ull);
            al = nl;
        }
        const long long ac = run_c, aq = run_q;
        const long long nb = st->n_bank + st->r_lead;
        const long long nbirth = st->remap_W > 0 ? n_hist : 0;
        const long long N = nb + nbirth;
        const int krw = scale_exponent((double)(N > 0 ? N : 1) * st->w_ref, 125);
        const double wsum = acc128_to_double(al, ah, ldexp(1.0, -krw));
        st->comb_total_alive = ac;
        st->comb_T = aq;
        const int comb = ac > cap ? 1 : 0;
        st->comb_on = comb;
        const unsigned long long ua = (unsigned long long)aq, ux = (unsigned long long)x_off;
        st->comb_o = (long long)((__umul64hi(ux, ua) << 32) | ((ux * ua) >> 32));
        st->wcopy = comb ? wsum / (double)cap : 0.0;
        // a comb needs a positive quantised total; otherwise every survivor is below the
        // quantum 2^-33 w_ref and the census is empty
        st->out_count = comb ? (aq > 0 ? cap : 0) : ac;
        st->r_alive = (unsigned long long)ac;
        st->bank_wsum = wsum;
        st->bank_wmax = comb ? st->wcopy : 0.0;   // non-comb: max gathered in pass B
    }
}

// ceil(num / T) for num = hi 2^64 + lo >= 0 with quotient < 2^40, 0 < T < 2^63, without FP64: a
// float estimate (relative error below 2^-21) is refined once from the exact 128-bit remainder
// (leaving an error of at most one) and finished by exact integer steps.
__device__ __forceinline__ long long ceil_div(unsigned long long hi, unsigned long long lo, unsigned long long T) {
    const float fT = u64_to_f(T);
    const float fN = fmaf(u64_to_f(hi), 0x1p64f, u64_to_f(lo));
    long long q = f2ll_rn(fN / fT);
    if (q < 0) q = 0;
    {
        const unsigned long long plo = (unsigned long long)q * T, phi = __umul64hi((unsigned long long)q, T);
        unsigned long long rlo = lo - plo;
        unsigned long long rhi = hi - phi - (lo < plo ? 1ull : 0ull);
        const bool neg = (long long)rhi < 0;
        if (neg) {                       // |r| of the two's-complement remainder
            rlo = ~rlo + 1ull;
            rhi = ~rhi + (rlo == 0ull ? 1ull : 0ull);
        }
        const float fr = fmaf(u64_to_f(rhi), 0x1p64f, u64_to_f(rlo));
        const long long dq = f2ll_rn(fr / fT);
        q = neg ? q - dq : q + dq;
        if (q < 0) q = 0;
    }
    for (int it = 0; it < 16; ++it) {
        // prod = q T
        const unsigned long long plo = (unsigned long long)q * T, phi = __umul64hi((unsigned long long)q, T);
        const bool gt = phi > hi || (phi == hi && plo > lo);
        if (gt) { --q; continue; }
        // rem = num - prod >= 0; if rem >= T then q++
        const unsigned long long rlo = lo - plo;
        const unsigned long long rhi = hi - phi - (lo < plo ? 1ull : 0ull);
        if (rhi > 0 || rlo >= T) { ++q; continue; }
        return (rhi == 0 && rlo == 0) ? q : q + 1;
    }
    return q;
}

// first tooth index at or after cumulative weight S: ceil((S M - o) / T), 0 if S M <= o
__device__ __forceinline__ long long first_tooth(long long S, long long M, long long o, long long T) {
    unsigned long long lo = (unsigned long long)S * (unsigned long long)M;
    unsigned long long hi = __umul64hi((unsigned long long)S, (unsigned long long)M);
    const unsigned long long uo = (unsigned long long)o;
    if (hi == 0 && lo <= uo) return 0;
    const unsigned long long nlo = lo - uo;
    hi -= (lo < uo ? 1ull : 0ull);
    return ceil_div(hi, nlo, (unsigned long long)T);
}

// block exclusive scan of a (count, sum) pair per thread; totals in *tc, *tq
__device__ __forceinline__ void block_exclusive_scan2(long long c, long long q, long long* ec, long long* eq,
                                                      long long* tc, long long* tq) {
    __shared__ long long s2c[kTile / 32], s2q[kTile / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long ic = c, iq = q;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long vc = __shfl_up_sync(0xffffffffu, ic, off), vq = __shfl_up_sync(0xffffffffu, iq, off);
        if (lane >= off) { ic += vc; iq += vq; }
    }
    if (lane == 31) { s2c[wid] = ic; s2q[wid] = iq; }
    __syncthreads();
    long long wc = 0, wq = 0, ac = 0, aq = 0;
#pragma unroll
    for (int ww = 0; ww < kTile / 32; ++ww) {
        if (ww < wid) { wc += s2c[ww]; wq += s2q[ww]; }
        ac += s2c[ww]; aq += s2q[ww];
    }
    *ec = wc + ic - c; *eq = wq + iq - q;
    *tc = ac; *tq = aq;
}

// teeth of a position whose q M - ph exceeds T or 64 bits (a weight far above the mean tooth
// spacing): the exact 128-bit form, kept out of line
__device__ __noinline__ long long comb_teeth_wide(long long S, long long q, long long M, long long o, long long T,
                                                 long long t, unsigned long long ph) {
    const unsigned long long uq = (unsigned long long)q, uM = (unsigned long long)M;
    if (__umul64hi(uq, uM) != 0ull) return first_tooth(S + q, M, o, T) - t;
    return ceil_div(0ull, uq * uM - ph, (unsigned long long)T);
}

// Pass B. Thread i of block b takes the kRounds consecutive census positions starting at
// b kSlotsPerBlock + i kRounds (census order: slot order, or the sorted order of perm).
// Comb: position j with cumulative quantised weight S_j before it and q_j of its own takes the
// teeth t in [first_tooth(S_j), first_tooth(S_j + q_j)), tooth t standing at t T + o on the axis
// S M. With the phase ph = t T + o - S M of the next tooth t (in [0, T)), position j takes
// n = ceil((q_j M - ph) / T) teeth when q_j M > ph and none otherwise, so a thread divides 128-bit
// numbers once (its first tooth) and advances t by 64-bit comparisons: the same teeth as a
// first_tooth per position.
template <typename T>
__global__ void __launch_bounds__(kTile) remap_write_kernel(RemapArgs<T> a) {
    pdl_wait();
    pdl_trigger();
    __shared__ RemapScal s_rs;
    if (threadIdx.x == 0) s_rs = a.st->rs;
    __syncthreads();
    const long long N = s_rs.N;
    const double w_ref = s_rs.w_ref;
    const float qsc = s_rs.qsc;
    const int comb = a.st->comb_on;
    const long long M = a.cap, o = a.st->comb_o, Ttot = a.st->comb_T;
    const T wcopy = (T)a.st->wcopy;
    const bool combing = comb && Ttot > 0;
    const long long j0 = (long long)blockIdx.x * kSlotsPerBlock + (long long)threadIdx.x * kRounds;
    int cell[kRounds];
    T w[kRounds];
    if (!a.perm && j0 + kRounds <= N) {
        // slot order, all kRounds positions in range: 16-byte loads (the stage arrays start on
        // 16-byte boundaries and j0 is a multiple of kRounds)
        const int4* pc = reinterpret_cast<const int4*>(a.stg.cell + j0);
#pragma unroll
        for (int v = 0; v < kRounds / 4; ++v) {
            const int4 c4 = pc[v];
            cell[4 * v] = c4.x; cell[4 * v + 1] = c4.y; cell[4 * v + 2] = c4.z; cell[4 * v + 3] = c4.w;
        }
        if constexpr (sizeof(T) == 4) {
            const float4* pw = reinterpret_cast<const float4*>(a.stg.w + j0);
#pragma unroll
            for (int v = 0; v < kRounds / 4; ++v) {
                const float4 w4 = pw[v];
                w[4 * v] = w4.x; w[4 * v + 1] = w4.y; w[4 * v + 2] = w4.z; w[4 * v + 3] = w4.w;
            }
        } else {
            const double2* pw = reinterpret_cast<const double2*>(a.stg.w + j0);
#pragma unroll
            for (int v = 0; v < kRounds / 2; ++v) {
                const double2 w2 = pw[v];
                w[2 * v] = w2.x; w[2 * v + 1] = w2.y;
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const long long j = j0 + r;
            cell[r] = -1;
            w[r] = T(0);
            if (j < N) {
                const long long js = a.perm ? (long long)(uint32_t)a.perm[j] : j;
                cell[r] = a.stg.cell[js];
                w[r] = a.stg.w[js];
            }
        }
    }
    long long q[kRounds];
    long long c = 0, qt = 0;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const bool alive = cell[r] >= 0;
        q[r] = alive ? quant<T>(w[r], w_ref, qsc) : 0;
        c += alive ? 1 : 0;
        qt += q[r];
    }
    long long ec, eq, tc, tq;
    block_exclusive_scan2(c, qt, &ec, &eq, &tc, &tq);
    const size_t b0 = 4 * (size_t)blockIdx.x * kPartsPerBlock;   // the block's first census piece
    long long pos = a.blk[b0] + ec;
    long long S = a.blk[b0 + 1] + eq;
    T wmax = 0;
    if (combing) {
        const unsigned long long uT = (unsigned long long)Ttot, uM = (unsigned long long)M, uo = (unsigned long long)o;
        long long t = first_tooth(S, M, o, Ttot);
        // phase of tooth t, exact modulo 2^64 (its value lies in [0, T))
        unsigned long long ph = (unsigned long long)t * uT + uo - (unsigned long long)S * uM;
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            if (q[r] <= 0) continue;
            const unsigned long long uq = (unsigned long long)q[r], qm = uq * uM;
            long long n;
            if (__umul64hi(uq, uM) == 0ull && qm <= ph) n = 0;
            else if (__umul64hi(uq, uM) == 0ull && qm - ph <= uT) n = 1;
            else n = comb_teeth_wide(S, q[r], M, o, Ttot, t, ph);
            S += q[r];
            if (n > 0) {
                const long long js = a.perm ? (long long)(uint32_t)a.perm[j0 + r] : j0 + r;
                const T fx = a.stg.fx[js], fy = a.stg.fy[js], ox = a.stg.ox[js], oy = a.stg.oy[js];
                const T wc_ = w[r] < T(0) ? -wcopy : wcopy;
                const long long te = t + n < M ? t + n : M;
                for (long long u = t; u < te; ++u) {
                    a.out.cell[u] = cell[r]; a.out.fx[u] = fx; a.out.fy[u] = fy;
                    a.out.ox[u] = ox; a.out.oy[u] = oy; a.out.w[u] = wc_;
                }
                t += n;
            }
            ph = (unsigned long long)t * uT + uo - (unsigned long long)S * uM;
        }
    } else {
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            if (cell[r] < 0) continue;
            if (pos < M) {
                const long long js = a.perm ? (long long)(uint32_t)a.perm[j0 + r] : j0 + r;
                a.out.cell[pos] = cell[r]; a.out.fx[pos] = a.stg.fx[js]; a.out.fy[pos] = a.stg.fy[js];
                a.out.ox[pos] = a.stg.ox[js]; a.out.oy[pos] = a.stg.oy[js]; a.out.w[pos] = w[r];
                wmax = fmax(wmax, fabs(w[r]));
            }
            ++pos;
        }
    }
    const int lane = threadIdx.x & 31;
    for (int off = 16; off > 0; off >>= 1) wmax = fmax(wmax, __shfl_down_sync(0xffffffffu, wmax, off));
    if (lane == 0 && wmax > T(0))
        atomicMax((unsigned long long*)&a.st->bank_wmax, (unsigned long long)__double_as_longlong((double)wmax));
    // the last block to finish: the new bank's size, and the census of t_{n+1} makes the next
    // leg and remap those of step n + 1
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.st->write_done, 1u) == gridDim.x - 1u) {
            __threadfence();
            a.st->n_bank = a.st->out_count;
            a.st->step += 1;
            a.st->write_done = 0u;
        }
    }
}


// the arguments of the remap passes (census in slot order, every slot streamed)
template <typename T>
static RemapArgs<T> remap_args(hyb_problem* p) {
    RemapArgs<T> a;
    a.nx = p->nx; a.ny = p->ny;
    a.dx = (T)p->dx; a.dy = (T)p->dy;
    a.cdt = (T)(p->d.c * p->d.dt);
    a.w_min = (T)p->d.w_min;
    a.split = make_cell_split(p->nx);
    a.sig = (const T*)p->sig;
    a.in = bank_view<T>(p, p->cur);
    a.out = bank_view<T>(p, 1 - p->cur);
    a.cdf = p->rem_cdf;
    a.f = p->rem_f;
    a.f32 = p->rem_f32;
    a.fpos = p->rem_pos;
    a.n_hist = p->d.n_hist;
    a.cap = p->d.census_cap > 0 ? p->d.census_cap : p->d.n_hist;
    if (a.cap > p->bank_cap) a.cap = p->bank_cap;
    a.V = p->point_tab;
    a.ntab = p->d.sampler != HYB_PRNG ? 5 : 0;
    a.bt = p->byte_tab;
    a.nbt = p->d.sampler == HYB_SOBOL_DS && p->byte_tab ? a.ntab : 0;
    a.sampler = p->d.sampler;
    a.seed = p->d.seed;
    a.st = p->st;
    a.blk = p->blk;
    a.stg = stage_view<T>(p);
    a.perm = nullptr;
    a.nslots = p->stage_slots;
    a.perm_slots = census_sorted_now(p) ? 1 : 0;
    a.lead_staged = 0;
    a.mode = 0;
    return a;
}

// Bank pre-pass: zero the remap counters, form the bank's scalars and re-stream slots [0, n_bank)
// into the staging buffer, all on p->side after the work queued on p->stream so far (the leg that
// last used the staging buffer for its births)
// the SM count the pre-pass sizes its grid from (queried once per device)
struct PrepassLimits { int dev = -1, sms = 0; };
static PrepassLimits g_prepass;

static cudaError_t prepass_limits() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || (g_prepass.sms > 0 && g_prepass.dev == dev)) return e;
    g_prepass.dev = dev;
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) g_prepass.sms = sms;
    return e;
}

// resident blocks of pass A on this device (blocks per SM at its shared memory, times the SMs)
template <typename T>
static cudaError_t count_grid(size_t smem, int* blocks) {
    static int per_sm[2] = {0, 0};
    static size_t per_smem[2] = {0, 0};
    cudaError_t e = prepass_limits();
    if (e != cudaSuccess) return e;
    const int t = sizeof(T) == 4 ? 0 : 1;
    if (per_sm[t] == 0 || per_smem[t] != smem) {
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, remap_count_kernel<T>, kTile, smem);
        if (e != cudaSuccess) return e;
        per_sm[t] = n > 0 ? n : 1;
        per_smem[t] = smem;
    }
    *blocks = per_sm[t] * g_prepass.sms;
    return cudaSuccess;
}

template <typename T>
static cudaError_t bank_prepass_t(hyb_problem* p) {
    cudaStream_t s = p->side;
    cudaError_t e = prepass_limits();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(p->ev_fork, p->stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamWaitEvent(s, p->ev_fork, 0);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&p->st->r_histories, 0, (char*)&p->st->n_bank - (char*)&p->st->r_histories, s);
    if (e != cudaSuccess) return e;
    remap_bank_prep_kernel<<<1, 1, 0, s>>>(p->st);
    RemapArgs<T> a = remap_args<T>(p);
    a.mode = 1;
    // One block per SM, each looping over slot blocks: the solve's kernels always find room beside
    // it (a full-occupancy grid delays the first sweep until its blocks drain; measured: +18 us of
    // solve per step against +7 us this way)
    const int nblk = (int)std::min<long long>((p->bank_cap + kSlotsPerBlock - 1) / kSlotsPerBlock, (long long)g_prepass.sms);
    if (nblk > 0) remap_count_kernel<T><<<nblk, kTile, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(p->ev_join, s);
    if (e != cudaSuccess) return e;
    p->bank_prepass = true;
    return cudaSuccess;
}

cudaError_t launch_remap_bank_prepass(hyb_problem* p) {
    cudaError_t e = drop_bank_prepass(p);
    if (e != cudaSuccess) return e;
    return p->prec == HYB_FP64 ? bank_prepass_t<double>(p) : bank_prepass_t<float>(p);
}

cudaError_t drop_bank_prepass(hyb_problem* p) {
    if (!p->bank_prepass) return cudaSuccess;
    p->bank_prepass = false;
    return cudaStreamWaitEvent(p->stream, p->ev_join, 0);
}

template <typename T>
static cudaError_t remap_t(hyb_problem* p) {
    cudaStream_t s = p->stream;
    // a bank pre-pass of this step (launch_remap_bank_prepass) zeroed the remap counters and
    // staged the bank slots' end states; otherwise the density launch zeroes them (no memset
    // separates the programmatically launched kernels below)
    const bool pre = p->bank_prepass;
    p->bank_prepass = false;
    const bool additive = p->d.remap_variant == 1;
    // the remap density with the CDF's reduction (and the zeroing of pass A's census pieces),
    // then the CDF rows, whose last block also forms the per-step scalars
    double* part = p->cell_scratch;
    long long* row_tot = (long long*)(p->cell_scratch + kCdfParts);
    double* part_max = p->cell_scratch + kCdfParts + p->ny + p->ncells;
    const long long blk_words = 4 * ((p->stage_slots + kPartSlots - 1) / kPartSlots);
    cudaError_t e = launch_pdl(p->pdl, remap_density_cdf_kernel, dim3(kCdfParts), dim3(256), 0, s, p->ncells,
                               p->area * p->d.dt, (const double*)p->Q_d, (const double*)p->ss_d,
                               (const double*)p->pre_raw, (const double*)p->post_raw, (const double*)p->sn_phi_d,
                               p->rem_f, p->rem_f32, p->rem_pos, p->rem_q, p->st, additive ? 0 : 1, p->area,
                               p->d.dt, part, part_max, part_max + kCdfParts, p->blk, blk_words, pre ? 0 : 1);
    if (e != cudaSuccess) return e;
    // steps 3'/4': the leg's census (bank slots, then its n_hist source births) leads the slots
    const long long lead = additive && p->has_src ? p->d.n_hist : 0;
    const double w_lead = additive && p->has_src ? p->w_src / (double)p->d.n_hist : 0.0;
    e = launch_pdl(p->pdl, cdf_rows_kernel, dim3(p->ny), dim3(256), 0, s, (const double*)p->rem_q,
                   (const double*)&p->st->remap_qmax, p->nx, p->ny, p->rem_cdf, row_tot,
                   reinterpret_cast<unsigned*>(part), p->st, (long long)p->d.n_hist, lead, w_lead);
    if (e != cudaSuccess) return e;

    RemapArgs<T> a = remap_args<T>(p);
    const long long maxN = p->stage_slots;
    a.lead_staged = additive ? 1 : 0;
    a.mode = pre ? 2 : 0;
    const int nblk = (int)((maxN + kSlotsPerBlock - 1) / kSlotsPerBlock);    // pass B blocks
    const int nparts = (int)((maxN + kPartSlots - 1) / kPartSlots);          // census pieces
    const size_t smem = (size_t)(remap_table_words(a.ntab, a.nbt) + a.ntab + 1) * sizeof(uint32_t);
    int resident = 0;
    e = count_grid<T>(smem, &resident);
    if (e != cudaSuccess) return e;
    if (pre) {
        e = cudaStreamWaitEvent(s, p->ev_join, 0);
        if (e != cudaSuccess) return e;
    }
    e = launch_pdl(p->pdl, remap_count_kernel<T>, dim3(std::min(nparts, resident)), dim3(kTile), smem, s, a);
    if (e != cudaSuccess) return e;
    p->bank_sorted = census_sorted_now(p);
    if (p->bank_sorted) {
        // survivors in cell (or phase-space) order, stable: the comb and the census write follow it
        e = sort_census<T>(p, a.stg, maxN, s, &a.perm);
        if (e != cudaSuccess) return e;
        remap_partials_kernel<T><<<nparts, kTile, 0, s>>>(a);
    }
    e = launch_pdl(p->pdl, remap_scan_kernel, dim3(1), dim3(1024), 0, s, p->blk, nparts, p->st, a.cap, a.seed,
                   a.sampler, (long long)p->d.n_hist);
    if (e != cudaSuccess) return e;
    e = launch_pdl(p->pdl, remap_write_kernel<T>, dim3(nblk), dim3(kTile), 0, s, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_remap(hyb_problem* p) { return p->prec == HYB_FP64 ? remap_t<double>(p) : remap_t<float>(p); }

// N_s = infinity: the census scalars. N = bank + births (remap_W stands for the birth weight),
// w_ref = the power of two at or above max(|w| of the step-start bank, source weight per birth).
__global__ void census_prep_kernel(DevState* st, double w_src, long long n_hist) {
    st->remap_W = w_src;
    st->r_lead = 0;
    const double wmax = fmax(st->bank_wmax, w_src > 0 ? w_src / (double)n_hist : 0.0);
    st->w_ref = wmax > 0 ? pow2_ceil(wmax) : 1.0;
    st->rs = remap_scalars(st, n_hist);
}

// staging slots past the leg's histories hold nothing: mark them dead (they sort last)
__global__ void stage_tail_kernel(int32_t* cell, const DevState* st, long long n_src, long long nslots) {
    const long long N = st->n_bank + n_src;
    for (long long j = N + (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nslots;
         j += (long long)gridDim.x * blockDim.x)
        cell[j] = -1;
}

// N_s = infinity (pure (Q)MC, no hand-off, no collided stage, no remap births): the leg staged
// every history's end state at its index (census survivors alive, the rest dead); the census of
// t_{n+1} is those survivors in slot order or in cell order, combed to census_cap with the
// remap's comb (Sec. 2.2 with the remap replaced by the MC census).
template <typename T>
static cudaError_t census_t(hyb_problem* p) {
    cudaStream_t s = p->stream;
    census_prep_kernel<<<1, 1, 0, s>>>(p->st, p->has_src ? p->w_src : 0.0, p->d.n_hist);
    RemapArgs<T> a;
    a.out = bank_view<T>(p, 1 - p->cur);
    a.stg = stage_view<T>(p);
    a.n_hist = p->d.n_hist;
    a.cap = p->d.census_cap > 0 ? p->d.census_cap : p->d.n_hist;
    if (a.cap > p->bank_cap) a.cap = p->bank_cap;
    a.sampler = p->d.sampler;
    a.seed = p->d.seed;
    a.st = p->st;
    a.blk = p->blk;
    a.perm = nullptr;
    const long long maxN = p->stage_slots;
    a.nslots = maxN;
    a.perm_slots = 0;
    a.lead_staged = 0;
    a.mode = 0;
    const int nblk = (int)((maxN + kSlotsPerBlock - 1) / kSlotsPerBlock);
    const int nparts = (int)((maxN + kPartSlots - 1) / kPartSlots);
    cudaError_t e = cudaMemsetAsync(&p->st->r_histories, 0, (char*)&p->st->n_bank - (char*)&p->st->r_histories, s);
    if (e != cudaSuccess) return e;
    p->bank_sorted = census_sorted_now(p);
    if (p->bank_sorted) {
        stage_tail_kernel<<<152, 256, 0, s>>>(a.stg.cell, p->st, p->has_src ? p->d.n_hist : 0, maxN);
        e = sort_census<T>(p, a.stg, maxN, s, &a.perm);
        if (e != cudaSuccess) return e;
    }
    remap_partials_kernel<T><<<nparts, kTile, 0, s>>>(a);
    remap_scan_kernel<<<1, 1024, 0, s>>>(p->blk, nparts, p->st, a.cap, a.seed, a.sampler, p->d.n_hist);
    remap_write_kernel<T><<<nblk, kTile, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_census(hyb_problem* p) { return p->prec == HYB_FP64 ? census_t<double>(p) : census_t<float>(p); }

// step flux phi_pre + phi_post + phi_c0 (cell averages)
__global__ void flux_kernel(int ncells, const double* pre, const double* post, const double* phi, double* flux) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ncells) flux[k] = pre[k] + post[k] + phi[4 * k];
}

cudaError_t launch_flux(hyb_problem* p) {
    flux_kernel<<<(p->ncells + 255) / 256, 256, 0, p->stream>>>(p->ncells, p->pre_d, p->post_d, p->sn_phi_d,
                                                                p->flux_d);
    return cudaGetLastError();
}

}  // namespace hyb
