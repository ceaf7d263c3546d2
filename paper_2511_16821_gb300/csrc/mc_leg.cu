// mc_leg.cu -- the scatter-limited (Q)MC leg (Sec. 2.2 step 1; Sec. 2.3) on sm_103a.
//
// One thread per history, grid-stride over [bank slots | source births]. Per history: pick-up
// from the SoA census bank or birth from the integer source CDF (implicit capture, isotropic
// direction, uniform time in the step), then the segment loop: distance to the x face, the y face,
// the next candidate collision (pre-limit only) and census; the shortest wins (collision over
// face over census). Pre-limit segments (n < N_s) tally w l g(sigma_a l) into <Psi>_pre and
// attenuate with sigma_a; post-limit segments (n = N_s) tally into <Psi>_post, attenuate with
// sigma_t and deposit the (N_s+1)-th collision density sigma_s int w P_j ds into four Legendre
// moments per cell. Tallies are fixed-point integer atomics (order-free, deterministic).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <type_traits>

#include "hyb_device.cuh"

namespace hyb {

template <typename T>
struct LegArgs {
    int nx, ny;
    T dx, dy, cdt;
    const T* sig;               // (sigma_a, sigma_s) per cell
    const float4* sig_inv;      // FP32 path: per cell two float4: (1/sigma_a, 1/sigma_s, 1/sigma_t, limit bits)
                                // (0 where sigma = 0), then (sigma_a, sigma_s, 0, 0)
    int n_s, sampler, handoff_full, ntab;
    T w_min;
    const uint32_t* V;
    const uint32_t* bt;         // Sobol byte tables of the births' dimensions (kByteDims x kByteWords), or null
    uint64_t seed;              // keys of the census and source point sets come from (seed, step)
    BankView<T> bank;
    BirthView<T> births;        // staged source births (cell == nullptr: drawn inside the leg)
    int spread_bank;            // 1: bank slots taken in transposed order (the bank is sorted by cell)
    BankView<T> cens;           // N_s = infinity: end state of history j at slot j (cell -1 unless census)
    int stage_census;
    const int32_t* ns_cell;     // per-cell scatter limits (space-dependent N_s), or null: n_s everywhere
    CellSplit split;            // cell index -> (ix, iy)
    Cdf2DView cdf;
    long long n_src;
    T w0;
    typename Prec<T>::acc_t *pre, *post, *mom;   // ncopy copies, ncells (pre, post) / 4 ncells (mom) apart
    int ncopy;                  // tally copies: each warp adds into copy (global warp index mod ncopy)
    DevState* st;
    int32_t* hist;
    double sig_s_max, w_src_total, cdt_d;
    long long h0, h1;           // history index range tracked: [h0, h1) of [bank slots | births]
    long long birth_step;       // step index of the births drawn by mc_birth_kernel (-1: the device's step)
    int seg_limit;              // segments per history before the history ends as an error
    int wx0, wy0, wside;        // privatised window of cells (single-problem fused leg; wside 0: none)
};

// State of one live history in a lane.
template <typename T>
struct Hist {
    int ix, iy, n, seg;
    T fx, fy, ox, oy, w, w_start, srem, tau;
    T rox, roy;                 // 1/ox, 1/oy (FP32 face distances)
    uint32_t idx;               // point index: bank slot or birth index (global index: idx, or nb + idx)
    bool census_stream;
};

// The phased leg (leg_sort_every = K >= 1): every history advances at most K segments per phase;
// the histories still alive at the end of a phase are saved here (compacted), sorted by cell, and
// taken up again by the next phase. A saved history is exactly its lane state (a scatter's new
// direction and optical depth already drawn), so the phases do the fused leg's arithmetic.
template <typename T>
struct LiveView {
    uint32_t* id;               // point index, census stream in bit 31
    int32_t* cell;
    T *fx, *fy, *ox, *oy, *w, *w0, *srem, *tau;
    int32_t *n, *seg;
};

template <typename T>
struct PhaseArgs {
    LiveView<T> in, out;                  // in: the phase's histories (later phases); out: those alive after it
    unsigned long long* out_count;        // histories saved to `out`
    const unsigned long long* in_count;   // histories in `in`
    int first;                            // 1: the histories start from the bank and the births
    int budget;                           // segments per history per phase (K)
};

// Per-thread statistics of the histories a thread finished (integers: order-free sums).
struct LegTally {
    unsigned int c[9];         // histories, segments, collisions, leaked, census, killed, reached, errors,
                               // fixed-point tally additions issued
    Acc128 f[4];               // fixed-point weights (128-bit sums): source, leaked, census, killed (the
                               // absorbed and handed-off weights are derived from the tallies by the
                               // normalisation)
    int status;
};

__device__ __forceinline__ void leg_tally_zero(LegTally& t) {
#pragma unroll
    for (int q = 0; q < 9; ++q) t.c[q] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) t.f[q] = Acc128{0ull, 0ull};
    t.status = 0;
}

// a += v (v a signed 64-bit value, a a 128-bit two's-complement sum)
__device__ __forceinline__ void add128(unsigned long long* lo, unsigned long long* hi, long long v) {
    const unsigned long long nl = *lo + (unsigned long long)v;
    *hi += (v < 0 ? ~0ull : 0ull) + (nl < *lo ? 1ull : 0ull);
    *lo = nl;
}

// Scales of one leg (fixed point of the tallies and of the weight totals). Tallies: sums over the
// whole leg are bounded by the step's starting weight W (x c dt, x sigma_s,max for the moments),
// so the scale is 2^(kbits - ceil(log2 bound)). Weight statistics: every value one history adds is
// at most its starting weight, bounded by the largest bank weight or the birth weight, so each is an
// int64 at scale 2^(62 - ceil(log2 w_max)) and the sums are 128-bit: the resolution is set by a
// single history's weight, not by the step total (many identical small birth weights would
// otherwise round alike). On the FP32 path the exponents are capped at 126 so that every scale is a
// finite float: a float product by a power of two is exact, and the per-segment bookkeeping then
// needs no FP64 arithmetic.
struct LegScales {
    int kt, km, kw;
    double scw, sct, scm;     // 2^kw, 2^kt, 2^km
};

template <typename T>
__device__ __forceinline__ LegScales leg_scales(const LegArgs<T>& a) {
    const double Wstep = a.st->bank_wsum + a.w_src_total;
    LegScales s;
    s.kt = scale_exponent(Wstep * a.cdt_d, Prec<T>::kbits);
    s.km = scale_exponent(Wstep * a.cdt_d * a.sig_s_max, Prec<T>::kbits);
    const double w0 = a.n_src > 0 ? a.w_src_total / (double)a.n_src : 0.0;
    s.kw = scale_exponent(fmax(a.st->bank_wmax, w0), 62);
    if (sizeof(T) == 4) {
        s.kt = min(s.kt, 126);
        s.km = min(s.km, 126);
        s.kw = min(s.kw, 126);
    }
    s.scw = ldexp(1.0, s.kw);
    s.sct = ldexp(1.0, s.kt);
    s.scm = ldexp(1.0, s.km);
    return s;
}

// weight x in the fixed point of scale 2^kw: FP32 by an exact float product, FP64 as before
__device__ __forceinline__ long long fix_w(float x, double, float scw_f) { return f2ll_rn(x * scw_f); }
__device__ __forceinline__ long long fix_w(double x, double scw, float) { return __double2ll_rn(x * scw); }

// Start state of source birth i (Sec. 2.3): cell and in-cell position from the integer source CDF
// (dims 0, 1), remaining flight c dt (1 - u) from the birth time (dim 2), isotropic direction
// (dims 3, 4), first optical depth -log u (dim 5) when N_s > 0. Used by the birth kernel and by
// the leg when births are not staged, so both give the same state bit for bit.
template <typename T, typename Pts>
__device__ __forceinline__ void birth_state(const LegArgs<T>& a, const Pts& pts, uint32_t i, int* ix, int* iy, T* fx,
                                            T* fy, T* ox, T* oy, T* srem, T* tau) {
    using P = Prec<T>;
    T frx, fry;
    const int k = sample_cell<T>(a.cdf, a.nx, a.ny, pts(i, 0), pts(i, 1), &frx, &fry);
    a.split(k, ix, iy);
    *fx = frx * a.dx; *fy = fry * a.dy;
    iso_dir<T>(pts(i, 3), pts(i, 4), ox, oy);
    *srem = a.cdt * P::unit_c(pts(i, 2));
    *tau = a.n_s > 0 ? P::neglog(P::unit(pts(i, 5))) : T(0);
}

// Work sources of a warp: chunks of kWarpChunk histories taken from a counter (the single-problem
// leg: warps that drew short histories take more and none waits at the end; the batched leg: the
// CTA's share of one work-queue chunk). Global history index = base + counter value, below `end`.
// Integer tallies make the results independent of which warp runs which history.
constexpr long long kWarpChunk = 64;

struct CounterChunks {
    unsigned long long* counter;
    long long base, end;
    __device__ bool operator()(long long* next, long long* last) {
        long long s = 0;
        if ((threadIdx.x & 31) == 0) s = (long long)atomicAdd(counter, (unsigned long long)kWarpChunk);
        s = base + __shfl_sync(0xffffffffu, s, 0);
        if (s >= end) return false;
        *next = s;
        *last = s + kWarpChunk < end ? s + kWarpChunk : end;
        return true;
    }
};

// Processing order of the bank slots when the bank is sorted by cell: with nb = 32 q + r, index
// i < 32 q goes to slot (i mod 32) q + i / 32, so the 32 lanes that take consecutive indices hold
// particles a 32nd of the bank apart (different cells: no lanes adding to one tally address at
// once); the last r slots keep their place. A bijection, and the results do not depend on which
// lane runs which history (integer tallies; the point index is the slot).
__device__ __forceinline__ long long spread_slot(long long i, long long nb) {
    const long long q = nb >> 5;
    return i < (q << 5) ? (i & 31) * q + (i >> 5) : i;
}

// sigma_a, sigma_s of cell k (one vector load through the read-only path)
__device__ __forceinline__ void load_sig(const float* sig, int k, float* sa, float* ss) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(sig) + k);
    *sa = v.x; *ss = v.y;
}
__device__ __forceinline__ void load_sig(const double* sig, int k, double* sa, double* ss) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(sig) + k);
    *sa = v.x; *ss = v.y;
}

// The histories of one problem that `src` hands out, tracked by the calling warp with lane refill:
// a lane whose history ends takes the next index at once (ranks by ballot, deterministic order),
// so the warp keeps its lanes on segments instead of waiting for its longest history.
// kStaged: the births were staged by the birth kernel (every leg but the ones that keep their
// census as particles, N_s = infinity and steps 3'/4', whose staging buffer holds that census);
// the kernel without the in-loop birth code keeps the loop body small
// kPhased: histories of one phase of the phased leg (ph): they start from the bank and births
// (first phase) or from the saved states, and a history that completes its phase's budget of
// segments alive is saved for the next phase.
// kPriv: the tallies of the cells in the window (a.wx0, a.wy0, a.wside) go to the block's copy in
// shared memory (tile: pre, post, then the 4 moments per cell of the window), flushed by the caller.
template <typename T, bool kStaged, typename Src, bool kPhased = false, bool kPriv = false>
__device__ void leg_warp_range(const LegArgs<T>& a, Src src, long long nb, const uint32_t* sV, const uint32_t* sShC,
                               const uint32_t* sShS, uint64_t key_c, uint64_t key_s, const LegScales& sc,
                               LegTally& t, const PhaseArgs<T>* ph = nullptr,
                               typename Prec<T>::acc_t* tile = nullptr) {
    // this thread's 128-bit weight sums (source, leaked, census, killed) live in shared memory,
    // not in registers: the segment loop then fits its register budget without spills
    __shared__ unsigned long long s_wl[4][kTile], s_wh[4][kTile];
#pragma unroll
    for (int q = 0; q < 4; ++q) { s_wl[q][threadIdx.x] = 0ull; s_wh[q][threadIdx.x] = 0ull; }
    using P = Prec<T>;
    const T sc_t = (T)sc.sct, sc_m = (T)sc.scm;
    const double scw = sc.scw;
    const float scw_f = (float)sc.scw;     // used on the FP32 path only (kw <= 126 there)
    constexpr bool kF32 = sizeof(T) == 4;
    const T DX = a.dx, DY = a.dy;
    const T INF = (T)INFINITY;
    const int Ns = a.n_s;
    const int nx = a.nx, ny = a.ny;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // this warp's tally copy: adds to a hot cell spread over ncopy addresses (integer sums, so
    // the total does not depend on which copy an add lands in)
    const size_t cp = (size_t)(((int)blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5)) % a.ncopy);
    typename P::acc_t* const pre_b = a.pre + cp * (size_t)nx * ny;
    typename P::acc_t* const post_b = a.post + cp * (size_t)nx * ny;
    typename P::acc_t* const mom_b = a.mom + cp * 4 * (size_t)nx * ny;

    Points pts;
    pts.NT = sV;
    pts.sampler = a.sampler;
    pts.ntab = a.ntab;
    Hist<T> h;
    bool alive = false;
    bool pending = false;   // scattered, waiting for its new direction and optical depth
    long long next = 0, last = 0;
    bool exhausted = false;
    bool to_save = false;   // phased leg: the lane's history completed its phase alive
    int seg0 = 0;           // phased leg: the history's segments before this phase

    for (;;) {
        if constexpr (kPhased) {
            // histories that completed the phase's segments alive: saved (compacted) for the next
            const unsigned sv = __ballot_sync(0xffffffffu, to_save);
            if (sv) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(ph->out_count, (unsigned long long)__popc(sv));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (to_save) {
                    const size_t o = (size_t)(base + (unsigned long long)__popc(sv & lt_mask));
                    ph->out.id[o] = h.idx | (h.census_stream ? 0x80000000u : 0u);
                    ph->out.cell[o] = h.iy * nx + h.ix;
                    ph->out.fx[o] = h.fx; ph->out.fy[o] = h.fy; ph->out.ox[o] = h.ox; ph->out.oy[o] = h.oy;
                    ph->out.w[o] = h.w; ph->out.w0[o] = h.w_start; ph->out.srem[o] = h.srem; ph->out.tau[o] = h.tau;
                    ph->out.n[o] = h.n; ph->out.seg[o] = h.seg;
                    to_save = false;
                    alive = false;
                }
            }
        }
        unsigned need = __ballot_sync(0xffffffffu, !alive);
        while (need && !exhausted) {
            if (next >= last && !src(&next, &last)) { exhausted = true; break; }
            const int cnt = __popc(need);
            const int take = last - next < (long long)cnt ? (int)(last - next) : cnt;
            const int rank = __popc(need & lt_mask);
            const bool mine = ((need >> lane) & 1u) && rank < take;
            long long j = next + rank;
            if (a.spread_bank && j < nb && !(kPhased && !ph->first)) j = spread_slot(j, nb);
            next += take;
            need &= ~__ballot_sync(0xffffffffu, mine);
            if (mine) {
                // ---- start a history: bank pick-up or birth from Q -----------------------------
                bool ok = true, resumed = false;
                if (kPhased && !ph->first) {
                    // a history of the previous phase, taken up where it stopped
                    const uint32_t id = ph->in.id[j];
                    h.idx = id & 0x7fffffffu;
                    h.census_stream = (id >> 31) != 0u;
                    a.split(ph->in.cell[j], &h.ix, &h.iy);
                    h.fx = ph->in.fx[j]; h.fy = ph->in.fy[j]; h.ox = ph->in.ox[j]; h.oy = ph->in.oy[j];
                    h.w = ph->in.w[j]; h.w_start = ph->in.w0[j]; h.srem = ph->in.srem[j]; h.tau = ph->in.tau[j];
                    h.n = ph->in.n[j]; h.seg = ph->in.seg[j];
                    resumed = true;
                } else if (j < nb) {
                    h.idx = (uint32_t)j;
                    h.census_stream = true;
                    const int k = a.bank.cell[j];
                    if (k < 0 || k >= nx * ny) { t.status |= kStBounds; ok = false; }
                    else {
                        a.split(k, &h.ix, &h.iy);
                        h.fx = a.bank.fx[j]; h.fy = a.bank.fy[j];
                        h.ox = a.bank.ox[j]; h.oy = a.bank.oy[j];
                        h.w = a.bank.w[j];
                        h.srem = a.cdt;
                    }
                } else {
                    h.idx = (uint32_t)(j - nb);
                    h.census_stream = false;
                    if constexpr (kStaged) {
                        const int k = a.births.cell[h.idx];
                        a.split(k, &h.ix, &h.iy);
                        h.fx = a.births.fx[h.idx]; h.fy = a.births.fy[h.idx];
                        h.ox = a.births.ox[h.idx]; h.oy = a.births.oy[h.idx];
                        h.srem = a.births.srem[h.idx];
                        h.tau = a.births.tau[h.idx];
                    } else {
                        pts.key = key_s; pts.shift = sShS;
                        birth_state<T, Points>(a, pts, h.idx, &h.ix, &h.iy, &h.fx, &h.fy, &h.ox, &h.oy, &h.srem, &h.tau);
                    }
                    h.w = a.w0;
                }
                if (resumed) {
                    if constexpr (kF32) { h.rox = P::rcp(h.ox); h.roy = P::rcp(h.oy); }
                    seg0 = h.seg;
                    alive = true;
                } else if (ok) {
                    seg0 = 0;
                    pts.key = h.census_stream ? key_c : key_s;
                    pts.shift = h.census_stream ? sShC : sShS;
                    if constexpr (kF32) { h.rox = P::rcp(h.ox); h.roy = P::rcp(h.oy); }
                    ++t.c[0];
                    h.w_start = h.w;
                    add128(&s_wl[0][threadIdx.x], &s_wh[0][threadIdx.x], fix_w(h.w, scw, scw_f));
                    h.n = 0;
                    h.seg = 0;
                    if ((a.ns_cell ? __ldg(a.ns_cell + h.iy * nx + h.ix) : Ns) == 0) ++t.c[6];
                    if (h.census_stream) h.tau = Ns > 0 ? P::neglog(P::unit(pts(h.idx, 5))) : T(0);
                    alive = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, alive)) {
            if (exhausted) break;
            continue;
        }
        pts.key = h.census_stream ? key_c : key_s;
        pts.shift = h.census_stream ? sShC : sShS;
        // a scatter's new direction and optical depth (three point dimensions, the direction map
        // and a logarithm) are drawn for the warp's scattered histories together, once 6 have
        // collected or no other lane could run a segment, instead of for one or two lanes in every
        // iteration (a scatter ends ~5 % of the segments on the benchmark)
        {
            const unsigned pend = __ballot_sync(0xffffffffu, pending);
            if (pend) {
                const unsigned runnable = __ballot_sync(0xffffffffu, alive && !pending);
                if (__popc(pend) >= 6 || __popc(runnable) < 6) {
                    if (pending) {
                        const int base = 5 + 3 * (h.n - 1);
                        iso_dir<T>(pts(h.idx, base + 1), pts(h.idx, base + 2), &h.ox, &h.oy);
                        if constexpr (kF32) { h.rox = P::rcp(h.ox); h.roy = P::rcp(h.oy); }
                        h.tau = h.n < Ns ? P::neglog(P::unit(pts(h.idx, 5 + 3 * h.n))) : T(0);
                        pending = false;
                    }
                }
            }
        }
        if (!alive || pending) continue;

        // ---- one segment ----------------------------------------------------------------------
        ++h.seg;
        const int k = h.iy * nx + h.ix;
        typename P::acc_t* pre_p = &pre_b[k];
        typename P::acc_t* post_p = &post_b[k];
        typename P::acc_t* mom_p = &mom_b[4 * k];
        if constexpr (kPriv) {
            const unsigned lx = (unsigned)(h.ix - a.wx0), ly = (unsigned)(h.iy - a.wy0);
            if (lx < (unsigned)a.wside && ly < (unsigned)a.wside) {
                const int kl = (int)(ly * (unsigned)a.wside + lx), w2 = a.wside * a.wside;
                pre_p = tile + kl;
                post_p = tile + w2 + kl;
                mom_p = tile + 2 * w2 + 4 * kl;
            }
        }
        T sa, ss;
        load_sig(a.sig, k, &sa, &ss);
        const T st = sa + ss;
        T dxf, dyf, dcol, isa = 0, iss = 0, ist = 0;
        int Nk = Ns;   // the scatter limit of this cell (space-dependent N_s) or n_s
        if constexpr (kF32) {
            // FP32: products with per-cell and per-flight reciprocals instead of divisions; the
            // fourth word of the reciprocal record carries the cell's scatter limit
            const float4 iv = __ldg(a.sig_inv + 2 * (size_t)k);
            isa = iv.x; iss = iv.y; ist = iv.z;
            if (a.ns_cell) Nk = __float_as_int(iv.w);
            dxf = h.ox > T(0) ? (DX - h.fx) * h.rox : (h.ox < T(0) ? h.fx * (-h.rox) : INF);
            dyf = h.oy > T(0) ? (DY - h.fy) * h.roy : (h.oy < T(0) ? h.fy * (-h.roy) : INF);
            dcol = (h.n < Nk && ss > T(0)) ? h.tau * iss : INF;
        } else {
            // FP64: the same divisions as the oracle (bit-identical geometry)
            if (a.ns_cell) Nk = __ldg(a.ns_cell + k);
            dxf = h.ox > T(0) ? (DX - h.fx) / h.ox : (h.ox < T(0) ? h.fx / (-h.ox) : INF);
            dyf = h.oy > T(0) ? (DY - h.fy) / h.oy : (h.oy < T(0) ? h.fy / (-h.oy) : INF);
            dcol = (h.n < Nk && ss > T(0)) ? h.tau / ss : INF;
        }
        T l;
        int ev;
        bool xc = false, yc = false;
        if (dcol <= dxf && dcol <= dyf && dcol <= h.srem) { l = dcol; ev = 0; }
        else if (dxf <= h.srem || dyf <= h.srem) {
            l = dxf < dyf ? dxf : dyf; ev = 1; xc = (dxf == l); yc = (dyf == l);
        } else { l = h.srem; ev = 2; }

        if (h.n < Nk) {
            // implicit capture with sigma_a (a pure scatterer keeps its weight and scores w l)
            T pre_c = h.w * l;
            if (sa > T(0)) {
                T att, e;
                P::att_e(sa * l, &att, &e);
                pre_c = kF32 ? h.w * att * isa : h.w * att / sa;
                h.w = h.w * e;
            }
            t.c[8] += P::add(pre_p, pre_c, sc_t);
            h.tau = P::msub(h.tau, ss, l);
        } else {
            T att, e;
            P::att_e(st * l, &att, &e);
            const T post_c = st > T(0) ? (kF32 ? h.w * att * ist : h.w * att / st) : h.w * l;
            t.c[8] += P::add(post_p, post_c, sc_t);
            if (ss > T(0)) {
                T g0, g1, g2;
                gfun<T>(st * l, e, att, &g0, &g1, &g2);
                const T I0 = l * g0, I1 = l * l * g1, I2 = l * l * l * g2;
                const T sw = ss * h.w;
                t.c[8] += P::add(mom_p + 0, sw * I0, sc_m);
                if (a.handoff_full) {
                    const T xi0 = T(2) * h.fx / DX - T(1), eta0 = T(2) * h.fy / DY - T(1);
                    const T axi = T(2) * h.ox / DX, aeta = T(2) * h.oy / DY;
                    // explicit fused forms: the same rounding in every kernel this is inlined into
                    t.c[8] += P::add(mom_p + 1, sw * P::fma_(xi0, I0, axi * I1), sc_m);
                    t.c[8] += P::add(mom_p + 2, sw * P::fma_(eta0, I0, aeta * I1), sc_m);
                    t.c[8] += P::add(mom_p + 3,
                           sw * P::fma_(xi0 * eta0, I0, P::fma_(P::fma_(xi0, aeta, eta0 * axi), I1, axi * aeta * I2)),
                           sc_m);
                }
            }
            h.w = h.w * e;
        }
        h.fx = P::madd(h.ox, l, h.fx);
        h.fy = P::madd(h.oy, l, h.fy);
        h.srem = h.srem - l;

        int fate = -1;
        if (ev == 2) {
            fate = kFateCensus;
        } else if (ev == 1) {
            if (xc) { h.ix += h.ox > T(0) ? 1 : -1; h.fx = h.ox > T(0) ? T(0) : DX; }
            else h.fx = clamp_(h.fx, T(0), DX);
            if (yc) { h.iy += h.oy > T(0) ? 1 : -1; h.fy = h.oy > T(0) ? T(0) : DY; }
            else h.fy = clamp_(h.fy, T(0), DY);
            if (h.ix < 0 || h.ix >= nx || h.iy < 0 || h.iy >= ny) {
                fate = kFateLeaked;
                h.ix = h.ix < 0 ? 0 : (h.ix >= nx ? nx - 1 : h.ix);
                h.iy = h.iy < 0 ? 0 : (h.iy >= ny ? ny - 1 : h.iy);
            }
        } else {
            h.fx = clamp_(h.fx, T(0), DX);
            h.fy = clamp_(h.fy, T(0), DY);
            ++h.n; ++t.c[2];
            pending = true;
            if (h.n >= Nk) ++t.c[6];
        }
        if (fate < 0 && a.w_min > T(0) && h.w < a.w_min * h.w_start) fate = kFateKilled;
        if (fate < 0 && h.seg >= a.seg_limit) fate = kFateError;
        if (fate >= 0) {
            // ---- end of the history ------------------------------------------------------------
            const long long fw = fix_w(h.w, scw, scw_f);
            if (a.stage_census) {
                // N_s = infinity or steps 3'/4': the census survivors are kept (history order)
                const long long j = h.census_stream ? (long long)h.idx : nb + (long long)h.idx;
                if (fate == kFateCensus) {
                    a.cens.cell[j] = h.iy * nx + h.ix;
                    a.cens.fx[j] = clamp_(h.fx, T(0), DX); a.cens.fy[j] = clamp_(h.fy, T(0), DY);
                    a.cens.ox[j] = h.ox; a.cens.oy[j] = h.oy; a.cens.w[j] = h.w;
                } else {
                    a.cens.cell[j] = -1;
                }
            }
            if (fate == kFateCensus) { ++t.c[4]; add128(&s_wl[2][threadIdx.x], &s_wh[2][threadIdx.x], fw); }
            else if (fate == kFateLeaked) { ++t.c[3]; add128(&s_wl[1][threadIdx.x], &s_wh[1][threadIdx.x], fw); }
            else if (fate == kFateKilled) { ++t.c[5]; add128(&s_wl[3][threadIdx.x], &s_wh[3][threadIdx.x], fw); }
            else { ++t.c[7]; t.status |= kStSegments; }
            t.c[1] += (unsigned int)h.seg;
            if (a.hist) {
                const int4 r = make_int4(h.iy * nx + h.ix, fate, h.n, h.seg);
                reinterpret_cast<int4*>(a.hist)[h.census_stream ? (long long)h.idx : nb + (long long)h.idx] = r;
            }
            alive = false;
        } else if constexpr (kPhased) {
            if (h.seg - seg0 >= ph->budget) {
                // the phase's segments done: saved at the top of the next iteration, with a
                // scatter's new direction and optical depth drawn now (as the fused leg draws them)
                if (pending) {
                    const int base = 5 + 3 * (h.n - 1);
                    iso_dir<T>(pts(h.idx, base + 1), pts(h.idx, base + 2), &h.ox, &h.oy);
                    h.tau = h.n < Ns ? P::neglog(P::unit(pts(h.idx, 5 + 3 * h.n))) : T(0);
                    pending = false;
                }
                to_save = true;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned long long nl = t.f[q].lo + s_wl[q][threadIdx.x];
        t.f[q].hi += s_wh[q][threadIdx.x] + (nl < t.f[q].lo ? 1ull : 0ull);
        t.f[q].lo = nl;
    }
}

// 128-bit warp sum (lane 0 gets the total)
__device__ __forceinline__ Acc128 warp_sum_128(Acc128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        const unsigned long long hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        const unsigned long long nl = v.lo + lo;
        v.hi += hi + (nl < v.lo ? 1ull : 0ull);
        v.lo = nl;
    }
    return v;
}

// Block reduction of the per-thread statistics into the problem's counters (all threads call).
__device__ void leg_flush(DevState* st, LegTally& t, const LegScales& sc, bool write_scales) {
    __shared__ unsigned long long s_c[kTile / 32][9];
    __shared__ Acc128 s_w[kTile / 32][4];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    unsigned long long cs[9];
    Acc128 ws[4];
#pragma unroll
    for (int q = 0; q < 9; ++q) cs[q] = warp_sum_u64((unsigned long long)t.c[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) ws[q] = warp_sum_128(t.f[q]);
    if (lane == 0) {
        for (int q = 0; q < 9; ++q) s_c[wl][q] = cs[q];
        for (int q = 0; q < 4; ++q) s_w[wl][q] = ws[q];
    }
    if (t.status) atomicOr(&st->status, t.status);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* cdst[9] = {&st->histories, &st->segments, &st->collisions, &st->leaked,
                                       &st->census, &st->killed, &st->reached, &st->errors, &st->tally_adds};
        Acc128* wdst[4] = {&st->w_source, &st->w_leaked, &st->w_census, &st->w_killed};
        const int nw = (int)(blockDim.x >> 5);
        for (int q = 0; q < 9; ++q) {
            unsigned long long v = 0;
            for (int ww = 0; ww < nw; ++ww) v += s_c[ww][q];
            if (v) atomicAdd(cdst[q], v);
        }
        for (int q = 0; q < 4; ++q) {
            unsigned long long lo = 0, hi = 0;
            for (int ww = 0; ww < nw; ++ww) {
                const unsigned long long nl = lo + s_w[ww][q].lo;
                hi += s_w[ww][q].hi + (nl < lo ? 1ull : 0ull);
                lo = nl;
            }
            if (lo || hi) atomic_add128(wdst[q], lo, hi);
        }
        if (write_scales) {
            st->k_track = sc.kt;
            st->k_mom = sc.km;
            st->k_w = sc.kw;
        }
    }
    __syncthreads();
}

// Single problem: a persistent grid whose warps take chunks of the history index range [h0, h1)
// (clamped to [0, bank + births)) from the problem's counter.
// FP32: four CTAs of 256 threads per SM (64 registers; a few bytes spill outside the segment loop,
// measured 5 % faster than three CTAs without spills); FP64: two
// byte offset of the privatised tile in the leg kernel's dynamic shared memory (after the point
// tables and the two digital-shift vectors, 16-byte aligned)
__host__ __device__ __forceinline__ size_t leg_tile_offset(int ntab) {
    return ((size_t)(ntab * kNibbleWords + 2 * ntab) * sizeof(uint32_t) + 15) & ~(size_t)15;
}

// kPhased: one phase of the phased leg (ph), over the bank and births (first phase) or the saved
// histories of the previous phase. kPriv: the block keeps the tallies of the window's cells in
// shared memory (after the point tables) and adds them to its global copy at the end, one
// coalesced atomic per nonzero entry.
template <typename T, bool kStaged, bool kPhased, bool kPriv>
__global__ void __launch_bounds__(kTile, sizeof(T) == 4 ? 4 : 2) mc_leg_kernel(LegArgs<T> a, PhaseArgs<T> ph) {
    using acc_t = typename Prec<T>::acc_t;
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* sV = sm;
    acc_t* tile = nullptr;
    if constexpr (kPriv) {
        tile = reinterpret_cast<acc_t*>(reinterpret_cast<char*>(sm) + leg_tile_offset(a.ntab));
        const int ne = 6 * a.wside * a.wside;
        for (int i = threadIdx.x; i < ne; i += blockDim.x) tile[i] = acc_t{};
    }
    uint32_t* sShC = sm + a.ntab * kNibbleWords;
    uint32_t* sShS = sShC + a.ntab;
    const uint64_t step = (uint64_t)a.st->step;
    const uint64_t key_c = dstream_key(a.seed, step, HYB_STREAM_LEG_CENSUS);
    const uint64_t key_s = dstream_key(a.seed, step, HYB_STREAM_LEG_SOURCE);
    build_point_tables(a.V, a.ntab, sV, a.sampler);
    for (int d = threadIdx.x; d < a.ntab; d += blockDim.x) {
        sShC[d] = dshift(key_c, (uint64_t)d);
        sShS[d] = dshift(key_s, (uint64_t)d);
    }
    __shared__ LegScales s_sc;   // formed once per block (FP64 work)
    if (threadIdx.x == 0) s_sc = leg_scales<T>(a);
    __syncthreads();
    const LegScales sc = s_sc;
    LegTally t;
    leg_tally_zero(t);
    if constexpr (kPhased) {
        // nb: the bank size in every phase (a finished history's record and census slot follow
        // [bank slots | births]); later phases take up saved histories [0, in_count)
        const long long nb = a.st->n_bank;
        const long long N = ph.first ? nb + a.n_src : (long long)*ph.in_count;
        leg_warp_range<T, kStaged, CounterChunks, true>(a, CounterChunks{&a.st->leg_next, 0, N}, nb, sV, sShC, sShS,
                                                        key_c, key_s, sc, t, &ph);
    } else {
        const long long nb = a.st->n_bank;
        const long long N = nb + a.n_src;
        const long long h1 = a.h1 < N ? a.h1 : N;
        leg_warp_range<T, kStaged, CounterChunks, false, kPriv>(a, CounterChunks{&a.st->leg_next, a.h0, h1}, nb, sV,
                                                                sShC, sShS, key_c, key_s, sc, t, nullptr, tile);
    }
    if constexpr (kPriv) {
        // the window's tallies into the block's global copy (integer sums: any copy, any order)
        __syncthreads();
        const int ws = a.wside, w2 = ws * ws;
        const size_t nc = (size_t)a.nx * a.ny, cb = (size_t)(blockIdx.x % a.ncopy);
        for (int i = threadIdx.x; i < 6 * w2; i += blockDim.x) {
            const acc_t v = tile[i];
            const int kl = i < 2 * w2 ? i % w2 : (i - 2 * w2) >> 2;
            const size_t cell = (size_t)(a.wy0 + kl / ws) * a.nx + (size_t)(a.wx0 + kl % ws);
            acc_t* dst = i < w2 ? a.pre + cb * nc + cell
                       : i < 2 * w2 ? a.post + cb * nc + cell
                                    : a.mom + cb * 4 * nc + 4 * cell + ((i - 2 * w2) & 3);
            if constexpr (sizeof(T) == 4) {
                if (v) atomicAdd(dst, v);
            } else {
                if (v.lo || v.hi) atomic_add128(dst, v.lo, v.hi);
            }
        }
    }
    leg_flush(a.st, t, sc, blockIdx.x == 0);
}

// Many problems: a persistent grid pulls (problem, [j0, j1)) chunks from a work queue; per chunk
// the CTA's warps split the range, then flush the chunk's statistics to its problem.
struct LegChunk { int p; int pad; long long j0, j1; };

template <typename T>
__global__ void __launch_bounds__(kTile, 2)
mc_leg_batch_kernel(const LegArgs<T>* __restrict__ args, const LegChunk* __restrict__ chunks, int nchunks,
                    int* head, const uint32_t* V, int ntab_max) {
    extern __shared__ uint32_t sm[];
    uint32_t* sV = sm;
    uint32_t* sShC = sm + ntab_max * kNibbleWords;
    uint32_t* sShS = sShC + ntab_max;
    __shared__ int s_chunk;
    // the chunk's problem descriptor lives in shared memory (read on use, not held in registers)
    __shared__ __align__(16) unsigned int s_args[(sizeof(LegArgs<T>) + 3) / 4];
    __shared__ unsigned long long s_next;   // warps take kWarpChunk histories of the chunk at a time
    __shared__ LegScales s_sc;              // the chunk problem's scales, formed by one thread
    build_nibble_tables(V, ntab_max, sV);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(head, 1);
        __syncthreads();
        const int c = s_chunk;
        if (c >= nchunks) break;
        const LegChunk ch = chunks[c];
        const unsigned int* src = reinterpret_cast<const unsigned int*>(args + ch.p);
        for (int i = threadIdx.x; i < (int)(sizeof(LegArgs<T>) / 4); i += blockDim.x) s_args[i] = src[i];
        if (threadIdx.x == 0) s_next = 0ull;
        __syncthreads();
        const LegArgs<T>& a = *reinterpret_cast<const LegArgs<T>*>(s_args);
        const uint64_t step = (uint64_t)a.st->step;
        const uint64_t key_c = dstream_key(a.seed, step, HYB_STREAM_LEG_CENSUS);
        const uint64_t key_s = dstream_key(a.seed, step, HYB_STREAM_LEG_SOURCE);
        for (int d = threadIdx.x; d < a.ntab; d += blockDim.x) {
            sShC[d] = dshift(key_c, (uint64_t)d);
            sShS[d] = dshift(key_s, (uint64_t)d);
        }
        if (threadIdx.x == 0) s_sc = leg_scales<T>(a);
        __syncthreads();
        const long long nb = a.st->n_bank;
        const long long N = nb + a.n_src;
        const long long e = ch.j1 < N ? ch.j1 : N;
        const LegScales sc = s_sc;
        LegTally t;
        leg_tally_zero(t);
        if (ch.j0 < e)   // batches always stage their births (no N_s = infinity or steps 3'/4' in a batch)
            leg_warp_range<T, true>(a, CounterChunks{&s_next, ch.j0, e}, nb, sV, sShC, sShS, key_c, key_s, sc, t);
        leg_flush(a.st, t, sc, ch.j0 == 0);
    }
}

// Source births of one problem, [i0, i1) of its birth indices, into its birth staging arrays.
template <typename T, typename Pts>
__device__ __forceinline__ void births_range(const LegArgs<T>& a, const Pts& pts, long long i0, long long i1,
                                             long long stride) {
    for (long long i = i0; i < i1; i += stride) {
        int ix, iy;
        T fx, fy, ox, oy, srem, tau;
        birth_state<T, Pts>(a, pts, (uint32_t)i, &ix, &iy, &fx, &fy, &ox, &oy, &srem, &tau);
        a.births.cell[i] = iy * a.nx + ix;
        a.births.fx[i] = fx; a.births.fy[i] = fy;
        a.births.ox[i] = ox; a.births.oy[i] = oy;
        a.births.srem[i] = srem; a.births.tau[i] = tau;
    }
}

// The births of a leg, one per thread: every lane does the same work (no divergence between
// births and bank pick-ups, no refill), and the leg then reads them like bank particles.
template <typename T>
__global__ void __launch_bounds__(kTile) mc_birth_kernel(LegArgs<T> a) {
    __shared__ __align__(16) uint32_t sV[kByteDims * kByteWords];   // byte tables, or Halton tables
    __shared__ uint32_t sSh[6];
    const int nt = a.ntab < 6 ? a.ntab : 6;
    const uint64_t key = dstream_key(a.seed, (uint64_t)(a.birth_step >= 0 ? a.birth_step : a.st->step),
                                     HYB_STREAM_LEG_SOURCE);
    const int nbt = a.sampler == HYB_SOBOL_DS && a.bt ? nt : 0;
    if (nbt) copy_byte_tables(a.bt, nbt, sV);
    else build_point_tables(a.V, nt, sV, a.sampler);
    if (threadIdx.x < nt) sSh[threadIdx.x] = dshift(key, (uint64_t)threadIdx.x);
    __syncthreads();
    const PointsB pts{sV, nbt, Points{sV, sSh, key, a.sampler, nt}};
    // the births inside the leg's history range [h0, h1) of [bank slots | births]
    const long long nb = a.st->n_bank;
    const long long i0 = a.h0 > nb ? a.h0 - nb : 0;
    const long long i1 = a.h1 - nb < a.n_src ? a.h1 - nb : a.n_src;
    births_range<T>(a, pts, i0 + (long long)blockIdx.x * blockDim.x + threadIdx.x, i1, (long long)gridDim.x * blockDim.x);
}

// The births of many problems: CTAs pull (problem, [i0, i1)) chunks from a queue.
template <typename T>
__global__ void __launch_bounds__(kTile)
mc_birth_batch_kernel(const LegArgs<T>* __restrict__ args, const LegChunk* __restrict__ chunks, int nchunks,
                      int* head) {
    __shared__ uint32_t sV[6 * kNibbleWords];
    __shared__ uint32_t sSh[6];
    __shared__ int s_chunk;
    bool have_tables = false;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(head, 1);
        __syncthreads();
        const int c = s_chunk;
        if (c >= nchunks) break;
        const LegChunk ch = chunks[c];
        const LegArgs<T> a = args[ch.p];
        const int nt = a.ntab < 6 ? a.ntab : 6;
        const uint64_t key = dstream_key(a.seed, (uint64_t)a.st->step, HYB_STREAM_LEG_SOURCE);
        if (!have_tables) {           // the direction numbers are the same for every problem
            build_nibble_tables(a.V, 6, sV);
            have_tables = true;
        }
        if (threadIdx.x < nt) sSh[threadIdx.x] = dshift(key, (uint64_t)threadIdx.x);
        __syncthreads();
        const Points pts{sV, sSh, key, a.sampler, nt};
        const long long e = ch.j1 < a.n_src ? ch.j1 : a.n_src;
        births_range<T>(a, pts, ch.j0 + threadIdx.x, e, blockDim.x);
    }
}

// fixed point -> FP64: raw track-length sums, step-average fluxes and hand-off moments, each the
// exact integer sum of the ncopy tally copies
// The leg's absorbed and handed-off weights follow from its tallies: a pre-limit segment scores
// w (1 - e^{-sigma_a l}) / sigma_a (w l where sigma_a = 0) and loses sigma_a times that to
// absorption; a post-limit one scores w (1 - e^{-sigma_t l}) / sigma_t and loses sigma_a and
// sigma_s times that to absorption and to the hand-off. So w_absorbed = sum_k sigma_a,k (pre_k +
// post_k) and w_handoff = sum_k sigma_s,k post_k, each cell's product added in 128-bit fixed point
// (order-free) at the weight statistics' scale.
template <typename T>
__global__ void leg_normalise_kernel(typename Prec<T>::acc_t* pre, typename Prec<T>::acc_t* post,
                                     typename Prec<T>::acc_t* mom, int ncopy, DevState* st, int ncells,
                                     double inv_adt, const double* sa, const double* ss, double* pre_raw,
                                     double* post_raw, double* pre_d, double* post_d, double* mom_d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    Acc128 wa{0ull, 0ull}, wh{0ull, 0ull};
    if (k < ncells) {
        const double it = ldexp(1.0, -st->k_track), im = ldexp(1.0, -st->k_mom);
        const size_t n1 = (size_t)ncells, n4 = 4 * (size_t)ncells;
        const double a = Prec<T>::sum_to_double(&pre[k], n1, ncopy, it), b = Prec<T>::sum_to_double(&post[k], n1, ncopy, it);
        pre_raw[k] = a;
        post_raw[k] = b;
        pre_d[k] = a * inv_adt;
        post_d[k] = b * inv_adt;
        for (int j = 0; j < 4; ++j) mom_d[4 * k + j] = Prec<T>::sum_to_double(&mom[4 * k + j], n4, ncopy, im);
        // the fixed-point copies are read: zero them for the next leg (which then needs no memset)
        const typename Prec<T>::acc_t z{};
        for (int c = 0; c < ncopy; ++c) {
            pre[k + c * n1] = z;
            post[k + c * n1] = z;
            for (int j = 0; j < 4; ++j) mom[4 * k + j + c * n4] = z;
        }
        const double scw = ldexp(1.0, st->k_w);
        to_i128(sa[k] * (a + b) * scw, &wa.lo, &wa.hi);
        to_i128(ss[k] * b * scw, &wh.lo, &wh.hi);
    }
    wa = warp_sum_128(wa);
    wh = warp_sum_128(wh);
    if ((threadIdx.x & 31) == 0) {
        if (wa.lo || wa.hi) atomic_add128(&st->w_absorbed, wa.lo, wa.hi);
        if (wh.lo || wh.hi) atomic_add128(&st->w_handoff, wh.lo, wh.hi);
    }
}

// initial bank: n particles from the initial-weight CDF (stream INIT, step 0), isotropic, t = 0
template <typename T>
__global__ void init_bank_kernel(BankView<T> b, Cdf2DView cdf, int nx, int ny, T dx, T dy, long long n, T w0,
                                 const uint32_t* V, int ntab, int sampler, uint64_t key) {
    __shared__ uint32_t sV[5 * kNibbleWords];
    __shared__ uint32_t sSh[5];
    const int nt = ntab < 5 ? ntab : 5;
    build_point_tables(V, nt, sV, sampler);
    if (threadIdx.x < nt) sSh[threadIdx.x] = dshift(key, threadIdx.x);
    __syncthreads();
    Points pts{sV, sSh, key, sampler, nt};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T frx, fry, ox, oy;
        const int k = sample_cell<T>(cdf, nx, ny, pts((uint32_t)i, 0), pts((uint32_t)i, 1), &frx, &fry);
        iso_dir<T>(pts((uint32_t)i, 3), pts((uint32_t)i, 4), &ox, &oy);
        b.cell[i] = k;
        b.fx[i] = frx * dx;
        b.fy[i] = fry * dy;
        b.ox[i] = ox;
        b.oy[i] = oy;
        b.w[i] = w0;
    }
}

// bank statistics: max |w| (exact, bitwise atomic max) and sum |w| (block order)
template <typename T>
__global__ void bank_wmax_kernel(const T* w, DevState* st) {
    const long long n = st->n_bank;
    double m = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)w[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax((unsigned long long*)&st->bank_wmax, (unsigned long long)__double_as_longlong(m));
}

template <typename T>
__global__ void bank_wsum_kernel(const T* w, DevState* st) {
    const long long n = st->n_bank;
    const int kw = scale_exponent((double)n * st->bank_wmax, 125);
    const double sc = ldexp(1.0, kw);
    double s = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += fabs((double)w[i]);
    s = warp_sum(s);
    __shared__ double sw[32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sw[q];
        unsigned long long lo, hi;
        to_i128(t * sc, &lo, &hi);
        atomic_add128(&st->bank_wsum_acc, lo, hi);
    }
}

__global__ void bank_wsum_final_kernel(DevState* st) {
    const int kw = scale_exponent((double)st->n_bank * st->bank_wmax, 125);
    st->bank_wsum = acc128_to_double(st->bank_wsum_acc.lo, st->bank_wsum_acc.hi, ldexp(1.0, -kw));
}

__global__ void points_kernel(uint64_t key, int sampler, const uint32_t* V, long long i0, long long n, int ndims,
                              uint32_t* out) {
    extern __shared__ uint32_t sm[];
    const int ntab = ndims < HYB_SOBOL_DIMS ? ndims : HYB_SOBOL_DIMS;
    uint32_t* sV = sm;
    uint32_t* sSh = sm + ntab * kNibbleWords;
    build_point_tables(V, ntab, sV, sampler);
    for (int d = threadIdx.x; d < ntab; d += blockDim.x) sSh[d] = dshift(key, (uint64_t)d);
    __syncthreads();
    Points pts{sV, sSh, key, sampler, ntab};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(i0 + t);
        for (int d = 0; d < ndims; ++d) out[t * ndims + d] = pts(i, d);
    }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
// grid of the grid-stride kernels: up to 8 CTAs of kTile threads per SM
static int stride_grid(long long work) {
    long long g = (work + kTile - 1) / kTile;
    const long long cap = 152LL * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// resident CTAs of kTile threads per SM: the single-problem leg keeps its descriptor in constant
// memory and fits 4 (FP32); the batched leg holds a chunk's descriptor in registers and runs 2
static int leg_ctas_per_sm(int prec) { return prec == HYB_FP64 ? 2 : 4; }

// persistent grid: every CTA resident at once (warps then take history chunks from the counter)
static int leg_grid(long long work, int prec) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = (work + kTile - 1) / kTile;
    const long long cap = (long long)sms * leg_ctas_per_sm(prec);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// persistent grid of the privatised leg: as many CTAs per SM as its shared memory leaves resident
static int leg_grid_priv(long long work, int prec, size_t smem, const void* kernel) {
    int dev = 0, sms = 152, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kTile, smem) != cudaSuccess || per < 1) per = 1;
    if (per > leg_ctas_per_sm(prec)) per = leg_ctas_per_sm(prec);
    long long g = (work + kTile - 1) / kTile;
    const long long cap = (long long)sms * per;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T>
LegArgs<T> leg_args(hyb_problem* p, int32_t* hist, int cur) {
    LegArgs<T> a;
    a.nx = p->nx; a.ny = p->ny;
    a.dx = (T)p->dx; a.dy = (T)p->dy;
    a.cdt = (T)(p->d.c * p->d.dt);
    a.cdt_d = p->d.c * p->d.dt;
    a.sig = (const T*)p->sig;
    a.sig_inv = (const float4*)p->sig_inv;
    a.n_s = p->d.n_s; a.sampler = p->d.sampler; a.handoff_full = p->d.handoff_full;
    a.ns_cell = p->ns_cell;
    a.split = make_cell_split(p->nx);
    a.ntab = p->ndims < HYB_SOBOL_DIMS ? p->ndims : HYB_SOBOL_DIMS;
    a.w_min = (T)p->d.w_min;
    a.V = p->point_tab;
    a.bt = p->byte_tab;
    a.seed = p->d.seed;
    a.bank = bank_view<T>(p, cur);
    a.births = birth_view<T>(p);
    a.birth_step = -1;
    a.spread_bank = p->bank_sorted ? 1 : 0;
    // N_s = infinity and steps 3'/4' keep the leg's census as particles
    a.stage_census = p->d.n_s == HYB_NS_INF || p->d.remap_variant == 1 ? 1 : 0;
    a.cens = stage_view<T>(p);
    if (a.stage_census) a.births.cell = nullptr;   // the staging buffer holds the census instead
    a.cdf = p->src_cdf;
    a.n_src = p->has_src ? p->d.n_hist : 0;
    a.w0 = (T)(p->has_src ? p->w_src / (double)p->d.n_hist : 0.0);
    a.pre = (typename Prec<T>::acc_t*)p->acc_pre;
    a.ncopy = p->tally_copies;
    a.post = (typename Prec<T>::acc_t*)p->acc_post;
    a.mom = (typename Prec<T>::acc_t*)p->acc_mom;
    a.st = p->st;
    a.hist = hist;
    a.sig_s_max = p->sig_s_max;
    a.w_src_total = p->has_src ? p->w_src : 0.0;
    a.h0 = 0;
    a.h1 = LLONG_MAX;
    a.seg_limit = p->d.seg_limit > 0 ? p->d.seg_limit : (int)kMaxSegments;
    a.wx0 = p->priv_x0;
    a.wy0 = p->priv_y0;
    a.wside = p->priv_side;
    return a;
}

// the leg kernels' dynamic shared memory (point tables: up to 65 dimensions) beside their static
// per-thread weight sums exceeds the default 48 KB per block: raise the kernel's limit once
template <typename K>
static cudaError_t allow_smem(K kernel, size_t dynamic_bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes + dynamic_bytes <= (48u << 10)) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynamic_bytes);
}

template <typename T>
static cudaError_t mc_leg_t(hyb_problem* p, int32_t* hist, long long h0, long long h1) {
    LegArgs<T> a = leg_args<T>(p, hist, p->cur);
    a.h0 = h0;
    a.h1 = h1;
    const size_t smem = (size_t)(a.ntab * kNibbleWords + 2 * a.ntab) * sizeof(uint32_t);
    const long long work = (h1 < p->bank_cap + a.n_src ? h1 : p->bank_cap + a.n_src) - h0;
    if (a.n_src > 0 && a.births.cell && p->births_step != p->step) {
        // births not drawn ahead (beside the previous step's collided solve): draw them now
        const long long g = (a.n_src + kTile - 1) / kTile;
        mc_birth_kernel<T><<<(unsigned)(g < 152 * 8 ? g : 152 * 8), kTile, 0, p->stream>>>(a);
        p->births_step = h0 == 0 && h1 == LLONG_MAX ? p->step : -1;   // a range leg draws only its share
    }
    const bool staged = a.births.cell != nullptr;
    const PhaseArgs<T> none{};
    cudaError_t e;
    if (a.wside > 0) {
        // the privatised window: its tile after the tables (allow_smem raises the limit as needed)
        const size_t smem_t = leg_tile_offset(a.ntab) + (size_t)6 * a.wside * a.wside * sizeof(typename Prec<T>::acc_t);
        e = staged ? allow_smem(mc_leg_kernel<T, true, false, true>, smem_t)
                   : allow_smem(mc_leg_kernel<T, false, false, true>, smem_t);
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(p->evk[0], p->stream);
        if (e != cudaSuccess) return e;
        const int g = leg_grid_priv(work, p->prec, smem_t, staged ? (const void*)mc_leg_kernel<T, true, false, true>
                                                                  : (const void*)mc_leg_kernel<T, false, false, true>);
        if (staged) mc_leg_kernel<T, true, false, true><<<g, kTile, smem_t, p->stream>>>(a, none);
        else mc_leg_kernel<T, false, false, true><<<g, kTile, smem_t, p->stream>>>(a, none);
    } else {
        e = staged ? allow_smem(mc_leg_kernel<T, true, false, false>, smem)
                   : allow_smem(mc_leg_kernel<T, false, false, false>, smem);
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(p->evk[0], p->stream);
        if (e != cudaSuccess) return e;
        if (staged) mc_leg_kernel<T, true, false, false><<<leg_grid(work, p->prec), kTile, smem, p->stream>>>(a, none);
        else mc_leg_kernel<T, false, false, false><<<leg_grid(work, p->prec), kTile, smem, p->stream>>>(a, none);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaEventRecord(p->evk[1], p->stream);
}

// Live-state buffer b (0, 1) of the phased leg: the eight T arrays first (8-byte alignment on the
// FP64 path), then id, cell, n and seg
template <typename T>
static LiveView<T> live_view(hyb_problem* p, int b) {
    const size_t n = (size_t)p->live_cap;
    T* f = static_cast<T*>(p->live_buf[b]);
    LiveView<T> v;
    v.fx = f; v.fy = f + n; v.ox = f + 2 * n; v.oy = f + 3 * n;
    v.w = f + 4 * n; v.w0 = f + 5 * n; v.srem = f + 6 * n; v.tau = f + 7 * n;
    uint32_t* u = reinterpret_cast<uint32_t*>(f + 8 * n);
    v.id = u;
    v.cell = reinterpret_cast<int32_t*>(u + n);
    v.n = reinterpret_cast<int32_t*>(u + 2 * n);
    v.seg = reinterpret_cast<int32_t*>(u + 3 * n);
    return v;
}

size_t live_buf_bytes(long long cap, int prec) {
    return (size_t)cap * (8 * (prec == HYB_FP64 ? sizeof(double) : sizeof(float)) + 4 * sizeof(uint32_t));
}

// the saved histories in cell order: dst[q] = src[perm[q]] (low half of the sorted pair)
template <typename T>
__global__ void __launch_bounds__(kTile) live_gather_kernel(LiveView<T> src, LiveView<T> dst,
                                                            const unsigned long long* perm, long long n) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)perm[q];
        dst.id[q] = src.id[j]; dst.cell[q] = src.cell[j];
        dst.fx[q] = src.fx[j]; dst.fy[q] = src.fy[j]; dst.ox[q] = src.ox[j]; dst.oy[q] = src.oy[j];
        dst.w[q] = src.w[j]; dst.w0[q] = src.w0[j]; dst.srem[q] = src.srem[j]; dst.tau[q] = src.tau[j];
        dst.n[q] = src.n[j]; dst.seg[q] = src.seg[j];
    }
}

// The phased leg (leg_sort_every = K >= 1): phase 0 starts every history (bank slots, then
// births) and runs each for at most K segments; the histories alive after a phase are saved
// (compacted), sorted by cell (stable radix sort of their cells), and the next phase takes them up
// in that order, until none is left. The host reads the live count after each phase. Every
// history does the fused leg's arithmetic on the same points, and every sum is an order-free
// integer sum, so the tallies, counters and weight statistics equal the fused leg's bit for bit.
template <typename T>
static cudaError_t mc_leg_phased_t(hyb_problem* p, int32_t* hist) {
    LegArgs<T> a = leg_args<T>(p, hist, p->cur);
    const size_t smem = (size_t)(a.ntab * kNibbleWords + 2 * a.ntab) * sizeof(uint32_t);
    if (a.n_src > 0 && a.births.cell && p->births_step != p->step) {
        const long long g = (a.n_src + kTile - 1) / kTile;
        mc_birth_kernel<T><<<(unsigned)(g < 152 * 8 ? g : 152 * 8), kTile, 0, p->stream>>>(a);
        p->births_step = p->step;
    }
    const bool staged = a.births.cell != nullptr;
    cudaError_t e = staged ? allow_smem(mc_leg_kernel<T, true, true, false>, smem)
                           : allow_smem(mc_leg_kernel<T, false, true, false>, smem);
    if (e != cudaSuccess) return e;
    PhaseArgs<T> ph{};
    ph.budget = p->d.leg_sort_every;
    ph.out_count = &p->st->live_count;
    ph.in_count = &p->st->live_in;
    ph.in = live_view<T>(p, 1);
    ph.out = live_view<T>(p, 0);
    // every phase adds at least K segments to each history it saves, and a history ends (as an
    // error) at the segment bound: the phases are bounded
    const long long max_phases = (long long)a.seg_limit / ph.budget + 2;
    const int wait = p->d.wait_limit > 0 ? p->d.wait_limit : (1 << 22);
    long long work = p->bank_cap + a.n_src;
    e = cudaEventRecord(p->evk[0], p->stream);
    if (e != cudaSuccess) return e;
    for (long long phase = 0;; ++phase) {
        if (phase > max_phases) return cudaErrorIllegalState;
        ph.first = phase == 0 ? 1 : 0;
        e = cudaMemsetAsync(&p->st->leg_next, 0, 2 * sizeof(unsigned long long), p->stream);   // leg_next, live_count
        if (e != cudaSuccess) return e;
        if (staged) mc_leg_kernel<T, true, true, false><<<leg_grid(work, p->prec), kTile, smem, p->stream>>>(a, ph);
        else mc_leg_kernel<T, false, true, false><<<leg_grid(work, p->prec), kTile, smem, p->stream>>>(a, ph);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(&p->st_host->live_count, &p->st->live_count, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return e;
        const long long n = (long long)p->st_host->live_count;
        if (n == 0) break;
        const unsigned long long* perm = nullptr;
        e = launch_census_sort(ph.out.cell, n, (uint32_t)p->ncells, p->live_pairs, p->live_scratch, wait,
                               &p->st->status, p->stream, &perm);
        if (e != cudaSuccess) return e;
        const long long g = (n + kTile - 1) / kTile;
        live_gather_kernel<T><<<(unsigned)(g < 152 * 8 ? g : 152 * 8), kTile, 0, p->stream>>>(ph.out, ph.in, perm, n);
        e = cudaMemcpyAsync(&p->st->live_in, &p->st->live_count, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                            p->stream);
        if (e != cudaSuccess) return e;
        work = n;
    }
    return cudaEventRecord(p->evk[1], p->stream);
}

size_t leg_args_bytes(int prec) { return prec == HYB_FP64 ? sizeof(LegArgs<double>) : sizeof(LegArgs<float>); }

void leg_args_host(hyb_problem* p, int cur, void* out) {
    if (p->prec == HYB_FP64) *(LegArgs<double>*)out = leg_args<double>(p, nullptr, cur);
    else *(LegArgs<float>*)out = leg_args<float>(p, nullptr, cur);
}

int leg_ntab(const hyb_problem* p) { return p->ndims < HYB_SOBOL_DIMS ? p->ndims : HYB_SOBOL_DIMS; }

int leg_batch_ctas_per_sm(int) { return 2; }

cudaError_t launch_mc_leg_batch(int prec, const void* d_args, const void* d_chunks, int nchunks, int* d_head,
                                const uint32_t* V, int ntab_max, int grid, int block, cudaStream_t s,
                                const void* d_bchunks, int nbchunks, int* d_bhead) {
    const size_t smem = (size_t)(ntab_max * kNibbleWords + 2 * ntab_max) * sizeof(uint32_t);
    if (nbchunks > 0) {
        const int bg = grid < nbchunks ? grid : nbchunks;
        if (prec == HYB_FP64)
            mc_birth_batch_kernel<double><<<bg, kTile, 0, s>>>((const LegArgs<double>*)d_args,
                                                               (const LegChunk*)d_bchunks, nbchunks, d_bhead);
        else
            mc_birth_batch_kernel<float><<<bg, kTile, 0, s>>>((const LegArgs<float>*)d_args,
                                                              (const LegChunk*)d_bchunks, nbchunks, d_bhead);
    }
    cudaError_t e = prec == HYB_FP64 ? allow_smem(mc_leg_batch_kernel<double>, smem)
                                     : allow_smem(mc_leg_batch_kernel<float>, smem);
    if (e != cudaSuccess) return e;
    if (prec == HYB_FP64)
        mc_leg_batch_kernel<double><<<grid, block, smem, s>>>((const LegArgs<double>*)d_args,
                                                             (const LegChunk*)d_chunks, nchunks, d_head, V, ntab_max);
    else
        mc_leg_batch_kernel<float><<<grid, block, smem, s>>>((const LegArgs<float>*)d_args,
                                                            (const LegChunk*)d_chunks, nchunks, d_head, V, ntab_max);
    return cudaGetLastError();
}

// The next step's births on the side stream, one block per SM (the collided solve's kernels keep
// room beside them), then ev_join again so that the remap (and every later use of the staging
// side) is ordered after them.
template <typename T>
static cudaError_t births_ahead_t(hyb_problem* p) {
    LegArgs<T> a = leg_args<T>(p, nullptr, p->cur);
    a.h0 = 0;
    a.h1 = LLONG_MAX;
    a.birth_step = p->step + 1;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long g = (a.n_src + kTile - 1) / kTile;
    mc_birth_kernel<T><<<(unsigned)(g < sms ? g : sms), kTile, 0, p->side>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(p->ev_join, p->side);
    if (e != cudaSuccess) return e;
    p->births_step = p->step + 1;
    return cudaSuccess;
}

cudaError_t launch_births_ahead(hyb_problem* p) {
    // only beside a bank pre-pass (the side stream is then ordered after this step's leg, which
    // read the births buffer, and the remap waits for ev_join)
    if (!p->bank_prepass || !p->births_buf || !p->has_src || p->d.n_hist <= 0) return cudaSuccess;
    return p->prec == HYB_FP64 ? births_ahead_t<double>(p) : births_ahead_t<float>(p);
}

cudaError_t launch_mc_leg(hyb_problem* p, int32_t* hist_dev, long long h0, long long h1) {
    if (p->d.leg_sort_every > 0 && h0 == 0 && h1 == LLONG_MAX)   // a whole leg: phases sorted by cell
        return p->prec == HYB_FP64 ? mc_leg_phased_t<double>(p, hist_dev) : mc_leg_phased_t<float>(p, hist_dev);
    return p->prec == HYB_FP64 ? mc_leg_t<double>(p, hist_dev, h0, h1) : mc_leg_t<float>(p, hist_dev, h0, h1);
}

// ---------------------------------------------------------------------------------------------
// Exchange block of a history-sharded leg: the raw integer results of a leg over one index range,
// laid out so that the element-wise int64 sum of the blocks of ranges that partition [0, N) is
// the block of the whole leg (an all-reduce with a plain integer sum). Words: [0, 12) counters
// (histories, segments, collisions, leaked, census, killed, reached, errors, tally adds, then how
// many ranges raised the bounds / segments / capacity status bits); [12, 36) the six weight sums,
// four 32-bit limbs each (value = sum_i limb_i 2^(32 i) mod 2^128, top limb signed); then the
// tallies pre, post (ncells each) and the moments (4 ncells): FP32 path one int64 word per value
// (two's-complement sums wrap consistently), FP64 path four limbs per 128-bit accumulator.
// ---------------------------------------------------------------------------------------------
constexpr int kXHead = 12 + 6 * 4;

__host__ __device__ inline size_t xblk_words(int prec, long long ncells) {
    return (size_t)kXHead + (size_t)6 * ncells * (prec == HYB_FP64 ? 4 : 1);
}

__device__ __forceinline__ void to_limbs(unsigned long long lo, unsigned long long hi, long long* w) {
    w[0] = (long long)(lo & 0xffffffffull);
    w[1] = (long long)(lo >> 32);
    w[2] = (long long)(hi & 0xffffffffull);
    w[3] = (long long)(int)(unsigned int)(hi >> 32);
}

// sum_i w_i 2^(32 i) mod 2^128 for signed 64-bit limb sums w_i
__device__ __forceinline__ void from_limbs(const long long* w, unsigned long long* lo, unsigned long long* hi) {
    unsigned long long L = 0, H = 0;
    auto add = [&](unsigned long long al, unsigned long long ah) {
        const unsigned long long nl = L + al;
        H += ah + (nl < L ? 1ull : 0ull);
        L = nl;
    };
    add((unsigned long long)w[0], w[0] < 0 ? ~0ull : 0ull);
    add((unsigned long long)w[1] << 32, (unsigned long long)(w[1] >> 32));
    add(0ull, (unsigned long long)w[2]);
    add(0ull, (unsigned long long)w[3] << 32);
    *lo = L;
    *hi = H;
}

__device__ __forceinline__ void acc_fold(const unsigned long long* p, size_t stride, int n, long long* w) {
    unsigned long long v = 0;
    for (int c = 0; c < n; ++c) v += p[c * stride];
    w[0] = (long long)v;
}
__device__ __forceinline__ void acc_fold(const Acc128* p, size_t stride, int n, long long* w) {
    unsigned long long lo = 0, hi = 0;
    for (int c = 0; c < n; ++c) {
        const Acc128 v = p[c * stride];
        const unsigned long long nl = lo + v.lo;
        hi += v.hi + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
    to_limbs(lo, hi, w);
}
__device__ __forceinline__ void acc_put(unsigned long long* p, const long long* w) { *p = (unsigned long long)w[0]; }
__device__ __forceinline__ void acc_put(Acc128* p, const long long* w) { from_limbs(w, &p->lo, &p->hi); }

template <typename T>
__global__ void leg_pack_kernel(const typename Prec<T>::acc_t* pre, const typename Prec<T>::acc_t* post,
                                const typename Prec<T>::acc_t* mom, int ncopy, int ncells, const DevState* st,
                                long long* x) {
    constexpr int L = sizeof(T) == 8 ? 4 : 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n1 = (size_t)ncells, n4 = 4 * (size_t)ncells;
    long long* t = x + kXHead;
    if (k < ncells) {
        acc_fold(pre + k, n1, ncopy, t + (size_t)L * k);
        acc_fold(post + k, n1, ncopy, t + (size_t)L * (n1 + k));
        for (int j = 0; j < 4; ++j) acc_fold(mom + 4 * (size_t)k + j, n4, ncopy, t + (size_t)L * (2 * n1 + 4 * (size_t)k + j));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long c[9] = {st->histories, st->segments, st->collisions, st->leaked, st->census,
                                         st->killed, st->reached, st->errors, st->tally_adds};
        for (int i = 0; i < 9; ++i) x[i] = (long long)c[i];
        x[9] = (st->status & kStBounds) ? 1 : 0;
        x[10] = (st->status & kStSegments) ? 1 : 0;
        x[11] = (st->status & kStCapacity) ? 1 : 0;
        const Acc128* ws[6] = {&st->w_source, &st->w_absorbed, &st->w_leaked, &st->w_census, &st->w_handoff,
                               &st->w_killed};
        for (int i = 0; i < 6; ++i) to_limbs(ws[i]->lo, ws[i]->hi, x + 12 + 4 * i);
    }
}

// the (summed) block into tally copy 0 (other copies zero) and the leg counters
template <typename T>
__global__ void leg_unpack_kernel(typename Prec<T>::acc_t* pre, typename Prec<T>::acc_t* post,
                                  typename Prec<T>::acc_t* mom, int ncopy, int ncells, DevState* st,
                                  const long long* x) {
    using acc_t = typename Prec<T>::acc_t;
    constexpr int L = sizeof(T) == 8 ? 4 : 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n1 = (size_t)ncells, n4 = 4 * (size_t)ncells;
    const long long* t = x + kXHead;
    if (k < ncells) {
        acc_t z;
        memset(&z, 0, sizeof(z));
        acc_put(pre + k, t + (size_t)L * k);
        acc_put(post + k, t + (size_t)L * (n1 + k));
        for (int j = 0; j < 4; ++j) acc_put(mom + 4 * (size_t)k + j, t + (size_t)L * (2 * n1 + 4 * (size_t)k + j));
        for (int c = 1; c < ncopy; ++c) {
            pre[c * n1 + k] = z;
            post[c * n1 + k] = z;
            for (int j = 0; j < 4; ++j) mom[c * n4 + 4 * (size_t)k + j] = z;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long* c[9] = {&st->histories, &st->segments, &st->collisions, &st->leaked, &st->census,
                                    &st->killed, &st->reached, &st->errors, &st->tally_adds};
        for (int i = 0; i < 9; ++i) *c[i] = (unsigned long long)x[i];
        st->status = (x[9] ? kStBounds : 0) | (x[10] ? kStSegments : 0) | (x[11] ? kStCapacity : 0);
        Acc128* ws[6] = {&st->w_source, &st->w_absorbed, &st->w_leaked, &st->w_census, &st->w_handoff,
                         &st->w_killed};
        for (int i = 0; i < 6; ++i) from_limbs(x + 12 + 4 * i, &ws[i]->lo, &ws[i]->hi);
    }
}

size_t leg_exchange_words(const hyb_problem* p) { return xblk_words(p->prec, p->ncells); }

cudaError_t launch_leg_pack(hyb_problem* p, long long* x) {
    const int g = (p->ncells + 255) / 256;
    if (p->prec == HYB_FP64)
        leg_pack_kernel<double><<<g, 256, 0, p->stream>>>((const Acc128*)p->acc_pre, (const Acc128*)p->acc_post,
                                                          (const Acc128*)p->acc_mom, p->tally_copies, p->ncells, p->st, x);
    else
        leg_pack_kernel<float><<<g, 256, 0, p->stream>>>((const unsigned long long*)p->acc_pre,
                                                         (const unsigned long long*)p->acc_post,
                                                         (const unsigned long long*)p->acc_mom, p->tally_copies,
                                                         p->ncells, p->st, x);
    return cudaGetLastError();
}

cudaError_t launch_leg_unpack(hyb_problem* p, const long long* x) {
    const int g = (p->ncells + 255) / 256;
    if (p->prec == HYB_FP64)
        leg_unpack_kernel<double><<<g, 256, 0, p->stream>>>((Acc128*)p->acc_pre, (Acc128*)p->acc_post,
                                                            (Acc128*)p->acc_mom, p->tally_copies, p->ncells, p->st, x);
    else
        leg_unpack_kernel<float><<<g, 256, 0, p->stream>>>((unsigned long long*)p->acc_pre,
                                                           (unsigned long long*)p->acc_post,
                                                           (unsigned long long*)p->acc_mom, p->tally_copies,
                                                           p->ncells, p->st, x);
    return cudaGetLastError();
}

cudaError_t launch_leg_normalise(hyb_problem* p) {
    const double inv_adt = 1.0 / (p->area * p->d.dt);
    const int g = (p->ncells + 255) / 256;
    if (p->prec == HYB_FP64)
        leg_normalise_kernel<double><<<g, 256, 0, p->stream>>>((Acc128*)p->acc_pre, (Acc128*)p->acc_post,
                                                               (Acc128*)p->acc_mom, p->tally_copies, p->st,
                                                               p->ncells, inv_adt, p->sa_d, p->ss_d,
                                                               p->pre_raw, p->post_raw, p->pre_d, p->post_d, p->mom_d);
    else
        leg_normalise_kernel<float><<<g, 256, 0, p->stream>>>(
            (unsigned long long*)p->acc_pre, (unsigned long long*)p->acc_post,
            (unsigned long long*)p->acc_mom, p->tally_copies, p->st, p->ncells, inv_adt, p->sa_d, p->ss_d,
            p->pre_raw, p->post_raw, p->pre_d, p->post_d, p->mom_d);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) p->acc_clean = true;
    return e;
}

cudaError_t launch_init_bank(hyb_problem* p, const Cdf2DView& cdf, double w0) {
    const uint64_t key = stream_key(p->d.seed, 0, HYB_STREAM_INIT);
    const int ntab = p->d.sampler != HYB_PRNG ? 5 : 0;
    const long long n = p->d.n_hist;
    const int g = stride_grid(n);
    if (p->prec == HYB_FP64)
        init_bank_kernel<double><<<g, kTile, 0, p->stream>>>(bank_view<double>(p, p->cur), cdf, p->nx, p->ny, p->dx,
                                                             p->dy, n, w0, p->point_tab, ntab, p->d.sampler, key);
    else
        init_bank_kernel<float><<<g, kTile, 0, p->stream>>>(bank_view<float>(p, p->cur), cdf, p->nx, p->ny,
                                                            (float)p->dx, (float)p->dy, n, (float)w0, p->point_tab, ntab,
                                                            p->d.sampler, key);
    return cudaGetLastError();
}

cudaError_t launch_bank_stats(hyb_problem* p) {
    cudaError_t e = cudaMemsetAsync(&p->st->bank_wmax, 0, sizeof(double), p->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&p->st->bank_wsum_acc, 0, sizeof(Acc128), p->stream);
    if (e != cudaSuccess) return e;
    const int g = stride_grid(p->bank_cap);
    if (p->prec == HYB_FP64) {
        BankView<double> b = bank_view<double>(p, p->cur);
        bank_wmax_kernel<double><<<g, kTile, 0, p->stream>>>(b.w, p->st);
        bank_wsum_kernel<double><<<g, kTile, 0, p->stream>>>(b.w, p->st);
    } else {
        BankView<float> b = bank_view<float>(p, p->cur);
        bank_wmax_kernel<float><<<g, kTile, 0, p->stream>>>(b.w, p->st);
        bank_wsum_kernel<float><<<g, kTile, 0, p->stream>>>(b.w, p->st);
    }
    bank_wsum_final_kernel<<<1, 1, 0, p->stream>>>(p->st);
    return cudaGetLastError();
}

cudaError_t launch_points(uint64_t key, int sampler, const uint32_t* V, int64_t i0, int64_t n, int ndims,
                          uint32_t* out, cudaStream_t s) {
    const int ntab = ndims < HYB_SOBOL_DIMS ? ndims : HYB_SOBOL_DIMS;
    const size_t smem = (size_t)(ntab * kNibbleWords + ntab) * sizeof(uint32_t);
    points_kernel<<<stride_grid(n), kTile, smem, s>>>(key, sampler, V, i0, n, ndims, out);
    return cudaGetLastError();
}

}  // namespace hyb
