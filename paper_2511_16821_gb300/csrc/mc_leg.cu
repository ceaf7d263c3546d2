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

#include <cmath>

#include "hyb_device.cuh"

namespace hyb {

template <typename T>
struct LegArgs {
    int nx, ny;
    T dx, dy, cdt;
    const T* sig;               // (sigma_a, sigma_s) per cell
    int n_s, sampler, handoff_full, ntab;
    T w_min;
    const uint32_t* V;
    uint64_t seed;              // keys of the census and source point sets come from (seed, step)
    BankView<T> bank;
    Cdf2DView cdf;
    long long n_src;
    T w0;
    typename Prec<T>::acc_t *pre, *post, *mom;
    DevState* st;
    int32_t* hist;
    double sig_s_max, w_src_total, cdt_d;
};

// State of one live history in a lane.
template <typename T>
struct Hist {
    int ix, iy, n, seg;
    T fx, fy, ox, oy, w, w_start, srem, tau;
    uint32_t idx;
    long long j;
    bool census_stream;
};

// Per-thread statistics of the histories a thread finished (integers: order-free sums).
struct LegTally {
    unsigned long long c[9];   // histories, segments, collisions, leaked, census, killed, reached, errors,
                               // fixed-point tally additions issued
    long long f[6];            // fixed-point weights: source, absorbed, leaked, census, handoff, killed
    int status;
};

__device__ __forceinline__ void leg_tally_zero(LegTally& t) {
#pragma unroll
    for (int q = 0; q < 9; ++q) t.c[q] = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) t.f[q] = 0;
    t.status = 0;
}

// Scales of one leg (fixed point of the tallies and of the weight totals). On the FP32 path the
// exponents are capped at 126 so that every scale is a finite float: a float product by a power of
// two is exact, and the per-segment bookkeeping then needs no FP64 arithmetic.
struct LegScales {
    int kt, km, kw;
    double scw;
};

template <typename T>
__device__ __forceinline__ LegScales leg_scales(const LegArgs<T>& a) {
    const double Wstep = a.st->bank_wsum + a.w_src_total;
    LegScales s;
    s.kt = scale_exponent(Wstep * a.cdt_d, Prec<T>::kbits);
    s.km = scale_exponent(Wstep * a.cdt_d * a.sig_s_max, Prec<T>::kbits);
    s.kw = scale_exponent(Wstep, 61);
    if (sizeof(T) == 4) {
        s.kt = min(s.kt, 126);
        s.km = min(s.km, 126);
        s.kw = min(s.kw, 126);
    }
    s.scw = ldexp(1.0, s.kw);
    return s;
}

// weight x in the fixed point of scale 2^kw: FP32 by an exact float product, FP64 as before
__device__ __forceinline__ long long fix_w(float x, double, float scw_f) { return __float2ll_rn(x * scw_f); }
__device__ __forceinline__ long long fix_w(double x, double scw, float) { return __double2ll_rn(x * scw); }

// The histories [next, last) of one problem, tracked by the calling warp with lane refill: a lane
// whose history ends takes the next index at once (ranks by ballot, deterministic order), so the
// warp keeps its lanes on segments instead of waiting for its longest history.
template <typename T>
__device__ void leg_warp_range(const LegArgs<T>& a, long long next, long long last, long long nb,
                               const uint32_t* sV, const uint32_t* sShC, const uint32_t* sShS, uint64_t key_c,
                               uint64_t key_s, const LegScales& sc, LegTally& t) {
    using P = Prec<T>;
    const T sc_t = (T)ldexp(1.0, sc.kt), sc_m = (T)ldexp(1.0, sc.km);
    const double scw = sc.scw;
    const float scw_f = (float)sc.scw;     // used on the FP32 path only (kw <= 126 there)
    constexpr bool kF32 = sizeof(T) == 4;
    const T DX = a.dx, DY = a.dy;
    const T INF = (T)INFINITY;
    const int Ns = a.n_s;
    const int nx = a.nx, ny = a.ny;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    Points pts;
    pts.NT = sV;
    pts.sampler = a.sampler;
    pts.ntab = a.ntab;
    Hist<T> h;
    bool alive = false;
    double d_abs = 0, d_hand = 0;   // FP64 path: weight removed from the live history so far

    for (;;) {
        const unsigned need = __ballot_sync(0xffffffffu, !alive);
        if (need) {
            const long long j = next + __popc(need & lt_mask);
            next += __popc(need);
            if (!alive && j < last) {
                // ---- start a history: bank pick-up or birth from Q -----------------------------
                h.j = j;
                bool ok = true;
                if (j < nb) {
                    h.idx = (uint32_t)j;
                    h.census_stream = true;
                    const int k = a.bank.cell[j];
                    if (k < 0 || k >= nx * ny) { t.status |= kStBounds; ok = false; }
                    else {
                        h.ix = k % nx; h.iy = k / nx;
                        h.fx = a.bank.fx[j]; h.fy = a.bank.fy[j];
                        h.ox = a.bank.ox[j]; h.oy = a.bank.oy[j];
                        h.w = a.bank.w[j];
                        h.srem = a.cdt;
                    }
                } else {
                    h.idx = (uint32_t)(j - nb);
                    h.census_stream = false;
                    pts.key = key_s; pts.shift = sShS;
                    T frx, fry;
                    const int k = sample_cell<T>(a.cdf, nx, ny, pts(h.idx, 0), pts(h.idx, 1), &frx, &fry);
                    h.ix = k % nx; h.iy = k / nx;
                    h.fx = frx * DX; h.fy = fry * DY;
                    iso_dir<T>(pts(h.idx, 3), pts(h.idx, 4), &h.ox, &h.oy);
                    h.w = a.w0;
                    h.srem = a.cdt * P::unit_c(pts(h.idx, 2));
                }
                if (ok) {
                    pts.key = h.census_stream ? key_c : key_s;
                    pts.shift = h.census_stream ? sShC : sShS;
                    ++t.c[0];
                    h.w_start = h.w;
                    t.f[0] += fix_w(h.w, scw, scw_f);
                    d_abs = 0; d_hand = 0;
                    h.n = 0;
                    h.seg = 0;
                    if (Ns == 0) ++t.c[6];
                    h.tau = Ns > 0 ? P::neglog(P::unit(pts(h.idx, 5))) : T(0);
                    alive = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, alive)) break;
        if (!alive) continue;
        pts.key = h.census_stream ? key_c : key_s;
        pts.shift = h.census_stream ? sShC : sShS;

        // ---- one segment ----------------------------------------------------------------------
        ++h.seg;
        const int k = h.iy * nx + h.ix;
        const T sa = a.sig[2 * k], ss = a.sig[2 * k + 1], st = sa + ss;
        const T dxf = h.ox > T(0) ? (DX - h.fx) / h.ox : (h.ox < T(0) ? h.fx / (-h.ox) : INF);
        const T dyf = h.oy > T(0) ? (DY - h.fy) / h.oy : (h.oy < T(0) ? h.fy / (-h.oy) : INF);
        const T dcol = (h.n < Ns && ss > T(0)) ? h.tau / ss : INF;
        T l;
        int ev;
        bool xc = false, yc = false;
        if (dcol <= dxf && dcol <= dyf && dcol <= h.srem) { l = dcol; ev = 0; }
        else if (dxf <= h.srem || dyf <= h.srem) {
            l = dxf < dyf ? dxf : dyf; ev = 1; xc = (dxf == l); yc = (dyf == l);
        } else { l = h.srem; ev = 2; }

        if (h.n < Ns) {
            const T att = -P::exm1(-sa * l);
            t.c[8] += P::add(&a.pre[k], sa > T(0) ? h.w * att / sa : h.w * l, sc_t);
            if constexpr (kF32) t.f[1] += fix_w(h.w * att, scw, scw_f);
            else d_abs += (double)(h.w * att);
            h.w = h.w * P::ex(-sa * l);
            h.tau = P::msub(h.tau, ss, l);
        } else {
            const T att = -P::exm1(-st * l);
            t.c[8] += P::add(&a.post[k], st > T(0) ? h.w * att / st : h.w * l, sc_t);
            if (ss > T(0)) {
                T g0, g1, g2;
                gfun<T>(st * l, &g0, &g1, &g2);
                const T I0 = l * g0, I1 = l * l * g1, I2 = l * l * l * g2;
                const T sw = ss * h.w;
                t.c[8] += P::add(&a.mom[4 * k + 0], sw * I0, sc_m);
                if (a.handoff_full) {
                    const T xi0 = T(2) * h.fx / DX - T(1), eta0 = T(2) * h.fy / DY - T(1);
                    const T axi = T(2) * h.ox / DX, aeta = T(2) * h.oy / DY;
                    // explicit fused forms: the same rounding in every kernel this is inlined into
                    t.c[8] += P::add(&a.mom[4 * k + 1], sw * P::fma_(xi0, I0, axi * I1), sc_m);
                    t.c[8] += P::add(&a.mom[4 * k + 2], sw * P::fma_(eta0, I0, aeta * I1), sc_m);
                    t.c[8] += P::add(&a.mom[4 * k + 3],
                           sw * P::fma_(xi0 * eta0, I0, P::fma_(P::fma_(xi0, aeta, eta0 * axi), I1, axi * aeta * I2)),
                           sc_m);
                }
            }
            if (st > T(0)) {
                if constexpr (kF32) {
                    t.f[4] += fix_w(h.w * att * (ss / st), scw, scw_f);
                    t.f[1] += fix_w(h.w * att * (sa / st), scw, scw_f);
                } else {
                    d_hand += (double)(h.w * att * (ss / st));
                    d_abs += (double)(h.w * att * (sa / st));
                }
            }
            h.w = h.w * P::ex(-st * l);
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
            const int base = 5 + 3 * (h.n - 1);
            iso_dir<T>(pts(h.idx, base + 1), pts(h.idx, base + 2), &h.ox, &h.oy);
            if (h.n < Ns) h.tau = P::neglog(P::unit(pts(h.idx, 5 + 3 * h.n)));
            else { h.tau = T(0); ++t.c[6]; }
        }
        if (fate < 0 && a.w_min > T(0) && h.w < a.w_min * h.w_start) fate = kFateKilled;
        if (fate < 0 && h.seg >= (int)kMaxSegments) fate = kFateError;
        if (fate >= 0) {
            // ---- end of the history ------------------------------------------------------------
            const long long fw = fix_w(h.w, scw, scw_f);
            if (fate == kFateCensus) { ++t.c[4]; t.f[3] += fw; }
            else if (fate == kFateLeaked) { ++t.c[3]; t.f[2] += fw; }
            else if (fate == kFateKilled) { ++t.c[5]; t.f[5] += fw; }
            else { ++t.c[7]; t.status |= kStSegments; }
            if constexpr (!kF32) {
                t.f[1] += __double2ll_rn(d_abs * scw);
                t.f[4] += __double2ll_rn(d_hand * scw);
            }
            t.c[1] += (unsigned long long)h.seg;
            if (a.hist) {
                const int4 r = make_int4(h.iy * nx + h.ix, fate, h.n, h.seg);
                reinterpret_cast<int4*>(a.hist)[h.j] = r;
            }
            alive = false;
        }
    }
}

// Block reduction of the per-thread statistics into the problem's counters (all threads call).
__device__ void leg_flush(DevState* st, LegTally& t, const LegScales& sc, bool write_scales) {
    __shared__ unsigned long long s_c[kTile / 32][15];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    unsigned long long cs[15];
#pragma unroll
    for (int q = 0; q < 9; ++q) cs[q] = t.c[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) cs[9 + q] = (unsigned long long)t.f[q];
#pragma unroll
    for (int q = 0; q < 15; ++q) cs[q] = warp_sum_u64(cs[q]);
    if (lane == 0)
        for (int q = 0; q < 15; ++q) s_c[wl][q] = cs[q];
    if (t.status) atomicOr(&st->status, t.status);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* cdst[9] = {&st->histories, &st->segments, &st->collisions, &st->leaked,
                                       &st->census, &st->killed, &st->reached, &st->errors, &st->tally_adds};
        Acc128* wdst[6] = {&st->w_source, &st->w_absorbed, &st->w_leaked, &st->w_census,
                           &st->w_handoff, &st->w_killed};
        const int nw = (int)(blockDim.x >> 5);
        for (int q = 0; q < 15; ++q) {
            unsigned long long v = 0;
            for (int ww = 0; ww < nw; ++ww) v += s_c[ww][q];
            if (q < 9) { if (v) atomicAdd(cdst[q], v); }
            else if (v) {
                const long long sv = (long long)v;
                atomic_add128(wdst[q - 9], (unsigned long long)sv, sv < 0 ? ~0ull : 0ull);
            }
        }
        if (write_scales) {
            st->k_track = sc.kt;
            st->k_mom = sc.km;
            st->k_w = sc.kw;
        }
    }
    __syncthreads();
}

// Single problem: the grid's warps split [bank slots | births] into contiguous slices.
template <typename T>
__global__ void __launch_bounds__(kTile, sizeof(T) == 4 ? 3 : 2) mc_leg_kernel(LegArgs<T> a) {
    extern __shared__ uint32_t sm[];
    uint32_t* sV = sm;
    uint32_t* sShC = sm + a.ntab * kNibbleWords;
    uint32_t* sShS = sShC + a.ntab;
    const uint64_t step = (uint64_t)a.st->step;
    const uint64_t key_c = dstream_key(a.seed, step, HYB_STREAM_LEG_CENSUS);
    const uint64_t key_s = dstream_key(a.seed, step, HYB_STREAM_LEG_SOURCE);
    build_nibble_tables(a.V, a.ntab, sV);
    for (int d = threadIdx.x; d < a.ntab; d += blockDim.x) {
        sShC[d] = dshift(key_c, (uint64_t)d);
        sShS[d] = dshift(key_s, (uint64_t)d);
    }
    __syncthreads();
    const long long nb = a.st->n_bank;
    const long long N = nb + a.n_src;
    const LegScales sc = leg_scales<T>(a);
    LegTally t;
    leg_tally_zero(t);
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long per = (N + nwarps - 1) / nwarps;
    const long long j0 = wid * per;
    const long long j1 = j0 + per < N ? j0 + per : N;
    leg_warp_range<T>(a, j0, j1, nb, sV, sShC, sShS, key_c, key_s, sc, t);
    leg_flush(a.st, t, sc, blockIdx.x == 0);
}

// Many problems: a persistent grid pulls (problem, [j0, j1)) chunks from a work queue; per chunk
// the CTA's warps split the range, then flush the chunk's statistics to its problem.
struct LegChunk { int p; int pad; long long j0, j1; };

template <typename T>
__global__ void __launch_bounds__(kTile, sizeof(T) == 4 ? 3 : 2)
mc_leg_batch_kernel(const LegArgs<T>* __restrict__ args, const LegChunk* __restrict__ chunks, int nchunks,
                    int* head, const uint32_t* V, int ntab_max) {
    extern __shared__ uint32_t sm[];
    uint32_t* sV = sm;
    uint32_t* sShC = sm + ntab_max * kNibbleWords;
    uint32_t* sShS = sShC + ntab_max;
    __shared__ int s_chunk;
    build_nibble_tables(V, ntab_max, sV);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_chunk = atomicAdd(head, 1);
        __syncthreads();
        const int c = s_chunk;
        if (c >= nchunks) break;
        const LegChunk ch = chunks[c];
        const LegArgs<T> a = args[ch.p];
        const uint64_t step = (uint64_t)a.st->step;
        const uint64_t key_c = dstream_key(a.seed, step, HYB_STREAM_LEG_CENSUS);
        const uint64_t key_s = dstream_key(a.seed, step, HYB_STREAM_LEG_SOURCE);
        for (int d = threadIdx.x; d < a.ntab; d += blockDim.x) {
            sShC[d] = dshift(key_c, (uint64_t)d);
            sShS[d] = dshift(key_s, (uint64_t)d);
        }
        __syncthreads();
        const long long nb = a.st->n_bank;
        const long long N = nb + a.n_src;
        const long long e = ch.j1 < N ? ch.j1 : N;
        const LegScales sc = leg_scales<T>(a);
        LegTally t;
        leg_tally_zero(t);
        if (ch.j0 < e) {
            const long long nw = blockDim.x >> 5, w = threadIdx.x >> 5;
            const long long per = (e - ch.j0 + nw - 1) / nw;
            const long long j0 = ch.j0 + w * per;
            const long long j1 = j0 + per < e ? j0 + per : e;
            leg_warp_range<T>(a, j0, j1, nb, sV, sShC, sShS, key_c, key_s, sc, t);
        }
        leg_flush(a.st, t, sc, ch.j0 == 0);
    }
}

// fixed point -> FP64: raw track-length sums, step-average fluxes and hand-off moments
template <typename T>
__global__ void leg_normalise_kernel(const typename Prec<T>::acc_t* pre, const typename Prec<T>::acc_t* post,
                                     const typename Prec<T>::acc_t* mom, const DevState* st, int ncells,
                                     double inv_adt, double* pre_raw, double* post_raw, double* pre_d,
                                     double* post_d, double* mom_d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncells) return;
    const double it = ldexp(1.0, -st->k_track), im = ldexp(1.0, -st->k_mom);
    const double a = Prec<T>::to_double(&pre[k], it), b = Prec<T>::to_double(&post[k], it);
    pre_raw[k] = a;
    post_raw[k] = b;
    pre_d[k] = a * inv_adt;
    post_d[k] = b * inv_adt;
    for (int j = 0; j < 4; ++j) mom_d[4 * k + j] = Prec<T>::to_double(&mom[4 * k + j], im);
}

// initial bank: n particles from the initial-weight CDF (stream INIT, step 0), isotropic, t = 0
template <typename T>
__global__ void init_bank_kernel(BankView<T> b, Cdf2DView cdf, int nx, int ny, T dx, T dy, long long n, T w0,
                                 const uint32_t* V, int ntab, int sampler, uint64_t key) {
    __shared__ uint32_t sV[5 * kNibbleWords];
    __shared__ uint32_t sSh[5];
    const int nt = ntab < 5 ? ntab : 5;
    build_nibble_tables(V, nt, sV);
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
    build_nibble_tables(V, ntab, sV);
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
static int leg_grid(long long work) {
    long long g = (work + kTile - 1) / kTile;
    const long long cap = 152LL * 8;
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
    a.n_s = p->d.n_s; a.sampler = p->d.sampler; a.handoff_full = p->d.handoff_full;
    a.ntab = p->ndims < HYB_SOBOL_DIMS ? p->ndims : HYB_SOBOL_DIMS;
    a.w_min = (T)p->d.w_min;
    a.V = p->sobolV;
    a.seed = p->d.seed;
    a.bank = bank_view<T>(p, cur);
    a.cdf = p->src_cdf;
    a.n_src = p->has_src ? p->d.n_hist : 0;
    a.w0 = (T)(p->has_src ? p->w_src / (double)p->d.n_hist : 0.0);
    a.pre = (typename Prec<T>::acc_t*)p->acc_pre;
    a.post = (typename Prec<T>::acc_t*)p->acc_post;
    a.mom = (typename Prec<T>::acc_t*)p->acc_mom;
    a.st = p->st;
    a.hist = hist;
    a.sig_s_max = p->sig_s_max;
    a.w_src_total = p->has_src ? p->w_src : 0.0;
    return a;
}

template <typename T>
static cudaError_t mc_leg_t(hyb_problem* p, int32_t* hist) {
    const LegArgs<T> a = leg_args<T>(p, hist, p->cur);
    const size_t smem = (size_t)(a.ntab * kNibbleWords + 2 * a.ntab) * sizeof(uint32_t);
    const long long work = p->bank_cap + a.n_src;
    mc_leg_kernel<T><<<leg_grid(work), kTile, smem, p->stream>>>(a);
    return cudaGetLastError();
}

size_t leg_args_bytes(int prec) { return prec == HYB_FP64 ? sizeof(LegArgs<double>) : sizeof(LegArgs<float>); }

void leg_args_host(hyb_problem* p, int cur, void* out) {
    if (p->prec == HYB_FP64) *(LegArgs<double>*)out = leg_args<double>(p, nullptr, cur);
    else *(LegArgs<float>*)out = leg_args<float>(p, nullptr, cur);
}

int leg_ntab(const hyb_problem* p) { return p->ndims < HYB_SOBOL_DIMS ? p->ndims : HYB_SOBOL_DIMS; }

int leg_batch_ctas_per_sm(int prec) { return prec == HYB_FP64 ? 2 : 3; }

cudaError_t launch_mc_leg_batch(int prec, const void* d_args, const void* d_chunks, int nchunks, int* d_head,
                                const uint32_t* V, int ntab_max, int grid, int block, cudaStream_t s) {
    const size_t smem = (size_t)(ntab_max * kNibbleWords + 2 * ntab_max) * sizeof(uint32_t);
    if (prec == HYB_FP64)
        mc_leg_batch_kernel<double><<<grid, block, smem, s>>>((const LegArgs<double>*)d_args,
                                                             (const LegChunk*)d_chunks, nchunks, d_head, V, ntab_max);
    else
        mc_leg_batch_kernel<float><<<grid, block, smem, s>>>((const LegArgs<float>*)d_args,
                                                            (const LegChunk*)d_chunks, nchunks, d_head, V, ntab_max);
    return cudaGetLastError();
}

cudaError_t launch_mc_leg(hyb_problem* p, int32_t* hist_dev) {
    return p->prec == HYB_FP64 ? mc_leg_t<double>(p, hist_dev) : mc_leg_t<float>(p, hist_dev);
}

cudaError_t launch_leg_normalise(hyb_problem* p) {
    const double inv_adt = 1.0 / (p->area * p->d.dt);
    const int g = (p->ncells + 255) / 256;
    if (p->prec == HYB_FP64)
        leg_normalise_kernel<double><<<g, 256, 0, p->stream>>>((const Acc128*)p->acc_pre, (const Acc128*)p->acc_post,
                                                               (const Acc128*)p->acc_mom, p->st, p->ncells, inv_adt,
                                                               p->pre_raw, p->post_raw, p->pre_d, p->post_d, p->mom_d);
    else
        leg_normalise_kernel<float><<<g, 256, 0, p->stream>>>(
            (const unsigned long long*)p->acc_pre, (const unsigned long long*)p->acc_post,
            (const unsigned long long*)p->acc_mom, p->st, p->ncells, inv_adt, p->pre_raw, p->post_raw, p->pre_d,
            p->post_d, p->mom_d);
    return cudaGetLastError();
}

cudaError_t launch_init_bank(hyb_problem* p, const Cdf2DView& cdf, double w0) {
    const uint64_t key = stream_key(p->d.seed, 0, HYB_STREAM_INIT);
    const int ntab = p->d.sampler == HYB_SOBOL_DS ? 5 : 0;
    const long long n = p->d.n_hist;
    const int g = leg_grid(n);
    if (p->prec == HYB_FP64)
        init_bank_kernel<double><<<g, kTile, 0, p->stream>>>(bank_view<double>(p, p->cur), cdf, p->nx, p->ny, p->dx,
                                                             p->dy, n, w0, p->sobolV, ntab, p->d.sampler, key);
    else
        init_bank_kernel<float><<<g, kTile, 0, p->stream>>>(bank_view<float>(p, p->cur), cdf, p->nx, p->ny,
                                                            (float)p->dx, (float)p->dy, n, (float)w0, p->sobolV, ntab,
                                                            p->d.sampler, key);
    return cudaGetLastError();
}

cudaError_t launch_bank_stats(hyb_problem* p) {
    cudaError_t e = cudaMemsetAsync(&p->st->bank_wmax, 0, sizeof(double), p->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&p->st->bank_wsum_acc, 0, sizeof(Acc128), p->stream);
    if (e != cudaSuccess) return e;
    const int g = leg_grid(p->bank_cap);
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
    points_kernel<<<leg_grid(n), kTile, smem, s>>>(key, sampler, V, i0, n, ndims, out);
    return cudaGetLastError();
}

}  // namespace hyb
