// hyb_device.cuh -- device helpers shared by the sm_103a kernels: counter hashing and point
// sets (Sec. 2.4), isotropic directions, segment integrals, fixed-point tally accumulation and
// the integer 2-D CDF pick used for births (Sec. 2.3) and the remap (Sec. 2.2, Eq. (R)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hyb_internal.h"

namespace hyb {

// SoA bank layout inside a bank buffer: cell (int32, padded to 256 B), then fx, fy, ox, oy, w
inline size_t bank_cell_bytes(int64_t cap) { return (size_t)(((cap * 4 + 255) / 256) * 256); }

template <typename T>
inline BankView<T> bank_view(hyb_problem* p, int which) {
    BankView<T> b;
    const int64_t cap = p->bank_cap;
    char* bk = (char*)p->bank[which];
    b.cell = (int32_t*)bk;
    T* f = (T*)(bk + bank_cell_bytes(cap));
    b.fx = f; b.fy = f + cap; b.ox = f + 2 * cap; b.oy = f + 3 * cap; b.w = f + 4 * cap;
    return b;
}

// The remap staging SoA: one end state per slot (p->stage_slots: bank capacity + n_hist, plus
// n_hist more for steps 3'/4'), same layout as a bank (cell -1 = not alive)
template <typename T>
inline BankView<T> stage_view(hyb_problem* p) {
    BankView<T> b;
    const int64_t n = p->stage_slots;
    char* base = (char*)p->stage;
    b.cell = (int32_t*)base;
    T* f = (T*)(base + bank_cell_bytes(n));
    b.fx = f; b.fy = f + n; b.ox = f + 2 * n; b.oy = f + 3 * n; b.w = f + 4 * n;
    return b;
}

// Birth staging (its own buffer, so that the next step's births can be drawn while this step's
// remap uses the staging buffer): cell (int32, n_hist, padded to 256 B), then fx, fy, ox, oy,
// srem, tau (n_hist each). cell is null when the problem stages no births.
template <typename T>
inline BirthView<T> birth_view(hyb_problem* p) {
    BirthView<T> b;
    const int64_t n = p->d.n_hist;
    char* base = (char*)p->births_buf;
    if (!base) {
        b.cell = nullptr;
        b.fx = b.fy = b.ox = b.oy = b.srem = b.tau = nullptr;
        return b;
    }
    b.cell = (int32_t*)base;
    T* f = (T*)(base + bank_cell_bytes(n));
    b.fx = f; b.fy = f + n; b.ox = f + 2 * n; b.oy = f + 3 * n; b.srem = f + 4 * n; b.tau = f + 5 * n;
    return b;
}

// ---------------------------------------------------------------------------------------------
// splitmix64 output function (Steele, Lea & Flood 2014) and the point-set keys
// ---------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t dmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint32_t dshift(uint64_t key, uint64_t d) {
    return (uint32_t)(dmix64(key ^ (d + kGamma)) >> 32);
}

// key of the point set (seed, step, stream)
__host__ __device__ __forceinline__ uint64_t dstream_key(uint64_t seed, uint64_t step, uint64_t stream) {
    uint64_t z = dmix64(seed + kGamma);
    z = dmix64(z ^ (step + kGamma));
    return dmix64(z ^ (stream + kGamma));
}

// first point of a set (index 0, dimension 0): Sobol(0) = Halton(0) = 0 leaves the shift; else
// the hash
__host__ __device__ __forceinline__ uint32_t first_point(uint64_t key, int sampler) {
    return sampler != HYB_PRNG ? dshift(key, 0)
                                   : (uint32_t)(dmix64(dmix64(key ^ (0ull + kGamma)) ^ (0ull + kGamma)) >> 32);
}

// Sobol direction numbers as nibble tables: for dimension d and nibble k of the index, entry v is
// the XOR of the direction numbers of the set bits of v (bits 4k..4k+3 of the index). A point is
// then eight table reads whatever the index, and the 16 entries of one nibble table sit in 16
// distinct shared-memory banks, so a warp's reads never conflict.
constexpr int kNibbleWords = 128;   // 8 nibbles x 16 entries per dimension
static_assert(kNibbleWords == kHaltonWords, "Sobol and Halton tables share the per-dimension stride");

// builds the tables of dimensions [0, ntab) from the direction numbers V (ntab x 32) into sNT
// (ntab x kNibbleWords); all threads of the block call it, the caller synchronises
__device__ __forceinline__ void build_nibble_tables(const uint32_t* __restrict__ V, int ntab, uint32_t* sNT) {
    for (int e = threadIdx.x; e < ntab * kNibbleWords; e += blockDim.x) {
        const int d = e / kNibbleWords, k = (e / 16) & 7, v = e & 15;
        const uint32_t* vd = V + d * 32 + 4 * k;
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if ((v >> j) & 1) x ^= __ldg(vd + j);
        sNT[e] = x;
    }
}

// the shared-memory tables of a point set: Sobol nibble tables built from the direction numbers,
// or the Halton tables copied as they are (tab: the problem's point table, ntab x 32 Sobol
// direction numbers or ntab x kNibbleWords Halton words)
__device__ __forceinline__ void build_point_tables(const uint32_t* __restrict__ tab, int ntab, uint32_t* sNT,
                                                   int sampler) {
    if (sampler == HYB_HALTON) {
        for (int e = threadIdx.x; e < ntab * kNibbleWords; e += blockDim.x) sNT[e] = __ldg(tab + e);
    } else if (sampler == HYB_SOBOL_DS) {
        build_nibble_tables(tab, ntab, sNT);
    }
}

// ---------------------------------------------------------------------------------------------
// Halton coordinates. Dimension d uses the d-th prime b; the radical inverse phi_b(i) is formed in
// base B = b^m (the largest power of b up to 256, so m base-b digits per chunk): with i's base-B
// chunks c_0 (least significant) .. c_{J-1} and C_j = c_j with its m base-b digits reversed,
// phi = (C_0 + (C_1 + ... (C_{J-1})/B ...)/B)/B. The 32-bit value floor(2^32 phi) is built from the
// innermost chunk outwards, u <- floor((C 2^32 + u) / B): the fraction dropped at each level is
// below one and cannot change a later floor, so the result is exact. Divisions by B use the
// direct-computation method of Lemire, Kaser and Kurz (2019): n / B = floor(c n / 2^64) for all
// 32-bit n with c = ceil(2^64 / B).
// Per-dimension table (kNibbleWords words): [0] b, [1] B, [2] m, [3] floor(2^32 / B),
// [4] 2^32 mod B, [5..6] c (low, high), [7] bits per packed chunk, then the chunk reversal as
// bytes (m > 1 only).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t div_direct(uint32_t c_lo, uint32_t c_hi, uint32_t n) {
    return (uint32_t)(((unsigned long long)c_hi * n + __umulhi(c_lo, n)) >> 32);
}

// Cell index k -> (ix, iy) for a mesh nx wide, without an integer division: iy = k / nx by the
// same direct computation (c = ceil(2^64 / nx), exact for every 32-bit k); nx = 1 (c would not
// fit in 64 bits) is the identity.
struct CellSplit {
    uint32_t c_lo, c_hi;
    int nx;
    __device__ __forceinline__ void operator()(int k, int* ix, int* iy) const {
        const uint32_t q = nx == 1 ? (uint32_t)k : div_direct(c_lo, c_hi, (uint32_t)k);
        *iy = (int)q;
        *ix = k - (int)q * nx;
    }
};

inline CellSplit make_cell_split(int nx) {
    CellSplit s;
    s.nx = nx;
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned long long c = nx > 1 ? (unsigned long long)((two64 + (unsigned)nx - 1) / (unsigned)nx) : 0ull;
    s.c_lo = (uint32_t)c;
    s.c_hi = (uint32_t)(c >> 32);
    return s;
}

__device__ __forceinline__ uint32_t halton_u(const uint32_t* t, uint32_t i) {
    if (t[0] == 2u) return __brev(i);   // base 2: the bit reversal is floor(2^32 phi_2(i))
    const uint32_t B = t[1], QB = t[3], RB = t[4], c_lo = t[5], c_hi = t[6], fb = t[7];
    const bool rev = t[2] > 1u;
    const unsigned char* rv = reinterpret_cast<const unsigned char*>(t + 8);
    unsigned long long pk = 0;   // chunks, least significant first, fb bits each
    int J = 0;
    for (uint32_t n = i; n != 0u; ++J) {
        const uint32_t q = div_direct(c_lo, c_hi, n);
        pk |= (unsigned long long)(n - q * B) << (fb * J);
        n = q;
    }
    const uint32_t mask = (1u << fb) - 1u;
    uint32_t u = 0;
    for (int j = J - 1; j >= 0; --j) {
        uint32_t C = (uint32_t)(pk >> (fb * j)) & mask;
        if (rev) C = rv[C];
        // floor((C 2^32 + u) / B) with 2^32 = QB B + RB and u = uq B + ur
        const uint32_t uq = div_direct(c_lo, c_hi, u), ur = u - uq * B;
        u = C * QB + uq + div_direct(c_lo, c_hi, C * RB + ur);
    }
    return u;
}

// A point set in shared memory: per-dimension tables of ntab dims (Sobol nibble tables or Halton
// tables) and per-dimension shifts; dimensions beyond the table (or sampler == PRNG) use the
// counter hash.
struct Points {
    const uint32_t* NT;
    const uint32_t* shift;
    uint64_t key;
    int sampler;
    int ntab;
    __device__ __forceinline__ uint32_t operator()(uint32_t i, int d) const {
        if (sampler == HYB_SOBOL_DS && d < ntab) {
            const uint32_t* t = NT + d * kNibbleWords;
            uint32_t x = shift[d];
#pragma unroll
            for (int k = 0; k < 6; ++k) x ^= t[16 * k + ((i >> (4 * k)) & 15u)];
            if (i >> 24) {
                x ^= t[96 + ((i >> 24) & 15u)];
                x ^= t[112 + (i >> 28)];
            }
            return x;
        }
        if (sampler == HYB_HALTON && d < ntab) return halton_u(NT + d * kNibbleWords, i) + shift[d];
        const uint64_t h = dmix64(key ^ ((uint64_t)i + kGamma));
        return (uint32_t)(dmix64(h ^ ((uint64_t)d + kGamma)) >> 32);
    }
};

// Sobol byte tables: for dimension d < kByteDims and byte k of the index, entry v is the XOR of the
// direction numbers of the set bits of v (bits 8k..8k+7 of the index): a point is four table
// reads (three below 2^24). Consecutive indices differ in their low byte, so a warp's reads of the
// first table hit distinct banks; the other three are broadcasts. The births' dimensions use them.
constexpr int kByteDims = 6;
constexpr int kByteWords = 1024;   // 4 bytes x 256 entries per dimension

// A point set whose first nbt dimensions come from byte tables BT (Sobol with digital shift), the
// rest as in Points (nbt = 0 for the other samplers)
struct PointsB {
    const uint32_t* BT;
    int nbt;
    Points base;
    __device__ __forceinline__ uint32_t operator()(uint32_t i, int d) const {
        if (d < nbt) {
            const uint32_t* t = BT + d * kByteWords;
            return base.shift[d] ^ t[i & 255u] ^ t[256 + ((i >> 8) & 255u)] ^ t[512 + ((i >> 16) & 255u)] ^
                   t[768 + (i >> 24)];
        }
        return base(i, d);
    }
};

// copies the byte tables of nbt dimensions (global, nbt x kByteWords words) into sBT; all threads
// of the block call it, the caller synchronises
__device__ __forceinline__ void copy_byte_tables(const uint32_t* __restrict__ bt, int nbt, uint32_t* sBT) {
    const uint4* src = reinterpret_cast<const uint4*>(bt);
    uint4* dst = reinterpret_cast<uint4*>(sBT);
    for (int e = threadIdx.x; e < nbt * kByteWords / 4; e += blockDim.x) dst[e] = __ldg(src + e);
}

// ---------------------------------------------------------------------------------------------
// Integer <-> float conversions on the integer pipe. The conversion instructions count against
// the FP64 pipe on this GPU (a small fraction of the FP32 rate; measured as FP64-pipe activity in
// FP32-only kernels), so the FP32 path composes the values from IEEE-754 fields instead.
// ---------------------------------------------------------------------------------------------
// float -> int64, rounding to nearest, ties to even (|x| < 2^63; equals __float2ll_rn there)
__device__ __forceinline__ long long f2ll_rn(float x) {
    const uint32_t u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xFFu);
    const uint32_t m = (u & 0x7FFFFFu) | 0x800000u;
    int sh = e - 150;                       // x = +-m 2^sh for normal x
    long long v = 0;
    if (sh >= 0) {
        sh = sh > 39 ? 39 : sh;             // |x| < 2^63 keeps sh <= 39
        v = (long long)((unsigned long long)m << sh);
    } else if (sh >= -24) {
        const int r = -sh;                  // 1..24 fraction bits
        const uint32_t q = m >> r, rem = m & ((1u << r) - 1u), half = 1u << (r - 1);
        v = (long long)(q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u));
    }                                       // else |x| < 1/2 (or 0, subnormal): 0
    return (u >> 31) ? -v : v;
}

// uint32 -> float rounded toward zero (equals __uint2float_rz): the leading bit gives the
// exponent, the next 23 bits the fraction
__device__ __forceinline__ float u32_to_f_rz(uint32_t x) {
    if (x == 0u) return 0.0f;
    const int p = 31 - __clz(x);                              // leading bit
    const uint32_t m = p >= 23 ? (x >> (p - 23)) : (x << (23 - p));
    return __uint_as_float(((uint32_t)(127 + p) << 23) | (m & 0x7FFFFFu));
}

// uint64 -> float rounded toward zero (within 1 ulp)
__device__ __forceinline__ float u64_to_f(unsigned long long x) {
    if (x == 0ull) return 0.0f;
    const int p = 63 - __clzll(x);
    const uint32_t m = p >= 23 ? (uint32_t)(x >> (p - 23)) : (uint32_t)(x << (23 - p));
    return __uint_as_float(((uint32_t)(127 + p) << 23) | (m & 0x7FFFFFu));
}

// ---------------------------------------------------------------------------------------------
// precision traits: FP32 path (int64 fixed point), FP64 path (128-bit fixed point)
// ---------------------------------------------------------------------------------------------
template <typename T> struct Prec;

template <> struct Prec<float> {
    using acc_t = unsigned long long;
    static constexpr int kbits = 61;
    // u in (0,1): x 2^-32 + 2^-33 with x rounded toward zero to 24 bits, so u keeps 2^-24
    // relative precision near 0 (-log u stays accurate) and never rounds up to 1
    static __device__ __forceinline__ float unit(uint32_t x) { return fmaf(u32_to_f_rz(x), 0x1p-32f, 0x1p-33f); }
    // 1 - u with the same relative precision: the complement ~x maps to 1 - u exactly
    static __device__ __forceinline__ float unit_c(uint32_t x) { return unit(~x); }
    static __device__ __forceinline__ float neglog(float u) { return -logf(u); }
    static __device__ __forceinline__ float ex(float x) { return expf(x); }
    static __device__ __forceinline__ float exm1(float x) { return expm1f(x); }
    // e = e^{-x} and att = 1 - e^{-x} for x = sigma l >= 0 in one evaluation: below x = 1/4 the
    // Taylor series of 1 - e^{-x} in nested form (nine terms, truncation below 1e-10 relative),
    // above it the hardware exponential (relative error ~1e-7 for the x of a few mean free paths
    // that carry weight)
    static __device__ __forceinline__ void att_e(float x, float* att, float* e) {
        if (x < 0.25f) {
            float s = 1.0f - x * (1.0f / 9.0f);
            s = 1.0f - x * (1.0f / 8.0f) * s;
            s = 1.0f - x * (1.0f / 7.0f) * s;
            s = 1.0f - x * (1.0f / 6.0f) * s;
            s = 1.0f - x * (1.0f / 5.0f) * s;
            s = 1.0f - x * (1.0f / 4.0f) * s;
            s = 1.0f - x * (1.0f / 3.0f) * s;
            s = 1.0f - x * 0.5f * s;
            *att = x * s;
            *e = 1.0f - *att;
        } else {
            *e = __expf(-x);
            *att = 1.0f - *e;
        }
    }
    // reciprocal of a flight direction component (used for face distances on the FP32 path)
    static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
    static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    // exact-order a*b + c (FP32 path: contraction allowed)
    static __device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float msub(float c, float a, float b) { return fmaf(-a, b, c); }
    // a*b + c with one rounding, spelled out so every inlined copy evaluates it the same way
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
    // returns the number of global additions issued (0 or 1)
    static __device__ __forceinline__ int add(acc_t* p, float c, float scale) {
        const long long v = f2ll_rn(c * scale);
        if (v) atomicAdd(p, (unsigned long long)v);
        return v != 0;
    }
    static __device__ __forceinline__ double to_double(const acc_t* p, double inv_scale) {
        return (double)(long long)(*p) * inv_scale;
    }
    // the sum of n copies stride apart, exact (int64 two's complement), as a double
    static __device__ __forceinline__ double sum_to_double(const acc_t* p, size_t stride, int n, double inv_scale) {
        unsigned long long v = 0;
        for (int c = 0; c < n; ++c) v += p[c * stride];
        return (double)(long long)v * inv_scale;
    }
    static constexpr int kSeries = 11;
};

__device__ __forceinline__ void to_i128(double v, unsigned long long* lo, unsigned long long* hi) {
    const bool neg = v < 0.0;
    const double a = fabs(v);
    const double h = floor(a * 0x1p-64);
    unsigned long long H = (unsigned long long)h;
    unsigned long long L = __double2ull_rn(a - h * 0x1p64);
    if (neg) {
        L = ~L + 1ull;
        H = ~H + (L == 0ull ? 1ull : 0ull);
    }
    *lo = L;
    *hi = H;
}

// returns the number of global additions issued (0 to 2)
__device__ __forceinline__ int atomic_add128(Acc128* p, unsigned long long lo, unsigned long long hi) {
    if (lo) {
        const unsigned long long old = atomicAdd(&p->lo, lo);
        if (old + lo < old) hi += 1ull;
    }
    if (hi) atomicAdd(&p->hi, hi);
    return (lo != 0ull) + (hi != 0ull);
}

__host__ __device__ __forceinline__ double acc128_to_double(unsigned long long lo, unsigned long long hi,
                                                            double inv_scale) {
    const bool neg = (hi >> 63) != 0ull;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const double v = ((double)hi * 0x1p64 + (double)lo) * inv_scale;
    return neg ? -v : v;
}

// FP64 direction and optical-depth maps by explicit series in separately rounded operations, so the
// FP64 geometry is reproducible bit for bit by any implementation of the same recipe:
//   sin/cos(2 pi u): q = rint(4u), r = u - q/4 (exact), a = 2 pi r, Taylor series to a^17 / a^18
//   (coefficients 1/n! from exact factorials), quadrant rotation by q mod 4;
//   -log u: u = m 2^e, m in [1/sqrt2, sqrt2), log m = 2 s sum_k s^2k/(2k+1), s = (m-1)/(m+1).
__device__ __forceinline__ void sincos_2pi_series(double u, double* s_out, double* c_out) {
    const double q = rint(4.0 * u);
    const double r = __dsub_rn(u, __dmul_rn(0.25, q));
    const double a = __dmul_rn(6.283185307179586, r);
    const double a2 = __dmul_rn(a, a);
    constexpr double ks[9] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0,
                              1.0 / 6227020800.0, -1.0 / 1307674368000.0, 1.0 / 355687428096000.0};
    constexpr double kc[10] = {1.0, -1.0 / 2.0, 1.0 / 24.0, -1.0 / 720.0, 1.0 / 40320.0, -1.0 / 3628800.0,
                               1.0 / 479001600.0, -1.0 / 87178291200.0, 1.0 / 20922789888000.0,
                               -1.0 / 6402373705728000.0};
    double S = ks[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) S = __dadd_rn(__dmul_rn(S, a2), ks[k]);
    double Cc = kc[9];
#pragma unroll
    for (int k = 8; k >= 0; --k) Cc = __dadd_rn(__dmul_rn(Cc, a2), kc[k]);
    const double sa = __dmul_rn(a, S), ca = Cc;
    switch (((int)q) & 3) {
        case 0: *s_out = sa; *c_out = ca; break;
        case 1: *s_out = ca; *c_out = -sa; break;
        case 2: *s_out = -sa; *c_out = -ca; break;
        default: *s_out = -ca; *c_out = sa; break;
    }
}

__device__ __forceinline__ double neg_log_series(double u) {
    int e = 0;
    double m = frexp(u, &e);
    if (m < 0.7071067811865476) { m = 2.0 * m; e -= 1; }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double s2 = __dmul_rn(s, s);
    constexpr double kl[12] = {1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0, 1.0 / 9.0, 1.0 / 11.0,
                               1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0, 1.0 / 23.0};
    double P = kl[11];
#pragma unroll
    for (int k = 10; k >= 0; --k) P = __dadd_rn(__dmul_rn(P, s2), kl[k]);
    const double lm = __dmul_rn(__dmul_rn(2.0, s), P);
    return -__dadd_rn(__dmul_rn((double)e, 0.6931471805599453), lm);
}

template <> struct Prec<double> {
    using acc_t = Acc128;
    static constexpr int kbits = 125;
    static __device__ __forceinline__ double unit(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }
    static __device__ __forceinline__ double unit_c(uint32_t x) { return 1.0 - unit(x); }   // exact in FP64
    static __device__ __forceinline__ double neglog(double u) { return neg_log_series(u); }
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double exm1(double x) { return expm1(x); }
    static __device__ __forceinline__ void att_e(double x, double* att, double* e) {
        *att = -expm1(-x);
        *e = exp(-x);
    }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincos_2pi_series(u, s, c); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    // separately rounded product and sum: FP64 geometry follows IEEE order exactly
    static __device__ __forceinline__ double madd(double a, double b, double c) { return __dadd_rn(__dmul_rn(a, b), c); }
    static __device__ __forceinline__ double msub(double c, double a, double b) { return __dsub_rn(c, __dmul_rn(a, b)); }
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
    static __device__ __forceinline__ int add(acc_t* p, double c, double scale) {
        unsigned long long lo, hi;
        to_i128(c * scale, &lo, &hi);
        return atomic_add128(p, lo, hi);
    }
    static __device__ __forceinline__ double to_double(const acc_t* p, double inv_scale) {
        return acc128_to_double(p->lo, p->hi, inv_scale);
    }
    // the sum of n copies stride apart, exact (128-bit two's complement), as a double
    static __device__ __forceinline__ double sum_to_double(const acc_t* p, size_t stride, int n, double inv_scale) {
        unsigned long long lo = 0, hi = 0;
        for (int c = 0; c < n; ++c) {
            const acc_t v = p[c * stride];
            const unsigned long long nl = lo + v.lo;
            hi += v.hi + (nl < lo ? 1ull : 0ull);
            lo = nl;
        }
        return acc128_to_double(lo, hi, inv_scale);
    }
    static constexpr int kSeries = 19;
};

// scale 2^(kbits - ceil(log2 B)) so that sums bounded by B fit the accumulator; 0 if B == 0
__host__ __device__ __forceinline__ int scale_exponent(double B, int kbits) {
    if (!(B > 0.0)) return 0;
    int e = 0;
    const double m = frexp(B, &e);
    const int cl = (m == 0.5) ? e - 1 : e;
    int k = kbits - cl;
    if (k > 1000) k = 1000;
    return k;
}

// ---------------------------------------------------------------------------------------------
// g_n(x) = int_0^1 t^n e^{-x t} dt, n = 0,1,2: series below x = 1, closed form above
// ---------------------------------------------------------------------------------------------
// coefficient of x^k in g_n(x) = int_0^1 t^n e^{-x t} dt = sum_k (-x)^k / (k! (n + k + 1))
__host__ __device__ constexpr double gcoef(int n, int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return ((k & 1) ? -1.0 : 1.0) / (f * (double)(n + k + 1));
}

// Horner steps k = K, K-1, ..., 0 for g_0, g_1, g_2 together (coefficients fixed at compile time)
template <typename T, int K>
struct GHorner {
    static __device__ __forceinline__ void run(T x, T* s0, T* s1, T* s2) {
        constexpr double c0 = gcoef(0, K), c1 = gcoef(1, K), c2 = gcoef(2, K);
        *s0 = Prec<T>::fma_(*s0, x, T(c0));
        *s1 = Prec<T>::fma_(*s1, x, T(c1));
        *s2 = Prec<T>::fma_(*s2, x, T(c2));
        GHorner<T, K - 1>::run(x, s0, s1, s2);
    }
};
template <typename T>
struct GHorner<T, -1> {
    static __device__ __forceinline__ void run(T, T*, T*, T*) {}
};

// g_0, g_1, g_2 at x = sigma l >= 0, given e = e^{-x} and att = 1 - e^{-x} of the same x:
// the power series (Horner, kSeries terms) below x = 1, the closed forms above
template <typename T>
__device__ __forceinline__ void gfun(T x, T e, T att, T* g0, T* g1, T* g2) {
    if (x < T(1)) {
        constexpr int K = Prec<T>::kSeries - 1;
        T s0 = T(gcoef(0, K)), s1 = T(gcoef(1, K)), s2 = T(gcoef(2, K));
        GHorner<T, K - 1>::run(x, &s0, &s1, &s2);
        *g0 = s0; *g1 = s1; *g2 = s2;
    } else if (sizeof(T) == 4) {
        const T rx = T(1) / x;
        *g0 = att * rx;
        *g1 = (*g0 - e) * rx;
        *g2 = Prec<T>::fma_(T(2), *g1, -e) * rx;
    } else {
        *g0 = att / x;
        *g1 = (*g0 - e) / x;
        *g2 = Prec<T>::fma_(T(2), *g1, -e) / x;
    }
}

// isotropic direction from two point integers: mu = 2u - 1, phi = 2 pi u'; returns the in-plane
// components, sin(theta) = 2 sqrt(u (1 - u)) with 1 - u formed without cancellation
template <typename T>
__device__ __forceinline__ void iso_dir(uint32_t x_mu, uint32_t x_phi, T* ox, T* oy) {
    const T st = T(2) * Prec<T>::sqrt_(Prec<T>::unit(x_mu) * Prec<T>::unit_c(x_mu));
    T s, c;
    Prec<T>::sincos2pi(Prec<T>::unit(x_phi), &s, &c);
    *ox = st * c;
    *oy = st * s;
}

// ---------------------------------------------------------------------------------------------
// integer CDF pick: bin j of pre[0..n] with pre[j] 2^33 <= (2x+1) total < pre[j+1] 2^33, searched
// in [lo, hi] (which must hold it); a, b: the remainder split as rem = a 2^33 + b; W: the bin weight.
// With P = (2x+1) total < 2^95 and Tx = floor(P / 2^33) < 2^62, pre[j] 2^33 <= P is pre[j] <= Tx
// (pre[j] an integer), so the search compares 64-bit integers, and rem = (Tx - pre[j]) 2^33 +
// (P mod 2^33): a = Tx - pre[j], b = P mod 2^33.
__device__ __forceinline__ int pick_bin(const long long* __restrict__ pre, int n, uint32_t x, int lo, int hi,
                                        unsigned long long* a, unsigned long long* b, unsigned long long* W) {
    const unsigned long long total = (unsigned long long)pre[n];
    const unsigned long long m = 2ull * (unsigned long long)x + 1ull;
    const unsigned long long Plo = m * total, Phi = __umul64hi(m, total);
    const unsigned long long Tx = (Phi << 31) | (Plo >> 33);
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)pre[mid] <= Tx) lo = mid; else hi = mid - 1;
    }
    const unsigned long long v = (unsigned long long)pre[lo];
    *a = Tx - v;
    *b = Plo & ((1ull << 33) - 1ull);
    *W = (unsigned long long)pre[lo + 1] - v;
    return lo;
}

// the search range of point x from a guide table of 2^g buckets (the whole range without one)
__device__ __forceinline__ void guide_range(const int* guide, int g, int n, uint32_t x, int* lo, int* hi) {
    if (guide) {
        const uint32_t bkt = g ? (x >> (32 - g)) : 0u;
        *lo = __ldg(guide + bkt);
        *hi = __ldg(guide + bkt + 1);
    } else {
        *lo = 0;
        *hi = n - 1;
    }
}

template <typename T>
__device__ __forceinline__ T bin_frac(unsigned long long a, unsigned long long b, unsigned long long W) {
    return (T)(((double)a + (double)b * 0x1p-33) / (double)W);
}

template <>
__device__ __forceinline__ float bin_frac<float>(unsigned long long a, unsigned long long b, unsigned long long W) {
    return fmaf(u64_to_f(b), 0x1p-33f, u64_to_f(a)) / u64_to_f(W);
}

// cell and in-cell fractions from the 2-D CDF: row from x1, column within the row from x0
template <typename T>
__device__ __forceinline__ int sample_cell(const Cdf2DView& C, int nx, int ny, uint32_t x0, uint32_t x1,
                                           T* frx, T* fry) {
    unsigned long long a, b, W;
    int lo, hi;
    guide_range(C.row_g, C.gr, ny, x1, &lo, &hi);
    const int iy = pick_bin(C.row_pre, ny, x1, lo, hi, &a, &b, &W);
    *fry = bin_frac<T>(a, b, W);
    guide_range(C.col_g ? C.col_g + (size_t)iy * ((1 << C.gc) + 1) : nullptr, C.gc, nx, x0, &lo, &hi);
    const int ix = pick_bin(C.col_pre + (size_t)iy * (nx + 1), nx, x0, lo, hi, &a, &b, &W);
    *frx = bin_frac<T>(a, b, W);
    return iy * nx + ix;
}

template <typename T>
__device__ __forceinline__ T clamp_(T v, T lo, T hi) { return v < lo ? lo : (v > hi ? hi : v); }

// deterministic block reduction of a double (fixed tree order for a fixed block size)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace hyb
