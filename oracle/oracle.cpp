// oracle.cpp -- TEST INFRASTRUCTURE ONLY: the parity oracle for the scatter-limited
// hybrid (Q)MC / S_N method of Krotz & McClarren, "Scatter-Limited Hybrid Monte Carlo,
// Deterministic Transport with Quasi-Monte Carlo Sampling" (PHYSOR 2026).
//
// Plain, slow, single-threaded FP64 C++. It shares no code, header, table or constant
// generator with the CUDA library: only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / --impl reference legs may load it. Each function cites the passage of the
// paper it restates; where the paper is silent the reading taken is stated in the comment.
//
// Paper map:
//   Sec. 2.1, Eq. (1)          transport equation, isotropic kernel S[Psi] = <Psi>/4pi - Psi
//   Sec. 2.2, Eq. (n-split)    n-collision fluxes; Eq. (ceil N_s)/(floor N_s+1) the N_s split
//   Sec. 2.2, steps 1-4        one hybrid time step: MC leg, collided S_N solve, remap, census
//   Sec. 2.2, Eq. (R)          scatter-free remap with the full scattering source
//   Sec. 2.3                   implicit capture, pre/post-limit legs, two track-length tallies
//   Sec. 2.4                   QMC: low-discrepancy points inside the same inverse-CDF maps
//   App. B                     Erlang law of the (N_s+1)-th scatter time (used as a test pin)
//
// Units: Q is the angle-integrated emission rate density (particles / area / time), so one
// step emits Q*A*dt per cell. phi = int Psi dOmega; a track-length sum T = sum w*l over a cell
// and a step equals the space-time integral of phi, so the step-average flux is T/(A*dt).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <algorithm>
#include <limits>

namespace {

// ------------------------------------------------------------------------------------------
// Constants of this restatement
// ------------------------------------------------------------------------------------------
constexpr int kDimMax = 65;               // Sobol dimensions tabulated (5 + 3*20)
constexpr int kStreamInit = 0;            // initial-condition particles
constexpr int kStreamLegCensus = 1;       // MC leg, particles picked up from the census bank
constexpr int kStreamLegSource = 2;       // MC leg, particles born from Q
constexpr int kStreamRemapSource = 3;     // remap, particles born from the remap source
constexpr int kStreamRemapComb = 4;       // remap, offset of the census comb
constexpr int32_t kNsInf = 2147483647;    // N_s = infinity (pure (Q)MC, no remap)
constexpr int64_t kMaxSegments = 1 << 20; // bound on segments per history
constexpr int kFateLeaked = 0, kFateCensus = 1, kFateKilled = 2, kFateError = 3;
const double kInf = std::numeric_limits<double>::infinity();
const double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------------------------------
// Counter-based hashing: the splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014).
// ------------------------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Key of one point set: (seed, step, stream).
uint64_t stream_key(uint64_t seed, uint64_t step, uint64_t stream) {
    uint64_t z = mix64(seed + kGamma);
    z = mix64(z ^ (step + kGamma));
    z = mix64(z ^ (stream + kGamma));
    return z;
}

// Digital shift of dimension d (top 32 bits of one more hash round).
uint32_t digital_shift(uint64_t key, uint64_t d) {
    return (uint32_t)(mix64(key ^ (d + kGamma)) >> 32);
}

// Pseudorandom 32-bit integer for (history i, dimension d).
uint32_t prng_int(uint64_t key, uint64_t i, uint64_t d) {
    uint64_t h = mix64(key ^ (i + kGamma));
    return (uint32_t)(mix64(h ^ (d + kGamma)) >> 32);
}

// ------------------------------------------------------------------------------------------
// Sobol direction numbers, generated here (no published table is used).
//   dim 0: van der Corput, V_b = 2^(31-b).
//   dim d>=1: the d-th primitive polynomial over GF(2), in increasing (degree, value) order,
//   found by brute force (x has multiplicative order 2^s - 1 modulo p). Initial numbers m_j
//   (odd, < 2^j) chosen one at a time, j = 1..s: the value for which the fewest earlier
//   dimensions d' fail the (0, j, 2)-net test of the pair (d', d) on the first 2^j points;
//   ties go to the smallest m_j. Later numbers by the Bratley-Fox recurrence.
// ------------------------------------------------------------------------------------------
uint32_t g_V[kDimMax][32];
bool g_V_ready = false;

int poly_degree(uint32_t p) { int s = 0; while ((p >> (s + 1)) != 0) ++s; return s; }

bool is_primitive(uint32_t p, int s) {
    // order of x modulo p must be exactly 2^s - 1
    uint32_t r = 1, period = (1u << s) - 1;
    for (uint32_t k = 1; k <= period; ++k) {
        r <<= 1;
        if ((r >> s) & 1u) r ^= p;
        if (r == 1u) return k == period;
    }
    return false;
}

// generator-matrix entry: row r (bit 31-r of V), column b (bit b of the index)
inline int gen_bit(const uint32_t* V, int r, int b) { return (int)((V[b] >> (31 - r)) & 1u); }

// rank over GF(2) of rows given as bit masks
int gf2_rank(std::vector<uint64_t> rows, int ncols) {
    int rank = 0;
    for (int c = 0; c < ncols && rank < (int)rows.size(); ++c) {
        int piv = -1;
        for (int i = rank; i < (int)rows.size(); ++i) if ((rows[i] >> c) & 1u) { piv = i; break; }
        if (piv < 0) continue;
        std::swap(rows[rank], rows[piv]);
        for (int i = 0; i < (int)rows.size(); ++i)
            if (i != rank && ((rows[i] >> c) & 1u)) rows[i] ^= rows[rank];
        ++rank;
    }
    return rank;
}

// (0, m, 2)-net test of the first 2^m points of the pair (A, B): for every split k + (m-k)
// the m x m matrix made of the first k rows of A and the first m-k rows of B (columns 0..m-1)
// must be nonsingular.
bool pair_is_0m2_net(const uint32_t* A, const uint32_t* B, int m) {
    for (int k = 0; k <= m; ++k) {
        std::vector<uint64_t> rows;
        for (int r = 0; r < k; ++r) {
            uint64_t mask = 0;
            for (int c = 0; c < m; ++c) mask |= (uint64_t)gen_bit(A, r, c) << c;
            rows.push_back(mask);
        }
        for (int r = 0; r < m - k; ++r) {
            uint64_t mask = 0;
            for (int c = 0; c < m; ++c) mask |= (uint64_t)gen_bit(B, r, c) << c;
            rows.push_back(mask);
        }
        if (gf2_rank(rows, m) < m) return false;
    }
    return true;
}

void direction_numbers(uint32_t poly, int s, const std::vector<uint32_t>& m, uint32_t* V) {
    for (int j = 1; j <= s; ++j) V[j - 1] = m[j - 1] << (32 - j);
    for (int j = s + 1; j <= 32; ++j) {
        uint32_t x = V[j - s - 1] ^ (V[j - s - 1] >> s);
        for (int k = 1; k < s; ++k)
            if ((poly >> (s - k)) & 1u) x ^= V[j - k - 1];
        V[j - 1] = x;
    }
}

void build_sobol_table() {
    if (g_V_ready) return;
    for (int b = 0; b < 32; ++b) g_V[0][b] = 1u << (31 - b);
    int d = 1;
    for (int s = 1; d < kDimMax; ++s) {
        for (uint32_t p = (1u << s) | 1u; p < (1u << (s + 1)) && d < kDimMax; p += 2) {
            if (!is_primitive(p, s)) continue;
            std::vector<uint32_t> m;
            for (int j = 1; j <= s; ++j) {
                uint32_t best_m = 1; int best_fail = 1 << 30;
                for (uint32_t cand = 1; cand < (1u << j); cand += 2) {
                    std::vector<uint32_t> trial = m;
                    trial.push_back(cand);
                    while ((int)trial.size() < s) trial.push_back(1);
                    uint32_t V[32];
                    direction_numbers(p, s, trial, V);
                    int fails = 0;
                    for (int e = 0; e < d; ++e) fails += pair_is_0m2_net(g_V[e], V, j) ? 0 : 1;
                    if (fails < best_fail) { best_fail = fails; best_m = cand; }
                }
                m.push_back(best_m);
            }
            direction_numbers(p, s, m, g_V[d]);
            ++d;
        }
    }
    g_V_ready = true;
}

uint32_t sobol_int(int d, uint64_t i) {
    uint32_t x = 0;
    for (int b = 0; b < 32; ++b)
        if ((i >> b) & 1u) x ^= g_V[d][b];
    return x;
}

// ------------------------------------------------------------------------------------------
// Halton points (the paper's QMC, Sec. 2.4). Coordinate d of point i is the radical inverse of
// i in the d-th prime base b: for i = sum_k a_k b^k (digits 0 <= a_k < b, K of them),
// phi_b(i) = sum_k a_k b^-(k+1) = R / b^K with R the digits read in reverse. It is kept as the
// 32-bit fixed-point value floor(2^32 phi_b(i)), formed exactly in 128-bit integers. A replica
// is randomised by a shift modulo 1 (Cranley & Patterson 1976) of that value by the same
// per-(key, dimension) 32-bit hash the Sobol sets use as their digital shift.
// ------------------------------------------------------------------------------------------
uint32_t g_prime[kDimMax];
bool g_prime_ready = false;

void build_primes() {
    if (g_prime_ready) return;
    int n = 0;
    for (uint32_t c = 2; n < kDimMax; ++c) {
        bool prime = true;
        for (uint32_t q = 2; q * q <= c; ++q)
            if (c % q == 0) { prime = false; break; }
        if (prime) g_prime[n++] = c;
    }
    g_prime_ready = true;
}

uint32_t halton_int(int d, uint64_t i) {
    const uint64_t b = g_prime[d];
    unsigned __int128 R = 0, D = 1;
    for (uint64_t n = i; n > 0; n /= b) {
        R = R * b + n % b;
        D *= b;
    }
    return (uint32_t)((R << 32) / D);
}

// One point coordinate as a 32-bit integer (Sec. 2.4: the low-discrepancy points replace the
// pseudorandom draws inside the same maps). Sobol + digital shift, Halton + shift modulo 1, or
// the counter PRNG. Dimensions beyond the tables fall back to the counter PRNG.
struct Points {
    uint64_t key; int sampler;
    uint32_t operator()(uint64_t i, int d) const {
        if (sampler == 0 && d < kDimMax) return sobol_int(d, i) ^ digital_shift(key, (uint64_t)d);
        if (sampler == 2 && d < kDimMax) return halton_int(d, i) + digital_shift(key, (uint64_t)d);
        return prng_int(key, i, (uint64_t)d);
    }
};

// u in (0,1): (x + 1/2) 2^-32, exact in FP64
inline double unit(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

// ------------------------------------------------------------------------------------------
// Problem, bank, statistics (oracle-side layouts)
// ------------------------------------------------------------------------------------------
}  // namespace

extern "C" {

typedef struct {
    int32_t nx, ny;
    double lx, ly;
    const double* sigma_a;  // nx*ny, idx = iy*nx + ix
    const double* sigma_s;
    const double* Q;        // nx*ny emission rate density, may be NULL
    double c, dt;
    int32_t n_s;            // N_s, kNsInf = unlimited
    int32_t sampler;        // 0 Sobol + digital shift, 1 counter PRNG, 2 Halton + shift modulo 1
    int64_t n_hist;         // births per step (MC-leg source and remap source)
    uint64_t seed;
    int32_t sn_order;       // 4 or 8
    int32_t handoff_full;   // 1: four Legendre moments, 0: moment 0 only
    double w_min;           // relative kill threshold (0 = never)
    int64_t census_cap;     // 0 = n_hist
    double sn_tol;          // source-iteration relative-change tolerance
    int32_t sn_max_iter;
    int32_t census_order;   // 0: slot order (bank slots, then births); 1: stable by cell; 2: by cell, then
                            // phase space (Morton order of in-cell x, y and direction angle)
    int32_t remap_variant;  // 0: Eq. (R) relabelling remap; 1: steps 3'/4' (additive, previous hybrids)
    const int32_t* n_s_cell;  // nx*ny scatter limits per cell in [0, n_s] (space-dependent N_s), or NULL
    int32_t elem;             // evaluation of sin/cos(2 pi u) and -log u: 0 host libm, 1 explicit series
    int32_t sort_every;       // census_order >= 1 applies on the steps n with n mod sort_every == 0 (0, 1: all)
} or_problem;

typedef struct {
    int64_t n, cap;
    int32_t* cell;
    double *fx, *fy, *ox, *oy, *w;
} or_bank;

typedef struct {
    int64_t histories, segments, collisions, leaked, census, killed, reached_limit, errors;
    double w_source, w_absorbed, w_leaked, w_census, w_handoff, w_killed;
    int32_t sn_iterations, pad;
} or_stats;

}  // extern "C"

namespace {

struct Mesh {
    int nx, ny; double dx, dy, area;
    explicit Mesh(const or_problem* P)
        : nx(P->nx), ny(P->ny), dx(P->lx / P->nx), dy(P->ly / P->ny), area(0.0) {
        area = dx * dy;
    }
};

bool bank_push(or_bank* b, int32_t cell, double fx, double fy, double ox, double oy, double w) {
    if (!b) return true;
    if (b->n >= b->cap) return false;
    int64_t k = b->n++;
    b->cell[k] = cell; b->fx[k] = fx; b->fy[k] = fy; b->ox[k] = ox; b->oy[k] = oy; b->w[k] = w;
    return true;
}

// ------------------------------------------------------------------------------------------
// Integer 2-D CDF over cells (row marginal, then the column conditional within the row).
// Weights are quantised q_k = rint(|w_k| / max|w| * 2^B) with B = min(40, 62 - ceil(log2 ncells)),
// so the total stays below 2^62 on every mesh (B = 40 up to 2^22 cells); a point x (32-bit) selects by the
// exact product (2x+1) * total / 2^33, so selection is exact integer arithmetic and the
// remainder gives the uniform in-cell fraction.
// ------------------------------------------------------------------------------------------
struct Cdf2D {
    int nx = 0, ny = 0;
    std::vector<int64_t> q, row_pre, col_pre;  // row_pre: ny+1; col_pre: ny*(nx+1)
    int64_t total = 0;
};

Cdf2D build_cdf(const Mesh& M, const std::vector<double>& w) {
    Cdf2D C; C.nx = M.nx; C.ny = M.ny;
    double wmax = 0.0;
    for (double v : w) wmax = std::max(wmax, std::fabs(v));
    C.q.assign(w.size(), 0);
    int lg = 0;
    while (((size_t)1 << lg) < w.size()) ++lg;
    const double scale = std::ldexp(1.0, std::min(40, 62 - lg));
    if (wmax > 0.0)
        for (size_t k = 0; k < w.size(); ++k)
            C.q[k] = (int64_t)std::nearbyint((std::fabs(w[k]) / wmax) * scale);
    C.row_pre.assign(M.ny + 1, 0);
    C.col_pre.assign((size_t)M.ny * (M.nx + 1), 0);
    for (int iy = 0; iy < M.ny; ++iy) {
        int64_t acc = 0;
        for (int ix = 0; ix < M.nx; ++ix) {
            C.col_pre[(size_t)iy * (M.nx + 1) + ix] = acc;
            acc += C.q[(size_t)iy * M.nx + ix];
        }
        C.col_pre[(size_t)iy * (M.nx + 1) + M.nx] = acc;
        C.row_pre[iy + 1] = C.row_pre[iy] + acc;
    }
    C.total = C.row_pre[M.ny];
    return C;
}

// Pick the bin j of a prefix array pre[0..n] (pre[n] = total) for the point x and return
// the in-bin fraction in [0,1].
int pick_bin(const int64_t* pre, int n, uint32_t x, double* frac) {
    typedef unsigned __int128 u128;
    u128 total = (u128)(uint64_t)pre[n];
    u128 P = (u128)(2ull * x + 1ull) * total;  // u * total * 2^33
    int lo = 0, hi = n - 1;                    // largest j with pre[j] * 2^33 <= P
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (((u128)(uint64_t)pre[mid] << 33) <= P) lo = mid; else hi = mid - 1;
    }
    u128 rem = P - ((u128)(uint64_t)pre[lo] << 33);
    uint64_t W = (uint64_t)(pre[lo + 1] - pre[lo]);
    uint64_t a = (uint64_t)(rem >> 33);
    uint64_t b = (uint64_t)(rem & ((((u128)1) << 33) - 1));
    *frac = ((double)a + (double)b * 0x1p-33) / (double)W;
    return lo;
}

// Sample a cell and in-cell fractions (fx/dx, fy/dy) from the 2-D CDF with points x0 (column)
// and x1 (row).
int sample_cell(const Cdf2D& C, uint32_t x0, uint32_t x1, double* frac_x, double* frac_y) {
    int iy = pick_bin(C.row_pre.data(), C.ny, x1, frac_y);
    int ix = pick_bin(&C.col_pre[(size_t)iy * (C.nx + 1)], C.nx, x0, frac_x);
    return iy * C.nx + ix;
}

// Second evaluation mode (elem = 1) of sin and cos of 2 pi u for a point uniform u, and of -log u:
// explicit series with IEEE operations in a fixed order, so that any implementation written to the
// same recipe gives the same bits (the GPU FP64 path evaluates the maps this way; comparing it with
// this mode checks the rest of its arithmetic bit for bit, comparing it with the libm mode shows
// how often a last-bit difference in a direction or optical depth changes a decision):
//   2 pi u = 2 pi r + q pi/2 with q = rint(4u), r = u - q/4 in [-1/8, 1/8] (both exact), Taylor
//   series of sin and cos of a = 2 pi r to a^17 / a^18, then the quadrant rotation;
//   u = m 2^e with m in [1/sqrt2, sqrt2), log m = 2 atanh(s), s = (m-1)/(m+1), series to s^23.
struct SeriesCoef {
    double sinc[9], cosc[10], logc[12];
    SeriesCoef() {
        double f = 1.0;  // n!, exact in FP64 up to 18!
        for (int n = 1; n <= 18; ++n) {
            f *= n;
            if (n % 2 == 1) sinc[(n - 1) / 2] = (((n - 1) / 2) % 2 ? -1.0 : 1.0) / f;
            else cosc[n / 2] = ((n / 2) % 2 ? -1.0 : 1.0) / f;
        }
        cosc[0] = 1.0;
        for (int k = 0; k < 12; ++k) logc[k] = 1.0 / (2.0 * k + 1.0);
    }
};
const SeriesCoef kSer;

// Which evaluation of the direction and optical-depth maps the current call uses (set from the
// problem's `elem` field at every entry point; the oracle is single-threaded): 0 = the host libm
// (std::sin, std::cos of the rounded product 2 pi u, std::log), the plain reading of Sec. 2.3-2.4;
// 1 = the explicit series below.
int g_elem = 0;

void sincos_2pi_series(double u, double* s_out, double* c_out) {
    const double q = std::nearbyint(4.0 * u);
    const double r = u - 0.25 * q;
    const double a = 6.283185307179586 * r;
    const double a2 = a * a;
    double S = kSer.sinc[8];
    for (int k = 7; k >= 0; --k) S = S * a2 + kSer.sinc[k];
    double Cc = kSer.cosc[9];
    for (int k = 8; k >= 0; --k) Cc = Cc * a2 + kSer.cosc[k];
    const double sa = a * S, ca = Cc;
    switch (((int)q) & 3) {
        case 0: *s_out = sa; *c_out = ca; break;
        case 1: *s_out = ca; *c_out = -sa; break;
        case 2: *s_out = -sa; *c_out = -ca; break;
        default: *s_out = -ca; *c_out = sa; break;
    }
}

double neg_log_series(double u) {
    int e = 0;
    double m = std::frexp(u, &e);
    if (m < 0.7071067811865476) { m = 2.0 * m; e -= 1; }
    const double s = (m - 1.0) / (m + 1.0);
    const double s2 = s * s;
    double P = kSer.logc[11];
    for (int k = 10; k >= 0; --k) P = P * s2 + kSer.logc[k];
    const double lm = 2.0 * s * P;
    return -((double)e * 0.6931471805599453 + lm);
}

void sincos_2pi(double u, double* s_out, double* c_out) {
    if (g_elem == 1) { sincos_2pi_series(u, s_out, c_out); return; }
    const double a = 2.0 * kPi * u;
    *s_out = std::sin(a);
    *c_out = std::cos(a);
}

double neg_log(double u) { return g_elem == 1 ? neg_log_series(u) : -std::log(u); }

// Isotropic direction: mu = 2u - 1, phi = 2 pi u'; the 2-D motion uses (Omega_x, Omega_y) and
// the path length is the 3-D one (the domain is extruded in z).
void iso_direction(double u_mu, double u_phi, double* ox, double* oy) {
    double sin_theta = 2.0 * std::sqrt(u_mu * (1.0 - u_mu));
    double sp, cp;
    sincos_2pi(u_phi, &sp, &cp);
    *ox = sin_theta * cp;
    *oy = sin_theta * sp;
}

// g_n(x) = int_0^1 t^n e^{-x t} dt, n = 0, 1, 2 (exact segment integrals of the decaying weight)
void gfun(double x, double* g0, double* g1, double* g2) {
    if (x < 1.0) {
        // series sum_k (-x)^k / (k! (n + k + 1))
        double s0 = 0, s1 = 0, s2 = 0, term = 1.0;
        for (int k = 0; k < 30; ++k) {
            s0 += term / (k + 1); s1 += term / (k + 2); s2 += term / (k + 3);
            term *= -x / (k + 1);
        }
        *g0 = s0; *g1 = s1; *g2 = s2;
    } else {
        double e = std::exp(-x);
        *g0 = -std::expm1(-x) / x;
        *g1 = (*g0 - e) / x;
        *g2 = (2.0 * *g1 - e) / x;
    }
}

// ------------------------------------------------------------------------------------------
// The scatter-limited MC leg, Sec. 2.3 (pseudocode paragraph): one history.
// ------------------------------------------------------------------------------------------
struct Leg {
    const or_problem* P; Mesh M; Points pts;
    std::vector<long double> pre, post, mom;
    std::vector<int64_t> pre_n, post_n;   // segments scored per cell (statistical support of a tally)
    long double w_source = 0, w_absorbed = 0, w_leaked = 0, w_census = 0, w_handoff = 0, w_killed = 0;
    int64_t segments = 0, collisions = 0, leaked = 0, census = 0, killed = 0, reached = 0, errors = 0;
    or_bank* census_out = nullptr;
    bool census_overflow = false;
    explicit Leg(const or_problem* p) : P(p), M(p), pts{0, p->sampler} {
        size_t nc = (size_t)M.nx * M.ny;
        pre.assign(nc, 0); post.assign(nc, 0); mom.assign(nc * 4, 0);
        pre_n.assign(nc, 0); post_n.assign(nc, 0);
    }

    // Track one history from its start state to termination; returns the fate and fills the
    // record (final cell, fate, final scatter count, segments).
    // Space-dependent N_s (the paper's outlook, Sec. 4): a segment in cell k is pre-limit while
    // the history's scatter count n is below N_s(k), post-limit otherwise; the optical depth to the
    // next scatter is kept across post-limit stretches (exponential, so memoryless). Uniform N_s:
    // N_s(k) = n_s everywhere.
    int limit(int k) const { return P->n_s_cell ? P->n_s_cell[k] : P->n_s; }

    // Decision margin of one segment: the event is the smallest of the candidate distances
    // (collision, x face, y face, census); the relative gap (d2 - d1) / d2 between the two smallest
    // says how far the decision is from a tie (0: an exact tie such as a corner; 1: one finite
    // candidate). A last-bit change of a distance can only change a decision whose gap is of the
    // order of the rounding error.
    static double decision_gap(double dcol, double dxf, double dyf, double dcen) {
        double d[4] = {dcol, dxf, dyf, dcen};
        std::sort(d, d + 4);
        if (!(d[1] < kInf)) return 1.0;
        if (d[1] <= 0.0) return 0.0;
        return (d[1] - d[0]) / d[1];
    }

    void run(uint64_t idx, int ix, int iy, double fx, double fy, double ox, double oy,
             double w, double s_rem, int32_t* rec, double* margin = nullptr) {
        double gap = 1.0;
        const int Ns = P->n_s;   // the largest limit: sets the point dimensions
        const double DX = M.dx, DY = M.dy;
        const double w_start = w;
        w_source += w;
        int n = 0;
        if (limit(iy * M.nx + ix) == 0) ++reached;
        double tau = 0.0;
        if (Ns > 0) tau = neg_log(unit(pts(idx, 5)));
        int64_t seg = 0;
        int fate = kFateError;
        while (seg < kMaxSegments) {
            ++seg;
            const int k = iy * M.nx + ix;
            const int Nk = limit(k);
            const double sa = P->sigma_a[k], ss = P->sigma_s[k], st = sa + ss;
            const double dxf = ox > 0 ? (DX - fx) / ox : (ox < 0 ? fx / (-ox) : kInf);
            const double dyf = oy > 0 ? (DY - fy) / oy : (oy < 0 ? fy / (-oy) : kInf);
            const double dcol = (n < Nk && ss > 0) ? tau / ss : kInf;
            const double dcen = s_rem;
            if (margin) gap = std::min(gap, decision_gap(dcol, dxf, dyf, dcen));
            // event: collision wins ties over faces, faces over census
            double l; int ev; bool xc = false, yc = false;
            if (dcol <= dxf && dcol <= dyf && dcol <= dcen) { l = dcol; ev = 0; }
            else if (dxf <= dcen || dyf <= dcen) {
                l = std::min(dxf, dyf); ev = 1; xc = (dxf == l); yc = (dyf == l);
            } else { l = dcen; ev = 2; }

            if (n < Nk) {
                // pre-limit: implicit capture with sigma_a, tally <Psi>_pre
                const double att = -std::expm1(-sa * l);
                pre[k] += (sa > 0) ? (long double)(w * att / sa) : (long double)(w * l);
                ++pre_n[k];
                w_absorbed += w * att;
                w = w * std::exp(-sa * l);
                tau -= ss * l;
            } else {
                // post-limit: no collisions, attenuation with sigma_t, tally <Psi>_post and
                // deposit the (N_s+1)-th collision density into the bilinear moments
                const double att = -std::expm1(-st * l);
                post[k] += (st > 0) ? (long double)(w * att / st) : (long double)(w * l);
                ++post_n[k];
                double g0, g1, g2;
                gfun(st * l, &g0, &g1, &g2);
                const double I0 = l * g0, I1 = l * l * g1, I2 = l * l * l * g2;
                const double xi0 = 2.0 * fx / DX - 1.0, eta0 = 2.0 * fy / DY - 1.0;
                const double axi = 2.0 * ox / DX, aeta = 2.0 * oy / DY;
                mom[4 * k + 0] += ss * w * I0;
                if (P->handoff_full) {
                    mom[4 * k + 1] += ss * w * (xi0 * I0 + axi * I1);
                    mom[4 * k + 2] += ss * w * (eta0 * I0 + aeta * I1);
                    mom[4 * k + 3] += ss * w * (xi0 * eta0 * I0 + (xi0 * aeta + eta0 * axi) * I1
                                                + axi * aeta * I2);
                }
                if (st > 0) {
                    w_handoff += w * att * (ss / st);
                    w_absorbed += w * att * (sa / st);
                }
                w = w * std::exp(-st * l);
            }
            fx += ox * l; fy += oy * l;
            s_rem -= l;

            if (ev == 2) {  // census at t_{n+1}
                fx = std::min(std::max(fx, 0.0), DX); fy = std::min(std::max(fy, 0.0), DY);
                fate = kFateCensus; ++census; w_census += w;
                if (!bank_push(census_out, k, fx, fy, ox, oy, w)) census_overflow = true;
                break;
            }
            if (ev == 1) {
                if (xc) { ix += ox > 0 ? 1 : -1; fx = ox > 0 ? 0.0 : DX; }
                else fx = std::min(std::max(fx, 0.0), DX);
                if (yc) { iy += oy > 0 ? 1 : -1; fy = oy > 0 ? 0.0 : DY; }
                else fy = std::min(std::max(fy, 0.0), DY);
                if (ix < 0 || ix >= M.nx || iy < 0 || iy >= M.ny) {
                    fate = kFateLeaked; ++leaked; w_leaked += w;
                    ix = std::min(std::max(ix, 0), M.nx - 1); iy = std::min(std::max(iy, 0), M.ny - 1);
                    break;
                }
            } else {  // collision: isotropic re-emission, n <- n + 1
                fx = std::min(std::max(fx, 0.0), DX); fy = std::min(std::max(fy, 0.0), DY);
                ++n; ++collisions;
                const int base = 5 + 3 * (n - 1);
                iso_direction(unit(pts(idx, base + 1)), unit(pts(idx, base + 2)), &ox, &oy);
                tau = n < Ns ? neg_log(unit(pts(idx, 5 + 3 * n))) : 0.0;
                if (n >= Nk) ++reached;
            }
            if (margin && P->w_min > 0) gap = std::min(gap, std::fabs(w - P->w_min * w_start) / (P->w_min * w_start));
            if (P->w_min > 0 && w < P->w_min * w_start) {
                fate = kFateKilled; ++killed; w_killed += w;
                break;
            }
        }
        segments += seg;
        if (fate == kFateError) ++errors;
        if (rec) { rec[0] = iy * M.nx + ix; rec[1] = fate; rec[2] = n; rec[3] = (int32_t)seg; }
        if (margin) *margin = gap;
    }
};

void fill_stats(const Leg& L, int64_t hist, or_stats* st) {
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    st->histories = hist; st->segments = L.segments; st->collisions = L.collisions;
    st->leaked = L.leaked; st->census = L.census; st->killed = L.killed;
    st->reached_limit = L.reached; st->errors = L.errors;
    st->w_source = (double)L.w_source; st->w_absorbed = (double)L.w_absorbed;
    st->w_leaked = (double)L.w_leaked; st->w_census = (double)L.w_census;
    st->w_handoff = (double)L.w_handoff; st->w_killed = (double)L.w_killed;
}

// ------------------------------------------------------------------------------------------
// Level-symmetric S_N quadrature on the upper hemisphere (2-D, z-symmetric).
//   levels mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2); points (mu_i, mu_j, mu_k) with
//   i + j + k = N/2 + 2; one weight per point class (sorted index triple), fixed by matching
//   the sphere moments <mu^0>, <mu^4>, <mu^6>, ... ; mu_1 is the root for which the next even
//   moment <mu^N> is integrated exactly too. Weights sum to 4 pi over the sphere; the upper
//   hemisphere carries twice its weight in 2-D.
// ------------------------------------------------------------------------------------------
struct Quad { std::vector<double> ox, oy, oz, w; };

bool solve_dense(std::vector<double> A, std::vector<double> b, int n, std::vector<double>* x) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) { for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]); std::swap(b[c], b[piv]); }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    x->assign(n, 0.0);
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * (*x)[k];
        (*x)[r] = s / A[r * n + r];
    }
    return true;
}

// class weights for a given mu_1^2; returns the residual of the <mu^N> moment
double ls_weights(int N, double mu1sq, std::vector<double>* mu, std::vector<std::vector<int>>* pts,
                  std::vector<int>* cls, std::vector<double>* wcls) {
    int h = N / 2;
    mu->assign(h, 0.0);
    for (int i = 0; i < h; ++i) (*mu)[i] = std::sqrt(mu1sq + i * 2.0 * (1.0 - 3.0 * mu1sq) / (N - 2));
    pts->clear(); cls->clear();
    std::vector<std::vector<int>> classes;
    for (int i = 1; i <= h; ++i) for (int j = 1; j <= h; ++j) for (int k = 1; k <= h; ++k) {
        if (i + j + k != h + 2) continue;
        std::vector<int> p = {i, j, k}, s = p;
        std::sort(s.begin(), s.end());
        int ci = -1;
        for (size_t c = 0; c < classes.size(); ++c) if (classes[c] == s) ci = (int)c;
        if (ci < 0) { classes.push_back(s); ci = (int)classes.size() - 1; }
        pts->push_back(p); cls->push_back(ci);
    }
    int nc = (int)classes.size();
    std::vector<int> powers = {0};
    for (int p = 2; (int)powers.size() < nc; ++p) powers.push_back(p);  // <mu^0>, <mu^4>, <mu^6>...
    std::vector<double> A(nc * nc, 0.0), b(nc, 0.0);
    for (int e = 0; e < nc; ++e) {
        b[e] = 1.0 / (2 * powers[e] + 1);
        for (size_t q = 0; q < pts->size(); ++q)
            A[e * nc + (*cls)[q]] += std::pow((*mu)[(*pts)[q][2] - 1], 2 * powers[e]);
    }
    solve_dense(A, b, nc, wcls);
    double mN = 0.0;
    for (size_t q = 0; q < pts->size(); ++q)
        mN += (*wcls)[(*cls)[q]] * std::pow((*mu)[(*pts)[q][2] - 1], N);
    return mN - 1.0 / (N + 1);
}

bool build_quadrature(int N, Quad* Q) {
    if (N != 4 && N != 8) return false;
    std::vector<double> mu, wcls; std::vector<std::vector<int>> pts; std::vector<int> cls;
    // bisection for mu_1^2 in (0, 1/3): the smaller root of the <mu^N> residual
    double lo = 1e-6, hi = N == 4 ? 0.3 : 0.1;
    double flo = ls_weights(N, lo, &mu, &pts, &cls, &wcls);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = ls_weights(N, mid, &mu, &pts, &cls, &wcls);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
    }
    ls_weights(N, 0.5 * (lo + hi), &mu, &pts, &cls, &wcls);
    Q->ox.clear(); Q->oy.clear(); Q->oz.clear(); Q->w.clear();
    const int sx[4] = {1, -1, -1, 1}, sy[4] = {1, 1, -1, -1};
    for (int quad = 0; quad < 4; ++quad)
        for (size_t q = 0; q < pts.size(); ++q) {
            Q->ox.push_back(sx[quad] * mu[pts[q][0] - 1]);
            Q->oy.push_back(sy[quad] * mu[pts[q][1] - 1]);
            Q->oz.push_back(mu[pts[q][2] - 1]);
            Q->w.push_back(wcls[cls[q]] * (4.0 * kPi / 8.0) * 2.0);
        }
    return true;
}

// ------------------------------------------------------------------------------------------
// Bilinear discontinuous Galerkin upwind sweep for one ordinate (collided stage, Eq. (floor
// N_s+1), backward Euler). Per cell, psi = a0 + a1 xi + a2 eta + a3 xi eta (Legendre on
// [-1,1]^2); the weak form against each basis function P_i is
//   sig* A n_i a_i - Ox dy/2 Vx_i(a) - Oy dx/2 Vy_i(a) + Ox dy/2 Fx_i + Oy dx/2 Fy_i = S_i,
// n = (1, 1/3, 1/3, 1/9), Vx/Vy the volume terms of int psi dP_i, Fx/Fy the face integrals of
// P_i times the upwind trace. The 4x4 system is assembled column by column by applying the
// operator to unit vectors and solved by Gaussian elimination.
// ------------------------------------------------------------------------------------------
const double kNorm[4] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 9.0};

// face integral  int_{-1}^{1} P_i(side, s) (b0 + b1 s) ds  for a face normal to xi (x-face) or
// eta (y-face); side = +1 or -1
void face_int_x(double side, double b0, double b1, double out[4]) {
    out[0] = 2.0 * b0; out[1] = side * 2.0 * b0; out[2] = (2.0 / 3.0) * b1; out[3] = side * (2.0 / 3.0) * b1;
}
void face_int_y(double side, double c0, double c1, double out[4]) {
    out[0] = 2.0 * c0; out[1] = (2.0 / 3.0) * c1; out[2] = side * 2.0 * c0; out[3] = side * (2.0 / 3.0) * c1;
}

// residual operator L(a; inflow) = lhs(a) with the given inflow traces (x-inflow (bx0,bx1),
// y-inflow (by0,by1)); returns L_i
void dg_operator(const double a[4], double sig, double ox, double oy, double DX, double DY,
                 double bx0, double bx1, double by0, double by1, double out[4]) {
    const double A = DX * DY;
    const double cx = ox * DY / 2.0, cy = oy * DX / 2.0;
    double volx[4] = {0.0, 4.0 * a[0], 0.0, (4.0 / 3.0) * a[2]};
    double voly[4] = {0.0, 0.0, 4.0 * a[0], (4.0 / 3.0) * a[1]};
    double fr[4], fl[4], ft[4], fb[4];
    // x faces: right (xi=+1) and left (xi=-1); the outflow face carries the own trace
    if (ox > 0) {
        face_int_x(+1.0, a[0] + a[1], a[2] + a[3], fr);
        face_int_x(-1.0, bx0, bx1, fl);
    } else {
        face_int_x(+1.0, bx0, bx1, fr);
        face_int_x(-1.0, a[0] - a[1], a[2] - a[3], fl);
    }
    if (oy > 0) {
        face_int_y(+1.0, a[0] + a[2], a[1] + a[3], ft);
        face_int_y(-1.0, by0, by1, fb);
    } else {
        face_int_y(+1.0, by0, by1, ft);
        face_int_y(-1.0, a[0] - a[2], a[1] - a[3], fb);
    }
    for (int i = 0; i < 4; ++i)
        out[i] = sig * A * kNorm[i] * a[i] - cx * volx[i] - cy * voly[i]
                 + cx * (fr[i] - fl[i]) + cy * (ft[i] - fb[i]);
}

void dg_cell_solve(double sig, double ox, double oy, double DX, double DY, const double S[4],
                   double bx0, double bx1, double by0, double by1, double a[4]) {
    std::vector<double> M(16), rhs(4);
    double zero[4] = {0, 0, 0, 0}, col[4], Lb[4];
    for (int j = 0; j < 4; ++j) {
        double e[4] = {0, 0, 0, 0}; e[j] = 1.0;
        dg_operator(e, sig, ox, oy, DX, DY, 0, 0, 0, 0, col);
        for (int i = 0; i < 4; ++i) M[i * 4 + j] = col[i];
    }
    dg_operator(zero, sig, ox, oy, DX, DY, bx0, bx1, by0, by1, Lb);
    for (int i = 0; i < 4; ++i) rhs[i] = S[i] - Lb[i];
    std::vector<double> x;
    solve_dense(M, rhs, 4, &x);
    for (int i = 0; i < 4; ++i) a[i] = x[i];
}

// Sweep one ordinate over the mesh. S: per-cell source integrals (4 per cell, test function
// P_i). in_x: inflow traces on the x-boundary the ordinate enters through (ny rows x 2 coeffs,
// NULL = vacuum); in_y likewise (nx columns x 2). psi out: 4 Legendre coefficients per cell.
void dg_sweep(const Mesh& M, const double* sig, double ox, double oy, const double* S,
              const double* in_x, const double* in_y, double* psi) {
    const int nx = M.nx, ny = M.ny;
    for (int jy = 0; jy < ny; ++jy) {
        const int iy = oy > 0 ? jy : ny - 1 - jy;
        for (int jx = 0; jx < nx; ++jx) {
            const int ix = ox > 0 ? jx : nx - 1 - jx;
            const int k = iy * nx + ix;
            double bx0 = 0, bx1 = 0, by0 = 0, by1 = 0;
            if (jx == 0) {
                if (in_x) { bx0 = in_x[2 * iy]; bx1 = in_x[2 * iy + 1]; }
            } else {
                const double* u = &psi[4 * (ox > 0 ? k - 1 : k + 1)];
                // upwind neighbour's trace on the shared face: its xi = +1 (or -1) side
                if (ox > 0) { bx0 = u[0] + u[1]; bx1 = u[2] + u[3]; }
                else { bx0 = u[0] - u[1]; bx1 = u[2] - u[3]; }
            }
            if (jy == 0) {
                if (in_y) { by0 = in_y[2 * ix]; by1 = in_y[2 * ix + 1]; }
            } else {
                const double* u = &psi[4 * (oy > 0 ? k - nx : k + nx)];
                if (oy > 0) { by0 = u[0] + u[2]; by1 = u[1] + u[3]; }
                else { by0 = u[0] - u[2]; by1 = u[1] - u[3]; }
            }
            dg_cell_solve(sig[k], ox, oy, M.dx, M.dy, &S[4 * k], bx0, bx1, by0, by1, &psi[4 * k]);
        }
    }
}

// Collided solve, step 2 of Sec. 2.2: backward Euler from zero initial data with vacuum
// boundaries, (sigma_t + 1/(c dt)) Psi_c + Omega.grad Psi_c = (sigma_s/4pi)(phi_c + phi_N_s).
// The hand-off moments m_i = sigma_s sum w int P_i ds are space-time integrals, so the
// fixed source integral against P_i is m_i / (4 pi dt). Source iteration on phi_c.
int sn_solve(const or_problem* P, const double* mom, double* phi, int* iters_out) {
    Mesh M(P);
    Quad Qd;
    if (!build_quadrature(P->sn_order, &Qd)) return 1;
    const size_t nc = (size_t)M.nx * M.ny;
    std::vector<double> sig(nc), S(4 * nc), psi(4 * nc), phi_new(4 * nc);
    for (size_t k = 0; k < nc; ++k) sig[k] = P->sigma_a[k] + P->sigma_s[k] + 1.0 / (P->c * P->dt);
    std::fill(phi, phi + 4 * nc, 0.0);
    int it = 0;
    for (it = 1; it <= P->sn_max_iter; ++it) {
        for (size_t k = 0; k < nc; ++k)
            for (int i = 0; i < 4; ++i)
                S[4 * k + i] = P->sigma_s[k] / (4.0 * kPi) * phi[4 * k + i] * M.area * kNorm[i]
                               + mom[4 * k + i] / (4.0 * kPi * P->dt);
        std::fill(phi_new.begin(), phi_new.end(), 0.0);
        for (size_t m = 0; m < Qd.w.size(); ++m) {
            dg_sweep(M, sig.data(), Qd.ox[m], Qd.oy[m], S.data(), nullptr, nullptr, psi.data());
            for (size_t q = 0; q < 4 * nc; ++q) phi_new[q] += Qd.w[m] * psi[q];
        }
        double num = 0, den = 0;
        for (size_t k = 0; k < nc; ++k)
            for (int i = 0; i < 4; ++i) {
                double d = phi_new[4 * k + i] - phi[4 * k + i];
                num += kNorm[i] * d * d; den += kNorm[i] * phi_new[4 * k + i] * phi_new[4 * k + i];
            }
        std::copy(phi_new.begin(), phi_new.end(), phi);
        if (den == 0.0 || std::sqrt(num) <= P->sn_tol * std::sqrt(den)) break;
    }
    if (iters_out) *iters_out = std::min(it, P->sn_max_iter);
    return 0;
}

// ------------------------------------------------------------------------------------------
// Within-cell sampling of a bilinear density f = f0 + f1 xi + f2 eta + f3 xi eta on [-1,1]^2:
// inverse CDF of the linear marginal in xi, then of the linear conditional in eta.
// ------------------------------------------------------------------------------------------
// inverse CDF on [-1,1] of the density proportional to a + b s (a > 0, |b| <= a)
double inv_linear(double a, double b, double u) {
    if (!(a > 0.0)) return 2.0 * u - 1.0;
    const double amb = a - b;
    const double t = 4.0 * a * u / (amb + std::sqrt(std::max(0.0, amb * amb + 4.0 * a * b * u)));
    return std::min(std::max(t - 1.0, -1.0), 1.0);
}

// ------------------------------------------------------------------------------------------
// Remap, step 3 of Sec. 2.2, Eq. (R): zero allowable scatters, sigma_t attenuation, the full
// source Q + sigma_s (phi_pre + phi_post + phi_c); initial data Psi[t_n] (the step-start bank).
// Bank particles are re-streamed straight from their step-start state (Sec. 2.2: particles from
// initial data are copied, source particles are re-born). New particles: n_hist births.
// The survivors form the new census; above census_cap a systematic comb on quantised |w|.
// ------------------------------------------------------------------------------------------
struct Streamed { bool alive; int cell; double fx, fy, ox, oy, w; };

Streamed stream_free(const or_problem* P, const Mesh& M, int ix, int iy, double fx, double fy,
                     double ox, double oy, double w, double s_rem, or_stats* st, long double* acc) {
    // acc: absorbed(+handoff-free) removed weight, leaked, killed
    const double w_start = w;
    Streamed r{false, iy * M.nx + ix, fx, fy, ox, oy, w};
    for (int64_t seg = 0; seg < kMaxSegments; ++seg) {
        const int k = iy * M.nx + ix;
        const double st_ = P->sigma_a[k] + P->sigma_s[k];
        const double dxf = ox > 0 ? (M.dx - fx) / ox : (ox < 0 ? fx / (-ox) : kInf);
        const double dyf = oy > 0 ? (M.dy - fy) / oy : (oy < 0 ? fy / (-oy) : kInf);
        double l; bool face = false, xc = false, yc = false;
        if (dxf <= s_rem || dyf <= s_rem) { l = std::min(dxf, dyf); face = true; xc = dxf == l; yc = dyf == l; }
        else l = s_rem;
        acc[0] += w * (-std::expm1(-st_ * l));
        w = w * std::exp(-st_ * l);
        fx += ox * l; fy += oy * l; s_rem -= l;
        if (st) st->segments += 1;
        if (!face) {
            fx = std::min(std::max(fx, 0.0), M.dx); fy = std::min(std::max(fy, 0.0), M.dy);
            r = Streamed{true, k, fx, fy, ox, oy, w};
            return r;
        }
        if (xc) { ix += ox > 0 ? 1 : -1; fx = ox > 0 ? 0.0 : M.dx; } else fx = std::min(std::max(fx, 0.0), M.dx);
        if (yc) { iy += oy > 0 ? 1 : -1; fy = oy > 0 ? 0.0 : M.dy; } else fy = std::min(std::max(fy, 0.0), M.dy);
        if (ix < 0 || ix >= M.nx || iy < 0 || iy >= M.ny) { acc[1] += w; if (st) st->leaked += 1; return r; }
        if (P->w_min > 0 && std::fabs(w) < P->w_min * std::fabs(w_start)) { acc[2] += w; if (st) st->killed += 1; return r; }
    }
    if (st) st->errors += 1;
    return r;
}

// Power of two at or above w (w > 0): the quantisation base of the comb.
double pow2_ceil(double w) {
    int e = 0;
    double m = std::frexp(w, &e);  // w = m 2^e, m in [0.5, 1)
    return m == 0.5 ? w : std::ldexp(1.0, e);
}

// Systematic comb of the particle list to exactly M copies (in list order). |w| is quantised
// as rint(|w| / w_ref * 2^32) with w_ref a power of two bounding every |w| before streaming
// (streaming only lowers |w|), so the quantisation does not depend on the survivors. The
// offset is the point (stream REMAP_COMB, index 0, dim 0); each copy carries sum|w| / M.
void comb(const std::vector<Streamed>& in, int64_t Mcap, uint32_t x_off, double w_ref,
          std::vector<Streamed>* out) {
    typedef unsigned __int128 u128;
    std::vector<int64_t> q(in.size());
    for (size_t j = 0; j < in.size(); ++j) q[j] = (int64_t)std::nearbyint((std::fabs(in[j].w) / w_ref) * 0x1p32);
    int64_t T = 0;
    for (auto v : q) T += v;
    out->clear();
    if (T == 0) return;
    long double wsum = 0;
    for (auto& p : in) wsum += std::fabs(p.w);
    const double wcopy = (double)(wsum / (long double)Mcap);
    const u128 o = ((u128)x_off * (u128)(uint64_t)T) >> 32;  // offset in [0, T)
    auto first_tooth = [&](int64_t S) -> u128 {             // ceil((S M - o) / T), >= 0
        u128 num = (u128)(uint64_t)S * (u128)(uint64_t)Mcap;
        if (num <= o) return 0;
        num -= o;
        return (num + (u128)(uint64_t)T - 1) / (u128)(uint64_t)T;
    };
    int64_t S = 0;
    for (size_t j = 0; j < in.size(); ++j) {
        u128 a = first_tooth(S), b = first_tooth(S + q[j]);
        for (u128 c = a; c < b; ++c) {
            Streamed p = in[j];
            p.w = in[j].w < 0 ? -wcopy : wcopy;
            out->push_back(p);
        }
        S += q[j];
    }
}

}  // namespace

// ==========================================================================================
// C entry points (oracle API; test infrastructure only)
// ==========================================================================================
extern "C" {

uint64_t or_mix64(uint64_t z) { return mix64(z); }

// the direction and optical-depth maps, exposed for their accuracy pins
void or_sincos_2pi(const double* u, int64_t n, double* s, double* c, int32_t elem) {
    g_elem = elem;
    for (int64_t i = 0; i < n; ++i) sincos_2pi(u[i], &s[i], &c[i]);
}
void or_neg_log(const double* u, int64_t n, double* out, int32_t elem) {
    g_elem = elem;
    for (int64_t i = 0; i < n; ++i) out[i] = neg_log(u[i]);
}

int or_sobol_table(int ndims, uint32_t* V) {
    if (ndims < 1 || ndims > kDimMax) return 1;
    build_sobol_table();
    build_primes();
    for (int d = 0; d < ndims; ++d) for (int b = 0; b < 32; ++b) V[d * 32 + b] = g_V[d][b];
    return 0;
}

// points for i in [i0, i0+n), dims [0, ndims): out[(i-i0)*ndims + d]
int or_points(uint64_t seed, int64_t step, int32_t stream, int32_t sampler, int64_t i0, int64_t n,
              int32_t ndims, uint32_t* out) {
    if (i0 < 0 || n < 0 || i0 + n > (int64_t)1 << 32) return 1;
    build_sobol_table();
    build_primes();
    Points pts{stream_key(seed, (uint64_t)step, (uint64_t)stream), sampler};
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < ndims; ++d) out[i * ndims + d] = pts((uint64_t)(i0 + i), d);
    return 0;
}

// The integer CDF of Sec. 2.3 births / Eq. (R) remap births (exposed for the CDF parity test).
int or_build_cdf(int32_t nx, int32_t ny, const double* w, int64_t* q, int64_t* row_pre, int64_t* col_pre) {
    or_problem P{}; P.nx = nx; P.ny = ny; P.lx = 1.0; P.ly = 1.0;
    Mesh M(&P);
    std::vector<double> wv(w, w + (size_t)nx * ny);
    Cdf2D C = build_cdf(M, wv);
    std::copy(C.q.begin(), C.q.end(), q);
    std::copy(C.row_pre.begin(), C.row_pre.end(), row_pre);
    std::copy(C.col_pre.begin(), C.col_pre.end(), col_pre);
    return 0;
}

int or_quadrature(int order, double* ox, double* oy, double* oz, double* w) {
    Quad Q;
    if (!build_quadrature(order, &Q)) return -1;
    for (size_t m = 0; m < Q.w.size(); ++m) { ox[m] = Q.ox[m]; oy[m] = Q.oy[m]; oz[m] = Q.oz[m]; w[m] = Q.w[m]; }
    return (int)Q.w.size();
}

// Initial bank (Sec. 2.2, Eq. (IC)): n_hist particles from the per-cell initial weight,
// uniform in each cell and isotropic, at t = 0 (stream INIT, dims 0-1 position, 3-4 direction).
int or_init_bank(const or_problem* P, const double* ic_cell_w, or_bank* out) {
    g_elem = P->elem;
    build_sobol_table();
    build_primes();
    Mesh M(P);
    const size_t nc = (size_t)M.nx * M.ny;
    std::vector<double> w(ic_cell_w, ic_cell_w + nc);
    double W = 0.0;
    for (double v : w) W += v;
    out->n = 0;
    if (W <= 0.0) return 0;
    if (out->cap < P->n_hist) return 2;
    Cdf2D C = build_cdf(M, w);
    Points pts{stream_key(P->seed, 0, kStreamInit), P->sampler};
    const double w0 = W / (double)P->n_hist;
    for (int64_t i = 0; i < P->n_hist; ++i) {
        double frx, fry, ox, oy;
        int k = sample_cell(C, pts(i, 0), pts(i, 1), &frx, &fry);
        iso_direction(unit(pts(i, 3)), unit(pts(i, 4)), &ox, &oy);
        bank_push(out, k, frx * M.dx, fry * M.dy, ox, oy, w0);
    }
    return 0;
}

// Source births of the MC leg (Sec. 2.3: (x, Omega, t) ~ q = Q / int Q, isotropic Omega,
// sum of w0 = int Q). Exposed for the uniform-source pin. t_frac = (t - t_n)/dt.
int or_sample_births(const or_problem* P, int64_t step, int64_t n, int32_t* cell, double* fx,
                     double* fy, double* ox, double* oy, double* t_frac, double* w0_out) {
    g_elem = P->elem;
    build_sobol_table();
    build_primes();
    Mesh M(P);
    const size_t nc = (size_t)M.nx * M.ny;
    std::vector<double> q(nc, 0.0);
    double W = 0.0;
    for (size_t k = 0; k < nc; ++k) { q[k] = (P->Q ? P->Q[k] : 0.0) * M.area * P->dt; W += q[k]; }
    if (W <= 0.0) return 1;
    Cdf2D C = build_cdf(M, q);
    Points pts{stream_key(P->seed, (uint64_t)step, kStreamLegSource), P->sampler};
    for (int64_t i = 0; i < n; ++i) {
        double frx, fry;
        int k = sample_cell(C, pts(i, 0), pts(i, 1), &frx, &fry);
        cell[i] = k; fx[i] = frx * M.dx; fy[i] = fry * M.dy;
        t_frac[i] = unit(pts(i, 2));
        iso_direction(unit(pts(i, 3)), unit(pts(i, 4)), &ox[i], &oy[i]);
    }
    *w0_out = W / (double)P->n_hist;
    return 0;
}

// The MC leg of step 1 (Sec. 2.2 step 1, Sec. 2.3). Histories: the census bank first (stream
// LEG_CENSUS, index = bank slot), then n_hist source births (stream LEG_SOURCE) when Q != 0.
// pre/post: track-length integrals sum w l g0 per cell; mom: hand-off moments (4 per cell).
// hist (optional): 4 int32 per history (final cell, fate, final n, segments).
// census_out (optional): the MC-leg census survivors.
// The general form: only the histories with global index h in [h0, h1) (index order: census bank
// slots, then source births) and skip[h] == 0 (skip may be NULL) are tracked, as one rank of a
// history-sharded leg would run them. hist and margin rows (when given) and the statistics cover
// the histories tracked, in index order. margin[r]: the smallest relative gap of the history's
// decisions (see Leg::run), to tell a decision that rounding can flip from a robust one.
int or_mc_leg_ex(const or_problem* P, int64_t step, const or_bank* census, int64_t h0, int64_t h1,
                 const uint8_t* skip, double* pre, double* post, double* mom, or_stats* st, int32_t* hist,
                 double* margin, or_bank* census_out, int64_t* pre_n, int64_t* post_n);

int or_mc_leg(const or_problem* P, int64_t step, const or_bank* census, double* pre, double* post,
              double* mom, or_stats* st, int32_t* hist, or_bank* census_out) {
    return or_mc_leg_ex(P, step, census, 0, INT64_MAX, nullptr, pre, post, mom, st, hist, nullptr, census_out,
                        nullptr, nullptr);
}

// The MC leg with, per cell, the number of segments scored into the pre and post tallies.
int or_mc_leg_counts(const or_problem* P, int64_t step, const or_bank* census, double* pre, double* post,
                     double* mom, or_stats* st, int32_t* hist, or_bank* census_out, int64_t* pre_n, int64_t* post_n) {
    return or_mc_leg_ex(P, step, census, 0, INT64_MAX, nullptr, pre, post, mom, st, hist, nullptr, census_out,
                        pre_n, post_n);
}

int or_mc_leg_range(const or_problem* P, int64_t step, const or_bank* census, int64_t h0, int64_t h1, double* pre,
                    double* post, double* mom, or_stats* st, int32_t* hist) {
    return or_mc_leg_ex(P, step, census, h0, h1, nullptr, pre, post, mom, st, hist, nullptr, nullptr, nullptr,
                        nullptr);
}

int or_mc_leg_ex(const or_problem* P, int64_t step, const or_bank* census, int64_t h0, int64_t h1,
                 const uint8_t* skip, double* pre, double* post, double* mom, or_stats* st, int32_t* hist,
                 double* margin, or_bank* census_out, int64_t* pre_n, int64_t* post_n) {

    g_elem = P->elem;
    build_sobol_table();
    build_primes();
    Leg L(P);
    const Mesh& M = L.M;
    const size_t nc = (size_t)M.nx * M.ny;
    L.census_out = census_out;
    if (census_out) census_out->n = 0;
    const double cdt = P->c * P->dt;
    int64_t h = 0, ran = 0;
    if (census && census->n > 0) {
        L.pts.key = stream_key(P->seed, (uint64_t)step, kStreamLegCensus);
        for (int64_t j = 0; j < census->n; ++j, ++h) {
            if (h < h0 || h >= h1 || (skip && skip[h])) continue;
            int k = census->cell[j];
            L.run((uint64_t)j, k % M.nx, k / M.nx, census->fx[j], census->fy[j], census->ox[j],
                  census->oy[j], census->w[j], cdt, hist ? hist + 4 * ran : nullptr, margin ? margin + ran : nullptr);
            ++ran;
        }
    }
    std::vector<double> q(nc, 0.0);
    double W = 0.0;
    for (size_t k = 0; k < nc; ++k) { q[k] = (P->Q ? P->Q[k] : 0.0) * M.area * P->dt; W += q[k]; }
    if (W > 0.0) {
        Cdf2D C = build_cdf(M, q);
        const double w0 = W / (double)P->n_hist;
        L.pts.key = stream_key(P->seed, (uint64_t)step, kStreamLegSource);
        for (int64_t i = 0; i < P->n_hist; ++i, ++h) {
            if (h < h0 || h >= h1 || (skip && skip[h])) continue;
            double frx, fry, ox, oy;
            int k = sample_cell(C, L.pts(i, 0), L.pts(i, 1), &frx, &fry);
            const double tf = unit(L.pts(i, 2));
            iso_direction(unit(L.pts(i, 3)), unit(L.pts(i, 4)), &ox, &oy);
            L.run((uint64_t)i, k % M.nx, k / M.nx, frx * M.dx, fry * M.dy, ox, oy, w0,
                  cdt * (1.0 - tf), hist ? hist + 4 * ran : nullptr, margin ? margin + ran : nullptr);
            ++ran;
        }
    }
    for (size_t k = 0; k < nc; ++k) {
        pre[k] = (double)L.pre[k]; post[k] = (double)L.post[k];
        for (int i = 0; i < 4; ++i) mom[4 * k + i] = (double)L.mom[4 * k + i];
        if (pre_n) pre_n[k] = L.pre_n[k];
        if (post_n) post_n[k] = L.post_n[k];
    }
    fill_stats(L, ran, st);
    if (L.census_overflow) return 3;
    return L.errors ? 4 : 0;
}

int or_sn_solve(const or_problem* P, const double* mom, double* phi, int32_t* iters) {
    int it = 0;
    int rc = sn_solve(P, mom, phi, &it);
    if (iters) *iters = it;
    return rc;
}

// One ordinate sweep with an explicit source and inflow boundary (for manufactured tests).
int or_dg_sweep(int32_t nx, int32_t ny, double lx, double ly, const double* sig, double ox,
                double oy, const double* S, const double* in_x, const double* in_y, double* psi) {
    or_problem P{}; P.nx = nx; P.ny = ny; P.lx = lx; P.ly = ly;
    Mesh M(&P);
    dg_sweep(M, sig, ox, oy, S, in_x, in_y, psi);
    return 0;
}

// Remap source per cell as Legendre coefficients of its emission density f (4 per cell):
// f0 = Q + sigma_s (T_pre + T_post)/(A dt) + sigma_s phi_c0, f_j = sigma_s phi_cj.
void or_remap_density(const or_problem* P, const double* pre, const double* post, const double* phi,
                      double* f) {
    Mesh M(P);
    const size_t nc = (size_t)M.nx * M.ny;
    for (size_t k = 0; k < nc; ++k) {
        const double ss = P->sigma_s[k];
        const double T = (pre ? pre[k] : 0.0) + (post ? post[k] : 0.0);
        f[4 * k + 0] = (P->Q ? P->Q[k] : 0.0) + ss * T / (M.area * P->dt) + ss * (phi ? phi[4 * k] : 0.0);
        for (int j = 1; j < 4; ++j) f[4 * k + j] = ss * (phi ? phi[4 * k + j] : 0.0);
    }
}

// Births of a remap (Eq. (R), or Eq. (R') for the additive variant): n_hist particles from the
// bilinear density f (4 Legendre coefficients per cell), stream REMAP_SOURCE, each streamed
// straight to t_{n+1} with sigma_t attenuation; survivors are appended to surv. Returns the total
// |q| (0: no births); *wmax is raised to bound the birth weights.
static double remap_births(const or_problem* P, const Mesh& M, int64_t step, const std::vector<double>& f,
                           std::vector<Streamed>* surv, long double* w_src, or_stats* st, long double* acc,
                           double* wmax) {
    const size_t nc = (size_t)M.nx * M.ny;
    const double cdt = P->c * P->dt;
    std::vector<double> qc(nc);
    double W = 0.0;
    for (size_t k = 0; k < nc; ++k) { qc[k] = f[4 * k] * M.area * P->dt; W += std::fabs(qc[k]); }
    if (!(W > 0.0)) return 0.0;
    Cdf2D C = build_cdf(M, qc);
    Points pts{stream_key(P->seed, (uint64_t)step, kStreamRemapSource), P->sampler};
    const double wbar = W / (double)P->n_hist;
    for (size_t k = 0; k < nc; ++k) {
        if (qc[k] == 0.0) continue;
        const double* fk = &f[4 * k];
        const bool pos = fk[0] - fk[1] - fk[2] + fk[3] >= 0 && fk[0] + fk[1] - fk[2] - fk[3] >= 0 &&
                         fk[0] - fk[1] + fk[2] - fk[3] >= 0 && fk[0] + fk[1] + fk[2] + fk[3] >= 0;
        const double r = pos ? 1.0 : (std::fabs(fk[0]) + std::fabs(fk[1]) + std::fabs(fk[2]) +
                                      std::fabs(fk[3])) / std::fabs(fk[0]);
        *wmax = std::max(*wmax, wbar * r);
    }
    for (int64_t i = 0; i < P->n_hist; ++i) {
        double frx, fry, ox, oy;
        int k = sample_cell(C, pts(i, 0), pts(i, 1), &frx, &fry);
        const double* fk = &f[4 * k];
        const double nod[4] = {fk[0] - fk[1] - fk[2] + fk[3], fk[0] + fk[1] - fk[2] - fk[3],
                               fk[0] - fk[1] + fk[2] - fk[3], fk[0] + fk[1] + fk[2] + fk[3]};
        double xi, eta, w;
        if (nod[0] >= 0 && nod[1] >= 0 && nod[2] >= 0 && nod[3] >= 0) {
            xi = inv_linear(fk[0], fk[1], frx);
            eta = inv_linear(fk[0] + fk[1] * xi, fk[2] + fk[3] * xi, fry);
            w = wbar;
        } else {
            xi = 2.0 * frx - 1.0; eta = 2.0 * fry - 1.0;
            w = wbar * (fk[0] + fk[1] * xi + fk[2] * eta + fk[3] * xi * eta) / std::fabs(fk[0]);
        }
        const double tf = unit(pts(i, 2));
        iso_direction(unit(pts(i, 3)), unit(pts(i, 4)), &ox, &oy);
        *w_src += w;
        Streamed r = stream_free(P, M, k % M.nx, k / M.nx, 0.5 * (xi + 1.0) * M.dx,
                                 0.5 * (eta + 1.0) * M.dy, ox, oy, w, cdt * (1.0 - tf), st, acc);
        if (r.alive) surv->push_back(r);
    }
    return W;
}

// Phase-space key of a census particle (census_order 2): the cell index, then a Morton (Z-order)
// interleave of b bits each of the in-cell position x, y and the direction's polar angle, taken
// as the "diamond angle" d in [0, 4) (monotone in the polar angle, one division, no arctangent);
// b = min(5, (31 - cell bits) / 3) so that the key and its end-of-list sentinel fit in 32 bits.
uint32_t phase_key_bits(int64_t ncells, int* cell_bits) {
    int cb = 0;
    while (((int64_t)1 << cb) < ncells) ++cb;
    *cell_bits = cb;
    const int b = (31 - cb) / 3;
    return (uint32_t)(b < 0 ? 0 : (b > 5 ? 5 : b));
}

uint32_t phase_key(const Mesh& M, int cell, double fx, double fy, double ox, double oy, int b) {
    const double s = (double)(1u << b);
    auto quant = [&](double v) {
        const double t = std::floor(v * s);
        return (uint32_t)std::min(std::max(t, 0.0), s - 1.0);
    };
    double d;
    if (ox == 0.0 && oy == 0.0) d = 0.0;
    else if (oy >= 0.0) d = ox >= 0.0 ? oy / (ox + oy) : 1.0 + (-ox) / (oy - ox);
    else d = ox < 0.0 ? 2.0 + (-oy) / (-ox - oy) : 3.0 + ox / (ox - oy);
    const uint32_t qx = quant(fx / M.dx), qy = quant(fy / M.dy), qa = quant(d * 0.25);
    uint32_t sub = 0;
    for (int i = 0; i < b; ++i)
        sub |= (((qx >> i) & 1u) << (3 * i)) | (((qy >> i) & 1u) << (3 * i + 1)) | (((qa >> i) & 1u) << (3 * i + 2));
    return ((uint32_t)cell << (3 * b)) | sub;
}

// The census order of step 4: slot order (0), cell order (1), or cell then in-cell phase-space order
// (2), each a stable sort, so that the systematic comb along it samples each cell (and, for 2, the
// position and direction within it) in strata. With sort_every > 1 the sorted orders apply on every
// sort_every-th step only (step n with n mod sort_every == 0), slot order on the others.
void order_census(const or_problem* P, int64_t step, std::vector<Streamed>& v) {
    const int order = (P->sort_every <= 1 || step % P->sort_every == 0) ? P->census_order : 0;
    if (order == 1) {
        std::stable_sort(v.begin(), v.end(), [](const Streamed& a, const Streamed& b) { return a.cell < b.cell; });
    } else if (order == 2) {
        Mesh M(P);
        int cb = 0;
        const int b = (int)phase_key_bits((int64_t)M.nx * M.ny, &cb);
        std::vector<std::pair<uint32_t, size_t>> key(v.size());
        for (size_t i = 0; i < v.size(); ++i) key[i] = {phase_key(M, v[i].cell, v[i].fx, v[i].fy, v[i].ox, v[i].oy, b), i};
        std::stable_sort(key.begin(), key.end(), [](const std::pair<uint32_t, size_t>& a,
                                                    const std::pair<uint32_t, size_t>& b2) { return a.first < b2.first; });
        std::vector<Streamed> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = v[key[i].second];
        v.swap(o);
    }
}

// Census of step 4 from the survivors, in the requested order (order_census), combed to
// census_cap (power-of-two quantisation base at or above wmax, offset = point (REMAP_COMB, 0, 0))
// when above it.
static int census_from(const or_problem* P, int64_t step, std::vector<Streamed>& surv, double wmax,
                       or_bank* out, int32_t* combed, long double* wc) {
    const int64_t cap = P->census_cap > 0 ? P->census_cap : P->n_hist;
    order_census(P, step, surv);
    std::vector<Streamed> fin;
    int did_comb = 0;
    if ((int64_t)surv.size() > cap) {
        Points pc{stream_key(P->seed, (uint64_t)step, kStreamRemapComb), P->sampler};
        comb(surv, cap, pc(0, 0), pow2_ceil(wmax), &fin);
        did_comb = 1;
    } else fin = surv;
    out->n = 0;
    if ((int64_t)fin.size() > out->cap) return 3;
    *wc = 0;
    for (auto& p : fin) { bank_push(out, p.cell, p.fx, p.fy, p.ox, p.oy, p.w); *wc += p.w; }
    if (combed) *combed = did_comb;
    return 0;
}

// Remap (step 3, Eq. (R)) and census (step 4). out receives the new bank (capacity >= census_cap
// or bank + births). combed: 1 if the comb ran.
int or_remap(const or_problem* P, int64_t step, const or_bank* census, const double* pre,
             const double* post, const double* phi, or_bank* out, or_stats* st, int32_t* combed) {
    g_elem = P->elem;
    build_sobol_table();
    build_primes();
    Mesh M(P);
    const size_t nc = (size_t)M.nx * M.ny;
    if (st) std::memset(st, 0, sizeof(*st));
    long double acc[3] = {0, 0, 0};
    std::vector<Streamed> surv;
    const double cdt = P->c * P->dt;
    long double w_src = 0;
    // (i) bank particles, copied and re-streamed from their step-start state
    if (census)
        for (int64_t j = 0; j < census->n; ++j) {
            int k = census->cell[j];
            w_src += census->w[j];
            Streamed r = stream_free(P, M, k % M.nx, k / M.nx, census->fx[j], census->fy[j],
                                     census->ox[j], census->oy[j], census->w[j], cdt, st, acc);
            if (r.alive) surv.push_back(r);
        }
    double wmax = 0.0;  // bound on every |w| entering the comb
    if (census)
        for (int64_t j = 0; j < census->n; ++j) wmax = std::max(wmax, std::fabs(census->w[j]));
    // (ii) births from the remap source Q + sigma_s (phi_pre + phi_post + phi_c)
    std::vector<double> f(4 * nc);
    or_remap_density(P, pre, post, phi, f.data());
    const double W = remap_births(P, M, step, f, &surv, &w_src, st, acc, &wmax);
    // (iii) census
    long double wc = 0;
    const int rc = census_from(P, step, surv, wmax, out, combed, &wc);
    if (rc) return rc;
    if (st) {
        st->histories = (census ? census->n : 0) + (W > 0.0 ? P->n_hist : 0);
        st->census = out->n;
        st->w_source = (double)w_src; st->w_absorbed = (double)acc[0];
        st->w_leaked = (double)acc[1]; st->w_killed = (double)acc[2];
        st->w_census = (double)wc;
    }
    return (st && st->errors) ? 4 : 0;
}

// The remap of the previous hybrids (steps 3' and 4' of Sec. 2.2): new particles from the
// collided emission sigma_s (phi_post + phi_c) only (Eq. (R'): no Q, no pre-limit scattering,
// zero initial data), streamed scatter-free with sigma_t; the new census is the MC leg's census
// (pre- and post-limit particles alive at t_{n+1}, kept as they are) followed by those births'
// survivors, combed like the census of Eq. (R). bank: the step-start bank (its max |w| bounds the
// leg census weights, as does the leg's birth weight int Q / n_hist); leg_census: the leg's
// census particles in history order.
int or_remap_additive(const or_problem* P, int64_t step, const or_bank* bank, const or_bank* leg_census,
                      const double* post, const double* phi, or_bank* out, or_stats* st, int32_t* combed) {
    g_elem = P->elem;
    build_sobol_table();
    build_primes();
    Mesh M(P);
    const size_t nc = (size_t)M.nx * M.ny;
    if (st) std::memset(st, 0, sizeof(*st));
    long double acc[3] = {0, 0, 0};
    std::vector<Streamed> surv;
    double wmax = 0.0;
    if (bank)
        for (int64_t j = 0; j < bank->n; ++j) wmax = std::max(wmax, std::fabs(bank->w[j]));
    double Wq = 0.0;
    for (size_t k = 0; k < nc; ++k) Wq += std::fabs(P->Q ? P->Q[k] : 0.0) * M.area * P->dt;
    if (Wq > 0.0) wmax = std::max(wmax, Wq / (double)P->n_hist);
    if (leg_census)
        for (int64_t j = 0; j < leg_census->n; ++j)
            surv.push_back(Streamed{true, leg_census->cell[j], leg_census->fx[j], leg_census->fy[j],
                                    leg_census->ox[j], leg_census->oy[j], leg_census->w[j]});
    std::vector<double> f(4 * nc);
    for (size_t k = 0; k < nc; ++k) {
        const double ss = P->sigma_s[k];
        f[4 * k + 0] = ss * (post ? post[k] : 0.0) / (M.area * P->dt) + ss * (phi ? phi[4 * k] : 0.0);
        for (int j = 1; j < 4; ++j) f[4 * k + j] = ss * (phi ? phi[4 * k + j] : 0.0);
    }
    long double w_src = 0;
    const double W = remap_births(P, M, step, f, &surv, &w_src, st, acc, &wmax);
    long double wc = 0;
    const int rc = census_from(P, step, surv, wmax, out, combed, &wc);
    if (rc) return rc;
    if (st) {
        st->histories = W > 0.0 ? P->n_hist : 0;
        st->census = out->n;
        st->w_source = (double)w_src; st->w_absorbed = (double)acc[0];
        st->w_leaked = (double)acc[1]; st->w_killed = (double)acc[2];
        st->w_census = (double)wc;
    }
    return (st && st->errors) ? 4 : 0;
}

// the phase-space census key (census_order 2), exposed for its pins
int or_phase_keys(const or_problem* P, const or_bank* b, uint32_t* keys) {
    g_elem = P->elem;
    Mesh M(P);
    int cb = 0;
    const int bits = (int)phase_key_bits((int64_t)M.nx * M.ny, &cb);
    for (int64_t i = 0; i < b->n; ++i) keys[i] = phase_key(M, b->cell[i], b->fx[i], b->fy[i], b->ox[i], b->oy[i], bits);
    return bits;
}

// One hybrid time step (Sec. 2.2, steps 1-4). bank -> out. flux: step-average scalar flux per
// cell, phi = (T_pre + T_post)/(A dt) + phi_c0. For N_s = infinity the remap is skipped and the
// MC-leg census (combed to census_cap) is the new bank.
int or_step(const or_problem* P, int64_t step, const or_bank* bank, or_bank* out, double* flux,
            double* pre, double* post, double* mom, double* phi, or_stats* leg_st,
            or_stats* remap_st) {
    g_elem = P->elem;
    Mesh M(P);
    const size_t nc = (size_t)M.nx * M.ny;
    int rc;
    if (P->n_s == kNsInf) {
        or_bank tmp;
        const int64_t capt = (bank ? bank->n : 0) + P->n_hist;
        std::vector<int32_t> c(capt); std::vector<double> a(capt), b(capt), d(capt), e(capt), g(capt);
        tmp.n = 0; tmp.cap = capt; tmp.cell = c.data(); tmp.fx = a.data(); tmp.fy = b.data();
        tmp.ox = d.data(); tmp.oy = e.data(); tmp.w = g.data();
        rc = or_mc_leg(P, step, bank, pre, post, mom, leg_st, nullptr, &tmp);
        if (rc) return rc;
        std::fill(phi, phi + 4 * nc, 0.0);
        std::vector<Streamed> s, fin;
        for (int64_t j = 0; j < tmp.n; ++j) s.push_back(Streamed{true, c[j], a[j], b[j], d[j], e[j], g[j]});
        order_census(P, step, s);
        const int64_t cap = P->census_cap > 0 ? P->census_cap : P->n_hist;
        if ((int64_t)s.size() > cap) {
            double wmax = 0.0;
            if (bank) for (int64_t j = 0; j < bank->n; ++j) wmax = std::max(wmax, std::fabs(bank->w[j]));
            double Wq = 0.0;
            for (size_t k = 0; k < nc; ++k) Wq += (P->Q ? P->Q[k] : 0.0) * M.area * P->dt;
            if (Wq > 0.0) wmax = std::max(wmax, Wq / (double)P->n_hist);
            Points pc{stream_key(P->seed, (uint64_t)step, kStreamRemapComb), P->sampler};
            comb(s, cap, pc(0, 0), pow2_ceil(wmax), &fin);
        } else fin = s;
        out->n = 0;
        if ((int64_t)fin.size() > out->cap) return 3;
        for (auto& p : fin) bank_push(out, p.cell, p.fx, p.fy, p.ox, p.oy, p.w);
        if (remap_st) std::memset(remap_st, 0, sizeof(*remap_st));
    } else if (P->remap_variant == 1) {
        // steps 3' and 4': the leg's census survives as particles beside the Eq. (R') births
        or_bank lc;
        const int64_t capt = (bank ? bank->n : 0) + P->n_hist;
        std::vector<int32_t> c(capt); std::vector<double> a(capt), b(capt), d(capt), e(capt), g(capt);
        lc.n = 0; lc.cap = capt; lc.cell = c.data(); lc.fx = a.data(); lc.fy = b.data();
        lc.ox = d.data(); lc.oy = e.data(); lc.w = g.data();
        rc = or_mc_leg(P, step, bank, pre, post, mom, leg_st, nullptr, &lc);
        if (rc) return rc;
        int32_t it = 0;
        rc = or_sn_solve(P, mom, phi, &it);
        if (rc) return rc;
        if (leg_st) leg_st->sn_iterations = it;
        rc = or_remap_additive(P, step, bank, &lc, post, phi, out, remap_st, nullptr);
        if (rc) return rc;
    } else {
        rc = or_mc_leg(P, step, bank, pre, post, mom, leg_st, nullptr, nullptr);
        if (rc) return rc;
        int32_t it = 0;
        rc = or_sn_solve(P, mom, phi, &it);
        if (rc) return rc;
        if (leg_st) leg_st->sn_iterations = it;
        rc = or_remap(P, step, bank, pre, post, phi, out, remap_st, nullptr);
        if (rc) return rc;
    }
    for (size_t k = 0; k < nc; ++k) flux[k] = (pre[k] + post[k]) / (M.area * P->dt) + phi[4 * k];
    return 0;
}

}  // extern "C"
