// host.cu -- C ABI entry points (include/hyb.h): validation, workspace layout, problem set-up,
// the hybrid time step driver (Sec. 2.2 steps 1-4), statistics and data movement.
//
// Set-up tables generated here: Sobol direction numbers (primitive polynomials over GF(2) in
// (degree, value) order, initial numbers chosen greedily for (0, j, 2)-net pairs with all earlier
// dimensions) and the level-symmetric S4/S8 quadrature (moment-matched class weights).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hyb_device.cuh"

namespace hyb {

uint64_t mix64(uint64_t z) { return dmix64(z); }

uint64_t stream_key(uint64_t seed, uint64_t step, uint64_t stream) { return dstream_key(seed, step, stream); }

// ---------------------------------------------------------------------------------------------
// Sobol direction numbers
// ---------------------------------------------------------------------------------------------
namespace sobolgen {

uint32_t g_tab[HYB_SOBOL_DIMS][32];
std::once_flag g_tab_once;

// row r of the generator matrix as a bit mask over columns: bit c = bit (31 - r) of V[c]
inline uint32_t gen_row(const uint32_t* V, int r, int m) {
    uint32_t mask = 0;
    for (int c = 0; c < m; ++c) mask |= ((V[c] >> (31 - r)) & 1u) << c;
    return mask;
}

bool full_rank(uint32_t* rows, int n, int m) {
    int rank = 0;
    for (int c = 0; c < m && rank < n; ++c) {
        const uint32_t bit = 1u << c;
        int piv = -1;
        for (int i = rank; i < n; ++i) if (rows[i] & bit) { piv = i; break; }
        if (piv < 0) return false;
        std::swap(rows[rank], rows[piv]);
        for (int i = 0; i < n; ++i) if (i != rank && (rows[i] & bit)) rows[i] ^= rows[rank];
        ++rank;
    }
    return rank == m;
}

// the first 2^m points of dims (A, B) form a (0, m, 2)-net
bool net_pair(const uint32_t* A, const uint32_t* B, int m) {
    uint32_t ra[32], rb[32], rows[32];
    for (int r = 0; r < m; ++r) { ra[r] = gen_row(A, r, m); rb[r] = gen_row(B, r, m); }
    for (int k = 1; k < m; ++k) {   // k = 0 and k = m are triangular with unit diagonal
        for (int r = 0; r < k; ++r) rows[r] = ra[r];
        for (int r = 0; r < m - k; ++r) rows[k + r] = rb[r];
        if (!full_rank(rows, m, m)) return false;
    }
    return true;
}

void fill_directions(uint32_t poly, int s, const uint32_t* mv, uint32_t* V) {
    for (int j = 0; j < s; ++j) V[j] = mv[j] << (31 - j);
    for (int j = s; j < 32; ++j) {
        uint32_t x = V[j - s] ^ (V[j - s] >> s);
        for (int k = 1; k < s; ++k)
            if ((poly >> (s - k)) & 1u) x ^= V[j - k];
        V[j] = x;
    }
}

bool primitive(uint32_t poly, int s) {
    const uint32_t period = (1u << s) - 1u;
    uint32_t r = 1u;
    for (uint32_t e = 1; e <= period; ++e) {
        r <<= 1;
        if (r & (1u << s)) r ^= poly;
        if (r == 1u) return e == period;
    }
    return false;
}

void build_table() {
    for (int b = 0; b < 32; ++b) g_tab[0][b] = 1u << (31 - b);
    int d = 1;
    for (int s = 1; d < HYB_SOBOL_DIMS; ++s) {
        for (uint32_t poly = (1u << s) + 1u; poly < (2u << s) && d < HYB_SOBOL_DIMS; poly += 2u) {
            if (!primitive(poly, s)) continue;
            uint32_t mv[32];
            for (int j = 0; j < s; ++j) mv[j] = 1u;
            for (int j = 1; j <= s; ++j) {
                int best = -1;
                uint32_t best_m = 1u;
                for (uint32_t cand = 1u; cand < (1u << j); cand += 2u) {
                    mv[j - 1] = cand;
                    uint32_t V[32];
                    fill_directions(poly, s, mv, V);
                    int fails = 0;
                    for (int e = 0; e < d; ++e) fails += net_pair(g_tab[e], V, j) ? 0 : 1;
                    if (best < 0 || fails < best) { best = fails; best_m = cand; }
                }
                mv[j - 1] = best_m;
            }
            fill_directions(poly, s, mv, g_tab[d]);
            ++d;
        }
    }
}

}  // namespace sobolgen

const uint32_t* sobol_table_host() {
    std::call_once(sobolgen::g_tab_once, sobolgen::build_table);
    return &sobolgen::g_tab[0][0];
}

// ---------------------------------------------------------------------------------------------
// Halton tables: per dimension d (prime base b, the d-th prime), kHaltonWords words: b, B = b^m
// (largest power of b not above 256), m, floor(2^32 / B), 2^32 mod B, ceil(2^64 / B) as two words,
// the bits per packed base-B chunk, then for m > 1 the reversal of m base-b digits as B bytes.
// ---------------------------------------------------------------------------------------------
namespace haltongen {

uint32_t g_tab[HYB_SOBOL_DIMS][kHaltonWords];
std::once_flag g_once;

void build_table() {
    uint32_t b = 1;
    for (int d = 0; d < HYB_SOBOL_DIMS; ++d) {
        bool prime;
        do {
            ++b;
            prime = true;
            for (uint32_t q = 2; q * q <= b; ++q)
                if (b % q == 0) { prime = false; break; }
        } while (!prime);
        uint32_t B = b, m = 1;
        while (B * b <= 256u) { B *= b; ++m; }
        const uint64_t two32 = 1ull << 32;
        const unsigned __int128 two64 = (unsigned __int128)1 << 64;
        const uint64_t c = (uint64_t)((two64 + B - 1) / B);
        uint32_t* t = g_tab[d];
        std::memset(t, 0, sizeof(g_tab[d]));
        t[0] = b; t[1] = B; t[2] = m;
        t[3] = (uint32_t)(two32 / B); t[4] = (uint32_t)(two32 % B);
        t[5] = (uint32_t)c; t[6] = (uint32_t)(c >> 32);
        t[7] = B > 256u ? 9u : 8u;
        if (m > 1) {
            unsigned char* rv = reinterpret_cast<unsigned char*>(t + 8);
            for (uint32_t v = 0; v < B; ++v) {
                uint32_t r = 0, x = v;
                for (uint32_t k = 0; k < m; ++k) { r = r * b + x % b; x /= b; }
                rv[v] = (unsigned char)r;
            }
        }
    }
}

}  // namespace haltongen

const uint32_t* halton_table_host() {
    std::call_once(haltongen::g_once, haltongen::build_table);
    return &haltongen::g_tab[0][0];
}

// the point table a problem uploads for its sampler (Sobol direction numbers or Halton tables)
static const uint32_t* point_table_host(int sampler, size_t* bytes) {
    if (sampler == HYB_HALTON) {
        *bytes = (size_t)HYB_SOBOL_DIMS * kHaltonWords * 4;
        return halton_table_host();
    }
    *bytes = (size_t)HYB_SOBOL_DIMS * 32 * 4;
    return sobol_table_host();
}

// ---------------------------------------------------------------------------------------------
// level-symmetric quadrature (upper hemisphere; weights summing to 4 pi)
// ---------------------------------------------------------------------------------------------
void quadrature_host(int order, double* ox, double* oy, double* w, int* m_out) {
    const int h = order / 2;
    // mu_1^2 integrating <mu^N> exactly: S4 root of 6x^2 - 4x + 2/5 = 0; S8: 1/21
    const double mu1sq = order == 4 ? (4.0 - std::sqrt(6.4)) / 12.0 : 1.0 / 21.0;
    std::vector<double> mu(h);
    for (int i = 0; i < h; ++i) mu[i] = std::sqrt(mu1sq + i * 2.0 * (1.0 - 3.0 * mu1sq) / (order - 2));
    struct Pt { int i, j, k, cls; };
    std::vector<Pt> pts;
    std::vector<std::vector<int>> classes;
    for (int i = 1; i <= h; ++i)
        for (int j = 1; j <= h; ++j)
            for (int k = 1; k <= h; ++k) {
                if (i + j + k != h + 2) continue;
                std::vector<int> key = {i, j, k};
                std::sort(key.begin(), key.end());
                int c = (int)(std::find(classes.begin(), classes.end(), key) - classes.begin());
                if (c == (int)classes.size()) classes.push_back(key);
                pts.push_back({i, j, k, c});
            }
    const int nc = (int)classes.size();
    std::vector<double> wc(nc, 0.0);
    if (nc == 1) {
        wc[0] = 1.0 / pts.size();
    } else {
        // moment equations for <mu^0>, <mu^4>, <mu^6> (three classes for S8), Cramer's rule
        double A[3][3] = {{0}}, b[3];
        const int pw[3] = {0, 4, 6};
        for (int e = 0; e < 3; ++e) {
            b[e] = 1.0 / (pw[e] + 1);
            for (const Pt& p : pts) A[e][p.cls] += std::pow(mu[p.k - 1], pw[e]);
        }
        auto det3 = [](double M[3][3]) {
            return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        };
        const double D = det3(A);
        for (int c = 0; c < 3; ++c) {
            double Mc[3][3];
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) Mc[r][q] = q == c ? b[r] : A[r][q];
            wc[c] = det3(Mc) / D;
        }
    }
    const double pi = 3.14159265358979323846;
    int m = 0;
    const int sx[4] = {1, -1, -1, 1}, sy[4] = {1, 1, -1, -1};
    for (int q = 0; q < 4; ++q)
        for (const Pt& p : pts) {
            ox[m] = sx[q] * mu[p.i - 1];
            oy[m] = sy[q] * mu[p.j - 1];
            w[m] = wc[p.cls] * pi;        // 4 pi / 8 per octant point, x2 for the z mirror
            ++m;
        }
    *m_out = m;
}

}  // namespace hyb

using namespace hyb;

// ---------------------------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------------------------
namespace hybh {

thread_local std::string g_err;

struct Layout {
    size_t off[64];
    int n = 0;
    size_t total = 0;
    size_t add(size_t bytes) {
        const size_t o = total;
        total += (bytes + 255) / 256 * 256;
        off[n++] = o;
        return o;
    }
};

// The leg's privatised window (priv_tile > 0): the square of priv_tile cells on a side (at most the
// mesh) holding the largest source weight sum Q (2-D prefix sums; the first such square in row
// order), or the initial weight where there is no source, else the mesh centre. Births and the
// census concentrate there, so their tally additions stay in each block's shared memory.
// priv_tile = -1 (automatic): a 16 x 16 window where every segment adds to five tallies (N_s = 0)
// and the source is concentrated there -- the window holds at least a quarter of the source
// weight and at least four times its share of the area (measured on the checkerboard: the leg
// 2.2x faster there; with N_s >= 1 the leg is issue-bound, and with a spread source the additions
// do not crowd any window, so a window does not pay).
void choose_priv_window(const hyb_problem_desc* d, int* x0, int* y0, int* side) {
    *x0 = *y0 = *side = 0;
    const bool automatic = d->priv_tile < 0;
    if (d->priv_tile == 0) return;
    const int nx = d->nx, ny = d->ny;
    if (automatic && (d->n_s != 0 || !d->Q || nx < 16 || ny < 16)) return;
    const int s = std::min(automatic ? 16 : d->priv_tile, std::min(nx, ny));
    const double* q = d->Q ? d->Q : d->ic_cell_w;
    *side = s;
    *x0 = (nx - s) / 2;
    *y0 = (ny - s) / 2;
    if (!q) return;
    std::vector<double> ps((size_t)(nx + 1) * (ny + 1), 0.0);   // ps[(y) (nx + 1) + x]: sum over [0, x) x [0, y)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            ps[(size_t)(y + 1) * (nx + 1) + x + 1] = q[(size_t)y * nx + x] + ps[(size_t)y * (nx + 1) + x + 1] +
                                                    ps[(size_t)(y + 1) * (nx + 1) + x] - ps[(size_t)y * (nx + 1) + x];
    double best = -1.0;
    for (int y = 0; y + s <= ny; ++y)
        for (int x = 0; x + s <= nx; ++x) {
            const double v = ps[(size_t)(y + s) * (nx + 1) + x + s] - ps[(size_t)y * (nx + 1) + x + s] -
                             ps[(size_t)(y + s) * (nx + 1) + x] + ps[(size_t)y * (nx + 1) + x];
            if (v > best) { best = v; *x0 = x; *y0 = y; }
        }
    const double total = ps[(size_t)ny * (nx + 1) + nx];
    const double area_share = (double)s * s / ((double)nx * ny);
    if (automatic && !(best > 0 && best >= 0.25 * total && best >= 4.0 * area_share * total)) *side = 0;
}

int64_t eff_cap(const hyb_problem_desc* d) {
    const int64_t cc = d->census_cap > 0 ? d->census_cap : d->n_hist;
    return std::max<int64_t>(cc, d->n_hist);
}

struct Sizes {
    size_t st, sobol, sig, sa, ss, Q, cdf_q, cdf_row, cdf_col, rem_f, rem_q, scratch, bank, stage, acc1, acc4, d1, d4,
        sn4, sn16, sntx, sntab, snqb, snnorm, blk, grow, gcol, remf32, rempos, sortkv, sortc, siginv, aah, aas, nscell,
        sortkey, btab, births, live, livekv, livesc;
    int64_t cap, nblk, slots, live_cap;
    int gr, gc;
};

// remap staging slots: the bank capacity and one per birth (Eq. (R)); for steps 3'/4' the MC leg
// stages its census there too (bank slots, then its source births), ahead of the remap births
static int64_t stage_slots(const hyb_problem_desc* d, int64_t cap) {
    return cap + d->n_hist * (d->remap_variant == 1 ? 2 : 1);
}

// Copies of the fixed-point tally arrays: the leg's warps add into copy (warp index mod copies),
// so the adds to a hot cell (the source region) spread over several addresses; the normalisation
// adds the copies exactly. Four copies (measured on the 112^2 benchmark: 1 copy 0.235 ms per leg,
// 4 copies 0.205, 8 0.207, 16 0.211, 32 0.223) while they take at most 32 MB, fewer above: the
// copies must stay in L2 with the rest of the leg's working set (on the 1024^2 mesh four copies,
// 192 MB, made the leg 6 % slower than one).
int tally_copies(const hyb_problem_desc* d) {
    if (d->tally_copies > 0) return d->tally_copies;
    const size_t acc = d->precision == HYB_FP64 ? 16 : 8;
    const size_t per = 6 * (size_t)d->nx * d->ny * acc;   // pre, post, 4 moments
    int c = 4;
    while (c > 1 && (size_t)c * per > ((size_t)32 << 20)) c >>= 1;
    return c;
}

Sizes sizes(const hyb_problem_desc* d) {
    Sizes z;
    const size_t nc = (size_t)d->nx * d->ny;
    const size_t T = d->precision == HYB_FP64 ? 8 : 4;
    const size_t acc = d->precision == HYB_FP64 ? 16 : 8;
    const int nord = d->sn_order == 8 ? 40 : 12;
    z.cap = eff_cap(d);
    z.st = sizeof(DevState);
    z.sobol = HYB_SOBOL_DIMS * kHaltonWords * 4;  // the larger of the two point tables
    z.sig = nc * 2 * T;
    z.sa = z.ss = z.Q = nc * 8;
    z.cdf_q = nc * 8;
    z.cdf_row = (d->ny + 1) * 8;
    z.cdf_col = (size_t)d->ny * (d->nx + 1) * 8;
    z.rem_f = 4 * nc * 8;
    z.rem_q = nc * 8;
    z.scratch = (256 + d->ny + nc + 2 * 256) * 8;   // CDF partials, row totals, cell weights, remap partials
    z.bank = bank_cell_bytes(z.cap) + 5 * (size_t)z.cap * T;
    z.slots = stage_slots(d, z.cap);
    z.stage = bank_cell_bytes(z.slots) + 5 * (size_t)z.slots * T;
    z.acc1 = (size_t)tally_copies(d) * nc * acc;
    z.acc4 = (size_t)tally_copies(d) * 4 * nc * acc;
    z.d1 = nc * 8;
    z.d4 = 4 * nc * 8;
    z.sn4 = 4 * nc * T;
    z.sn16 = hyb::sn_src_bytes(d->nx, d->ny, nord, d->precision == HYB_FP64, d->sn_layout);    // sweep sources
    z.sntx = hyb::sn_psi_bytes(d->nx, d->ny, nord, d->precision == HYB_FP64, d->sn_layout);    // psi per ordinate
    z.sntab = hyb::sn_table_bytes(d->nx, d->ny, nord, d->precision == HYB_FP64, d->sn_layout);   // cell-solve table or 0
    z.snqb = 7 * kMaxOrd * T;                     // ox, oy, w, then 4 signed weights per ordinate
    z.snnorm = hyb::sn_norm_bytes((int)nc);       // reduction partials per block and group, group counters
    z.nblk = (z.slots + 2047) / 2048;   // remap census pieces of 2048 slots (partials)
    z.blk = 4 * (size_t)z.nblk * 8;
    z.gr = hyb::guide_bits(d->ny);
    z.gc = hyb::guide_bits(d->nx);
    z.grow = ((size_t(1) << z.gr) + 1) * 4;
    z.gcol = (size_t)d->ny * ((size_t(1) << z.gc) + 1) * 4;
    z.remf32 = 4 * nc * 4;
    z.siginv = 8 * nc * 4;
    z.nscell = d->n_s_cell ? nc * 4 : 0;
    z.aah = d->sn_accel > 0 ? 2 * (size_t)(d->sn_accel + 1) * 4 * nc * T : 0;   // Anderson history
    z.aas = d->sn_accel > 0 ? sn_accel_state_bytes() : 0;
    z.rempos = nc * 4;
    const size_t nslots = (size_t)z.slots;
    z.sortkv = d->census_order >= 1 ? nslots * 8 : 0;                    // x2: (key, slot) pairs, ping-pong
    z.sortc = d->census_order >= 1
                  ? census_sort_scratch_bytes((long long)nslots, census_sort_sentinel(d->census_order, d->nx * d->ny))
                  : 0;
    z.sortkey = d->census_order == 2 ? nslots * 4 : 0;                   // phase-space keys per slot
    z.btab = d->sampler == HYB_SOBOL_DS ? (size_t)kByteDims * kByteWords * 4 : 0;   // births' Sobol byte tables
    // staged source births (the legs that keep no census of their own: N_s finite, Eq. (R))
    z.births = d->n_s != HYB_NS_INF && d->remap_variant == 0
                   ? bank_cell_bytes(d->n_hist) + 6 * (size_t)d->n_hist * T : 0;
    // phased leg: two buffers of saved histories (bank capacity + births), their sort by cell
    z.live_cap = z.cap + d->n_hist;
    z.live = d->leg_sort_every > 0 ? live_buf_bytes(z.live_cap, d->precision) : 0;
    z.livekv = d->leg_sort_every > 0 ? (size_t)z.live_cap * 8 : 0;
    z.livesc = d->leg_sort_every > 0 ? census_sort_scratch_bytes(z.live_cap, (uint32_t)(d->nx * d->ny)) : 0;
    return z;
}

size_t layout_bytes(const hyb_problem_desc* d) {
    const Sizes z = sizes(d);
    Layout L;
    const size_t parts[] = {z.st, z.sobol, z.sig, z.sa, z.ss, z.Q, z.cdf_q, z.cdf_row, z.cdf_col, z.cdf_q, z.cdf_row,
                            z.cdf_col, z.rem_f, z.rem_q, z.scratch, z.bank, z.bank, z.stage, z.acc1, z.acc1, z.acc4, z.d1,
                            z.d1, z.d4, z.d1, z.d1, z.d1, z.sn4, z.sn4, z.sn16, z.sntx, z.sntab, z.snqb, z.d4, z.d4,
                            z.snnorm, z.blk, z.grow, z.gcol, z.grow, z.gcol, z.remf32, z.rempos, z.sortkv,
                            z.sortkv, z.sortc, z.siginv, z.aah, z.aas, z.nscell, z.sortkey, z.btab, z.births, z.live,
                            z.live, z.livekv, z.livekv, z.livesc};
    for (size_t b : parts) L.add(b);
    return L.total;
}

void assign(hyb_problem* p) {
    const Sizes z = sizes(&p->d);
    Layout L;
    char* b = (char*)p->ws;
    auto take = [&](size_t bytes) { return (void*)(b + L.add(bytes)); };
    p->st = (DevState*)take(z.st);
    p->point_tab = (uint32_t*)take(z.sobol);
    p->sig = take(z.sig);
    p->sa_d = (double*)take(z.sa);
    p->ss_d = (double*)take(z.ss);
    p->Q_d = (double*)take(z.Q);
    p->src_cdf.q = (long long*)take(z.cdf_q);
    p->src_cdf.row_pre = (long long*)take(z.cdf_row);
    p->src_cdf.col_pre = (long long*)take(z.cdf_col);
    p->rem_cdf.q = (long long*)take(z.cdf_q);
    p->rem_cdf.row_pre = (long long*)take(z.cdf_row);
    p->rem_cdf.col_pre = (long long*)take(z.cdf_col);
    p->rem_f = (double*)take(z.rem_f);
    p->rem_q = (double*)take(z.rem_q);
    p->cell_scratch = (double*)take(z.scratch);
    p->bank[0] = take(z.bank);
    p->bank[1] = take(z.bank);
    p->stage = take(z.stage);
    p->tally_copies = tally_copies(&p->d);
    p->acc_pre = take(z.acc1);
    p->acc_post = take(z.acc1);
    p->acc_mom = take(z.acc4);
    p->pre_d = (double*)take(z.d1);
    p->post_d = (double*)take(z.d1);
    p->mom_d = (double*)take(z.d4);
    p->flux_d = (double*)take(z.d1);
    p->pre_raw = (double*)take(z.d1);
    p->post_raw = (double*)take(z.d1);
    p->sn_phi = take(z.sn4);
    p->sn_phi_old = take(z.sn4);
    p->sn_quad = take(z.sn16);
    p->sn_psi = take(z.sntx);
    p->sn_table = z.sntab ? take(z.sntab) : nullptr;
    p->sn_quadbuf = take(z.snqb);
    p->sn_phi_d = (double*)take(z.d4);
    p->sn_phi_d2 = (double*)take(z.d4);
    p->sn_norm = (double*)take(z.snnorm);
    p->blk = (long long*)take(z.blk);
    p->src_cdf.row_g = (int*)take(z.grow);
    p->src_cdf.col_g = (int*)take(z.gcol);
    p->rem_cdf.row_g = (int*)take(z.grow);
    p->rem_cdf.col_g = (int*)take(z.gcol);
    p->src_cdf.gr = p->rem_cdf.gr = z.gr;
    p->src_cdf.gc = p->rem_cdf.gc = z.gc;
    p->rem_f32 = (float*)take(z.remf32);
    p->rem_pos = (int*)take(z.rempos);
    for (int i = 0; i < 2; ++i) p->sort_pairs[i] = z.sortkv ? (unsigned long long*)take(z.sortkv) : nullptr;
    p->sort_scratch = z.sortc ? take(z.sortc) : nullptr;
    p->sig_inv = (float*)take(z.siginv);
    p->aa_hist = z.aah ? take(z.aah) : nullptr;
    p->aa_state = z.aas ? take(z.aas) : nullptr;
    p->ns_cell = z.nscell ? (int32_t*)take(z.nscell) : nullptr;
    p->sort_keys = z.sortkey ? (int32_t*)take(z.sortkey) : nullptr;
    p->byte_tab = z.btab ? (uint32_t*)take(z.btab) : nullptr;
    p->births_buf = z.births ? take(z.births) : nullptr;
    for (int i = 0; i < 2; ++i) p->live_buf[i] = z.live ? take(z.live) : nullptr;
    for (int i = 0; i < 2; ++i) p->live_pairs[i] = z.livekv ? (unsigned long long*)take(z.livekv) : nullptr;
    p->live_scratch = z.livesc ? take(z.livesc) : nullptr;
    p->live_cap = z.live_cap;
    p->births_step = -1;
    p->bank_sorted = p->d.census_order >= 1;   // the transposed pick-up order from the first leg on
    p->bank_cap = z.cap;
    p->stage_slots = z.slots;
    p->nblk_max = z.nblk;
}

hyb_status fail(hyb_problem* p, hyb_status s, const std::string& msg) {
    if (p) p->err = msg; else g_err = msg;
    return s;
}

hyb_status cuda_fail(hyb_problem* p, cudaError_t e, const char* where) {
    return fail(p, HYB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HYB_CU(p, call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(p, e_, #call); \
    } while (0)

hyb_status validate(const hyb_problem_desc* d, std::string* why) {
    if (!d) { *why = "null descriptor"; return HYB_EINVAL; }
    if (d->nx < 1 || d->ny < 1 || d->nx > 4096 || d->ny > 4096) { *why = "nx, ny must be in [1, 4096]"; return HYB_EINVAL; }
    if (!(d->lx > 0) || !(d->ly > 0) || !std::isfinite(d->lx) || !std::isfinite(d->ly)) { *why = "lx, ly must be finite and > 0"; return HYB_EINVAL; }
    if (!(d->c > 0) || !std::isfinite(d->c)) { *why = "c must be finite and > 0"; return HYB_EINVAL; }
    if (!(d->dt > 0) || !std::isfinite(d->dt)) { *why = "dt must be finite and > 0"; return HYB_EINVAL; }
    if (d->n_s < 0) { *why = "N_s must be >= 0"; return HYB_EINVAL; }
    if (d->n_s != HYB_NS_INF && d->n_s > (1 << 20)) { *why = "N_s must be <= 2^20 or HYB_NS_INF"; return HYB_EINVAL; }
    if (d->n_hist < 1 || d->n_hist >= (int64_t)1 << 31) { *why = "n_hist must be in [1, 2^31)"; return HYB_EINVAL; }
    if (d->census_cap < 0 || d->census_cap >= (int64_t)1 << 31) { *why = "census_cap must be in [0, 2^31)"; return HYB_EINVAL; }
    if (d->sampler != HYB_SOBOL_DS && d->sampler != HYB_PRNG && d->sampler != HYB_HALTON) {
        *why = "unknown sampler";
        return HYB_EINVAL;
    }
    if (d->precision != HYB_FP32 && d->precision != HYB_FP64) { *why = "unknown precision"; return HYB_EINVAL; }
    if (d->sn_order != 4 && d->sn_order != 8) { *why = "sn_order must be 4 or 8"; return HYB_EINVAL; }
    if (d->sn_max_iter < 1) { *why = "sn_max_iter must be >= 1"; return HYB_EINVAL; }
    if (d->census_order < 0 || d->census_order > 2) { *why = "census_order must be 0, 1 or 2"; return HYB_EINVAL; }
    if (d->census_order >= 1 && stage_slots(d, eff_cap(d)) >= ((int64_t)1 << 32)) {
        *why = "a sorted census holds fewer than 2^32 remap slots";   // 32-bit slot indices in the sort
        return HYB_EINVAL;
    }
    if (d->tally_copies < 0 || d->tally_copies > 64) { *why = "tally_copies must be in [0, 64]"; return HYB_EINVAL; }
    if (d->sort_every < 0) { *why = "sort_every must be >= 0"; return HYB_EINVAL; }
    if (d->leg_sort_every < 0) { *why = "leg_sort_every must be >= 0"; return HYB_EINVAL; }
    if (d->priv_tile < -1 || d->priv_tile > 32) { *why = "priv_tile must be in [-1, 32]"; return HYB_EINVAL; }
    if (d->leg_sort_every > 0 && eff_cap(d) + d->n_hist >= ((int64_t)1 << 31)) {
        *why = "the phased leg holds fewer than 2^31 histories (bank capacity + births)";   // 31-bit saved indices
        return HYB_EINVAL;
    }
    if (d->sn_accel < 0 || d->sn_accel > 8) { *why = "sn_accel must be in [0, 8]"; return HYB_EINVAL; }
    if (d->sn_warm_start < 0 || d->sn_warm_start > 2) { *why = "sn_warm_start must be 0, 1 or 2"; return HYB_EINVAL; }
    if (d->remap_variant != 0 && d->remap_variant != 1) { *why = "remap_variant must be 0 or 1"; return HYB_EINVAL; }
    if (d->sn_layout < 0 || d->sn_layout > 2) { *why = "sn_layout must be 0, 1 or 2"; return HYB_EINVAL; }
    if (d->seg_limit < 0 || d->seg_limit > (1 << 30)) { *why = "seg_limit must be in [0, 2^30]"; return HYB_EINVAL; }
    if (d->wait_limit < 0) { *why = "wait_limit must be >= 0"; return HYB_EINVAL; }
    if (d->remap_variant == 1 && d->n_s == HYB_NS_INF) {
        *why = "remap_variant 1 needs a finite N_s (N_s = infinity has no remap)";
        return HYB_EINVAL;
    }
    if (!(d->sn_tol >= 0) || !(d->w_min >= 0) || !(d->w_min < 1)) { *why = "sn_tol >= 0 and 0 <= w_min < 1 required"; return HYB_EINVAL; }
    if (!d->sigma_a || !d->sigma_s) { *why = "sigma_a and sigma_s are required"; return HYB_EINVAL; }
    const size_t nc = (size_t)d->nx * d->ny;
    if (d->n_s_cell) {
        if (d->n_s == HYB_NS_INF) { *why = "per-cell scatter limits need a finite n_s (their maximum)"; return HYB_EINVAL; }
        for (size_t k = 0; k < nc; ++k)
            if (d->n_s_cell[k] < 0 || d->n_s_cell[k] > d->n_s) {
                *why = "per-cell scatter limits must lie in [0, n_s]";
                return HYB_EINVAL;
            }
    }
    for (size_t k = 0; k < nc; ++k) {
        if (!std::isfinite(d->sigma_a[k]) || d->sigma_a[k] < 0 || !std::isfinite(d->sigma_s[k]) || d->sigma_s[k] < 0) {
            *why = "sigma_a, sigma_s must be finite and >= 0"; return HYB_EINVAL;
        }
        if (d->Q && (!std::isfinite(d->Q[k]) || d->Q[k] < 0)) { *why = "Q must be finite and >= 0"; return HYB_EINVAL; }
        if (d->ic_cell_w && (!std::isfinite(d->ic_cell_w[k]) || d->ic_cell_w[k] < 0)) { *why = "ic must be finite and >= 0"; return HYB_EINVAL; }
    }
    return HYB_OK;
}

template <typename T>
void put_sig(const hyb_problem_desc* d, std::vector<unsigned char>* out) {
    const size_t nc = (size_t)d->nx * d->ny;
    out->resize(nc * 2 * sizeof(T));
    T* s = (T*)out->data();
    for (size_t k = 0; k < nc; ++k) { s[2 * k] = (T)d->sigma_a[k]; s[2 * k + 1] = (T)d->sigma_s[k]; }
}

template <typename T>
void put_quad(const hyb_problem* p, std::vector<unsigned char>* out) {
    out->assign(7 * kMaxOrd * sizeof(T), 0);
    T* q = (T*)out->data();
    const int nq = p->n_ord / 4;
    for (int m = 0; m < p->n_ord; ++m) {
        q[m] = (T)p->quad_ox[m]; q[kMaxOrd + m] = (T)p->quad_oy[m]; q[2 * kMaxOrd + m] = (T)p->quad_w[m];
        // the sweep works in coordinates mirrored to +x, +y (quadrants 0..3: (+,+), (-,+), (-,-), (+,-));
        // its xi and eta coefficients change sign with the mirror
        const int quad = m / nq;
        const double sx = (quad == 0 || quad == 3) ? 1.0 : -1.0, sy = quad <= 1 ? 1.0 : -1.0;
        const double w = p->quad_w[m];
        T* wv = q + 3 * kMaxOrd + 4 * m;
        wv[0] = (T)w; wv[1] = (T)(w * sx); wv[2] = (T)(w * sy); wv[3] = (T)(w * sx * sy);
    }
}

// per-cell weight of one step's emission, (Q A) dt in that order of rounding
__global__ void cell_weight_kernel(const double* v, int n, double area, double dt, double* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = __dmul_rn(__dmul_rn(v[k], area), dt);
}

__global__ void set_nbank_kernel(DevState* st, long long n) { st->n_bank = n; }

double stat_w(const Acc128& a, int k) { return acc128_to_double(a.lo, a.hi, std::ldexp(1.0, -k)); }

void fill_leg_stats(const hyb_problem* p, hyb_leg_stats* s) {
    const DevState& h = *p->st_host;
    std::memset(s, 0, sizeof(*s));
    s->histories = (int64_t)h.histories; s->segments = (int64_t)h.segments; s->collisions = (int64_t)h.collisions;
    s->leaked = (int64_t)h.leaked; s->census = (int64_t)h.census; s->killed = (int64_t)h.killed;
    s->reached_limit = (int64_t)h.reached; s->errors = (int64_t)h.errors; s->tally_adds = (int64_t)h.tally_adds;
    s->w_source = stat_w(h.w_source, h.k_w); s->w_absorbed = stat_w(h.w_absorbed, h.k_w);
    s->w_leaked = stat_w(h.w_leaked, h.k_w); s->w_census = stat_w(h.w_census, h.k_w);
    s->w_handoff = stat_w(h.w_handoff, h.k_w); s->w_killed = stat_w(h.w_killed, h.k_w);
    s->bank_size = h.n_bank;
}

void fill_remap_stats(const hyb_problem* p, hyb_leg_stats* s) {
    const DevState& h = *p->st_host;
    std::memset(s, 0, sizeof(*s));
    s->histories = (int64_t)h.r_histories; s->segments = (int64_t)h.r_segments; s->leaked = (int64_t)h.r_leaked;
    s->killed = (int64_t)h.r_killed; s->errors = (int64_t)h.r_errors; s->census = h.out_count;
    // a bank pre-pass (if any) summed its slots at its own scale: zero accumulators otherwise
    s->w_source = stat_w(h.r_w_source, h.k_rw) + stat_w(h.r_wb[0], h.k_rwb);
    s->w_absorbed = stat_w(h.r_w_absorbed, h.k_rw) + stat_w(h.r_wb[1], h.k_rwb);
    s->w_leaked = stat_w(h.r_w_leaked, h.k_rw) + stat_w(h.r_wb[2], h.k_rwb);
    s->w_killed = stat_w(h.r_w_killed, h.k_rw) + stat_w(h.r_wb[3], h.k_rwb);
    s->w_census = h.bank_wsum;
    s->combed = h.comb_on;
    s->bank_size = h.n_bank;
}

hyb_status pull_state(hyb_problem* p) {
    HYB_CU(p, cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
    HYB_CU(p, cudaStreamSynchronize(p->stream));
    p->status_pending = false;   // every error bit set so far is in this read
    if (p->st_host->bank_bad) {   // reported once, by the first check after the upload
        HYB_CU(p, cudaMemsetAsync(&p->st->bank_bad, 0, sizeof(unsigned int), p->stream));
        return fail(p, HYB_EINVAL, "the bank set with hyb_set_bank_native holds particles outside the problem "
                                   "(cell index, in-cell offset, direction or weight)");
    }
    if (p->st_host->status & kStBounds) return fail(p, HYB_EBOUNDS, "device index check failed (bank cell out of range)");
    if (p->st_host->status & kStSegments)
        return fail(p, HYB_ETIMEOUT, "a device loop bound was exhausted (history segments, sweep or census-sort wait)");
    return HYB_OK;
}

template <typename T>
static hyb_status get_bank_t(hyb_problem* p, int32_t* cell, double* fx, double* fy, double* ox, double* oy, double* w,
                             int64_t* n_io) {
    HYB_CU(p, cudaMemcpyAsync(&p->st_host->n_bank, &p->st->n_bank, sizeof(long long), cudaMemcpyDeviceToHost, p->stream));
    HYB_CU(p, cudaStreamSynchronize(p->stream));
    const int64_t n = p->st_host->n_bank;
    if (*n_io < n) { *n_io = n; return fail(p, HYB_ECAPACITY, "host arrays too small for the bank"); }
    BankView<T> b = bank_view<T>(p, p->cur);
    std::vector<T> tmp((size_t)n);
    HYB_CU(p, cudaMemcpy(cell, b.cell, (size_t)n * 4, cudaMemcpyDeviceToHost));
    T* src[5] = {b.fx, b.fy, b.ox, b.oy, b.w};
    double* dst[5] = {fx, fy, ox, oy, w};
    for (int q = 0; q < 5; ++q) {
        if (n) HYB_CU(p, cudaMemcpy(tmp.data(), src[q], (size_t)n * sizeof(T), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) dst[q][i] = (double)tmp[(size_t)i];
    }
    *n_io = n;
    return HYB_OK;
}

// Particles of a bank outside the problem (the checks of hyb_set_bank, on the device): counted
// into st->bank_bad, which the next synchronising call reports.
template <typename T>
__global__ void bank_check_kernel(BankView<T> b, long long n, int ncells, T dx, T dy, DevState* st) {
    unsigned int bad = 0;
    const T tx = dx * T(1.000001), ty = dy * T(1.000001), one = T(1.000001);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = b.cell[i];
        const T fx = b.fx[i], fy = b.fy[i], ox = b.ox[i], oy = b.oy[i], w = b.w[i];
        const bool ok = c >= 0 && c < ncells && fx >= T(0) && fx <= tx && fy >= T(0) && fy <= ty && isfinite(ox) &&
                        isfinite(oy) && ox * ox + oy * oy <= one && isfinite(w);
        bad += ok ? 0u : 1u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&st->bank_bad, bad);
}

// Bank upload from device memory in three launches: the new size with the statistics zeroed;
// copy, checks and max |w| in one pass; sum |w| (at the scale its max fixes) with the final
// conversion in the last block.
__global__ void bank_begin_kernel(DevState* st, long long n) {
    st->n_bank = n;
    st->bank_bad = 0u;
    st->bank_wmax = 0.0;
    st->bank_wsum_acc.lo = 0ull;
    st->bank_wsum_acc.hi = 0ull;
}

template <typename T>
__global__ void bank_load_kernel(BankView<T> b, const int32_t* __restrict__ sc, const T* __restrict__ sfx,
                                 const T* __restrict__ sfy, const T* __restrict__ sox, const T* __restrict__ soy,
                                 const T* __restrict__ sw, long long n, int ncells, T dx, T dy, DevState* st) {
    unsigned int bad = 0;
    double m = 0;
    const T tx = dx * T(1.000001), ty = dy * T(1.000001), one = T(1.000001);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = sc[i];
        const T fx = sfx[i], fy = sfy[i], ox = sox[i], oy = soy[i], w = sw[i];
        b.cell[i] = c; b.fx[i] = fx; b.fy[i] = fy; b.ox[i] = ox; b.oy[i] = oy; b.w[i] = w;
        const bool ok = c >= 0 && c < ncells && fx >= T(0) && fx <= tx && fy >= T(0) && fy <= ty && isfinite(ox) &&
                        isfinite(oy) && ox * ox + oy * oy <= one && isfinite(w);
        bad += ok ? 0u : 1u;
        m = fmax(m, fabs((double)w));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_down_sync(0xffffffffu, bad, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(&st->bank_bad, bad);
        if (m > 0) atomicMax((unsigned long long*)&st->bank_wmax, (unsigned long long)__double_as_longlong(m));
    }
}

// sum |w| of the bank (block order, 128-bit fixed point at the scale n max|w| fixes), the last
// block converting it to bank_wsum
template <typename T>
__global__ void bank_wsum_last_kernel(const T* w, DevState* st) {
    const long long n = st->n_bank;
    const int kw = scale_exponent((double)n * st->bank_wmax, 125);
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
        to_i128(t * ldexp(1.0, kw), &lo, &hi);
        atomic_add128(&st->bank_wsum_acc, lo, hi);
        __threadfence();
        if (atomicAdd(&st->bank_done, 1u) == gridDim.x - 1u) {
            __threadfence();
            const unsigned long long alo = atomicAdd(&st->bank_wsum_acc.lo, 0ull);
            const unsigned long long ahi = atomicAdd(&st->bank_wsum_acc.hi, 0ull);
            st->bank_wsum = acc128_to_double(alo, ahi, ldexp(1.0, -kw));
            st->bank_done = 0u;
        }
    }
}

static bool on_device(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A bank already in the problem's layout and precision (host memory, pinned for an asynchronous
// copy, or device memory): copied on the problem's stream and checked on the device.
template <typename T>
static hyb_status set_bank_native_t(hyb_problem* p, const int32_t* cell, const void* const* f, int64_t n) {
    BankView<T> b = bank_view<T>(p, p->cur);
    if (n && on_device(cell) && on_device(f[0]) && on_device(f[1]) && on_device(f[2]) && on_device(f[3]) &&
        on_device(f[4])) {
        const int g = (int)std::min<long long>((n + 255) / 256, 152 * 8);
        bank_begin_kernel<<<1, 1, 0, p->stream>>>(p->st, n);
        bank_load_kernel<T><<<g, 256, 0, p->stream>>>(b, cell, (const T*)f[0], (const T*)f[1], (const T*)f[2],
                                                      (const T*)f[3], (const T*)f[4], n, p->ncells, (T)p->dx,
                                                      (T)p->dy, p->st);
        // the same grid as the statistics kernels of the other uploads (same block sums, same total)
        const int gs = (int)std::min<long long>((p->bank_cap + kTile - 1) / kTile, 152 * 8);
        bank_wsum_last_kernel<T><<<gs > 0 ? gs : 1, kTile, 0, p->stream>>>(b.w, p->st);
        HYB_CU(p, cudaGetLastError());
        return HYB_OK;
    }
    HYB_CU(p, cudaMemsetAsync(&p->st->bank_bad, 0, sizeof(unsigned int), p->stream));
    if (n) {
        HYB_CU(p, cudaMemcpyAsync(b.cell, cell, (size_t)n * 4, cudaMemcpyDefault, p->stream));
        T* dst[5] = {b.fx, b.fy, b.ox, b.oy, b.w};
        for (int q = 0; q < 5; ++q)
            HYB_CU(p, cudaMemcpyAsync(dst[q], f[q], (size_t)n * sizeof(T), cudaMemcpyDefault, p->stream));
        const long long g = (n + 255) / 256;
        bank_check_kernel<T><<<(unsigned)(g < 152 * 4 ? g : 152 * 4), 256, 0, p->stream>>>(b, n, p->ncells, (T)p->dx,
                                                                                            (T)p->dy, p->st);
        HYB_CU(p, cudaGetLastError());
    }
    set_nbank_kernel<<<1, 1, 0, p->stream>>>(p->st, n);
    HYB_CU(p, cudaGetLastError());
    HYB_CU(p, launch_bank_stats(p));
    return HYB_OK;
}

template <typename T>
static hyb_status set_bank_t(hyb_problem* p, const int32_t* cell, const double* fx, const double* fy, const double* ox,
                             const double* oy, const double* w, int64_t n) {
    HYB_CU(p, cudaStreamSynchronize(p->stream));
    HYB_CU(p, cudaMemsetAsync(&p->st->bank_bad, 0, sizeof(unsigned int), p->stream));
    BankView<T> b = bank_view<T>(p, p->cur);
    std::vector<T> tmp((size_t)n);
    if (n) HYB_CU(p, cudaMemcpy(b.cell, cell, (size_t)n * 4, cudaMemcpyHostToDevice));
    T* dst[5] = {b.fx, b.fy, b.ox, b.oy, b.w};
    const double* src[5] = {fx, fy, ox, oy, w};
    for (int q = 0; q < 5; ++q) {
        for (int64_t i = 0; i < n; ++i) tmp[(size_t)i] = (T)src[q][i];
        if (n) HYB_CU(p, cudaMemcpy(dst[q], tmp.data(), (size_t)n * sizeof(T), cudaMemcpyHostToDevice));
    }
    set_nbank_kernel<<<1, 1, 0, p->stream>>>(p->st, n);
    HYB_CU(p, cudaGetLastError());
    HYB_CU(p, launch_bank_stats(p));
    HYB_CU(p, cudaStreamSynchronize(p->stream));
    return HYB_OK;
}

}  // namespace hybh

using namespace hybh;

namespace hyb {
double sn_tol_eff(const hyb_problem* p) { return p->prec == HYB_FP64 ? p->d.sn_tol : std::max(p->d.sn_tol, 2e-6); }
}  // namespace hyb

extern "C" {

const char* hyb_status_string(hyb_status s) {
    switch (s) {
        case HYB_OK: return "ok";
        case HYB_EINVAL: return "invalid argument";
        case HYB_ENOMEM: return "out of memory / workspace too small";
        case HYB_ECUDA: return "CUDA error";
        case HYB_ETIMEOUT: return "bounded device loop exhausted";
        case HYB_ESTATE: return "call out of order";
        case HYB_EBOUNDS: return "device bounds check failed";
        case HYB_ECAPACITY: return "capacity exceeded";
    }
    return "unknown status";
}

const char* hyb_last_error(const hyb_problem* p) { return p ? p->err.c_str() : g_err.c_str(); }

hyb_status hyb_workspace_size(const hyb_problem_desc* d, size_t* bytes) {
    std::string why;
    hyb_status s = validate(d, &why);
    if (s != HYB_OK) return fail(nullptr, s, why);
    if (!bytes) return fail(nullptr, HYB_EINVAL, "bytes is NULL");
    *bytes = layout_bytes(d);
    return HYB_OK;
}

hyb_status hyb_priv_window(const hyb_problem_desc* d, int32_t* x0, int32_t* y0, int32_t* side) {
    std::string why;
    hyb_status s = validate(d, &why);
    if (s != HYB_OK) return fail(nullptr, s, why);
    if (!x0 || !y0 || !side) return fail(nullptr, HYB_EINVAL, "output is NULL");
    int a = 0, b = 0, c = 0;
    choose_priv_window(d, &a, &b, &c);
    *x0 = a; *y0 = b; *side = c;
    return HYB_OK;
}

hyb_status hyb_sobol_table(int32_t ndims, uint32_t* out) {
    if (ndims < 1 || ndims > HYB_SOBOL_DIMS || !out) return fail(nullptr, HYB_EINVAL, "ndims out of range");
    std::memcpy(out, sobol_table_host(), (size_t)ndims * 32 * sizeof(uint32_t));
    return HYB_OK;
}

hyb_status hyb_quadrature(int32_t order, double* ox, double* oy, double* w, int32_t* m) {
    if ((order != 4 && order != 8) || !m) return fail(nullptr, HYB_EINVAL, "order must be 4 or 8");
    const int need = order == 4 ? 12 : 40;
    if (*m < need) return fail(nullptr, HYB_EINVAL, "capacity too small");
    int mm = 0;
    quadrature_host(order, ox, oy, w, &mm);
    *m = mm;
    return HYB_OK;
}

hyb_status hyb_create_problem(const hyb_problem_desc* d, void* workspace, size_t ws_bytes, void* cuda_stream,
                              hyb_problem** out) {
    std::string why;
    hyb_status s = validate(d, &why);
    if (s != HYB_OK) return fail(nullptr, s, why);
    if (!out) return fail(nullptr, HYB_EINVAL, "out is NULL");
    *out = nullptr;
    const size_t need = layout_bytes(d);
    if (workspace && ws_bytes < need) return fail(nullptr, HYB_ENOMEM, "workspace smaller than hyb_workspace_size");
    if (workspace && ((uintptr_t)workspace & 255u)) return fail(nullptr, HYB_EINVAL, "workspace must be 256-byte aligned");
    hyb_problem* p = new (std::nothrow) hyb_problem();
    if (!p) return fail(nullptr, HYB_ENOMEM, "host allocation failed");
    p->d = *d;
    choose_priv_window(d, &p->priv_x0, &p->priv_y0, &p->priv_side);
    p->d.sigma_a = p->d.sigma_s = p->d.Q = p->d.ic_cell_w = nullptr;
    p->nx = d->nx; p->ny = d->ny; p->ncells = d->nx * d->ny;
    p->dx = d->lx / d->nx; p->dy = d->ly / d->ny; p->area = p->dx * p->dy;
    p->prec = d->precision;
    p->stream = (cudaStream_t)cuda_stream;
    p->step = 0;
    p->cur = 0;
    p->ndims = d->n_s == HYB_NS_INF ? HYB_SOBOL_DIMS : 5 + 3 * d->n_s;   // dims past the table: counter hash
    p->leg_done = p->sn_done = false;
    p->pdl = true;
    p->sn_warm = false;
    p->ev0 = p->ev1 = nullptr;
    for (auto& e : p->evs) e = nullptr;
    p->st_host = nullptr;
    if (workspace) { p->ws = workspace; p->ws_bytes = ws_bytes; p->owns_ws = false; }
    else {
        cudaError_t e = cudaMalloc(&p->ws, need);
        if (e != cudaSuccess) { delete p; return fail(nullptr, HYB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
        p->ws_bytes = need; p->owns_ws = true;
    }
    assign(p);
    auto bail = [&](hyb_status st) {
        g_err = p->err;
        hyb_destroy_problem(p);
        return st;
    };
    if (cudaMallocHost((void**)&p->st_host, sizeof(DevState)) != cudaSuccess) return bail(fail(p, HYB_ENOMEM, "pinned alloc"));
    if (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess)
        return bail(fail(p, HYB_ECUDA, "event create"));
    for (auto& e : p->evs)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(p, HYB_ECUDA, "event create"));
    for (auto& e : p->evk)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(p, HYB_ECUDA, "event create"));
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(p, HYB_ECUDA, "side stream create"));
    const size_t nc = (size_t)p->ncells;
    p->sig_s_max = 0;
    for (size_t k = 0; k < nc; ++k) p->sig_s_max = std::max(p->sig_s_max, d->sigma_s[k]);
    // device copies of the problem data
    std::vector<unsigned char> sig;
    if (p->prec == HYB_FP64) put_sig<double>(d, &sig); else put_sig<float>(d, &sig);
    std::vector<double> zeros(nc, 0.0);
    cudaStream_t st = p->stream;
    auto chk = [&](cudaError_t e, const char* w) { return e == cudaSuccess ? HYB_OK : cuda_fail(p, e, w); };
    if (chk(cudaMemsetAsync(p->st, 0, sizeof(DevState), st), "memset state") != HYB_OK) return bail(HYB_ECUDA);
    size_t ptab_bytes = 0;
    const uint32_t* ptab = point_table_host(d->sampler, &ptab_bytes);
    if (chk(cudaMemcpyAsync(p->point_tab, ptab, ptab_bytes, cudaMemcpyHostToDevice, st), "copy point table") != HYB_OK) return bail(HYB_ECUDA);
    std::vector<uint32_t> btab;
    if (p->byte_tab) {
        // Sobol byte tables of the births' dimensions: entry (d, k, v) = XOR of the direction numbers
        // of dimension d over the set bits of v, bits 8k..8k+7 of the index
        btab.assign((size_t)kByteDims * kByteWords, 0u);
        for (int dd = 0; dd < kByteDims; ++dd)
            for (int k = 0; k < 4; ++k)
                for (int v = 0; v < 256; ++v) {
                    uint32_t x = 0;
                    for (int j = 0; j < 8; ++j)
                        if ((v >> j) & 1) x ^= ptab[dd * 32 + 8 * k + j];
                    btab[(size_t)dd * kByteWords + 256 * k + v] = x;
                }
        if (chk(cudaMemcpyAsync(p->byte_tab, btab.data(), btab.size() * 4, cudaMemcpyHostToDevice, st), "copy byte tables") != HYB_OK)
            return bail(HYB_ECUDA);
    }
    if (chk(cudaMemcpyAsync(p->sig, sig.data(), sig.size(), cudaMemcpyHostToDevice, st), "copy sigma") != HYB_OK) return bail(HYB_ECUDA);
    // FP32 path: one 32-byte record per cell (a single memory sector): the reciprocals (1/sigma_a,
    // 1/sigma_s, 1/sigma_t), 0 where the cross section is 0, the cell's scatter limit as the bits of
    // the fourth word (space-dependent N_s), then sigma_a and sigma_s
    std::vector<float> sinv(8 * nc, 0.0f);
    for (size_t k = 0; k < nc; ++k) {
        const double sa = d->sigma_a[k], ss = d->sigma_s[k], stt = sa + ss;
        sinv[8 * k] = sa > 0 ? (float)(1.0 / sa) : 0.0f;
        sinv[8 * k + 1] = ss > 0 ? (float)(1.0 / ss) : 0.0f;
        sinv[8 * k + 2] = stt > 0 ? (float)(1.0 / stt) : 0.0f;
        const int32_t lim = d->n_s_cell ? d->n_s_cell[k] : 0;
        std::memcpy(&sinv[8 * k + 3], &lim, 4);
        sinv[8 * k + 4] = (float)sa;
        sinv[8 * k + 5] = (float)ss;
    }
    if (d->n_s_cell &&
        chk(cudaMemcpyAsync(p->ns_cell, d->n_s_cell, nc * 4, cudaMemcpyHostToDevice, st), "copy limits") != HYB_OK)
        return bail(HYB_ECUDA);
    p->d.n_s_cell = nullptr;   // the caller's array is not kept: p->ns_cell holds the copy
    if (chk(cudaMemcpyAsync(p->sig_inv, sinv.data(), sinv.size() * 4, cudaMemcpyHostToDevice, st), "copy 1/sigma") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(cudaMemcpyAsync(p->sa_d, d->sigma_a, nc * 8, cudaMemcpyHostToDevice, st), "copy sa") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(cudaMemcpyAsync(p->ss_d, d->sigma_s, nc * 8, cudaMemcpyHostToDevice, st), "copy ss") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(cudaMemcpyAsync(p->Q_d, d->Q ? d->Q : zeros.data(), nc * 8, cudaMemcpyHostToDevice, st), "copy Q") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(cudaMemsetAsync(p->sn_phi_d, 0, 4 * nc * 8, st), "memset phi") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(cudaMemsetAsync(p->sn_phi_d2, 0, 4 * nc * 8, st), "memset phi") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(sn_clear_counters(p), "memset reduction counters") != HYB_OK) return bail(HYB_ECUDA);
    // sweep-source entries that hold no cell stay zero (only cells are ever written)
    if (chk(cudaMemsetAsync(p->sn_quad, 0, sn_src_bytes(d->nx, d->ny, d->sn_order == 8 ? 40 : 12, p->prec == HYB_FP64, d->sn_layout), st), "memset sweep sources") != HYB_OK)
        return bail(HYB_ECUDA);
    // quadrature
    p->n_ord = 0;
    quadrature_host(d->sn_order, p->quad_ox, p->quad_oy, p->quad_w, &p->n_ord);
    std::vector<unsigned char> qb;
    if (p->prec == HYB_FP64) put_quad<double>(p, &qb); else put_quad<float>(p, &qb);
    if (chk(cudaMemcpyAsync(p->sn_quadbuf, qb.data(), qb.size(), cudaMemcpyHostToDevice, st), "copy quad") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(sn_build_table(p), "cell-solve table") != HYB_OK) return bail(HYB_ECUDA);
    // static source CDF: cell weights Q A dt
    double* cw = p->cell_scratch + 256 + p->ny;
    double* scal = (double*)p->rem_f;   // two scalars of scratch before the first remap
    double host_sc[2] = {0, 0};
    p->has_src = false;
    p->w_src = 0;
    if (d->Q) {
        if (chk(cudaMemcpyAsync(cw, d->Q, nc * 8, cudaMemcpyHostToDevice, st), "copy Q weights") != HYB_OK) return bail(HYB_ECUDA);
        cell_weight_kernel<<<(p->ncells + 255) / 256, 256, 0, st>>>(cw, p->ncells, p->area, d->dt, cw);
        if (chk(launch_cdf_build(p, cw, p->src_cdf, scal, scal + 1), "source cdf") != HYB_OK) return bail(HYB_ECUDA);
        if (chk(cudaMemcpyAsync(host_sc, scal, 16, cudaMemcpyDeviceToHost, st), "read W") != HYB_OK) return bail(HYB_ECUDA);
        if (chk(cudaStreamSynchronize(st), "sync") != HYB_OK) return bail(HYB_ECUDA);
        p->w_src = host_sc[0];
        p->has_src = host_sc[0] > 0;
    }
    // initial bank from the initial weight per cell (stream INIT)
    long long nb = 0;
    if (d->ic_cell_w) {
        double Wic = 0;
        for (size_t k = 0; k < nc; ++k) Wic += d->ic_cell_w[k];
        if (Wic > 0) {
            if (chk(cudaMemcpyAsync(cw, d->ic_cell_w, nc * 8, cudaMemcpyHostToDevice, st), "copy ic") != HYB_OK) return bail(HYB_ECUDA);
            if (chk(launch_cdf_build(p, cw, p->rem_cdf, scal, scal + 1), "ic cdf") != HYB_OK) return bail(HYB_ECUDA);
            if (chk(cudaMemcpyAsync(host_sc, scal, 16, cudaMemcpyDeviceToHost, st), "read Wic") != HYB_OK) return bail(HYB_ECUDA);
            if (chk(cudaStreamSynchronize(st), "sync") != HYB_OK) return bail(HYB_ECUDA);
            if (chk(launch_init_bank(p, p->rem_cdf, host_sc[0] / (double)d->n_hist), "init bank") != HYB_OK) return bail(HYB_ECUDA);
            nb = d->n_hist;
        }
    }
    set_nbank_kernel<<<1, 1, 0, st>>>(p->st, nb);
    if (chk(launch_bank_stats(p), "bank stats") != HYB_OK) return bail(HYB_ECUDA);
    if (chk(cudaStreamSynchronize(st), "sync") != HYB_OK) return bail(HYB_ECUDA);
    *out = p;
    return HYB_OK;
}

hyb_status hyb_destroy_problem(hyb_problem* p) {
    if (!p) return HYB_OK;
    if (p->stream) cudaStreamSynchronize(p->stream); else cudaDeviceSynchronize();
    if (p->side) { cudaStreamSynchronize(p->side); cudaStreamDestroy(p->side); }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->owns_ws && p->ws) cudaFree(p->ws);
    if (p->st_host) cudaFreeHost(p->st_host);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    for (auto e : p->evs)
        if (e) cudaEventDestroy(e);
    for (auto e : p->evk)
        if (e) cudaEventDestroy(e);
    delete p;
    return HYB_OK;
}

// step 1 launches over the history range [h0, h1) (no host synchronisation); normalise = false
// leaves the raw integer tallies (a shard of a history-sharded leg)
// zero the device status word for the call about to run, unless an unchecked asynchronous step
// may have set error bits there (they stay until a synchronising call reads them)
static cudaError_t clear_status(hyb_problem* p) {
    if (p->status_pending) return cudaSuccess;
    return cudaMemsetAsync(&p->st->status, 0, sizeof(int), p->stream);
}

static hyb_status leg_launch(hyb_problem* p, int32_t* hist, long long h0 = 0, long long h1 = LLONG_MAX,
                             bool normalise = true) {
    const size_t nc = (size_t)p->ncells;
    const size_t acc = p->prec == HYB_FP64 ? 16 : 8;
    const size_t ncp = (size_t)p->tally_copies;
    HYB_CU(p, drop_bank_prepass(p));   // the leg's births reuse the staging buffer
    if (!p->acc_clean) {   // else the last normalisation zeroed them
        HYB_CU(p, cudaMemsetAsync(p->acc_pre, 0, ncp * nc * acc, p->stream));
        HYB_CU(p, cudaMemsetAsync(p->acc_post, 0, ncp * nc * acc, p->stream));
        HYB_CU(p, cudaMemsetAsync(p->acc_mom, 0, ncp * 4 * nc * acc, p->stream));
    }
    p->acc_clean = false;
    HYB_CU(p, cudaMemsetAsync(p->st, 0, offsetof(DevState, r_histories), p->stream));
    HYB_CU(p, clear_status(p));
    HYB_CU(p, launch_mc_leg(p, hist, h0, h1));
    if (normalise) HYB_CU(p, launch_leg_normalise(p));
    p->leg_done = normalise;
    p->sn_done = false;
    return HYB_OK;
}

// device time of the last MC leg kernel (events around its launch; the stream has been synchronised)
static float leg_kernel_ms(hyb_problem* p) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p->evk[0], p->evk[1]) != cudaSuccess) {
        cudaGetLastError();   // events not recorded yet: report 0
        return 0.f;
    }
    return ms;
}

static hyb_status leg_impl(hyb_problem* p, int32_t* hist, hyb_leg_stats* out) {
    if (!p) return fail(nullptr, HYB_EINVAL, "null problem");
    HYB_CU(p, cudaEventRecord(p->ev0, p->stream));
    hyb_status s0 = leg_launch(p, hist);
    if (s0 != HYB_OK) return s0;
    HYB_CU(p, cudaEventRecord(p->ev1, p->stream));
    if (out) {
        hyb_status s = pull_state(p);
        fill_leg_stats(p, out);
        float ms = 0;
        cudaEventElapsedTime(&ms, p->ev0, p->ev1);
        out->ms = ms;
        out->ms_leg_kernel = leg_kernel_ms(p);
        if (s != HYB_OK) return s;
    }
    return HYB_OK;
}

hyb_status hyb_mc_leg(hyb_problem* p, hyb_leg_stats* out) { return leg_impl(p, nullptr, out); }
hyb_status hyb_mc_leg_trace(hyb_problem* p, int32_t* hist, hyb_leg_stats* out) { return leg_impl(p, hist, out); }

// history-sharded leg: a range of the history index space into an exchange block, and a summed
// block back into the problem's tallies
hyb_status hyb_leg_exchange_bytes(const hyb_problem* p, size_t* bytes) {
    if (!p || !bytes) return fail(nullptr, HYB_EINVAL, "null argument");
    *bytes = leg_exchange_words(p) * sizeof(long long);
    return HYB_OK;
}

hyb_status hyb_mc_leg_range(hyb_problem* p, int64_t h0, int64_t h1, void* x_dev, size_t x_bytes, int32_t* hist_dev) {
    if (!p) return fail(nullptr, HYB_EINVAL, "null problem");
    if (h0 < 0 || h1 < h0) return fail(p, HYB_EINVAL, "history range must satisfy 0 <= h0 <= h1");
    if (!x_dev || ((uintptr_t)x_dev & 7)) return fail(p, HYB_EINVAL, "exchange block must be an 8-byte aligned device pointer");
    if (x_bytes < leg_exchange_words(p) * sizeof(long long)) return fail(p, HYB_ENOMEM, "exchange block too small");
    hyb_status s = leg_launch(p, hist_dev, h0, h1, false);
    if (s != HYB_OK) return s;
    HYB_CU(p, launch_leg_pack(p, (long long*)x_dev));
    return HYB_OK;
}

hyb_status hyb_mc_leg_reduce_finish(hyb_problem* p, const void* x_dev, size_t x_bytes, hyb_leg_stats* out) {
    if (!p) return fail(nullptr, HYB_EINVAL, "null problem");
    if (!x_dev || ((uintptr_t)x_dev & 7)) return fail(p, HYB_EINVAL, "exchange block must be an 8-byte aligned device pointer");
    if (x_bytes < leg_exchange_words(p) * sizeof(long long)) return fail(p, HYB_ENOMEM, "exchange block too small");
    HYB_CU(p, launch_leg_unpack(p, (const long long*)x_dev));
    HYB_CU(p, launch_leg_normalise(p));
    p->leg_done = true;
    p->sn_done = false;
    if (out) {
        hyb_status s = pull_state(p);
        fill_leg_stats(p, out);
        if (s != HYB_OK) return s;
    }
    return HYB_OK;
}

// step 2: source iteration with a device-side stop test. With a warm start the previous step's
// count predicts this one: that many iterations are queued without a read-back (iterations after
// convergence return at once), then the flag is read once, and only a solve that needs more
// iterations reads it after each further one. *iters: iterations taken. keep_status: the status
// word still holds the leg's bits of this step (checked here together with the sweep's).
static hyb_status sn_run(hyb_problem* p, int* iters, bool keep_status) {
    if (!keep_status) HYB_CU(p, clear_status(p));
    HYB_CU(p, sn_start(p));
    const int unchecked = (p->sn_warm && p->last_sn_iters > 0) ? std::min(p->last_sn_iters, p->d.sn_max_iter) : 0;
    // one read-back brings the status word and the stop state together (the span from status to
    // sn_iters); the loop only ends right after such a read, so no further read is needed
    const size_t off = offsetof(DevState, status);
    const size_t len = offsetof(DevState, sn_iters) + sizeof(int) - off;
    for (int it = 1; it <= p->d.sn_max_iter; ++it) {
        HYB_CU(p, sn_iteration(p, it == 1));
        if (it < unchecked) continue;
        HYB_CU(p, cudaMemcpyAsync((char*)p->st_host + off, (const char*)p->st + off, len, cudaMemcpyDeviceToHost,
                                  p->stream));
        HYB_CU(p, cudaStreamSynchronize(p->stream));
        p->status_pending = false;   // the read holds every error bit set so far
        if (p->st_host->sn_conv) break;
    }
    if (p->st_host->status & kStBounds) return fail(p, HYB_EBOUNDS, "device index check failed (bank cell out of range)");
    if (p->st_host->status & kStSegments)
        return fail(p, HYB_ETIMEOUT, keep_status ? "a device loop bound was exhausted (history segments or sweep wait)"
                                                 : "S_N sweep pipeline wait exhausted");
    const int it = p->st_host->sn_iters;
    HYB_CU(p, sn_finish(p));
    p->last_sn_iters = it;
    p->sn_done = true;
    p->sn_warm = p->d.sn_warm_start != 0;
    *iters = it;
    return HYB_OK;
}

hyb_status hyb_collided_solve(hyb_problem* p, hyb_leg_stats* out) {
    if (!p) return fail(nullptr, HYB_EINVAL, "null problem");
    p->pdl = true;   // stepped alone (a batch sets its members' launches itself)
    if (!p->leg_done) return fail(p, HYB_ESTATE, "collided solve needs an MC leg of this step");
    if (p->d.n_s == HYB_NS_INF) {   // nothing is handed off: the collided flux stays zero
        p->sn_done = true;
        if (out) std::memset(out, 0, sizeof(*out));
        return HYB_OK;
    }
    HYB_CU(p, cudaEventRecord(p->ev0, p->stream));
    int it = 0;
    hyb_status s = sn_run(p, &it, false);
    if (s != HYB_OK) return s;
    HYB_CU(p, cudaEventRecord(p->ev1, p->stream));
    if (out) {
        std::memset(out, 0, sizeof(*out));
        HYB_CU(p, cudaEventSynchronize(p->ev1));
        float ms = 0;
        cudaEventElapsedTime(&ms, p->ev0, p->ev1);
        out->ms = ms;
        out->sn_iterations = it;
    }
    return HYB_OK;
}

// steps 3-4 launches (no host synchronisation); for N_s = infinity the MC-leg census is the new
// bank (no remap) and the step flux is the MC tally alone
static hyb_status remap_launch(hyb_problem* p) {
    HYB_CU(p, clear_status(p));
    if (p->d.n_s == HYB_NS_INF) {
        HYB_CU(p, launch_census(p));
        HYB_CU(p, launch_flux(p));
    } else {
        HYB_CU(p, launch_remap(p));
    }
    p->cur = 1 - p->cur;
    p->step += 1;           // the remap's last kernel advances the device step
    p->leg_done = p->sn_done = false;
    p->pdl = true;
    return HYB_OK;
}

hyb_status hyb_remap(hyb_problem* p, hyb_leg_stats* out) {
    if (!p) return fail(nullptr, HYB_EINVAL, "null problem");
    p->pdl = true;
    if (!p->leg_done || (!p->sn_done && p->d.n_s != HYB_NS_INF))
        return fail(p, HYB_ESTATE, "remap needs an MC leg and a collided solve of this step");
    HYB_CU(p, cudaEventRecord(p->ev0, p->stream));
    hyb_status s0 = remap_launch(p);
    if (s0 != HYB_OK) return s0;
    HYB_CU(p, cudaEventRecord(p->ev1, p->stream));
    if (out) {
        hyb_status s = pull_state(p);
        fill_remap_stats(p, out);
        float ms = 0;
        cudaEventElapsedTime(&ms, p->ev0, p->ev1);
        out->ms = ms;
        if (s != HYB_OK) return s;
    }
    return HYB_OK;
}

// A whole step synchronises with the host twice: once inside the source iteration (stop test)
// and, with statistics, once at the end, when the leg and remap counters (kept apart in the
// device state) are read together. The leg's status bits are checked with the remap's.
// One step's launches (steps 1-4). The host waits inside the collided solve (stop test) only;
// with events, the phase boundaries are recorded on the stream.
static hyb_status step_launch(hyb_problem* p, int* iters, bool events) {
    if (events) HYB_CU(p, cudaEventRecord(p->evs[0], p->stream));
    hyb_status s = leg_launch(p, nullptr);
    if (s != HYB_OK) return s;
    if (events) HYB_CU(p, cudaEventRecord(p->evs[1], p->stream));
    *iters = 0;
    if (p->d.n_s != HYB_NS_INF) {
        // Eq. (R): the step-start bank's re-stream needs neither the collided flux nor the remap
        // density, so it runs on the side stream beside the solve
        if (p->d.remap_variant == 0) {
            HYB_CU(p, launch_remap_bank_prepass(p));
            // and the next step's source births (they depend on the step index alone)
            HYB_CU(p, launch_births_ahead(p));
        }
        s = sn_run(p, iters, true);
        if (s != HYB_OK) return s;
    } else {
        p->sn_done = true;
    }
    if (events) HYB_CU(p, cudaEventRecord(p->evs[2], p->stream));
    s = remap_launch(p);
    if (s != HYB_OK) return s;
    if (events) HYB_CU(p, cudaEventRecord(p->evs[3], p->stream));
    return HYB_OK;
}

hyb_status hyb_step(hyb_problem* p, int32_t nsteps, hyb_leg_stats* per_step) {
    if (!p || nsteps < 0) return fail(p, HYB_EINVAL, "bad arguments");
    p->pdl = true;   // stepped alone (a batch sets its members' launches itself)
    for (int32_t i = 0; i < nsteps; ++i) {
        int it = 0;
        hyb_status s = step_launch(p, &it, true);
        if (s != HYB_OK) return s;
        if (per_step) {
            s = pull_state(p);
            hyb_leg_stats rs;
            fill_leg_stats(p, &per_step[i]);
            fill_remap_stats(p, &rs);
            float m0 = 0, m1 = 0, m2 = 0;
            cudaEventElapsedTime(&m0, p->evs[0], p->evs[1]);
            cudaEventElapsedTime(&m1, p->evs[1], p->evs[2]);
            cudaEventElapsedTime(&m2, p->evs[2], p->evs[3]);
            per_step[i].sn_iterations = it;
            per_step[i].combed = rs.combed;
            per_step[i].bank_size = rs.bank_size;
            per_step[i].ms = m0 + m1 + m2;
            per_step[i].pad = 0;
            per_step[i].ms_leg = m0; per_step[i].ms_sn = m1; per_step[i].ms_remap = m2;
            per_step[i].ms_leg_kernel = leg_kernel_ms(p);
            if (s != HYB_OK) return s;
        }
    }
    if (!per_step) return pull_state(p);
    return HYB_OK;
}

hyb_status hyb_step_async(hyb_problem* p, int32_t nsteps) {
    if (!p || nsteps < 0) return fail(p, HYB_EINVAL, "bad arguments");
    p->pdl = true;
    for (int32_t i = 0; i < nsteps; ++i) {
        int it = 0;
        hyb_status s = step_launch(p, &it, false);
        if (s != HYB_OK) return s;
        p->status_pending = true;   // this step's remap is unchecked
    }
    return HYB_OK;
}

hyb_status hyb_remap_stats(hyb_problem* p, hyb_leg_stats* out) {
    if (!p || !out) return fail(p, HYB_EINVAL, "null argument");
    hyb_status s = pull_state(p);
    fill_remap_stats(p, out);
    return s;
}

hyb_status hyb_get_tally(hyb_problem* p, int32_t which, double* dst, size_t n, int32_t on_dev) {
    if (!p || !dst) return fail(p, HYB_EINVAL, "null argument");
    const size_t nc = (size_t)p->ncells;
    const double* src = nullptr;
    size_t need = nc;
    switch (which) {
        case HYB_TALLY_PRE: src = p->pre_d; break;
        case HYB_TALLY_POST: src = p->post_d; break;
        case HYB_TALLY_HANDOFF: src = p->mom_d; need = 4 * nc; break;
        case HYB_TALLY_SN_PHI: src = p->sn_phi_d; need = 4 * nc; break;
        case HYB_TALLY_FLUX: src = p->flux_d; break;
        case HYB_TALLY_PRE_RAW: src = p->pre_raw; break;
        case HYB_TALLY_POST_RAW: src = p->post_raw; break;
        default: return fail(p, HYB_EINVAL, "unknown tally");
    }
    if (n != need) return fail(p, HYB_EINVAL, "n does not match the tally size");
    HYB_CU(p, cudaMemcpyAsync(dst, src, need * 8, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (!on_dev) HYB_CU(p, cudaStreamSynchronize(p->stream));   // device copies stay ordered on the stream
    return HYB_OK;
}

hyb_status hyb_set_sn_phi(hyb_problem* p, const double* phi, size_t n) {
    if (!p || !phi || n != 4 * (size_t)p->ncells) return fail(p, HYB_EINVAL, "bad arguments");
    HYB_CU(p, cudaMemcpyAsync(p->sn_phi_d, phi, n * 8, cudaMemcpyHostToDevice, p->stream));
    HYB_CU(p, launch_flux(p));
    HYB_CU(p, cudaStreamSynchronize(p->stream));
    p->sn_done = true;
    return HYB_OK;
}

hyb_status hyb_get_bank(hyb_problem* p, int32_t* cell, double* fx, double* fy, double* ox, double* oy, double* w,
                        int64_t* n_io) {
    if (!p || !n_io || !cell || !fx || !fy || !ox || !oy || !w) return fail(p, HYB_EINVAL, "null argument");
    return p->prec == HYB_FP64 ? get_bank_t<double>(p, cell, fx, fy, ox, oy, w, n_io)
                               : get_bank_t<float>(p, cell, fx, fy, ox, oy, w, n_io);
}

hyb_status hyb_set_bank(hyb_problem* p, const int32_t* cell, const double* fx, const double* fy, const double* ox,
                        const double* oy, const double* w, int64_t n) {
    if (!p || n < 0 || (n > 0 && (!cell || !fx || !fy || !ox || !oy || !w))) return fail(p, HYB_EINVAL, "bad arguments");
    if (n > p->bank_cap) return fail(p, HYB_ECAPACITY, "bank larger than its capacity");
    HYB_CU(p, drop_bank_prepass(p));
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || cell[i] >= p->ncells) return fail(p, HYB_EINVAL, "bank cell index out of range");
        // FP32 banks read back in FP64 carry float rounding: allow a few float ulps
        const double tx = p->dx * (1.0 + 1e-6), ty = p->dy * (1.0 + 1e-6);
        if (!(fx[i] >= 0 && fx[i] <= tx && fy[i] >= 0 && fy[i] <= ty))
            return fail(p, HYB_EINVAL, "bank in-cell offset out of [0, dx] x [0, dy]");
        if (!std::isfinite(ox[i]) || !std::isfinite(oy[i]) || ox[i] * ox[i] + oy[i] * oy[i] > 1.0 + 1e-6 || !std::isfinite(w[i]))
            return fail(p, HYB_EINVAL, "bank direction or weight invalid");
    }
    return p->prec == HYB_FP64 ? set_bank_t<double>(p, cell, fx, fy, ox, oy, w, n)
                               : set_bank_t<float>(p, cell, fx, fy, ox, oy, w, n);
}

hyb_status hyb_set_bank_native(hyb_problem* p, const int32_t* cell, const void* fx, const void* fy, const void* ox,
                               const void* oy, const void* w, int64_t n) {
    if (!p || n < 0 || (n > 0 && (!cell || !fx || !fy || !ox || !oy || !w))) return fail(p, HYB_EINVAL, "bad arguments");
    if (n > p->bank_cap) return fail(p, HYB_ECAPACITY, "bank larger than its capacity");
    HYB_CU(p, drop_bank_prepass(p));
    const void* f[5] = {fx, fy, ox, oy, w};
    return p->prec == HYB_FP64 ? set_bank_native_t<double>(p, cell, f, n) : set_bank_native_t<float>(p, cell, f, n);
}

hyb_status hyb_bank_capacity(const hyb_problem* p, int64_t* cap) {
    if (!p || !cap) return HYB_EINVAL;
    *cap = p->bank_cap;
    return HYB_OK;
}

hyb_status hyb_set_step(hyb_problem* p, int64_t step) {
    if (!p || step < 0) return fail(p, HYB_EINVAL, "bad arguments");
    HYB_CU(p, drop_bank_prepass(p));
    p->step = step;
    p->st_host->step = step;
    HYB_CU(p, cudaMemcpyAsync(&p->st->step, &p->st_host->step, sizeof(long long), cudaMemcpyHostToDevice, p->stream));
    HYB_CU(p, cudaStreamSynchronize(p->stream));
    p->leg_done = p->sn_done = false;
    p->pdl = true;
    return HYB_OK;
}

hyb_status hyb_get_step(const hyb_problem* p, int64_t* step) {
    if (!p || !step) return HYB_EINVAL;
    *step = p->step;
    return HYB_OK;
}

hyb_status hyb_cdf_scratch_bytes(int32_t nx, int32_t ny, size_t* bytes) {
    if (nx < 1 || ny < 1 || nx > 4096 || ny > 4096 || !bytes) return fail(nullptr, HYB_EINVAL, "nx, ny must be in [1, 4096]");
    *bytes = (size_t)(kCdfParts + ny) * 8;
    return HYB_OK;
}

hyb_status hyb_build_cdf(const double* w_dev, int32_t nx, int32_t ny, int64_t* q_dev, int64_t* row_pre_dev,
                         int64_t* col_pre_dev, double* W_qmax_dev, void* scratch_dev, size_t scratch_bytes,
                         void* cuda_stream) {
    size_t need = 0;
    hyb_status s = hyb_cdf_scratch_bytes(nx, ny, &need);
    if (s != HYB_OK) return s;
    if (!w_dev || !q_dev || !row_pre_dev || !col_pre_dev || !W_qmax_dev || !scratch_dev)
        return fail(nullptr, HYB_EINVAL, "null device pointer");
    if (scratch_bytes < need) return fail(nullptr, HYB_ENOMEM, "scratch smaller than hyb_cdf_scratch_bytes");
    Cdf2DView cdf{(long long*)q_dev, (long long*)row_pre_dev, (long long*)col_pre_dev};
    cudaError_t e = launch_cdf_build_raw(w_dev, nx, ny, cdf, W_qmax_dev, W_qmax_dev + 1, (double*)scratch_dev,
                                         (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(nullptr, HYB_ECUDA, cudaGetErrorString(e));
    return HYB_OK;
}

hyb_status hyb_points(uint64_t seed, int64_t step, int32_t stream_id, int32_t sampler, int64_t i0, int64_t n,
                      int32_t ndims, uint32_t* out_dev, void* cuda_stream) {
    if (i0 < 0 || n < 0 || i0 + n > ((int64_t)1 << 32) || ndims < 1 || ndims > 1024 || !out_dev ||
        (sampler != HYB_SOBOL_DS && sampler != HYB_PRNG && sampler != HYB_HALTON))
        return fail(nullptr, HYB_EINVAL, "bad point-set arguments");
    if (n == 0) return HYB_OK;
    static uint32_t* dev_tab[2][64] = {{nullptr}};   // Sobol, Halton tables per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(nullptr, HYB_EINVAL, "device index");
    const int h = sampler == HYB_HALTON ? 1 : 0;
    if (!dev_tab[h][dev]) {
        size_t bytes = 0;
        const uint32_t* tab = point_table_host(sampler, &bytes);
        cudaError_t e = cudaMalloc(&dev_tab[h][dev], bytes);
        if (e != cudaSuccess) return fail(nullptr, HYB_ENOMEM, "table alloc");
        e = cudaMemcpy(dev_tab[h][dev], tab, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(nullptr, HYB_ECUDA, cudaGetErrorString(e));
    }
    const uint64_t key = stream_key(seed, (uint64_t)step, (uint64_t)stream_id);
    cudaError_t e = launch_points(key, sampler, dev_tab[h][dev], i0, n, ndims, out_dev, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(nullptr, HYB_ECUDA, cudaGetErrorString(e));
    return HYB_OK;
}

}  // extern "C"
