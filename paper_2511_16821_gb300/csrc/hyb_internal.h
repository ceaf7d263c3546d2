// hyb_internal.h -- internal structures of the sm_103a hybrid (Q)MC / S_N library (not ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hyb.h"

namespace hyb {

constexpr int kTile = 256;               // threads per block of the streaming kernels
constexpr int64_t kMaxSegments = 1 << 20;
constexpr int kFateLeaked = 0, kFateCensus = 1, kFateKilled = 2, kFateError = 3;
constexpr int kMaxOrd = 40;              // S8 upper hemisphere
constexpr int kHaltonWords = 128;        // words per dimension of the Halton tables
constexpr int kCdfParts = 256;           // block partial sums of the CDF build
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

// status bits written by kernels (device status word)
constexpr int kStBounds = 1, kStSegments = 2, kStCapacity = 4;

// 128-bit two's-complement fixed-point accumulator cell (lo word carries into hi)
struct Acc128 { unsigned long long lo, hi; };

// Device-resident per-leg counters and scalars (one block of memory per problem).
// Per-step scalars of the remap passes, formed once per remap by one thread (FP64 work that
// every block repeating it would put on the critical path of its slots)
struct RemapScal {
    long long N;               // slots: bank + births
    double wbar, w_ref;        // birth weight, comb quantisation base
    float qsc, sca;            // FP32 comb scale 2^(32 - log2 w_ref), FP32 |w|-sum scale 2^kfa
    int krw, kw, kfa, kf;      // 128-bit scales of sum |w| and of the statistics; FP32 per-thread ones
};

struct DevState {
    // counters of the last MC leg
    unsigned long long histories, segments, collisions, leaked, census, killed, reached, errors;
    unsigned long long tally_adds;   // fixed-point tally additions (global atomics) issued
    unsigned long long leg_next;     // next history index handed to a warp (single-problem leg)
    unsigned long long live_count;   // phased leg: histories saved by the phase (alive after it)
    unsigned long long live_in;      // phased leg: histories the phase takes up
    Acc128 w_source, w_absorbed, w_leaked, w_census, w_handoff, w_killed;
    // counters of the last remap
    unsigned long long r_histories, r_segments, r_leaked, r_killed, r_errors, r_alive;
    Acc128 r_w_source, r_w_absorbed, r_w_leaked, r_w_killed, r_w_census;
    Acc128 r_wb[4];            // the bank pre-pass's source, absorbed, leaked, killed weights (scale k_rwb)
    int k_rwb, pad_rwb;
    // bank descriptors
    long long n_bank;          // particles in the current bank
    double bank_wmax;          // max |w| of the current bank
    double bank_wsum;          // sum |w| of the current bank
    // remap / comb scalars
    double remap_W;            // sum |q_cell|
    double remap_qmax;         // max |q_cell|
    double remap_rmax;         // max weight factor bound over source cells
    double w_ref;              // power-of-two quantisation base of the comb
    long long comb_T;          // total quantised |w|
    long long comb_o;          // tooth offset
    long long comb_total_alive;
    int comb_on;
    int status;                // kSt* bits
    double wcopy;              // comb copy weight
    double sn_norm_num, sn_norm_den;
    int k_track, k_mom, k_w;   // fixed-point scale exponents of the last MC leg
    int k_rw;                  // scale exponent of the remap weight sums
    Acc128 bank_wsum_acc;      // scratch of the bank-statistics kernels
    long long out_count;       // particles written by the last remap
    long long r_lead;          // remap slots ahead of the births that hold the MC leg's staged census
                               // (steps 3'/4'), after the step-start bank slots; 0 for Eq. (R)
    long long step;            // time-step index n of the next MC leg / remap (t_n = n dt)
    int sn_conv;               // collided solve: converged flag of the current solve
    int sn_iters;              // collided solve: iterations run in the current solve
    int sn_warm;               // solves finished with warm starts enabled (counted up to 2)
    unsigned int sn_blocks_done;   // source-iteration reduction: blocks finished (last one resets it)
    unsigned int dens_done;    // remap density + CDF reduction: blocks finished (the last one resets it)
    unsigned int write_done;   // remap pass B: blocks finished (the last one resets it)
    unsigned int bank_done;    // bank |w| sum of an upload: blocks finished (the last one resets it)
    unsigned int bank_bad;     // particles of a native-layout bank upload outside the problem's domain
    RemapScal rs;              // scalars of the current remap (remap_prep_body)
    RemapScal rsb;             // scalars of the bank pre-pass (remap_bank_prep_kernel)
};

template <typename T>
struct BankView { int32_t* cell; T *fx, *fy, *ox, *oy, *w; };

// Start states of a leg's source births (cell, in-cell position, direction, remaining flight
// c (t_{n+1} - t), first optical depth), written ahead of the leg by a converged kernel.
template <typename T>
struct BirthView { int32_t* cell; T *fx, *fy, *ox, *oy, *srem, *tau; };

// Integer 2-D CDF: per-cell integer weights q, row marginal row_pre (ny + 1), per-row column
// conditionals col_pre (ny x (nx + 1)). Optional guide tables (Chen & Asau 1974) narrow each pick:
// for 2^g equal buckets of the 32-bit point, entry b holds the bin picked by the bucket's smallest
// point, so the bin of any point in bucket b lies in [guide[b], guide[b + 1]] (the pick is
// monotone); row_g has 2^gr + 1 entries, col_g 2^gc + 1 per row. Null guides: full search.
struct Cdf2DView {
    long long* q; long long* row_pre; long long* col_pre;
    int* row_g = nullptr; int* col_g = nullptr;
    int gr = 0, gc = 0;
};

// guide table bits for n bins: the smallest g with 2^g >= n (at most 20)
inline int guide_bits(int n) {
    int g = 0;
    while ((1 << g) < n && g < 20) ++g;
    return g;
}

}  // namespace hyb

// Problem object behind the opaque hyb_problem handle.
struct hyb_problem {
    hyb_problem_desc d;       // copy of the descriptor (array pointers cleared)
    int nx, ny, ncells;
    double dx, dy, area;
    int prec;                 // HYB_FP32 / HYB_FP64
    int64_t bank_cap;
    int64_t stage_slots;      // remap staging slots: bank_cap + n_hist (+ n_hist for steps 3'/4')
    int64_t step;
    cudaStream_t stream;
    void* ws;                 // device workspace base
    size_t ws_bytes;
    bool owns_ws;
    int ndims;                // point dimensions used: 5 + 3 N_s (capped)
    double w_src;             // total source weight per step (sum Q A dt)
    bool has_src;
    int n_ord;                // S_N ordinates
    double quad_ox[hyb::kMaxOrd], quad_oy[hyb::kMaxOrd], quad_w[hyb::kMaxOrd];
    bool leg_done, sn_done;
    bool sn_warm;             // start source iteration from the previous step's collided flux
    int last_sn_iters;
    std::string err;
    // device pointers (into ws)
    uint32_t* point_tab;      // Sobol direction numbers (HYB_SOBOL_DIMS x 32) or Halton tables
                              // (HYB_SOBOL_DIMS x kHaltonWords), by the sampler
    void* sig;                // ncells x 2 (T): sigma_a, sigma_s
    float* sig_inv;           // ncells x 8 (FP32 leg): 1/sigma_a, 1/sigma_s, 1/sigma_t (0 where sigma = 0),
                              // the cell's scatter limit as int bits (space-dependent N_s), sigma_a,
                              // sigma_s, 0, 0
    int32_t* ns_cell;         // per-cell scatter limits (space-dependent N_s), or null
    int32_t* sort_keys;       // census in phase-space order: the sort key of every staging slot
    uint32_t* byte_tab;       // Sobol byte tables of the births' dimensions (Sobol sampler only)
    double *sa_d, *ss_d, *Q_d;  // FP64 copies for the remap density
    hyb::Cdf2DView src_cdf, rem_cdf;
    double* rem_f;            // 4 x ncells remap density coefficients
    float* rem_f32;           // the same in FP32 (FP32 path)
    unsigned long long* sort_pairs[2];   // census sort (census_order 1): ping-pong (cell, slot) pairs
    void* sort_scratch;                  //   digit counts, tile counters and look-back records; null for slot order
    void* live_buf[2];                   // phased leg (leg_sort_every >= 1): saved histories, ping-pong
    unsigned long long* live_pairs[2];   //   their (cell, index) pairs for the sort by cell
    void* live_scratch;                  //   and the sort's scratch; all null for the fused leg
    long long live_cap;                  //   histories a leg can hold (bank capacity + births)
    int priv_x0, priv_y0, priv_side;     // the leg's privatised window of cells (side 0: none)
    int* rem_pos;             // ncells: 1 where the bilinear remap density is non-negative
    double* rem_q;            // ncells signed remap cell weights q = f0 A dt
    double* cell_scratch;     // per-row partials for the CDF build
    void* bank[2];            // two SoA banks (T)
    void* stage;              // remap staging SoA, bank_cap + n_hist slots (T)
    int cur;                  // current bank index
    void* acc_pre; void* acc_post; void* acc_mom;   // fixed-point tallies, tally_copies copies each
    int tally_copies;         // copies of the tally arrays (spreads adds to hot cells over addresses)
    double *pre_d, *post_d, *mom_d, *flux_d;        // normalised tallies (FP64)
    double *pre_raw, *post_raw;                     // raw track-length sums (FP64)
    double sig_s_max;         // max sigma_s (bound of the hand-off moments)
    void* sn_phi; void* sn_phi_old;   // collided flux, 4 Legendre coefficients per cell (T)
    void* sn_quad;            // sweep sources: S_0..S_3 per entry, then sigma* A per entry (T); entries: the padded
                              //   mesh, or per direction the wavefront order (solves too large for L2)
    void* sn_psi;             // psi_m per ordinate, mirrored coordinates (T): plain mesh or wavefront order
    void* sn_table;           // cell-solve table per ordinate class and padded cell (T), or null
    bool pdl;                 // launch the source iteration's and the remap's kernels as programmatic
                              //   dependents (true when stepped alone; a batch turns it off)
    void* sn_quadbuf;         // ordinates (ox, oy, w) x kMaxOrd, then 4 signed weights per ordinate (T)
    double* sn_phi_d;         // collided flux, FP64 copy (4 x ncells)
    double* sn_phi_d2;        // the solution of the step before (extrapolated warm start only)
    double* sn_norm;          // per-block norm partials (Anderson: kAAMax + 2 per block)
    void* aa_hist;            // Anderson acceleration: (depth + 1) iterates g, then residuals f (T)
    void* aa_state;           // Anderson: slots, Gram matrix, mixing weights
    long long* blk;           // remap block partials (4 x nblk)
    int64_t nblk_max;
    void* births_buf;         // staged source births of one step (BirthView layout), or null
    long long births_step;    // the step index whose births births_buf holds in full, or -1
    hyb::DevState* st;        // device counters
    hyb::DevState* st_host;   // pinned host mirror
    cudaEvent_t ev0, ev1;
    cudaEvent_t evs[4];       // hyb_step phase boundaries: leg start, solve start, remap start, end
    cudaEvent_t evk[2];       // around the MC leg kernel alone (recorded at its launch)
    // bank pre-pass of the remap (Eq. (R) remaps stepped by hyb_step): the step-start bank slots are
    // re-streamed on `side` while the collided solve runs on `stream` (its sweeps leave most SMs
    // idle); ev_fork orders it after the leg, ev_join orders the remap's pass A after it
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    bool bank_prepass;        // a pre-pass of this step's bank is in flight or done (not yet consumed)
    bool acc_clean;           // the fixed-point tally copies are zero (the last normalisation cleared them)
    bool bank_sorted;         // the current bank is in cell (or phase-space) order: the leg takes it
                              // in transposed order (lanes in different cells)
    bool status_pending;      // a step launched by hyb_step_async has not been checked: the status word
                              // keeps its error bits until a synchronising call reads them
};

namespace hyb {

// launchers (defined in the .cu files)
// the leg over the history index range [h0, h1) of [bank slots | births] (0, LLONG_MAX: all)
// census_order >= 1: is the census of the step being remapped sorted (every sort_every-th step)?
inline bool census_sorted_now(const hyb_problem* p) {
    return p->d.census_order >= 1 && (p->d.sort_every <= 1 || p->step % p->d.sort_every == 0);
}

cudaError_t launch_mc_leg(hyb_problem* p, int32_t* hist_dev, long long h0, long long h1);
cudaError_t launch_leg_normalise(hyb_problem* p);
// the exchange block of a history-sharded leg (int64 words): size, pack after a range leg, and
// unpack of a summed block into the tallies and counters
size_t leg_exchange_words(const hyb_problem* p);
cudaError_t launch_leg_pack(hyb_problem* p, long long* x);
cudaError_t launch_leg_unpack(hyb_problem* p, const long long* x);
cudaError_t launch_remap(hyb_problem* p);
// Eq. (R) remap: re-stream the step-start bank's slots on p->side (after the work queued on
// p->stream so far) and mark the pre-pass pending; launch_remap consumes it. No-op for an empty bank.
cudaError_t launch_remap_bank_prepass(hyb_problem* p);
// order p->stream after a pending bank pre-pass and forget it (the bank, the step or the staging
// buffer is about to change)
cudaError_t drop_bank_prepass(hyb_problem* p);
// the source births of step p->step + 1 into births_buf on p->side, after the work queued there
// so far (launch_remap_bank_prepass, which records p->ev_join after them)
cudaError_t launch_births_ahead(hyb_problem* p);
cudaError_t launch_census(hyb_problem* p);   // N_s = infinity: MC-leg census -> new bank
size_t sn_accel_state_bytes();                // device bytes of the Anderson state
size_t sn_norm_bytes(int ncells);            // reduction scratch of the source iteration
cudaError_t sn_clear_counters(hyb_problem* p);
// the collided solve's memory (layout: the desc's sn_layout)
size_t sn_src_bytes(int nx, int ny, int nord, bool fp64, int layout);   // sweep sources
size_t sn_psi_bytes(int nx, int ny, int nord, bool fp64, int layout);   // per-ordinate solutions
bool sn_wave_layout(int nx, int ny, int nord, bool fp64, int layout);   // the wavefront order is kept
size_t sn_table_bytes(int nx, int ny, int nord, bool fp64, int layout);  // cell-solve table, 0 if none
cudaError_t sn_build_table(hyb_problem* p);
cudaError_t launch_cdf_build(hyb_problem* p, const double* cell_w_dev, Cdf2DView cdf, double* W_out_dev,
                             double* qmax_out_dev);
cudaError_t launch_flux(hyb_problem* p);
cudaError_t launch_cdf_build_raw(const double* cell_w, int nx, int ny, Cdf2DView cdf, double* W_out,
                                 double* qmax_out, double* scratch, cudaStream_t stream, bool pdl = false);
cudaError_t launch_init_bank(hyb_problem* p, const Cdf2DView& cdf, double w0);
// census sort: the scratch holds the digit counts and tile counters (kSortScratchHead bytes), then
// one record per (tile, digit)
constexpr size_t kSortScratchHead = 8192;
size_t census_sort_scratch_bytes(long long n, uint32_t sentinel);
cudaError_t launch_census_sort(const int32_t* keys, long long n, uint32_t sentinel, unsigned long long* const pairs[2],
                               void* scratch, int wait_limit, int* status, cudaStream_t s,
                               const unsigned long long** sorted);
// the sort key's sentinel (above every key): the cell count (census_order 1), or 2^(cell bits + 3 b)
// for the phase-space key of b bits per coordinate (census_order 2)
uint32_t census_sort_sentinel(int census_order, int ncells);
size_t live_buf_bytes(long long cap, int prec);   // one live-state buffer of the phased leg
cudaError_t launch_bank_stats(hyb_problem* p);
cudaError_t launch_points(uint64_t key, int sampler, const uint32_t* V, int64_t i0, int64_t n, int ndims,
                          uint32_t* out, cudaStream_t s);
size_t leg_args_bytes(int prec);
void leg_args_host(hyb_problem* p, int cur, void* out);
int leg_ntab(const hyb_problem* p);
// the batched births (chunks over each problem's birth indices, queue head d_bhead) and then the
// batched leg (chunks over [bank | births], queue head d_head)
cudaError_t launch_mc_leg_batch(int prec, const void* d_args, const void* d_chunks, int nchunks, int* d_head,
                                const uint32_t* V, int ntab_max, int grid, int block, cudaStream_t s,
                                const void* d_bchunks, int nbchunks, int* d_bhead);
int leg_batch_ctas_per_sm(int prec);
cudaError_t sn_start(hyb_problem* p);
cudaError_t sn_iteration(hyb_problem* p, int first);
double sn_tol_eff(const hyb_problem* p);
cudaError_t sn_finish(hyb_problem* p);

// host helpers (host.cu)
uint64_t mix64(uint64_t z);
uint64_t stream_key(uint64_t seed, uint64_t step, uint64_t stream);
const uint32_t* sobol_table_host();
const uint32_t* halton_table_host();          // HYB_SOBOL_DIMS x kHaltonWords
void quadrature_host(int order, double* ox, double* oy, double* w, int* m);

}  // namespace hyb
