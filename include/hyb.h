/* hyb.h -- C ABI of the GB300 (sm_103a) scatter-limited hybrid (Q)MC / S_N transport path.
 *
 * Method: Krotz & McClarren, "Scatter-Limited Hybrid Monte Carlo, Deterministic Transport with
 * Quasi-Monte Carlo Sampling" (PHYSOR 2026). One time step [t_n, t_{n+1}] is (Sec. 2.2, steps 1-4):
 *   1. MC leg: the step-start particles and the source Q are tracked with at most N_s isotropic
 *      scatters (Sec. 2.3), scoring the pre-limit (n < N_s) and post-limit (n = N_s) cell-average
 *      track-length flux; the (N_s+1)-th collision density is deposited as four Legendre moments
 *      per cell (the collided source of Eq. (floor N_s+1)).
 *   2. Collided solve: bilinear-DG S_N (level-symmetric S4/S8) of Eq. (floor N_s+1), backward
 *      Euler from zero data, source iteration.
 *   3. Remap, Eq. (R): scatter-free re-streaming of the step-start particles plus new births from
 *      Q + sigma_s (phi_pre + phi_post + phi_c), attenuated with sigma_t.
 *   4. The survivors (combed to census_cap) become the census of t_{n+1}.
 * Points are Sobol with a per-(seed, step, stream, dimension) digital shift, Halton with a
 * per-(seed, step, stream, dimension) shift modulo 1, or a counter PRNG (Sec. 2.4 replaces
 * pseudorandom draws with low-discrepancy points inside the same maps).
 *
 * Conventions (all entry points):
 *   - Every function returns hyb_status and never throws. Pointers are plain host or device
 *     pointers as stated per argument; no ownership passes unless stated.
 *   - Mesh arrays are row-major per cell, index k = iy*nx + ix, cell (ix,iy) covers
 *     [ix*lx/nx, (ix+1)*lx/nx] x [iy*ly/ny, (iy+1)*ly/ny]. Boundaries are vacuum.
 *   - Q is the angle-integrated emission rate density (particles / area / time); a step emits
 *     Q*A*dt per cell. phi denotes the scalar flux int Psi dOmega; <Psi> = phi / (4 pi).
 *   - A problem is bound to one CUDA stream; calls on one problem must not overlap. Different
 *     problems are independent.
 */
#ifndef HYB_H
#define HYB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HYB_API __attribute__((visibility("default")))
#else
#define HYB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYB_OK = 0,
    HYB_EINVAL = 1,     /* invalid argument or descriptor */
    HYB_ENOMEM = 2,     /* workspace too small or allocation failed */
    HYB_ECUDA = 3,      /* a CUDA runtime call failed (see hyb_last_error) */
    HYB_ETIMEOUT = 4,   /* a bounded device loop ran out (segments per history, SI cap) */
    HYB_ESTATE = 5,     /* call out of order (e.g. remap before an MC leg) */
    HYB_EBOUNDS = 6,    /* a device-side index check failed; the result is invalid */
    HYB_ECAPACITY = 7   /* a bank or buffer would overflow its capacity */
} hyb_status;

typedef enum { HYB_FP32 = 0, HYB_FP64 = 1 } hyb_precision;
/* HYB_SOBOL_DS: Sobol, XOR of a 32-bit digital shift. HYB_HALTON: Halton (Sec. 2.4), coordinate d
 * = floor(2^32 phi_b(i)) + shift mod 2^32, phi_b the radical inverse in the d-th prime base b.
 * HYB_PRNG: the counter hash. Both QMC sets use the counter hash past HYB_SOBOL_DIMS dims. */
typedef enum { HYB_SOBOL_DS = 0, HYB_PRNG = 1, HYB_HALTON = 2 } hyb_sampler;

/* N_s = infinity: pure (Q)MC, no hand-off, no collided solve, no remap (the MC-leg census is
 * the next bank); Sec. 3 non-hybrid runs. */
#define HYB_NS_INF 2147483647

/* point-set streams (key = (seed, step, stream)) */
#define HYB_STREAM_INIT 0          /* initial-condition particles, step 0 */
#define HYB_STREAM_LEG_CENSUS 1    /* MC leg, bank particles (index = bank slot) */
#define HYB_STREAM_LEG_SOURCE 2    /* MC leg, births from Q */
#define HYB_STREAM_REMAP_SOURCE 3  /* remap births */
#define HYB_STREAM_REMAP_COMB 4    /* census comb offset (index 0, dim 0) */

/* Largest tabulated QMC dimension count (Sobol and Halton); dims >= this use the counter PRNG. */
#define HYB_SOBOL_DIMS 65

/* Problem descriptor (Sec. 2.1: mesh, sigma_a, sigma_s, c, Q, initial data; Sec. 2.2: dt;
 * Sec. 2.3: N_s and the history count; Sec. 2.4: the point set). All host pointers; the
 * arrays are copied at creation. */
typedef struct {
    int32_t nx, ny;           /* mesh cells per axis, 1..4096 each */
    double lx, ly;            /* domain extent (> 0) */
    const double* sigma_a;    /* nx*ny absorption cross sections, finite, >= 0 */
    const double* sigma_s;    /* nx*ny scattering cross sections, finite, >= 0 */
    const double* Q;          /* nx*ny emission rate density, finite, >= 0; NULL = no source */
    const double* ic_cell_w;  /* nx*ny initial weight per cell (isotropic, uniform in the cell,
                                 t = 0); NULL = vacuum initial condition */
    double c;                 /* particle speed (> 0) */
    double dt;                /* time step (> 0) */
    int32_t n_s;              /* scatter limit N_s >= 0, or HYB_NS_INF */
    int32_t sampler;          /* hyb_sampler */
    int64_t n_hist;           /* births per step (MC-leg source, remap source, initial bank) */
    uint64_t seed;            /* point-set seed */
    int32_t precision;        /* hyb_precision of tracking, banks and the S_N stage */
    int32_t sn_order;         /* 4 or 8 (level-symmetric, 12 / 40 ordinates in 2-D) */
    int32_t handoff_full;     /* 1: deposit four Legendre moments; 0: moment 0 only */
    int32_t sn_max_iter;      /* source-iteration cap (>= 1) */
    double sn_tol;            /* SI stop: ||phi_new - phi_old|| <= sn_tol ||phi_new|| */
    double w_min;             /* relative kill threshold (w < w_min * w_start); 0 = never */
    int64_t census_cap;       /* census capacity after the comb; 0 = n_hist */
    int32_t sn_warm_start;    /* 1: source iteration starts from the previous step's collided
                                 flux (same fixed point, fewer iterations); 2: from the linear
                                 extrapolation 2 phi_{n-1} - phi_{n-2} of the last two steps'
                                 fluxes (the previous one on the first warm step); 0: from zero */
    int32_t census_order;     /* 0: the census keeps slot order (re-streamed bank slots, then
                                 births); 1: survivors in cell order (stable within a cell)
                                 before the comb, so the systematic comb samples each cell's
                                 weight to within one copy and the next leg's bank is
                                 cell-coherent; 2: by cell, then within a cell along a Morton
                                 curve over the in-cell position and the direction angle (b bits
                                 each, b = min(5, (31 - cell bits) / 3)), so the comb samples
                                 position and direction within a cell in strata too */
    int32_t sn_accel;         /* 0: plain source iteration (the paper); 1..8: Anderson acceleration
                                 of that depth (the same fixed point, fewer sweeps in diffusive
                                 problems) */
    int32_t remap_variant;    /* 0: the remap of Eq. (R) (Sec. 2.2 steps 3-4: re-stream the
                                 step-start bank, births from Q + sigma_s (phi_pre + phi_post +
                                 phi_c)); 1: steps 3'/4' of the previous hybrids (Eq. (R')):
                                 births from sigma_s (phi_post + phi_c) only, zero initial data,
                                 and the new census is the MC leg's census followed by those
                                 births' survivors. Finite N_s only; not in batches */
    const int32_t* n_s_cell;  /* nx*ny per-cell scatter limits in [0, n_s] (space-dependent N_s,
                                 the paper's Sec. 4 outlook), or NULL for n_s everywhere: a
                                 segment in cell k is pre-limit while the history's scatter count
                                 is below n_s_cell[k], post-limit otherwise; n_s (finite) is the
                                 largest limit and fixes the point dimensions. Host pointer,
                                 copied at creation */
    int32_t sn_layout;        /* memory layout of the collided solve's sweep (no counterpart in the
                                 paper; results are the same): 0 automatic (the padded mesh while
                                 the per-ordinate solutions fit in 48 MB, else the wavefront
                                 order), 1 padded mesh, 2 wavefront order */
    int32_t seg_limit;        /* bound on segments per history (a guard on every device loop): a
                                 history that reaches it ends as an error and the leg returns
                                 HYB_ETIMEOUT; 0 = 2^20; at most 2^30 */
    int32_t wait_limit;       /* polls (20 ns sleeps apart) of one device wait -- the collided
                                 solve's strip pipeline, the census sort's look-back -- before it
                                 gives up and the call returns HYB_ETIMEOUT; 0 = 2^22 (about
                                 0.1 s per wait) */
    int32_t tally_copies;     /* (no counterpart in the paper; results are the same) copies of the
                                 fixed-point tally arrays the leg's warps add into
                                 (warp index mod copies; the normalisation sums them exactly, so
                                 the tallies do not depend on it): 0 automatic (4 while they take
                                 at most 32 MB, fewer above), else 1..64 */
    int32_t sort_every;       /* with census_order >= 1: sort the census on the steps n with
                                 n mod sort_every == 0 only (0 or 1: every step); the other steps
                                 comb the census in slot order. A batch rejects sort_every > 1
                                 (its step graphs replay one sort decision) */
    int32_t leg_sort_every;   /* (no counterpart in the paper; results are the same)
                                 0: the fused MC leg (each warp lane takes a history to its end,
                                 then the next one). K >= 1: the phased leg -- every history
                                 advances at most K segments per phase, and between phases the
                                 live histories are compacted and sorted by cell (stable), so
                                 the lanes of a warp track histories in nearby cells. Results are
                                 the fused leg's bit for bit; the host waits once per phase. A
                                 leg over a history range (hyb_mc_leg_range) stays fused; a
                                 batch rejects K >= 1 */
    int32_t priv_tile;        /* (no counterpart in the paper; results are the same)
                                 0: every tally addition of the fused MC leg goes to the global
                                 tally copies. 1..32: each CTA keeps the tallies of a square window
                                 of priv_tile x priv_tile cells -- placed where the source weight
                                 Q (else the initial weight) is largest -- in shared memory and
                                 adds them to its global copy once, at its end (integer sums: the
                                 results do not change). -1: automatic -- a 16 x 16 window when
                                 n_s = 0 and it holds at least a quarter of the weight of Q and
                                 four times its share of the area, else none. Not used by the
                                 phased leg or batches */
    int32_t pad4;
} hyb_problem_desc;

/* Per-leg (or per-step) statistics. Weights are exact fixed-point sums converted to double. */
typedef struct {
    int64_t histories, segments, collisions, leaked, census, killed, reached_limit, errors;
    double w_source, w_absorbed, w_leaked, w_census, w_handoff, w_killed;
    int32_t sn_iterations;    /* collided solve: SI iterations taken */
    int32_t combed;           /* remap: 1 if the census comb ran */
    int64_t bank_size;        /* particles in the census bank after the call */
    float ms;                 /* device time of the call (events), 0 if not measured */
    int32_t pad;
    int64_t tally_adds;       /* MC leg: fixed-point tally additions issued (global 64-bit atomics;
                                 the FP64 path adds up to two words per contribution) */
    float ms_leg, ms_sn, ms_remap;   /* hyb_step: device time of steps 1, 2 and 3-4 */
    float ms_leg_kernel;      /* hyb_step, hyb_mc_leg: device time of the MC leg kernel alone
                                 (events around its launch), 0 if not measured */
} hyb_leg_stats;

typedef struct hyb_problem hyb_problem;

/* Tally selectors for hyb_get_tally. All are FP64, nx*ny values (x4 for moments):
 *  HYB_TALLY_PRE:    phi_pre = (sum over n < N_s segments of w l g(sigma_a l)) / (A dt)
 *  HYB_TALLY_POST:   phi_post, the same over n = N_s segments with sigma_t
 *  HYB_TALLY_HANDOFF: m_j = sigma_s sum w int P_j ds, P = (1, xi, eta, xi eta) (4 per cell)
 *  HYB_TALLY_SN_PHI: collided scalar flux, 4 Legendre coefficients per cell
 *  HYB_TALLY_FLUX:   step flux phi_pre + phi_post + phi_c (cell average)
 *  HYB_TALLY_*_RAW:  the un-normalised track-length sums (no 1/(A dt)) */
#define HYB_TALLY_PRE 0
#define HYB_TALLY_POST 1
#define HYB_TALLY_HANDOFF 2
#define HYB_TALLY_SN_PHI 3
#define HYB_TALLY_FLUX 4
#define HYB_TALLY_PRE_RAW 5
#define HYB_TALLY_POST_RAW 6

/* Device workspace bytes a problem needs (banks, mesh, tallies, CDFs, S_N state). */
HYB_API hyb_status hyb_workspace_size(const hyb_problem_desc* desc, size_t* bytes);

/* The window of cells whose tallies the fused MC leg keeps in each CTA's shared memory for this
 * descriptor (priv_tile; -1 resolved by its rule): first cell (*x0, *y0) and side *side (0: no
 * window). Host computation only (no device needed); EINVAL for an invalid descriptor or a NULL
 * output. */
HYB_API hyb_status hyb_priv_window(const hyb_problem_desc* desc, int32_t* x0, int32_t* y0, int32_t* side);

/* Create a problem. workspace: device memory of >= hyb_workspace_size bytes, 256-byte
 * aligned, owned by the caller and kept alive until hyb_destroy_problem; NULL lets the library
 * allocate (and later free) it. cuda_stream: a cudaStream_t (borrowed; NULL = legacy stream).
 * Builds the initial bank (stream INIT) and the source CDF on the device; step index = 0.
 * Errors: EINVAL (nx,ny out of range, non-finite or negative sigma/Q/ic, dt<=0, c<=0,
 * n_hist<1 or >= 2^32, sn_order not 4/8, N_s < 0), ENOMEM, ECUDA. */
HYB_API hyb_status hyb_create_problem(const hyb_problem_desc* desc, void* workspace, size_t ws_bytes,
                              void* cuda_stream, hyb_problem** out);
HYB_API hyb_status hyb_destroy_problem(hyb_problem* p);

/* Step 1 (Sec. 2.2; Sec. 2.3): the MC leg of the current step over the current bank and Q.
 * Tallies stay on the device. stats (host, may be NULL): if given, the call synchronises the
 * stream and fills it; if NULL the call is asynchronous. hist (device, may be NULL): per
 * history 4 int32 (final cell, fate 0 leaked/1 census/2 killed/3 error, final scatter count,
 * segments), histories ordered bank slots first, then births; capacity bank_size + n_hist. */
HYB_API hyb_status hyb_mc_leg(hyb_problem* p, hyb_leg_stats* stats);
HYB_API hyb_status hyb_mc_leg_trace(hyb_problem* p, int32_t* hist_dev, hyb_leg_stats* stats);

/* History-sharded MC leg (Sec. 2.3: histories are independent, each drawing its own point, so a
 * leg split by history index over several GPUs, with its integer results summed, is the one-GPU
 * leg bit for bit). Every rank holds the same problem (bank, step, sigma, Q) and tracks a disjoint
 * part of the index space [bank slots | births]:
 *   hyb_leg_exchange_bytes: bytes of the exchange block (int64 words, 8-byte aligned).
 *   hyb_mc_leg_range: the leg over the histories with global index h in [h0, h1) (clamped to the
 *     leg's count; an empty range is allowed), with the whole leg's fixed-point scales, written to
 *     the caller's device block x_dev (x_bytes >= hyb_leg_exchange_bytes) as raw integer tallies
 *     and counters; hist_dev as for hyb_mc_leg_trace (rows at global indices, may be NULL).
 *     Asynchronous on the problem's stream; the problem's tallies are not normalised after it.
 *   The caller sums the blocks of all ranks element-wise as int64 (an all-reduce with a plain
 *     integer sum; two's-complement wrap-around is part of the format: 128-bit values travel as
 *     four 32-bit limbs, value = sum_i limb_i 2^(32 i) mod 2^128).
 *   hyb_mc_leg_reduce_finish: the summed block becomes the problem's leg (tallies, hand-off
 *     moments, counters, normalisation), as after hyb_mc_leg; stats as for hyb_mc_leg.
 * Errors: EINVAL (range, null or misaligned block), ENOMEM (block too small), ECUDA; the device
 * status bits of any rank survive the sum and are reported by the finish. */
HYB_API hyb_status hyb_leg_exchange_bytes(const hyb_problem* p, size_t* bytes);
HYB_API hyb_status hyb_mc_leg_range(hyb_problem* p, int64_t h0, int64_t h1, void* x_dev, size_t x_bytes,
                                    int32_t* hist_dev);
HYB_API hyb_status hyb_mc_leg_reduce_finish(hyb_problem* p, const void* x_dev, size_t x_bytes,
                                            hyb_leg_stats* stats);

/* Step 2 (Sec. 2.2; Eq. (floor N_s+1)): the collided S_N-DG solve fed by the hand-off
 * moments of the last MC leg. Synchronises per SI iteration (convergence test). */
HYB_API hyb_status hyb_collided_solve(hyb_problem* p, hyb_leg_stats* stats);

/* Steps 3-4 (Sec. 2.2, Eq. (R)): remap into the new census bank and advance the step index.
 * Needs an MC leg and a collided solve of the same step. stats as for hyb_mc_leg. */
HYB_API hyb_status hyb_remap(hyb_problem* p, hyb_leg_stats* stats);

/* nsteps full steps (1-4, Sec. 2.2). per_step (host, may be NULL): nsteps entries, leg
 * statistics with sn_iterations / combed / bank_size of the step, ms = whole step and
 * ms_leg / ms_sn / ms_remap per phase. A step waits for the device once inside the source
 * iteration (stop test), after each phase of the phased leg (leg_sort_every >= 1) and, with
 * per_step, once at its end; without per_step the call
 * synchronises the stream at the end. Device loop bounds map to ETIMEOUT, index checks to
 * EBOUNDS. */
HYB_API hyb_status hyb_step(hyb_problem* p, int32_t nsteps, hyb_leg_stats* per_step);

/* nsteps full steps as hyb_step, without per-step statistics and without the final
 * synchronisation: the host waits only inside each source iteration (the stop test) and, with
 * the phased leg (leg_sort_every >= 1), after each of its phases, so the call
 * returns while the last step's remap may still run on the problem's stream, and work the caller
 * queues after it on that stream (the next bank upload with hyb_set_bank_native, a device copy
 * with hyb_get_tally) overlaps it. Errors of that remap (device loop bounds, index checks) stay in
 * the device status word and are returned by the next call that reads it: the next step's stop
 * test, hyb_step, hyb_mc_leg, hyb_remap_stats. */
HYB_API hyb_status hyb_step_async(hyb_problem* p, int32_t nsteps);

/* Statistics of the last remap (of hyb_step or hyb_remap): histories (slots streamed: bank +
 * births), segments, leaked, killed, errors, census (particles written), w_source / w_absorbed /
 * w_leaked / w_killed (weight of the slots' start states, removed by sigma_t attenuation, leaving
 * the domain, below the weight cut-off), w_census (sum |w| of the survivors before the comb),
 * combed, bank_size. Synchronises the problem's stream. Inside hyb_step, an Eq. (R) remap's bank
 * slots are re-streamed on an internal stream beside the collided solve; their weight sums are
 * formed at the bank's own fixed-point scale and added here (equal to the single-pass sums up to
 * the rounding of that scale). */
HYB_API hyb_status hyb_remap_stats(hyb_problem* p, hyb_leg_stats* stats);

/* Copy a tally (see HYB_TALLY_*) into dst (host if dst_on_device == 0, else device), n values.
 * A host copy synchronises the stream; a device copy is asynchronous, ordered on the problem's
 * stream. EINVAL if n is not the tally's size. */
HYB_API hyb_status hyb_get_tally(hyb_problem* p, int32_t which, double* dst, size_t n, int32_t dst_on_device);

/* Overwrite the collided flux (4 Legendre coefficients per cell, host FP64) -- parity
 * injection for the remap. */
HYB_API hyb_status hyb_set_sn_phi(hyb_problem* p, const double* phi_host, size_t n);

/* Census bank I/O (host arrays, FP64 values converted to the problem precision). get: n_io in
 * = capacity, out = particles copied. set: replaces the bank (n <= bank capacity). */
HYB_API hyb_status hyb_get_bank(hyb_problem* p, int32_t* cell, double* fx, double* fy, double* ox,
                        double* oy, double* w, int64_t* n_io);
HYB_API hyb_status hyb_set_bank(hyb_problem* p, const int32_t* cell, const double* fx, const double* fy,
                        const double* ox, const double* oy, const double* w, int64_t n);
/* Census bank input in the problem's own layout, for callers that stream banks in every step: cell
 * (n int32) and fx, fy, ox, oy, w (n values each of the problem precision: float for HYB_FP32,
 * double for HYB_FP64), in host memory (page-locked for an asynchronous copy) or device memory
 * (all six device-resident: one kernel copies and checks them, two more form the bank's statistics).
 * Copied asynchronously on the problem's stream; the particles are checked on the device (cell
 * index, in-cell offsets in [0, dx] x [0, dy], |Omega_xy| <= 1, finite weight) and a bank with
 * invalid particles makes the next fully synchronising call (hyb_step, hyb_mc_leg,
 * hyb_remap_stats) return EINVAL. The source arrays must stay valid until the stream has passed
 * the copy. ECAPACITY if n exceeds
 * the bank capacity. */
HYB_API hyb_status hyb_set_bank_native(hyb_problem* p, const int32_t* cell, const void* fx, const void* fy,
                                       const void* ox, const void* oy, const void* w, int64_t n);
HYB_API hyb_status hyb_bank_capacity(const hyb_problem* p, int64_t* cap);

/* Step index (t_n = step * dt) used by the next MC leg / remap. */
HYB_API hyb_status hyb_set_step(hyb_problem* p, int64_t step);
HYB_API hyb_status hyb_get_step(const hyb_problem* p, int64_t* step);

/* Point sets (Sec. 2.4): out_dev[(i - i0)*ndims + d] for i in [i0, i0+n), d < ndims, as 32-bit
 * integers; i0 + n <= 2^32; sampler a hyb_sampler. Asynchronous on cuda_stream. */
HYB_API hyb_status hyb_points(uint64_t seed, int64_t step, int32_t stream_id, int32_t sampler, int64_t i0,
                      int64_t n, int32_t ndims, uint32_t* out_dev, void* cuda_stream);

/* ---- batches: many problems advanced by one CUDA graph per step --------------------------------
 * The MC legs of all problems run as one persistent launch that pulls (problem, history range)
 * chunks from a device work queue; normalisation, collided solves and remaps follow as
 * independent graph branches on a pool of streams. Results are those of stepping each problem
 * alone (bit-identical integers and tallies). Problems must share one precision, be at a step
 * boundary, and not be stepped individually while the batch exists (the batch owns their
 * stream use). Source iteration runs up to a per-problem cap inside the graph and stops on a
 * device flag; a problem that reaches its cap gets a doubled cap from the next step on. Batched
 * problems use Sobol or PRNG points (HYB_HALTON returns HYB_EINVAL). */
typedef struct hyb_batch hyb_batch;
typedef struct {
    int32_t block;        /* threads per CTA of the batched MC leg: 128 or 256 */
    int32_t chunk;        /* histories per work-queue item (>= 32) */
    int32_t ctas_per_sm;  /* resident CTAs per SM of the persistent leg; 0 = register limit */
    int32_t streams;      /* streams for the per-problem branches (1..64) */
    int32_t use_graph;    /* 1: record each step as CUDA graphs and replay them (fixed membership);
                             0: issue the same work directly (cheap to build, for changing sets) */
    int32_t pad;
} hyb_batch_tuning;

/* problems: n handles (host array, borrowed; the problems must outlive the batch). cuda_stream:
 * the stream the graph is launched on (NULL: the batch creates its own; the legacy default stream
 * cannot record graphs). Allocates the work queue, graph and report buffers. */
HYB_API hyb_status hyb_batch_create(hyb_problem* const* problems, int32_t n, void* cuda_stream, hyb_batch** out);
/* Replace the tuning (rebuilds the work queue; graphs are re-recorded at the next step). */
HYB_API hyb_status hyb_batch_set_tuning(hyb_batch* b, const hyb_batch_tuning* tuning);
/* Replace the batch's problems (same rules as hyb_batch_create; the problems must share the
 * batch's precision). Streams, events and device buffers are kept (per-problem buffers grow
 * only), so a serving loop can change the resident set every step without re-creating them.
 * Synchronises the batch stream. */
HYB_API hyb_status hyb_batch_set_problems(hyb_batch* b, hyb_problem* const* problems, int32_t n);
/* nsteps steps of every problem; per_problem (host, n entries, may be NULL): the last step's leg
 * statistics with sn_iterations / combed / bank_size, ms = device time of the last step, ms_leg =
 * device time of its batched births and MC-leg launches (the same for every problem). */
HYB_API hyb_status hyb_batch_step(hyb_batch* b, int32_t nsteps, hyb_leg_stats* per_problem);
HYB_API hyb_status hyb_batch_destroy(hyb_batch* b);
HYB_API const char* hyb_batch_last_error(const hyb_batch* b);

/* Integer 2-D CDF over cells (the sampling map of Sec. 2.3 births and of the Eq. (R) remap):
 * q_k = rint(|w_k| / max|w| 2^B), B = min(40, 62 - ceil(log2(nx*ny))) so that the total stays below
 * 2^62 on every accepted mesh (B = 40 up to 2^22 cells); col_pre: per row the exclusive prefix of q over the row's cells
 * (ny x (nx+1), last entry = row total); row_pre: exclusive prefix of the row totals (ny+1).
 * w_dev: nx*ny FP64 cell weights (device, sign ignored). W_qmax_dev: two device doubles written
 * with sum|w| and max|w|. scratch_dev: caller-owned device scratch of >= hyb_cdf_scratch_bytes
 * bytes (block partial sums and row totals). Asynchronous on cuda_stream. EINVAL: nx, ny outside
 * [1, 4096] or a null pointer; ENOMEM: scratch too small. */
HYB_API hyb_status hyb_cdf_scratch_bytes(int32_t nx, int32_t ny, size_t* bytes);
HYB_API hyb_status hyb_build_cdf(const double* w_dev, int32_t nx, int32_t ny, int64_t* q_dev, int64_t* row_pre_dev,
                                 int64_t* col_pre_dev, double* W_qmax_dev, void* scratch_dev, size_t scratch_bytes,
                                 void* cuda_stream);

/* The same CDF build without any device allocation, for callers that cannot call cudaMalloc or
 * hand out scratch memory: serving loops that must not allocate on their hot path (an allocation
 * can synchronise the device or fail under memory pressure mid-request), and hosts whose device
 * memory is owned by another allocator with a fixed budget that this library may not draw from.
 * (This entry point has no counterpart in the paper.)
 * Its scratch is one fixed __device__ array of 34,816 bytes, resident on every GPU that loads the
 * library until the process exits; ny is limited to 4096 rows (EINVAL beyond, like nx). The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) and keeps it for the
 * life of the process, so make that first call before any stream capture, and do not call it on a
 * device after cudaDeviceReset (the reset ends the context that address belongs to). All calls
 * share the array: calls that overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller. Outputs as hyb_build_cdf; asynchronous on cuda_stream; allocates
 * nothing. */
HYB_API hyb_status hyb_build_cdf_noalloc(const double* w_dev, int32_t nx, int32_t ny, int64_t* q_dev,
                                         int64_t* row_pre_dev, int64_t* col_pre_dev, double* W_qmax_dev,
                                         void* cuda_stream);

/* The generated Sobol direction numbers, host out[d*32 + b], d < ndims <= HYB_SOBOL_DIMS. */
HYB_API hyb_status hyb_sobol_table(int32_t ndims, uint32_t* out_host);

/* The S_N quadrature used (upper hemisphere, weights summing to 4 pi); returns the count in
 * *m (capacity in, count out). */
HYB_API hyb_status hyb_quadrature(int32_t order, double* ox, double* oy, double* w, int32_t* m);

/* Measurement helper, no counterpart in the paper: throughput of 64-bit global integer atomic
 * additions (the MC leg's fixed-point tally updates) to n_addr addresses chosen uniformly at
 * random, about n_ops additions per timed launch (best of 3 after a warm-up), on `stream`.
 * Allocates and frees n_addr * 8 bytes; synchronises the stream. Result in *ops_per_s.
 * EINVAL: n_addr < 1 or n_ops < 1; ENOMEM / ECUDA on failure. */
HYB_API hyb_status hyb_atomic_rate(int64_t n_addr, int64_t n_ops, void* stream, double* ops_per_s);

HYB_API const char* hyb_status_string(hyb_status s);
/* Last error message of a problem (valid until the next call on it); p = NULL: the last error
 * of a call that had no problem. */
HYB_API const char* hyb_last_error(const hyb_problem* p);

#ifdef __cplusplus
}
#endif
#endif /* HYB_H */
