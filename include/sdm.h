/*
 * sdm.h -- C ABI of the B300 (sm_103a) Super-Droplet Method coalescence
 * library (libsdm.so).
 *
 * The library implements the coalescence step of the Super-Droplet Method as
 * organised in Bartman & Arabas, arXiv:2101.06318: the state of Sec. 3.1
 * (multiplicities, extensive attributes, cell segmentation; Fig. "lst:vars"),
 * and the per-timestep workflow of Sec. 3.2, Fig. "fig:algo" -- Step 0
 * removal of zero-multiplicity super-droplets, Step 1 cell-wise shuffling and
 * pairing, Step 2 collision probability, eq. (p), Step 3 collision triggering
 * (gamma, eq. (gamma2)) and attribute update (eqs. (coal_attr_0), (coal)).
 *
 * Conventions shared by every call:
 *  - Every call returns an sdm_status and never aborts, traps or exits.
 *  - Device work is enqueued on the CUDA stream given to sdm_alloc (a
 *    cudaStream_t passed as void*; NULL = legacy default stream).  Calls
 *    return once the work is enqueued unless stated otherwise; errors found
 *    by kernels (capacity overflow and similar) are latched in a device error
 *    word and returned by sdm_sync and by the next call that synchronises.
 *  - "ptrs_on_device" arguments say whether a pointer is device memory
 *    (non-zero) or host memory (0).  Host memory may be pageable or pinned;
 *    the library copies out of / into it before returning.
 *  - A state is not thread-safe: one host thread at a time per state.
 *    Different states are independent.
 *  - All arrays are structure-of-arrays: xi[n_slots], attr[n_attr][n_slots]
 *    (row-major, attribute 0 is the particle volume v in m^3).
 *
 * Slot model.  Storage is a fixed array of slots grouped by cell: cell c owns
 * slots [cell_start[c], cell_start[c+1]).  The live super-droplets of a cell
 * always occupy the first n_c of its slots, in list order; the other slots
 * hold xi = 0 and attributes 0.  When a super-droplet is removed (Sec. 2.2,
 * "the j-th super-droplet is removed") the cell is compacted stably at the end
 * of the step, which is the paper's Step 0 (remove_if_equal_0) of the next
 * step.  An SD's position in its cell's list is its identity for the random
 * number contract.
 *
 * Random number contract (Philox4x32-10, Salmon et al. SC'11; key = seed).
 * Position i in the list of cell c (n live SDs) at step s:
 *   phi of candidate pair m: x = philox(m>>1, c, s, 1),
 *       u53 = ((x[2(m&1)] << 32) | x[2(m&1)+1]) >> 11, phi = u53 * 2^-53
 *   Step 1 shuffle (sdm_shuffle), giving the shuffled list L':
 *   SDM_SHUFFLE_SORT: key(i) = philox(i>>2, c, s, 0)[i&3]; L' = L ordered by
 *       (key, i) ascending (the paper's GPU approach, Sec. 3.2).
 *   SDM_SHUFFLE_PRP: cells with n <= 256 as SORT; larger cells L'[q] = L[P(q)]
 *       with P the keyed bijection of [0, n) given by an eight-round
 *       alternating Feistel network on Z_A x Z_B, x = L B + R (n = 2^k:
 *       A = 2^floor(k/2), B = 2^(k - floor(k/2)); otherwise A = ceil(sqrt n),
 *       B = ceil(n / A)), rounds L = (L + floor(h A / 2^32)) mod A and
 *       R = (R + floor(h B / 2^32)) mod B with h = lowbias32(v ^ K_r) of the
 *       other half v without the hash's last step x ^= x >> 16, round keys
 *       K_0..3 = philox(0, c, s, 2), K_4..7 = philox(1, c, s, 2), and
 *       cycle-walking into [0, n).  No sort and no data exchange is needed.
 *   Pair m is (L'[2m], L'[2m+1]) (Sec. 2.2 Step 1, Fig. "pair_flag").
 */
#ifndef SDM_H
#define SDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDM_OK = 0,
    SDM_EINVAL = 1,     /* invalid argument or invalid initial state */
    SDM_ENOMEM = 2,     /* device or host allocation failed / workspace too small */
    SDM_ECAPACITY = 3,  /* a size limit was exceeded (slots, cells, bucket capacity) */
    SDM_ERANGE = 4,     /* a multiplicity >= 2^53 (xi must convert to double exactly) */
    SDM_ECUDA = 5,      /* a CUDA runtime call failed */
    SDM_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
    SDM_ENOTSUP = 7     /* option not supported by this build */
} sdm_status;

/* Coalescence kernel a(v1, v2) selected per cell (Sec. 4). */
typedef enum {
    SDM_KERNEL_GOLOVIN = 0,        /* a = b (v1 + v2), b = sdm_step_params.golovin_b */
    SDM_KERNEL_GRAVITATIONAL = 1,  /* pi (r1+r2)^2 |vt(r1) - vt(r2)| E(r1, r2) */
    /* Electric-field kernel.  Sec. 4 compares with Berry's case run with a
     * parametric kernel for electric-field effects on the collision
     * probability, without giving it; project definition: the gravitational
     * kernel with the efficiency raised toward one by the field parameter
     * eps = sdm_step_params.efield in [0, 1], E_eps = E + eps (1 - E)
     * (eps = 0: the gravitational kernel; eps = 1: the geometric sweep-out
     * kernel pi (r1+r2)^2 |vt(r1) - vt(r2)|). */
    SDM_KERNEL_ELECTRIC = 2
} sdm_kernel_id;

/* Arithmetic of the collision decision (Steps 2-3). */
typedef enum {
    /* Results identical, bit for bit, to an FP64 evaluation of eq. (p) and
     * gamma: the probability is first bounded in FP32 and only pairs whose
     * integer outcome the bound cannot settle are re-evaluated in FP64. */
    SDM_PREC_FP64 = 0,
    /* The decision is taken from the FP32 value of p and the leading 23 bits of phi;
     * multiplicities stay exact uint64 and the attribute update stays FP64. */
    SDM_PREC_FP32 = 1,
    /* As SDM_PREC_FP32, with the gravitational kernel taken from the surrogate
     * network attached by sdm_attach_surrogate wherever its fallback mask allows
     * (plain FP32 kernel elsewhere).  Not part of the paper; results are
     * approximate (see sdm_surrogate_build_mask).  SDM_EINVAL without an attached
     * surrogate or with the SORT shuffle contract. */
    SDM_PREC_SURROGATE = 2
} sdm_precision;

/* Step 1 shuffle contract (see the random number contract above). */
typedef enum {
    SDM_SHUFFLE_PRP = 0,    /* keyed bijection for cells of more than 256 SDs (default) */
    SDM_SHUFFLE_SORT = 1    /* sort by Philox key in every cell */
} sdm_shuffle;

typedef struct sdm_state sdm_state;   /* opaque, owned by the library */

typedef struct {
    double dt;                 /* time step [s] (> 0) */
    double golovin_b;          /* Golovin constant b [1/s] */
    uint64_t seed;             /* Philox key */
    uint32_t step;             /* index s of the first step enqueued by this call */
    uint32_t precision;        /* sdm_precision */
    uint32_t shuffle;          /* sdm_shuffle */
    uint32_t reserved;         /* must be 0 */
    /* Optional device pointer.  When non-NULL the step index is read from
     * *d_step on the device and incremented there after each step (the host
     * 'step' field is ignored), so a captured CUDA graph advances the random
     * stream on every replay. */
    uint32_t* d_step;
    double efield;             /* field parameter of SDM_KERNEL_ELECTRIC, in [0, 1] (else SDM_EINVAL) */
} sdm_step_params;

typedef struct {
    uint64_t n_pairs;        /* candidate pairs examined */
    uint64_t n_collisions;   /* pairs with gamma~ > 0 */
    uint64_t n_removed;      /* super-droplets whose multiplicity became 0 */
    uint64_t sum_gamma;      /* sum of gamma~ over pairs */
    uint64_t n_fp64;         /* pairs whose decision was re-evaluated in FP64 */
} sdm_step_stats;

/* Tunables of the device schedule.  They change speed only: results do not
 * depend on them (the random stream is keyed by cell and slot, not by tile). */
typedef struct {
    uint32_t tile_slots;      /* max slots of the cells packed into one CTA (power of 2, 256..4096) */
    uint32_t tile_threads;    /* threads per tile CTA (64..512, multiple of 32) */
    uint32_t bucket_target;   /* mean SDs per bucket in the large-cell sort (64..2048, power of 2) */
    uint32_t persistent;      /* 0: one CTA per tile; k > 0: k CTAs per SM pulling tiles */
} sdm_schedule;

/* Library version string. */
const char* sdm_version(void);

/* Human readable name of a status code. */
const char* sdm_status_str(sdm_status s);

/* Bytes of device workspace needed by a state of this size when the caller
 * provides the memory (an upper bound for any cell layout). */
size_t sdm_workspace_bytes(uint64_t n_slots_cap, uint32_t n_cell, uint32_t n_attr);

/* Create a state on the current CUDA device.
 *   n_slots_cap: maximum number of slots (< 2^32);  n_cell >= 1;  n_attr >= 1.
 *   cuda_stream: cudaStream_t (as void*) all device work is ordered on.
 *   workspace, ws_bytes: optional caller-owned device buffer (e.g. a torch
 *     tensor) from which all device memory is carved; NULL = the library
 *     allocates with cudaMalloc.  The library never frees caller memory; the
 *     buffer must outlive the state.
 * Errors: SDM_EINVAL (bad sizes), SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_alloc(sdm_state** out, uint64_t n_slots_cap, uint32_t n_cell, uint32_t n_attr,
                     void* cuda_stream, void* workspace, size_t ws_bytes);

/* Load the initial super-droplet population (Sec. 3.1 state; Sec. 4 set-ups).
 *   xi[n_sd]          multiplicities (0 = removed slot; removed slots are moved
 *                     behind the live ones of their cell)
 *   attr[n_attr][n_sd] extensive attributes, row-major, attr[0] = volume v > 0
 *   cell_id[n_sd]     cell of each SD (< n_cell); SDs are grouped by cell with a
 *                     stable counting sort, so slot order within a cell is the
 *                     input order.
 *   dv[n_cell]        cell volume Delta V [m^3] (> 0)
 *   kernel_id[n_cell] sdm_kernel_id per cell; NULL = all Golovin.
 * Errors: SDM_EINVAL (cell_id >= n_cell, v not finite and > 0 on a live slot,
 * dv <= 0, unknown kernel id), SDM_ERANGE (xi >= 2^53), SDM_ECAPACITY
 * (n_sd > n_slots_cap).  Synchronises the stream. */
sdm_status sdm_init_state(sdm_state* st, const uint64_t* xi, const double* attr,
                          const uint32_t* cell_id, uint64_t n_sd, const double* dv,
                          const uint8_t* kernel_id, int ptrs_on_device);

/* Same as sdm_init_state but the layout is given as cell_start[n_cell+1]
 * (slots already grouped by cell; cell_start[0] = 0, non-decreasing,
 * cell_start[n_cell] = n_sd).  No sorting is done. */
sdm_status sdm_init_state_segmented(sdm_state* st, const uint64_t* xi, const double* attr,
                                    const uint32_t* cell_start, uint64_t n_sd, const double* dv,
                                    const uint8_t* kernel_id, int ptrs_on_device);

/* Overwrite xi and attr of an initialised state in its own slot layout
 * (checkpoint restore, or host-resident state streamed in, e.g. the arrays
 * sdm_get_state returned).  The live SDs of every cell must come first (as
 * sdm_get_state returns them).  Validated on the device like sdm_init_state
 * plus that layout rule; a violation is reported by the next sdm_sync
 * (SDM_EINVAL or SDM_ERANGE).  Asynchronous. */
sdm_status sdm_set_state(sdm_state* st, const uint64_t* xi, const double* attr, int ptrs_on_device);

/* Copy the state out in slot layout: xi[n_sd], attr[n_attr][n_sd] (either may
 * be NULL), cell_start[n_cell+1] (may be NULL), *n_sd (may be NULL).  For
 * host pointers the call synchronises; removed SDs appear with xi = 0. */
sdm_status sdm_get_state(sdm_state* st, uint64_t* xi, double* attr, uint32_t* cell_start,
                         uint64_t* n_sd, int ptrs_on_device);

/* Enqueue n_steps coalescence timesteps (Fig. "fig:algo", Steps 0-3), step
 * indices params->step .. params->step + n_steps - 1 (or read from
 * params->d_step).  stats (nullable) receives the sums over the steps; when
 * non-NULL the call synchronises to read them.  Without stats the call is
 * asynchronous and capturable in a CUDA graph (use d_step for replays).
 * Step 0 (removal of xi = 0 SDs) of a large cell under the PRP contract runs
 * at the start of the next step: a PRP step compacts the large cells the
 * previous one flagged (its launch is cooperative, every block resident, so
 * that its blocks can wait for that compaction), and every call that reads or
 * re-lays out the state (sdm_get_state, sdm_totals, sdm_spectrum,
 * sdm_remove_zero, sdm_check_state, sdm_set_schedule, sdm_autotune, a SORT
 * step) compacts them first, so no caller sees the difference.
 * Under SDM_SHUFFLE_SORT a large cell's SDs are distributed over buckets of
 * about bucket_target SDs by the top bits of their keys; a bucket holds its
 * mean count plus ten standard deviations plus 32 records.  A step whose keys
 * overflow a bucket of a cell (probability below 1e-20 per bucket and step)
 * records SDM_ECAPACITY in the device error word, read by sdm_sync or the
 * next call that synchronises, and leaves that cell unchanged in that step
 * (no memory is overrun; the other cells are stepped). */
sdm_status sdm_coalescence_step(sdm_state* st, const sdm_step_params* params, uint32_t n_steps,
                                sdm_step_stats* stats);

/* Step 0 on its own (remove_if_equal_0): count the live SDs of every cell.
 * Removal is already applied inside every step, so this call changes no
 * result; it reports the total live count (nullable) and is idempotent.
 * Synchronises when n_live is non-NULL. */
sdm_status sdm_remove_zero(sdm_state* st, uint64_t* n_live);

/* Mass spectrum (Sec. 4): out[b] = rho * sum(xi v) / (V * ln(r[b+1]/r[b])) over
 * live SDs with (4 pi/3) r[b]^3 <= v < (4 pi/3) r[b+1]^3, rho = 1000 kg/m^3.
 * cell = index of one cell, or UINT32_MAX for all cells (V = sum of dV).
 * r_edges[n_bins+1] (host), increasing, > 0.  out[n_bins] host or device. */
sdm_status sdm_spectrum(sdm_state* st, const double* r_edges, uint32_t n_bins, uint32_t cell,
                        double* out, int out_on_device);

/* Displacement between steps: every live SD moves to the cell cell_id[i]
 * names (cell_id[n_sd], one entry per slot of the current layout, read for
 * live slots only; host or device pointer).  The paper keeps a cell index per
 * SD and regroups the SDs by it (Sec. 3, cell_start); here each cell keeps its
 * slot range, so its width is its capacity -- allocate spare slots for cells
 * that may gain SDs.  Within a cell the SDs keep their old slot order, live
 * ones first (a stable sort by the new index: radix passes of 8 bits, then a
 * gather).  SDM_EINVAL for an index >= n_cell, SDM_ECAPACITY when a cell would
 * receive more SDs than its width -- the state is unchanged in both cases;
 * SDM_ENOTSUP for a state on a caller's workspace (the sort needs scratch).
 * Synchronises once (to read the checks). */
sdm_status sdm_rebucket(sdm_state* st, const uint32_t* cell_id, int ptrs_on_device);

/* Consistency check of the state's invariants (a diagnostic; Step 0 of
 * Fig. "fig:algo" relies on the first, the early exit on the second):
 *   *n_bad_live = slots that break the live-prefix rule: within every cell the
 *                 slots [0, n_live) hold xi > 0 and the rest xi = 0;
 *   *n_bad_key  = slots of the large cells whose stored volume bin (the
 *                 early exit's quarter-octave bin of the volume, kept beside
 *                 the volumes so that the large-cell step gathers 1 byte per
 *                 SD) differs from the volume's.
 * Both are 0 for any state the library produced.  SDM_EINVAL for a NULL
 * pointer or an uninitialised state.  Synchronises. */
sdm_status sdm_check_state(sdm_state* st, uint64_t* n_bad_live, uint64_t* n_bad_key);

/* Totals over live SDs: *n_total = sum xi (exact), *mass = sum xi v (FP64,
 * summation order unspecified), *n_live.  Any pointer may be NULL.
 * Synchronises. */
sdm_status sdm_totals(sdm_state* st, uint64_t* n_total, double* mass, uint64_t* n_live);

/* Read or change the device schedule (speed only). */
sdm_status sdm_get_schedule(sdm_state* st, sdm_schedule* out);
sdm_status sdm_set_schedule(sdm_state* st, const sdm_schedule* sched);

/* Time candidate schedules on the current state (the state is saved and
 * restored around the trials) and keep the fastest.  n_steps per trial.
 * Synchronises.  best (nullable) receives the chosen schedule. */
sdm_status sdm_autotune(sdm_state* st, const sdm_step_params* params, uint32_t n_steps,
                        sdm_schedule* best);

/* Wait for all work enqueued on the state's stream; returns the first error
 * latched by a kernel since the last sdm_sync (then clears it), or SDM_ECUDA. */
sdm_status sdm_sync(sdm_state* st);

/* Failure-path self-tests (no counterpart in the paper; they exercise the
 * library's own error handling without faulting the GPU).
 *
 * sdm_debug_wait_timeout: a cooperative launch of a few blocks meets at the
 * library's grid barrier (the bounded wait a PRP step uses before its Step 0
 * compaction), giving up after spin_limit polls of at least 100 ns each; with
 * withhold != 0 the last block never arrives, so the others' wait runs out,
 * records SDM_ETIMEOUT in the state's device error word and returns.  The
 * next sdm_sync reports it (and clears it); the state's contents are not
 * touched and the state stays usable.  Asynchronous.  SDM_EINVAL for a NULL
 * state or spin_limit 0.
 *
 * sdm_debug_bucket_capacity: lower the SORT contract's records per bucket of
 * the current layout to cap (a multiple of 32, at least 32, at most the
 * current capacity; SDM_EINVAL otherwise), so that a test can make a bucket
 * overflow.  The next layout change (sdm_set_schedule, sdm_init_state*)
 * restores the computed capacity.
 *
 * sdm_debug_stage_shortfall: in the SORT contract's large-cell step, each
 * finishing warp stages a bucket's records in shared memory by a bulk copy
 * whose mbarrier expects the copy's bytes; with extra_bytes != 0 (at most
 * 4096) every copy announces extra_bytes more than it delivers, so that the
 * barrier's phase never completes and the warp's bounded wait runs out: the
 * warp records SDM_ETIMEOUT, waits once more (bounded), and stops without
 * queueing pairs; no copy is left in flight.  Each wait polls for
 * 2^wait_log2 SM cycles (10 <= wait_log2 <= 31), or about one second with
 * wait_log2 = 0.  Applies to the steps enqueued after the call (allocating
 * entry points only) until it is called again with extra_bytes = 0 and
 * wait_log2 = 0.  SDM_EINVAL for a NULL state or arguments out of range. */
sdm_status sdm_debug_wait_timeout(sdm_state* st, uint32_t spin_limit, int withhold);
sdm_status sdm_debug_bucket_capacity(sdm_state* st, uint32_t cap);
sdm_status sdm_debug_stage_shortfall(sdm_state* st, uint32_t extra_bytes, uint32_t wait_log2);

/* Release the state and the device memory the library allocated. NULL is a no-op. */
void sdm_free(sdm_state* st);

/* Kernel profiling.  While enabled, every kernel launch of the coalescence step
 * is bracketed by CUDA events on the state's stream; sdm_get_profile
 * synchronises and reports, per kernel kind (0 = small-cell kernels: one warp
 * per cell up to 512 slots, tiles of cells above,
 * 1 = large-cell scatter, 2 = large-cell finish), the number of launches and
 * their summed device time in ms since profiling was enabled.  Arrays have
 * SDM_N_KERNEL_KINDS entries (kind 3 = large-cell kernel of the PRP contract).
 * Not for use inside CUDA graph capture. */
#define SDM_N_KERNEL_KINDS 4
sdm_status sdm_set_profiling(sdm_state* st, int enable);
sdm_status sdm_get_profile(sdm_state* st, uint32_t* launches, double* ms);

/* Number of kernel launches one timestep enqueues with the current schedule
 * and the given shuffle contract (sdm_shuffle); a d_step step adds one more
 * for the counter.  SDM_EINVAL for a null pointer or an unknown contract. */
sdm_status sdm_launches_per_step(sdm_state* st, uint32_t shuffle, uint32_t* n);

/* Evaluate, for n pairs (v1[i], v2[i]) with multiplicities (xi1[i], xi2[i]) in
 * a cell of n_cell_sd live SDs and volume dv, the collision kernel and eq.
 * (p) the ways the library does: p64[i] is the FP64 value the library uses
 * when it re-evaluates a pair (bit-identical to the documented operation
 * order); p32[i], err32[i] the FP32 value and its error bound,
 * |p64 - p32| <= err32; plite[i], errlite[i] (nullable; gravitational kernel)
 * the second filter's FP64 value from refined FP32 seeds and its bound,
 * |p64 - plite| <= errlite (errlite < 0: not applicable to this pair); pup[i]
 * (nullable) the early exit's upper bound of p from the table of the two
 * volumes' bins and the power of two above max(xi1, xi2), >= p64 and >= p32
 * (+inf for volumes beyond the table).  efield: the electric-field kernel's
 * parameter (SDM_EINVAL outside [0, 1]).  All arrays are device pointers.
 * Exposes Step 2 alone for testing (dependency injection, Sec. 5). */
sdm_status sdm_eval_pairs(sdm_state* st, uint32_t kernel_id, const double* v1, const double* v2,
                          const uint64_t* xi1, const uint64_t* xi2, uint64_t n, uint32_t n_cell_sd, double dv,
                          double dt, double golovin_b, double efield, double* p64, float* p32, float* err32,
                          double* plite, double* errlite, float* pup);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the gravitational kernel (no counterpart in the paper).
 *
 * A multilayer perceptron (inputs z = ((ln R - c0)/c1, (ln r - c0)/c1) for the
 * pair's radii R >= r, three hidden layers of 64 SiLU units, one output y)
 * stands in for the plain kernel: K^ = exp(mu + sigma y) - k_floor (clamped at
 * 0), where c0, c1 centre and scale ln r over the training range and mu, sigma
 * standardise ln(K + k_floor) of the training targets (k_floor = 1e-6 times the
 * median K of the first 65536 training pairs).  Parameters are kept in FP32 for
 * the optimiser and used rounded to BF16 in every pass; activations and sums
 * are FP32.  Training data: pair i has radii drawn log-uniform in
 * [r_min, r_max] from Philox (counter (i lo, i hi, 0, 3), key = seed), target
 * from the plain FP64 kernel; the loss is the mean squared error of the
 * standardised target.  All work runs in the library's own CUDA kernels on the
 * caller's stream (the state's device).
 * ------------------------------------------------------------------------- */
typedef struct sdm_surrogate sdm_surrogate;   /* opaque, owned by the library */

typedef struct {
    uint64_t n_train;      /* training set size (pairs); sample indices run modulo n_train */
    uint64_t seed;         /* Philox key of the training pairs and of the initial weights */
    double r_min, r_max;   /* radius range of the training pairs [m], 0 < r_min < r_max */
} sdm_surrogate_params;

/* Allocate a surrogate with randomly initialised weights and compute its
 * normalisation (one pass over 65536 training pairs).  *out NULL on error.
 * Errors: SDM_EINVAL (bad params), SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_surrogate_create(sdm_surrogate** out, const sdm_surrogate_params* p, void* cuda_stream);
void sdm_surrogate_free(sdm_surrogate* s);

/* Run n_steps Adam steps (lr decaying on a half cosine from lr to lr/20 over
 * these steps), each on the next 'batch' training pairs (batch a multiple of
 * 64).  loss (nullable host array of n_steps floats) receives each step's loss.
 * Blocks until the steps are done. */
sdm_status sdm_surrogate_train(sdm_surrogate* s, uint32_t n_steps, uint32_t batch, float lr, float* loss);

/* Build the fallback mask on a 256 x 256 grid of z over [-1, 1]^2: a tile uses
 * the network when its relative error against the FP64 kernel is <= tol at 4 x 4
 * points inside it; tiles with r > R or vanishing K keep the plain kernel.
 * frac (nullable host) receives the fraction of tiles with r <= R that use the
 * network; max_err (nullable host, 65536 floats) each tile's largest error. */
sdm_status sdm_surrogate_build_mask(sdm_surrogate* s, float tol, double* frac, float* max_err);

/* Copy the FP32 parameters (8577 floats, layout W1[64][2], b1, W2[64][64], b2,
 * W3[64][64], b3, w4[64], b4) to host memory (set = 0), or set them from host
 * memory (set = 1; the BF16 copy follows). */
sdm_status sdm_surrogate_params_io(sdm_surrogate* s, float* host_params, int set);

/* Normalisation constants: out[0..5] = c0, c1, mu, sigma, k_floor, r_max/r_min. */
sdm_status sdm_surrogate_info(const sdm_surrogate* s, double* out);

/* Loss and gradient at the current parameters for n samples given on the device
 * (x [n][2] network inputs, t [n] standardised targets): *loss and grad (host,
 * 8577 floats) receive mean((y - t)^2) and its gradient with respect to the
 * (BF16-rounded) parameters.  For testing the backward pass. */
sdm_status sdm_surrogate_loss_grad(sdm_surrogate* s, const float* x, const float* t, uint64_t n, float* loss,
                                   float* grad);

/* Surrogate kernel values for n pairs of radii (device arrays, metres): K[i] =
 * K^ where the mask lets the network answer, -1 where the plain kernel is used. */
sdm_status sdm_surrogate_eval(sdm_surrogate* s, const double* R, const double* r, uint64_t n, float* K);

/* Use s for SDM_PREC_SURROGATE steps of st (NULL detaches).  s must outlive its
 * use by st and live on the same device. */
sdm_status sdm_attach_surrogate(sdm_state* st, const sdm_surrogate* s);

/* ---------------------------------------------------------------------------
 * Allocation-free single-box step.  (No counterpart in the paper: this is a
 * deployment convenience of the library.)
 *
 * Some callers cannot allocate device memory at all: processes whose device
 * memory is fully owned by another pool or framework with a hard cap (a
 * cudaMalloc there fails or takes memory the pool counts on), and
 * latency-critical loops that must not hit the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.  sdm_alloc does not suit them, so
 * this entry point performs one coalescence timestep of a single
 * box (one cell, cell index 0 of the random-number contract) directly on the
 * caller's device arrays, with all scratch memory taken from a fixed array
 * compiled into the library (about 5 MB of device memory, held by every GPU
 * that loads the library until the process exits).  It calls no allocating
 * routine.
 *
 *   xi[n_sd]                    multiplicities (device, updated in place)
 *   attr[n_attr][attr_stride]   extensive attributes, row 0 = volume (device,
 *                               updated in place); attr_stride >= n_sd
 *   n_sd                        SDs in the box, at most SDM_NOALLOC_MAX_SD;
 *                               larger boxes return SDM_ECAPACITY
 *   dv, kernel_id               cell volume [m^3] and sdm_kernel_id
 *   params                      as for sdm_coalescence_step (d_step allowed)
 *   cuda_stream                 cudaStream_t the work is ordered on
 * The live SDs must come first in the arrays (as sdm_get_state returns them);
 * removals compact them at the end of the step.  Results are identical to
 * sdm_coalescence_step on a one-cell state holding the same arrays, for both
 * shuffle contracts.  The call copies its small descriptors from host memory,
 * enqueues the step, then blocks until the stream has drained to read the
 * step's error word, and returns it (SDM_ECAPACITY on a bucket overflow).
 * Because it synchronises the stream, it cannot be called while that stream
 * is being captured into a CUDA graph, nor from a host function or callback
 * enqueued on a stream (CUDA calls are not allowed there).  Every call looks
 * up the device address of the fixed scratch array in the current context
 * and, the first time in a context, uploads the library's constant tables.
 * All calls share the one scratch array, which keeps the last call's
 * contents: calls that overlap on the GPU (different streams, or several host
 * threads) race with each other and must be serialised by the caller. */
#define SDM_NOALLOC_MAX_SD (1u << 18)
sdm_status sdm_coalescence_step_noalloc(uint64_t* xi, double* attr, uint32_t n_attr, uint64_t attr_stride,
                                        uint32_t n_sd, double dv, uint32_t kernel_id,
                                        const sdm_step_params* params, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SDM_H */
