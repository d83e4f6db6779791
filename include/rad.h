/*
 * rad.h -- C ABI of the GB300 in-situ radiation-spectrum accumulator.
 *
 * The library computes, for every tracked particle j, observer direction n
 * and frequency omega, the Lienard-Wiechert far-field spectrum accumulated
 * over the PIC time steps, and sums it over particles (Frederiksen et al.,
 * "Radiation Spectral Synthesis of Relativistic Filamentation", Sec. 2.2:
 * the discretised integral P_omega ~ |int sum_j E_ret,j exp(i omega phi') dt'|^2
 * with phi' = t' - n.r(t')/c, multiple far-field observers at arbitrary
 * orientation, logarithmic or linear frequency bins, phase-coherent or
 * phase-incoherent synthesis, spectra recorded over windows of steps).  The
 * integrand is the Jackson retarded-time form the paper cites through
 * Rybicki & Lightman:
 *
 *   d^2W/(dw dOmega) = q^2/(4 pi^2 c) |sum_m n x ((n-beta) x betadot)/(1-n.beta)^2
 *                                        exp(i w (t_m - n.r_m/c)) dt|^2
 *
 * Units follow the paper's PIC scaling (Sec. 2.1): c = 1, time in 1/omega_pe,
 * frequencies in omega_pe; u = gamma*beta is the momentum per unit mass.
 *
 * Call protocol (leapfrog, the reading of Sec. 2.2's time integral): the call
 * for step s passes x_s (position at t = s dt, possibly wrapped into a
 * periodic box) and u_{s-1/2}.  Sample m uses r_m (unwrapped x_m),
 * beta_m = ubar/sqrt(1+ubar^2) with ubar = (u_{m-1/2}+u_{m+1/2})/2 and
 * betadot_m = (beta_{m+1/2} - beta_{m-1/2})/dt, so sample m is complete after
 * the call for step m+1.  A window [s0, s1) of samples therefore closes after
 * the call for step s1.  Steps start at 0 and increase by one.
 *
 * Memory: every pointer argument may point to host memory (pageable or
 * pinned) or device memory of the context's device; the library detects which
 * and copies what it needs.  The caller keeps ownership of everything it
 * passes.  Device-resident inputs are read on the context's stream, so the
 * caller may reuse them once work enqueued on that stream after the call has
 * completed.  Host-resident inputs may be reused as soon as the call returns.
 *
 * Errors: every int-returning call returns RAD_OK (0) or a negative RAD_E*
 * code; rad_last_error() gives a one-line description.  A failed call leaves
 * the context usable unless it returns RAD_ECUDA.  Every device-side wait is
 * bounded: if one expires the kernel raises an error word and returns, and
 * rad_finalize / rad_partial_sums report RAD_ETIMEOUT (rad_reset clears it).
 *
 * Failure-detection test hooks: the environment variable RAD_FAULT, read by
 * rad_init, holds comma-separated tokens (an unknown token makes rad_init
 * return RAD_EINVAL):
 *   alloc   rad_init fails as if an allocation had failed (RAD_ENOMEM);
 *   graph   step-graph capture fails: the context falls back to direct
 *           launches and rad_get_options reports use_graph = 0;
 *   step:N  the call starting at step N is lost once (returns RAD_OK, does
 *           nothing), so the next call returns RAD_ESTEP until N is resent;
 *   stall   in the next directly launched accumulation kernel, block 0 waits
 *           on a barrier nothing arrives on until the bounded wait expires,
 *           so rad_finalize returns RAD_ETIMEOUT (once).
 */
#ifndef RAD_H
#define RAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RAD_OK 0
#define RAD_EINVAL (-1)      /* bad argument */
#define RAD_ENOMEM (-2)      /* device or host allocation failed */
#define RAD_ECUDA (-3)       /* a CUDA call failed; see rad_last_error */
#define RAD_ESTEP (-4)       /* step is not previous step + 1 (first must be 0) */
#define RAD_EINCOMPLETE (-5) /* finalize before every window's last sample arrived */
#define RAD_ETIMEOUT (-6)    /* a bounded device-side wait expired; results invalid */
#define RAD_ENAN (-7)        /* non-finite input detected (check_inputs option) */
#define RAD_ESTATE (-8)      /* call not allowed in the context's current state */
#define RAD_ENOSPACE (-9)    /* problem larger than rad_spectrum_noalloc's fixed memory */

/* summation over particles (Sec. 2.2: "phase coherent or phase incoherent") */
#define RAD_INCOHERENT 0     /* S = 1/(4 pi^2) sum_j |q_j A_j|^2 */
#define RAD_COHERENT 1       /* S = 1/(4 pi^2) |sum_j q_j A_j|^2 */

/* arithmetic of the accumulation */
#define RAD_FP64 0           /* FP64 geometry, phase and sums; CUDA double sincos */
#define RAD_FP32_SPLIT 1     /* FP32 bulk; FP64 retarded-time anchor every K samples */

/* sincos engine of the FP32 split path */
#define RAD_VARIANT_AUTO 0   /* autotuned (or the cached choice) */
#define RAD_VARIANT_SFU 1    /* every e^{i theta} by the special-function unit */
#define RAD_VARIANT_MIX 2    /* some frequencies by an FMA-pipe polynomial (see reserved[1]) */
#define RAD_VARIANT_PRECISE 3 /* the offset phase nu dphi in float-float, reduced to one
                                 turn before the special-function unit: per-update phase
                                 error ~5e-7 rad instead of ~1e-7 |omega dphi|; 8
                                 frequencies per thread, anchor interval 32.  With a
                                 phase budget (reserved[3]) only the frequency tiles
                                 whose K = 32 rounding bound w_max 31 dt 2^-24 exceeds
                                 it take the precise phase, the others the SFU path */

typedef struct rad_ctx rad_ctx;

/* One particle species: `count` consecutive particles of the particle axis. */
typedef struct {
    int64_t count;   /* particles of this species (>= 0) */
    double charge;   /* q in units of the elementary charge (electron: -1) */
    double mass;     /* m in electron masses; informational (u is per unit mass) */
} rad_species;

/* One spectrum window: samples [s0, s1) of the species in species_mask (bit i
 * = species i), on frequency grid freq_grid, seen by the observers in dir_set
 * (Sec. 2.2: spectra "recorded every small multiple of a simulation timestep",
 * a cumulative snapshot being the window [0, t); "multiple far-field
 * observers at arbitrary orientation", so each window may take its own subset
 * of the context's directions).  The output holds, per window, a
 * [n_dirs][len(grid)] block whose rows follow dir_set (all D directions in
 * order when dir_set is NULL).  A zero-initialised window tail (dir_set NULL,
 * n_dir_set 0) selects every direction. */
typedef struct {
    int64_t s0, s1;
    uint32_t species_mask;
    int32_t freq_grid;
    const int32_t *dir_set;  /* NULL: every direction; else n_dir_set indices into
                                the directions given to rad_init (repeats allowed),
                                copied by rad_init                                 */
    int32_t n_dir_set;       /* entries of dir_set (>= 1 when dir_set is not NULL) */
    int32_t reserved;        /* must be 0                                          */
} rad_window;

/* Sample selectors (Sec. 2.2: "multiple regions for spectral collection in the
 * simulation volume"; the momentum pitch-cone selection of Sec. 3.2).  A window
 * that names a selector only sums the samples inside it (the other samples
 * contribute nothing, as if the particle did not radiate there). */
#define RAD_SEL_BOX 1        /* lo <= x_m < hi per component, x_m as handed over */
#define RAD_SEL_CONE 2       /* |angle(ubar_m, axis) - theta_c| <= dtheta       */

typedef struct {
    int32_t kind;            /* RAD_SEL_BOX or RAD_SEL_CONE */
    double lo[3], hi[3];     /* box corners (positions as the PIC hands them over) */
    double axis[3];          /* cone axis (normalised by the library) */
    double theta_c, dtheta;  /* cone centre angle and half width, radians */
} rad_selector;

/* Tuning knobs; zero-initialise for the defaults.  Set before the first step. */
typedef struct {
    int32_t variant;       /* RAD_VARIANT_*                                  */
    int32_t anchor_K;      /* FP32 path re-anchor interval: 8, 16 or 32 samples for
                              every frequency; 0 with the automatic kernel choice
                              or a phase budget in reserved[3]: the longest of 8,
                              16, 32 with w_max (K - 1) dt 2^-24 within the budget
                              (Sec. 2.2's phase as an FP32 offset), w_max the
                              highest frequency of all grids; where a lower
                              frequency tile can take a longer interval and the
                              kernel build is (or the automatic choice is then
                              restricted to) 8 SFU frequencies per thread, that
                              tile takes its own, from its own w_max
                              (rad_get_options reports the shortest, which
                              anchors the ring); 0 otherwise: 32              */
    int32_t freq_per_lane; /* 0 (auto), 4, 8 or 16 frequencies per thread      */
    int32_t defer;         /* 1: evaluate every window in one persistent launch at
                              finalize instead of when its last sample arrives */
    int32_t use_graph;     /* 1: FP32 path, one step per call, device inputs: replay
                              each step's launches (ingest; at a closing step also
                              the accumulation) as an instantiated CUDA graph    */
    int32_t check_inputs;  /* 1: flag non-finite x/u (RAD_ENAN at finalize)    */
    int32_t blocks_per_sm; /* 0 (auto), 2, 3 or 4: resident blocks per SM the FP32
                              kernel is built for (its register budget); 4
                              frequencies per thread go with 4, 16 with 2    */
    int32_t subcycle;      /* 0 or 1: none; n >= 2: n sub-samples per PIC sample
                              (Sec. 2.2 sub-cycling of the tracked particles):
                              u linear in time between the half-step states,
                              betadot its exact derivative, r by Simpson's rule;
                              updates and the ring grow n-fold               */
    int32_t reserved[8];   /* [0]: 1 = time the ingest launches (rad_timing);
                              [1]: MIX variant, frequencies of each thread on the
                              FMA-pipe polynomial (0: 2 of 8, 4 of 16); after the
                              first step rad_get_options reports the kernel build
                              in use here (0 for SFU); [2]: host inputs with
                              eager windows: MiB per staging buffer of the
                              particle-blocked transfer (0: 8192); [3]: FP32 path,
                              phase budget per update in nanoradians (0: 1e-4 rad),
                              see anchor_K; others must be 0                       */
} rad_options;

/*
 * rad_init -- create a context (Sec. 2.2: observers, frequency bins, tracked
 * particles, coherent/incoherent choice).
 *   out        : receives the context.
 *   dirs       : [D][3] observer directions (normalised by the library), D >= 1.
 *   freqs      : concatenation of n_grids frequency grids (any spacing; > 0
 *                not required), grid g has grid_len[g] >= 1 points.
 *   dt         : time step (> 0).
 *   sp         : n_species >= 1 species; particle axis = species concatenated.
 *   win        : n_win >= 1 windows, 0 <= s0 <= s1, grid index in range,
 *                species_mask within the species, dir_set entries in [0, D).
 *   mode       : RAD_INCOHERENT or RAD_COHERENT.
 *   precision  : RAD_FP64 or RAD_FP32_SPLIT.
 *   box_L      : periodic box side for unwrapping positions (0: no unwrap).
 *   cuda_stream: cudaStream_t to enqueue on (NULL: the legacy default stream).
 * Allocates all device memory the context needs (trajectory ring, state,
 * accumulators); returns RAD_ENOMEM if it does not fit.  On error *out is NULL.
 */
int rad_init(rad_ctx **out, const double *dirs, int32_t D, const double *freqs,
             const int32_t *grid_len, int32_t n_grids, double dt, const rad_species *sp,
             int32_t n_species, const rad_window *win, int32_t n_win, int32_t mode,
             int32_t precision, double box_L, void *cuda_stream);

/*
 * rad_set_selectors -- define n_sel <= 32 selectors and, for every window,
 * the selector it uses (window_selector[n_win]: index, or -1 for all samples).
 * The ingest tests each sample against every selector in FP64: the box on the
 * position x_m handed over for step m, the cone on
 * cos(angle) = (ubar_m . axis) / |ubar_m| against [cos(theta_c + dtheta),
 * cos(theta_c - dtheta)] (angles clamped to [0, pi]).  Call before the first
 * step (RAD_ESTATE after it); a later call replaces the earlier definition.
 */
int rad_set_selectors(rad_ctx *ctx, const rad_selector *sel, int32_t n_sel,
                      const int32_t *window_selector);

/* rad_set_options -- set tuning knobs; RAD_ESTATE after the first step. */
int rad_set_options(rad_ctx *ctx, const rad_options *opt);

/* rad_get_options -- the knobs in effect (after autotuning if it ran). */
int rad_get_options(const rad_ctx *ctx, rad_options *opt);

/*
 * rad_accumulate -- hand over one PIC step (Sec. 2.2: spectra are collected
 * at runtime).  x and u are SoA [3][N_total] FP64 (x: x_step, u: u_{step-1/2}).
 * Windows whose last sample completes with this step are evaluated now
 * (unless the defer option is set).  Returns before the device work is done.
 */
int rad_accumulate(rad_ctx *ctx, int64_t step, const double *x, const double *u);

/*
 * rad_accumulate_steps -- hand over n_steps consecutive steps at once:
 * x, u are [n_steps][3][N_total] FP64.  Equivalent to n_steps calls of
 * rad_accumulate, with fewer launches.  Host inputs are copied by the library
 * (the caller may reuse them when this returns); with eager windows and at
 * least 64 steps and 2048 particles, the particle axis (every species) is
 * streamed in blocks so that the transfer of later particles overlaps the
 * accumulation of earlier ones (results equal up to FP64 summation order).
 */
int rad_accumulate_steps(rad_ctx *ctx, int64_t step0, int64_t n_steps, const double *x,
                         const double *u);

/*
 * rad_finalize -- evaluate deferred windows, scale by 1/(4 pi^2 c) and write
 * the spectra: spectrum is [n_win][n_dirs of window][len(grid of window)] FP64
 * concatenated over windows (host or device).  Synchronises the context's stream.  Returns
 * RAD_EINCOMPLETE if a window's last sample has not arrived, RAD_ETIMEOUT or
 * RAD_ENAN if a device-side check failed.  May be called more than once.
 */
int rad_finalize(rad_ctx *ctx, double *spectrum);

/*
 * rad_partial_sums -- the unscaled FP64 particle sums behind the spectrum, for
 * combining the spectra of particle shards computed in different processes or
 * on different GPUs (Sec. 2.2: incoherent spectra of disjoint particle sets add;
 * coherent amplitudes add before the modulus is taken).  out holds, window
 * after window in rad_finalize's order:
 *   RAD_INCOHERENT: [n_bins] sum_j |A_j|^2;
 *   RAD_COHERENT:   [n_bins][4] Re, Im of sum_j A_j . e1 and of sum_j A_j . e2,
 *   where (e1, e2) is an orthonormal basis of the plane normal to the bin's
 *   direction that depends only on that direction (so shards with the same
 *   directions share it).
 * The spectrum of the union of shards is sum / (4 pi^2) (incoherent) or
 * (sum of each of the 4 components, squared and added) / (4 pi^2) (coherent).
 * Same preconditions, synchronisation and errors as rad_finalize.
 */
int rad_partial_sums(rad_ctx *ctx, double *out);

/*
 * rad_next_shard -- begin a further particle shard in the same context: the
 * step counter returns to 0 and the following calls hand over the leapfrog
 * states of another set of particles with the same species counts, whose
 * amplitudes are summed into the same accumulators (Sec. 2.2's sum over the
 * tracked particles j: incoherent spectra of disjoint particle sets add, and
 * coherent amplitudes add before the modulus is taken).  rad_finalize then
 * gives the spectrum of the union of every shard since rad_init or rad_reset.
 * This is how a population whose whole-window trajectory ring does not fit in
 * device memory at once is evaluated on one GPU: the context is sized for one
 * shard and the shards are handed over one after another.  Every window must
 * be complete for the current shard (RAD_EINCOMPLETE otherwise); deferred
 * windows are evaluated before the step counter is rewound.  Enqueues work on
 * the context's stream only; does not synchronise.
 */
int rad_next_shard(rad_ctx *ctx);

/*
 * rad_spectrum_from_sums -- the spectrum of the union of particle shards from
 * the element-wise sum of their rad_partial_sums outputs (Sec. 2.2: incoherent
 * spectra of disjoint particle sets add; coherent amplitudes add before the
 * modulus is taken), for the shards of several processes or GPUs once their
 * partial sums have been added (for example by an all-reduce):
 *   RAD_INCOHERENT: spectrum[i] = sums[i] / (4 pi^2)
 *   RAD_COHERENT:   spectrum[i] = (sums[4i]^2 + sums[4i+1]^2 + sums[4i+2]^2
 *                                  + sums[4i+3]^2) / (4 pi^2)
 * sums: [n_bins] or [n_bins][4] FP64 and spectrum: [n_bins] FP64, both in
 * device memory of the current device (or managed memory); anything else is
 * RAD_EINVAL.  Runs on cuda_stream (NULL: the legacy default stream) and
 * returns without synchronising; RAD_ECUDA if the launch fails.
 */
int rad_spectrum_from_sums(const double *sums, int64_t n_bins, int32_t mode, double *spectrum,
                           void *cuda_stream);

/* rad_reset -- forget all steps and zero the accumulators (same configuration). */
int rad_reset(rad_ctx *ctx);

/* rad_spectrum_size -- number of doubles rad_finalize writes (or -1). */
int64_t rad_spectrum_size(const rad_ctx *ctx);

/* rad_updates -- particle*sample*omega*direction updates over all windows. */
int64_t rad_updates(const rad_ctx *ctx);

/*
 * rad_timing -- device time (CUDA events on the context's stream) spent since
 * rad_init in the window accumulation kernels and (when enabled) in the
 * per-step ingest, and the number of accumulation and ingest launches.
 * rad_reset does not clear these totals.  Synchronises the stream.
 */
int rad_timing(rad_ctx *ctx, double *accum_ms, double *ingest_ms, int64_t *accum_launches,
               int64_t *ingest_launches);

/* rad_last_error -- description of the last failure on ctx (never NULL). */
const char *rad_last_error(const rad_ctx *ctx);

/* rad_destroy -- free the context (NULL is allowed). */
void rad_destroy(rad_ctx *ctx);

/*
 * rad_spectrum_noalloc -- the spectrum of one trajectory without allocating
 * any device memory.  The paper has no counterpart: this is a service of the
 * library for callers that may not allocate device memory, for example a
 * simulation that gives all GPU memory to its own pool at start-up and does
 * not let libraries call cudaMalloc, or a host program where allocation calls
 * are not available.  It computes what rad_init + rad_accumulate_steps +
 * rad_finalize compute for one species, one window of samples [0, n_calls-1)
 * and the FP32 split path (default kernel), using instead a fixed 96 MiB
 * device array that is part of this library: every GPU that loads the library
 * holds it until the process exits.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   dirs     : host [D][3] observer directions (normalised here), D >= 1.
 *   freqs    : host [F] frequencies, F >= 1.
 *   dt, charge, box_L, mode : as for rad_init / rad_species.
 *   N        : particles (>= 1); n_calls >= 2 steps of leapfrog states.
 *   x, u     : device [n_calls][3][N] FP64, x_s and u_{s-1/2} per step.
 *   spectrum : device [D][F] FP64, written by the call (the caller owns it).
 *   (x, u and spectrum in device memory of the current device, or managed
 *   memory; anything else is RAD_EINVAL.)
 *   cuda_stream : stream to run on (NULL: the legacy default stream).
 * Limit: the trajectory ring, anchor ring, per-particle state and
 * accumulators must fit in the 96 MiB array -- about
 *   (round_up(n_calls - 1, 32) + 64) * round_up(N, 8) * 40 bytes
 *   + (that many samples / 32) * round_up(N, 8) * 24 bytes + 72 * N bytes
 *   + 8 * D * F bytes (x4 for RAD_COHERENT) + small tables;
 * 1024 particles x 2000 samples fit, 8192 x 4096 do not.  Larger problems are
 * rejected with RAD_ENOSPACE before any device work.  RAD_EINVAL: bad
 * argument; RAD_ECUDA: a CUDA call failed; RAD_ETIMEOUT: a bounded device
 * wait expired (results invalid).
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so the address stays right
 * when a device reset re-creates the device's context.  The first call on a
 * device also loads the library's device code there, which is when the array
 * itself comes into being.  The call synchronises the stream and returns after
 * the spectrum is written, so it cannot be made while a stream is being
 * captured into a CUDA graph.  Every call uses the same array and leaves its
 * contents behind; each call clears what must start at zero.  Calls that
 * overlap on the same GPU (from several host threads or streams at once) race
 * on the array and corrupt each other: serialise them.
 */
int rad_spectrum_noalloc(const double *dirs, int32_t D, const double *freqs, int32_t F, double dt,
                         double charge, int64_t N, int64_t n_calls, const double *x,
                         const double *u, int32_t mode, double box_L, double *spectrum,
                         void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RAD_H */
