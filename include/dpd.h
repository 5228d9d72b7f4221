/*
 * dpd.h -- C ABI of the GB300 DPD fluid-step library (libdpd.so).
 *
 * The library advances a dissipative particle dynamics (DPD) fluid in
 * periodic boxes, following the method of the MiRheo paper:
 *   - Newton's equations of motion (Sec. 2.1, Eq. 1) with m the particle mass;
 *   - pair forces F_i = sum_j (F^C_ij + F^D_ij + F^R_ij) (Eq. 2):
 *       F^C = a w(r) e_ij,  w(r) = 1 - r/rc for r < rc, else 0  (Eqs. 3-4),
 *       F^D = -gamma w_D(r) (v_ij . e_ij) e_ij,
 *       F^R = sigma w_R(r) xi_ij e_ij / sqrt(dt)                  (Eq. 5),
 *     with sigma^2 = 2 gamma kT, w_D = w_R^2, w_R = w^k (Sec. 2.1);
 *   - the noise xi_ij is stateless and pair-symmetric: word 0 of
 *     Philox-4x32-10 on the counter (min id, max id, step lo, step hi) with key
 *     (seed lo, seed hi), mapped to xi = sqrt(3)(2U - 1),
 *     U = ((u >> 8) + 1/2) 2^-24 (zero mean, unit variance);
 *   - cell lists rebuilt every step (Sec. 3.2): counting sort of particles
 *     into cells of edge h_d = L_d / floor(L_d / rc) >= rc (each cut into 2
 *     slices along x), exclusive scan, reorder (stable by previous slot for
 *     the full stencil, by arrival for the half stencil); forces summed over
 *     the 27 neighbouring cells, or 13 of them plus the own cell with
 *     Newton's third law (half stencil);
 *   - velocity-Verlet with the velocity predicted at the half step (the fused
 *     leapfrog of Sec. 3.1, item 5): v += dt/2 F/m; x += dt v (wrapped into
 *     [0, L)); F = F(x, v); v += dt/2 F/m.
 *
 * Step index of the noise: the force computed by dpd_set_state uses step 0;
 * the force computed during the k-th call-counted step uses step k.
 *
 * Arithmetic: FP32 state and forces; box-level reductions sum in FP64 above
 * the GPU block (inside a block of 4096 particles, as unevaluated pairs of
 * FP32 numbers, about 2^-44 relative).
 *
 * Conventions for every call:
 *   - returns DPD_OK (0) or a negative DPD_ERR_* status; never aborts or
 *     exits; on failure dpd_last_error() gives a message (thread-local);
 *   - "where" arguments say whether a pointer is host memory
 *     (DPD_WHERE_HOST) or device memory of the current CUDA device
 *     (DPD_WHERE_DEVICE); the caller owns every buffer it passes and the
 *     library copies what it needs before returning;
 *   - arrays of 3-vectors are n x 3, row-major (x0 y0 z0 x1 y1 z1 ...);
 *   - a context lives on the CUDA device that was current at creation and
 *     enqueues all work on its stream (default: the legacy default stream);
 *     calls on one context are not thread-safe.
 */
#ifndef DPD_H
#define DPD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DPD_API __attribute__((visibility("default")))
#else
#define DPD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define DPD_OK 0
#define DPD_ERR_ARG (-1)      /* invalid argument                                  */
#define DPD_ERR_NOMEM (-2)    /* device or host allocation failed / budget exceeded */
#define DPD_ERR_CUDA (-3)     /* a CUDA runtime call failed                         */
#define DPD_ERR_STATE (-4)    /* call out of order (e.g. step before set_state)     */
#define DPD_ERR_NUMERIC (-5)  /* device flagged a non-finite position or force, a runaway particle, or (brick kernel) a cell row whose stencil exceeds its staging */
#define DPD_ERR_TIMEOUT (-6)  /* a bounded wait expired                              */
#define DPD_ERR_BUSY (-7)     /* resource in use (e.g. result not ready)            */
#define DPD_ERR_INTERNAL (-8) /* checked build only: a kernel's index check failed  */

#define DPD_WHERE_HOST 0
#define DPD_WHERE_DEVICE 1

/* Thread-local text of the last failure in this thread ("" if none). */
DPD_API const char *dpd_last_error(void);

/* Library version string. */
DPD_API const char *dpd_version(void);
/* Rounds R of the library's Philox-4x32-R noise generator: 10, unless the
 * library was built with another count for a round-count study. */
DPD_API int dpd_philox_rounds(void);

/* ================================================================ one box */
typedef struct dpd_ctx dpd_ctx;

/* Parameters settable after creation (dpd_set_param). */
#define DPD_PARAM_KEXP 1          /* weight exponent k in w_R = w^k, (0, 1]; default 1 (Sec. 2.1) */
#define DPD_PARAM_MASS 2          /* particle mass m > 0; default 1 (Eq. 1) */
#define DPD_PARAM_BODYFORCE 3     /* constant body force magnitude along DPD_PARAM_FLOW_AXIS */
#define DPD_PARAM_POISEUILLE_F 4  /* periodic Poiseuille force f (Sec. 4.2): -f where the
                                     coordinate on DPD_PARAM_GRAD_AXIS is <= L/2, +f above */
#define DPD_PARAM_FLOW_AXIS 5     /* 0, 1, 2: axis the body force points along; default 2 (z) */
#define DPD_PARAM_GRAD_AXIS 6     /* 0, 1, 2: axis the Poiseuille force switches on; default 0 (x) */
#define DPD_PARAM_STENCIL 7       /* DPD_STENCIL_FULL (default) or DPD_STENCIL_HALF */

#define DPD_PARAM_FORCE_TILES 8   /* full stencil: 1 stages each block's neighbourhood in shared
                                     memory; 0 (default) has one thread per particle read its
                                     neighbours through the L1 cache (faster on GB300) */
#define DPD_PARAM_TILE_CELLS 9    /* cells per staged tile, 1..64; 0 (default) = chosen by density */
#define DPD_PARAM_STAGE_CAP 10    /* staged particles per block, 64..4096; 0 (default) = by density;
                                     blocks whose neighbourhood exceeds it read global memory */

#define DPD_PARAM_FORCE_VARIANT 11 /* direct force-kernel variant 0..DPD_NUM_FORCE_VARIANTS-1, or -1
                                      (default) to pick per density band from the tuning table */

#define DPD_PARAM_NOISE 12        /* DPD_NOISE_UNIFORM (default) or DPD_NOISE_GAUSSIAN */

#define DPD_PARAM_FUSE 13         /* full stencil: 1 (default) lets each step's force kernel also
                                     kick, drift and bin every particle for the next step of the
                                     same dpd_step call (no separate integrate pass, no stored
                                     force in between); 0 runs them as separate kernels.  Both
                                     give the same bits.  Off for the half stencil, the staged
                                     tiles and steps followed by sampling. */

#define DPD_NOISE_UNIFORM 0   /* xi = sqrt(3)(2U - 1): uniform, unit variance, bit-exact on CPU */
#define DPD_NOISE_GAUSSIAN 1  /* xi Gaussian as Sec. 2.1 states: Box-Muller on words 0 and 1,
                                 sqrt(-2 ln U1) cos(2 pi U2); within rounding of libm */

#define DPD_STENCIL_FULL 0  /* 27 cells, each thread sums its own pairs: no atomics,
                               bitwise reproducible */
#define DPD_STENCIL_HALF 1  /* 13 cells + own cell, Newton's third law with atomics
                               (Sec. 3.2 notes the symmetric form is faster) */

/* Create a context for one periodic box.
 * box: three edges L_d, each >= 3 rc (so that the 27 neighbour cells are
 *      distinct) and at most 1023 cells per edge.
 * a, gamma, kT >= 0; rc > 0; dt > 0; seed: key of the pair noise.
 * Allocates nothing on the device until dpd_set_state.
 * Errors: DPD_ERR_ARG (bad value), DPD_ERR_CUDA (no device). */
DPD_API int dpd_create(dpd_ctx **out, const double box[3], double a, double gamma, double kT, double rc,
               double dt, uint64_t seed);

/* Release every resource of the context (synchronises its stream). NULL is a no-op. */
DPD_API int dpd_destroy(dpd_ctx *ctx);

/* Set one DPD_PARAM_* value.  Takes effect at the next dpd_set_state or
 * dpd_step.  Errors: DPD_ERR_ARG for an unknown key or bad value. */
DPD_API int dpd_set_param(dpd_ctx *ctx, int key, double value);

/* Read one DPD_PARAM_* value.  For DPD_PARAM_TILE_CELLS and
 * DPD_PARAM_STAGE_CAP the value in use is returned (after dpd_set_state,
 * the one chosen by density when the parameter was left at 0). */
DPD_API int dpd_get_param(const dpd_ctx *ctx, int key, double *value);

/* Enqueue all later work of the context on the given cudaStream_t
 * (e.g. torch.cuda.current_stream().cuda_stream).  NULL = legacy default stream. */
DPD_API int dpd_set_stream(dpd_ctx *ctx, void *stream);

/* Load n particles: pos and vel are n x 3 FP32 (positions anywhere; they are
 * wrapped into [0, L)).  Particle i receives id i, which keys its noise.  The
 * force at step 0 is computed here; the step counter is reset to 0.
 * n = 0 is allowed.  Errors: DPD_ERR_ARG, DPD_ERR_NOMEM, DPD_ERR_CUDA. */
DPD_API int dpd_set_state(dpd_ctx *ctx, int64_t n, const float *pos, const float *vel, int where);

/* ------------------------------------------------------------- species */
/* Several particle species in one box, each pair of species with its own
 * interaction (the particle vectors of Sec. 3.1, whose pairwise forces may
 * differ in parameters and cut-off; Sec. 3.2 keeps one cell list per
 * cut-off, here one list serves all, built for the context's rc).
 * a, gamma, rc: nspecies x nspecies row-major tables, symmetric, a and gamma
 * >= 0, 0 < rc_st <= the context's rc; sigma_st^2 = 2 gamma_st kT (Sec. 2.1).
 * All species share the mass and the weight exponent.  nspecies 2..4
 * (DPD_MAX_SPECIES); nspecies = 1 returns to one species with the scalar
 * parameters (the tables may then be NULL).  With a state loaded only the
 * table values may change, not the count.  The staged force tiles
 * (DPD_PARAM_FORCE_TILES) serve one species only.  Errors: DPD_ERR_ARG,
 * DPD_ERR_STATE. */
#define DPD_MAX_SPECIES 4
DPD_API int dpd_set_species(dpd_ctx *ctx, int nspecies, const double *a, const double *gamma,
                            const double *rc);
/* The species count and, when it is above 1, the tables (nspecies^2 each;
 * any table pointer may be NULL). */
DPD_API int dpd_get_species(const dpd_ctx *ctx, int *nspecies, double *a, double *gamma,
                            double *rc);
/* dpd_set_state with a species 0..nspecies-1 per particle (int32, in the same
 * memory as pos and vel; NULL = all species 0); a species out of range is
 * DPD_ERR_ARG.  n <= 2^26. */
DPD_API int dpd_set_state_species(dpd_ctx *ctx, int64_t n, const float *pos, const float *vel,
                                  const int32_t *species, int where);

/* Advance nsteps >= 0 steps.  Asynchronous on the context's stream.
 * Errors: DPD_ERR_STATE before dpd_set_state, DPD_ERR_CUDA. */
DPD_API int dpd_step(dpd_ctx *ctx, int64_t nsteps);

/* Current positions (in [0, L)) and full-step velocities, n x 3 FP32, in id
 * order.  Synchronises the stream.  Either pointer may be NULL.
 * Errors: DPD_ERR_STATE, DPD_ERR_NUMERIC (device flagged non-finite values;
 * the state is still returned), DPD_ERR_CUDA. */
DPD_API int dpd_get_state(dpd_ctx *ctx, float *pos, float *vel, int where);

/* Total force on each particle at the current step (pair sum + body force),
 * n x 3 FP32 in id order.  Synchronises the stream. */
DPD_API int dpd_get_forces(dpd_ctx *ctx, float *force, int where);

/* Box statistics at the current step, reduced in FP64. */
typedef struct {
    double momentum[3];  /* sum m v                                          */
    double kinetic;      /* sum m v^2 / 2                                    */
    double kT;           /* 2 kinetic / (3 (N - 1))                          */
    double virial;       /* sum over pairs i<j of r_ij . F^C_ij              */
    double pressure;     /* N kT / V + virial / (3 V)                        */
    int64_t step;        /* steps taken since dpd_set_state                  */
    int64_t n;           /* particles                                        */
} dpd_stats;

DPD_API int dpd_get_stats(dpd_ctx *ctx, dpd_stats *out);

/* ---------------------------------------------------------- checkpoints */
/* A checkpoint holds the context's internal state as the device keeps it:
 * positions, velocities (v(n - 1/2) after the first step), forces, in the
 * current cell order, with the step counter.  Loading it into a context
 * created with the same box and parameters continues the run exactly
 * (bitwise with the full stencil).  `buf` is host memory of
 * dpd_checkpoint_size() bytes; loading checks its header.
 * Errors: DPD_ERR_STATE (nothing loaded / mismatched header), DPD_ERR_ARG. */
DPD_API int64_t dpd_checkpoint_size(const dpd_ctx *ctx);
DPD_API int dpd_checkpoint_save(dpd_ctx *ctx, void *buf, int64_t bytes);
DPD_API int dpd_checkpoint_load(dpd_ctx *ctx, const void *buf, int64_t bytes);

/* Number of particles loaded (0 before dpd_set_state). */
DPD_API int64_t dpd_num_particles(const dpd_ctx *ctx);

/* ------------------------------------------------------- instrumentation */
#define DPD_NUM_STAGES 5       /* integrate+count, scan, key pass, reorder, force */
#define DPD_KERNELS_PER_STEP 7 /* kernel launches per step of one force band with the full
                                 * stencil (the scan takes three); the half stencil has no
                                 * key pass: one fewer */

/* Advance nsteps steps like dpd_step, launching each step's kernels directly
 * (no graph) with CUDA events recorded on the context's stream between the
 * stages, synchronising after every step.  stage_ms[DPD_NUM_STAGES] receives
 * the mean device milliseconds of each stage. */
DPD_API int dpd_profile_steps(dpd_ctx *ctx, int64_t nsteps, double *stage_ms);

/* ---------------------------------------------------------------- debug */
/* Raw noise words for n pairs (lo[k], hi[k]) at a step and seed: words 0
 * and 1 of Philox-4x32-10 on (min, max, step lo, step hi) keyed by (seed lo,
 * seed hi).  lo, hi, out0 are DEVICE pointers; out1 and xi may be NULL; xi
 * receives the FP32 noise of the given DPD_NOISE_* mode.  Runs on the given
 * stream (NULL = default) and synchronises it. */
DPD_API int dpd_debug_rng(const uint32_t *lo, const uint32_t *hi, int64_t n, uint64_t step, uint64_t seed,
                  int noise, uint32_t *out0, uint32_t *out1, float *xi, void *stream);

/* --------------------------------------------------------- kernel tuning */
/* The direct force kernel comes in variants that differ in threads per
 * block, pair-list entries per thread and how a warp drains its lists:
 * variants 0-6 per lane, 7-9 balanced over the warp in list order, 10-12
 * spread over the warp with atomic sums (half stencil only; with the full
 * stencil 10-12 drain per lane), 13 the brick kernel that stages cell rows
 * and their neighbours in shared memory (half stencil; with the full
 * stencil, and for boxes dense enough to fill half its staging with one
 * row's stencil, it runs variant 0).  Process-wide tables map density bands
 * (upper bounds of rho = N/V, increasing; the last band also takes every
 * higher density) to a variant.  There are four: table = stencil
 * (DPD_STENCIL_FULL/HALF) for a single box, stencil + DPD_TUNING_PACKED
 * for packed sets of several boxes, whose kernels differ (each lane looks
 * up its box); a packed table never set uses its stencil's single-box
 * table.  Contexts and batches pick their variants when their state is
 * laid out.  The package's autotuner measures the variants per band on the
 * GPU and sets the tables. */
#define DPD_NUM_FORCE_VARIANTS 14
#define DPD_MAX_DENSITY_BANDS 8
#define DPD_TUNING_PACKED 2
/* threads per block and list capacity of variant v; DPD_ERR_ARG if out of range */
DPD_API int dpd_force_variant_info(int v, int *threads, int *list_capacity);
/* set table 0..3 (see above): nbands in 1..DPD_MAX_DENSITY_BANDS */
DPD_API int dpd_tuning_set(int table, int nbands, const double *rho_upper, const int *variant);
/* copy at most `max` bands of the table in use; *nbands receives its length */
DPD_API int dpd_tuning_get(int table, int max, double *rho_upper, int *variant, int *nbands);

/* Measured issue rates on the current device, for the force kernel's
 * roofline (the paper has no counterpart): rates[0] FP32 fused
 * multiply-adds per second (lane operations, register-only loops, eight
 * resident blocks of 256 threads per SM), rates[1] Philox-4x32-R words per
 * second (the pair-noise generator).  Each is timed with CUDA events on
 * `stream` (NULL = legacy default) over one launch of a few milliseconds
 * after a warm-up launch; synchronises the stream.  Allocates 1 KB. */
DPD_API int dpd_issue_rates(double rates[2], void *stream);

/* ============================================================ many boxes */
/* A batch steps many independent periodic boxes together: their particles
 * and cells are packed into one set of arrays (per-box slot and cell
 * offsets, boxes ordered by density band), every stage of a step is one
 * launch over all boxes, and steps are replayed from CUDA graphs.  Each box
 * gives exactly the trajectory it would give alone in a dpd_ctx with the
 * same parameters and the same stencil/variant (bitwise for the full
 * stencil). */
typedef struct dpd_batch dpd_batch;

typedef struct {
    double box[3];       /* edges, each >= 3 rc */
    double a, gamma, kT, rc, dt;
    uint64_t seed;
    int64_t n;           /* particles in this box */
    int64_t steps;       /* steps this box takes in total; <= 0: no limit */
    double kexp;         /* weight exponent; 0 means 1 */
    double mass;         /* particle mass; 0 means 1 */
    double body_force;   /* body-force magnitude (0: none) */
    int body_mode;       /* 0 none, 1 constant, 2 periodic Poiseuille (Sec. 4.2) */
    int flow_axis;       /* axis of the body force */
    int grad_axis;       /* axis on which the Poiseuille force switches sign */
    int noise;           /* DPD_NOISE_UNIFORM or DPD_NOISE_GAUSSIAN */
    int nspecies;        /* 0 or 1: one species; 2..DPD_MAX_SPECIES: the tables below, as
                            for dpd_set_species, entry (s, t) at [DPD_MAX_SPECIES s + t] */
    double species_a[DPD_MAX_SPECIES * DPD_MAX_SPECIES];
    double species_gamma[DPD_MAX_SPECIES * DPD_MAX_SPECIES];
    double species_rc[DPD_MAX_SPECIES * DPD_MAX_SPECIES];
} dpd_box_desc;

/* Create a batch of nbox boxes and allocate its device memory.
 * Errors: DPD_ERR_ARG (a descriptor is invalid; the message names the box),
 * DPD_ERR_NOMEM, DPD_ERR_CUDA. */
DPD_API int dpd_batch_create(dpd_batch **out, int nbox, const dpd_box_desc *descs);
DPD_API int dpd_batch_destroy(dpd_batch *b);
DPD_API int dpd_batch_set_stream(dpd_batch *b, void *stream);
/* DPD_PARAM_STENCIL, DPD_PARAM_FORCE_TILES, DPD_PARAM_TILE_CELLS,
 * DPD_PARAM_STAGE_CAP, DPD_PARAM_FORCE_VARIANT, DPD_PARAM_FUSE, or DPD_BATCH_GRAPH_CHUNK
 * (steps per captured graph, >= 1) */
#define DPD_BATCH_GRAPH_CHUNK 100
DPD_API int dpd_batch_set_option(dpd_batch *b, int key, double value);
/* Load box `box` (n of its descriptor x 3 FP32, host or device); ids 0..n-1
 * within the box; the box's step counter restarts at 0.  The cell lists and
 * forces of loaded boxes are built at the next step or read. */
DPD_API int dpd_batch_set_state(dpd_batch *b, int box, const float *pos, const float *vel,
                                int where);
/* dpd_batch_set_state with a species per particle (see
 * dpd_set_state_species); the box's descriptor gives the tables. */
DPD_API int dpd_batch_set_state_species(dpd_batch *b, int box, const float *pos, const float *vel,
                                        const int32_t *species, int where);
/* Advance every box by nsteps (a box with a step limit stops at it).
 * Errors: DPD_ERR_STATE while some box has not been loaded. */
DPD_API int dpd_batch_step(dpd_batch *b, int64_t nsteps);
DPD_API int dpd_batch_get_state(dpd_batch *b, int box, float *pos, float *vel, int where);
DPD_API int dpd_batch_get_forces(dpd_batch *b, int box, float *force, int where);
/* Statistics of every box (out has nbox entries, in the order of the descriptors). */
DPD_API int dpd_batch_get_stats(dpd_batch *b, dpd_stats *out);
DPD_API int dpd_batch_profile_steps(dpd_batch *b, int64_t nsteps, double *stage_ms);
DPD_API int dpd_batch_num_boxes(const dpd_batch *b);

/* ================================================================ serving */
/* A queue admits independent DPD runs as they arrive and runs them on one
 * GPU with continuous batching: a worker thread steps the resident runs
 * together (one packed batch) in chunks; between chunks it returns the runs
 * that reached their step count and admits waiting ones while an HBM
 * budget and a resident-run limit allow.  Each run starts from an initial
 * state drawn on the device from its seed (uniform positions, Maxwellian
 * velocities, zero total momentum) and is stepped and sampled at its own
 * step indices, so its result does not depend on the other runs. */
typedef struct dpd_queue dpd_queue;

typedef struct {
    int64_t max_boxes;       /* resident runs at most (0: 4096) */
    int64_t chunk_steps;     /* steps between admission points (0: 100) */
    int64_t sample_every;    /* statistics sample interval in steps (0: 20) */
    int nbins;               /* velocity-profile slabs, 1..64 (0: 16) */
    int policy;              /* admission order: 0 first come first served, 1 smallest N x steps */
    int stencil;             /* DPD_STENCIL_FULL or DPD_STENCIL_HALF */
    int pad_;
    double chunk_timeout_s;  /* a chunk not finished after this long fails the queue (0: 600) */
} dpd_queue_opts;

typedef struct {
    double box[3];
    double rho;              /* number density; used when n <= 0 (n = round(rho V)) */
    int64_t n;
    double a, gamma, kT, rc, dt;
    uint64_t seed;           /* noise key and initial-state seed */
    int64_t steps;           /* steps to run (> 0) */
    double body_force;       /* 0: none */
    int body_mode;           /* 1 constant, 2 periodic Poiseuille (Sec. 4.2) */
    int flow_axis, grad_axis;
    int noise;               /* DPD_NOISE_UNIFORM or DPD_NOISE_GAUSSIAN */
} dpd_request;

typedef struct {
    int status;              /* DPD_OK, or the error that ended the run (DPD_ERR_STATE: cancelled) */
    int nbins;
    int64_t n, steps;
    int64_t samples;         /* statistics samples taken (second half of the run) */
    double kT_mean;          /* mean of 2 KE / (3 (N - 1)) over the samples */
    double pressure_mean;    /* mean of N kT / V + virial / (3 V) over the samples */
    double profile[64];      /* mean flow-axis velocity per slab along the gradient axis */
    double t_submit, t_admit, t_done;  /* seconds on the queue's clock */
} dpd_result;

typedef struct {
    int64_t pending, resident, admitted, completed;
    uint64_t bytes_in_use;   /* HBM ledger of resident runs */
    double particle_steps;   /* particle-steps run so far */
    double busy_seconds;     /* time spent in chunks */
    double clock_seconds;    /* queue clock now */
} dpd_queue_stats;

/* Start a queue (and its worker thread) on the current device.  Requests
 * whose estimated device footprint exceeds hbm_budget_bytes are refused at
 * submission (DPD_ERR_NOMEM). */
DPD_API int dpd_queue_create(dpd_queue **out, size_t hbm_budget_bytes, const dpd_queue_opts *opts);
/* Stop the worker (the current chunk finishes) and release everything. */
DPD_API int dpd_queue_destroy(dpd_queue *q);
/* Non-blocking; thread-safe.  *ticket identifies the run.  Its initial
 * state is drawn on the device from req->seed: uniform positions in the
 * box, velocities of variance kT/m with the mean removed. */
DPD_API int dpd_queue_submit(dpd_queue *q, const dpd_request *req, uint64_t *ticket);
/* As dpd_queue_submit, with the caller's initial state: pos, vel are
 * req->n x 3 FP32 HOST arrays (req->n > 0; particle i has id i), copied
 * before the call returns (the caller keeps ownership).  keep_final != 0
 * keeps the run's final state for dpd_queue_final_state. */
DPD_API int dpd_queue_submit_state(dpd_queue *q, const dpd_request *req, const float *pos,
                                   const float *vel, int keep_final, uint64_t *ticket);
/* The final state of a finished run submitted with keep_final: n x 3 FP32
 * HOST arrays in id order, full-step velocities.  DPD_ERR_BUSY until the
 * run has finished, DPD_ERR_STATE if it kept no state. */
DPD_API int dpd_queue_final_state(dpd_queue *q, uint64_t ticket, float *pos, float *vel);
DPD_API int dpd_queue_poll(dpd_queue *q, uint64_t ticket, int *done);
/* DPD_ERR_BUSY until the run has finished. */
DPD_API int dpd_queue_result(dpd_queue *q, uint64_t ticket, dpd_result *out);
/* A waiting run finishes at once; a resident one at the next chunk boundary. */
DPD_API int dpd_queue_cancel(dpd_queue *q, uint64_t ticket);
/* Wait until no run is waiting or resident; DPD_ERR_TIMEOUT after timeout_s. */
DPD_API int dpd_queue_wait_all(dpd_queue *q, double timeout_s);
DPD_API int dpd_queue_get_stats(dpd_queue *q, dpd_queue_stats *out);

/* ------------------------------------------------- forces without allocation */
/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory where they need forces (code inside a host
 * callback or a custom allocator, a framework that has given all device
 * memory to its own pool, a real-time loop that must not meet cudaMalloc's
 * implicit device synchronisation).
 *
 * Pair forces plus nothing else (no body force, k = 1, m = 1) on n particles
 * of one periodic box, at noise step `step`, from a caller-provided state.
 * pos, vel: n x 3 FP32 DEVICE pointers (particle i has id i); force: n x 3
 * FP32 DEVICE output, in the same order.  The result equals what
 * dpd_set_state + dpd_get_forces gives for the same state at step 0.
 *
 * Allocates nothing: the scratch (about 3.5 MB) is one static device array
 * of the library, held by every GPU that loads it until the process exits.
 * Limits: n <= DPD_NOALLOC_MAX_PARTICLES and at most DPD_NOALLOC_MAX_CELLS
 * cells (floor(L_d / rc) multiplied over the three axes); larger inputs
 * return DPD_ERR_ARG.  The first call on each device looks the scratch up
 * (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Work is enqueued on `stream` (NULL = legacy default) and the
 * call returns without synchronising.  All calls share the one scratch
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Because the call
 * does not wait for its work, a non-finite input position or velocity is
 * not reported by the normal build (the forces come back non-finite or
 * wrapped to 0); the checked build reads the device error word back and
 * reports failed index checks.  The scratch address of each device is
 * kept for the life of the process, so the call is not supported after
 * cudaDeviceReset on that device. */
#define DPD_NOALLOC_MAX_PARTICLES 32768
#define DPD_NOALLOC_MAX_CELLS 32767
DPD_API int dpd_forces_noalloc(int64_t n, const float *pos, const float *vel, const double box[3],
                               double a, double gamma, double kT, double rc, double dt,
                               uint64_t seed, uint64_t step, float *force, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DPD_H */
