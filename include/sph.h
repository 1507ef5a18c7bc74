/*
 * sph.h -- C ABI of libsph.so, the GB300 (sm_103a) weakly compressible SPH
 * hot path: cell list, pair interaction, CFL time step and symplectic (or the
 * paper's Verlet) update of a set of particles (Valdez-Balderas, Dominguez, Rogers, Crespo,
 * "Towards accelerating SPH simulations for free-surface flows on multi-GPU
 * clusters", single-GPU pipeline of Sec. 3).
 *
 * Conventions for every entry point
 *   - Return value: SPH_OK (0) or a negative SPH_ERR_* code.  The context's
 *     sph_last_error() then holds a one-line message.  A failed call leaves
 *     the context usable unless the code is SPH_ERR_CUDA.
 *   - Device memory: the caller allocates ONE device workspace of the size
 *     sph_query_sizes() reports and passes it to sph_init().  The library
 *     carves all its device buffers from it and never allocates or frees
 *     device memory.  The workspace must stay allocated until sph_destroy().
 *   - Host memory: arrays passed to sph_upload/sph_download/sph_read_array
 *     are owned by the caller and only touched during the call.
 *   - Streams: all work runs on the stream given to sph_init (a cudaStream_t
 *     passed as void*).  Calls marked "async" only enqueue work; calls marked
 *     "sync" wait for the stream.  On the legacy default stream (NULL) the
 *     step is launched kernel by kernel; on any other stream it is captured
 *     once into a CUDA graph and replayed.
 *   - Particle order: the library keeps particles sorted by (cell label,
 *     id).  Downloads return that order; ids identify particles.
 *   - Device-side faults of the data (non-finite rates, a bounded spin that
 *     gave up, a capacity overflow) never trap: they set bits of a device
 *     status word that sph_diagnostics() returns and sph_check() turns into
 *     an error code.
 *   - Sizes: n_particles < 2^26 (67,108,864); the cell grid must have fewer
 *     than 2^31 cells.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_OK                 0
#define SPH_ERR_INVALID_ARG   -1   /* bad pointer, size or parameter        */
#define SPH_ERR_CUDA          -2   /* a CUDA runtime call failed            */
#define SPH_ERR_WORKSPACE     -3   /* workspace too small or misaligned     */
#define SPH_ERR_TIMEOUT       -4   /* a bounded device spin gave up         */
#define SPH_ERR_NONFINITE     -5   /* NaN/Inf in the interaction results    */
#define SPH_ERR_CAPACITY      -6   /* a cell held more particles than the
                                      id tie-break handles (the order within
                                      it is then not the (label, id) order) */
#define SPH_ERR_STATE         -7   /* call out of order (e.g. no state yet) */
#define SPH_ERR_TOO_LARGE     -8   /* n above the fixed maximum of a call    */
#define SPH_ERR_BOUNDS        -9   /* checked build: a kernel index was out of
                                      range (the access was skipped)          */

/* Bits of the device status word. */
#define SPH_STATUS_TIMEOUT    1u
#define SPH_STATUS_NONFINITE  2u
#define SPH_STATUS_CAPACITY   4u
/* Set only by the checked build of the library (libsph_checked.so, compiled
 * with -DSPH_CHECKED), whose kernels test the indexes they compute and skip
 * an out-of-range access instead of making it. */
#define SPH_STATUS_BOUNDS     8u

/* Physical and numerical constants of one simulation (Sec. 2.2, 2.3, 3).
 *   dp        particle spacing [m]; mass is given separately
 *   h         smoothing length [m]; cells have size 2h (Sec. 3.1)
 *   rho0      reference density [kg/m^3] (1000 in the paper)
 *   gamma     Tait exponent; must be 7 (Sec. 2.2)
 *   c0        reference speed of sound [m/s]; B = c0^2 rho0 / gamma
 *   alpha     artificial-viscosity coefficient (Sec. 2.2)
 *   eta2_coef eta^2 = eta2_coef * h^2 (eta = 0.1 h in the paper -> 0.01)
 *   gravity   acceleration [m/s^2]
 *   cfl       CFL number of the variable time step (Sec. 3.3)
 *   mass      mass of every particle [kg]
 *   dmin,dmax cell-grid domain; ncx = ceil((dmax-dmin)/(2h)) per axis.
 *             Particles outside it are excluded from the interactions and
 *             frozen (counted in sph_diag.n_out)
 *   n_bound   particles with id < n_bound are dynamic boundary particles
 *             (Sec. 2.3): density evolves, position and velocity never do
 *   scheme    SPH_SCHEME_* bits; 0 = Wendland C2 kernel and the symplectic
 *             predictor-corrector
 *   dt_fixed  > 0: use this step size; otherwise the CFL step
 *   verlet_every  with SPH_SCHEME_VERLET: an Euler step every this many
 *             steps (0 = 40); see sph_verlet */
typedef struct sph_params {
    double dp, h, rho0, gamma, c0, alpha, eta2_coef;
    double gravity[3];
    double cfl, mass;
    double dmin[3], dmax[3];
    uint32_t n_bound;
    uint32_t scheme;
    double dt_fixed;
    uint32_t verlet_every;
    uint32_t reserved;     /* must be 0 */
} sph_params;

/* sph_params.scheme bits: the paper's own formulation.
 *   SPH_SCHEME_CUBIC   the cubic spline kernel of Sec. 2.2 (the kernel of
 *                      the paper's results) instead of Wendland C2:
 *                      W = aD (1 - 3/2 q^2 + 3/4 q^3) for q < 1,
 *                      aD/4 (2 - q)^3 for 1 <= q < 2, aD = 1/(pi h^3)
 *   SPH_SCHEME_VERLET  the second-order Verlet integrator of Sec. 3.3 (one
 *                      force evaluation per step) instead of the symplectic
 *                      predictor-corrector; see sph_verlet */
#define SPH_SCHEME_CUBIC   1u
#define SPH_SCHEME_VERLET  2u

typedef struct sph_sizes {
    uint64_t workspace_bytes;   /* device bytes sph_init needs            */
    uint64_t ncells;            /* ncx * ncy * ncz                        */
    uint32_t ncx, ncy, ncz;
    uint32_t sort_passes;       /* passes of the cell sort: 1 (a counting
                                   sort whose one digit is the whole label) */
} sph_sizes;

typedef struct sph_diag {
    double t;                   /* simulated time [s] (member 0)          */
    double dt;                  /* current step size (member 0)           */
    double mass;                /* total mass of in-domain particles      */
    double momentum[3];         /* fluid momentum                         */
    double kinetic;             /* fluid kinetic energy                   */
    double potential;           /* fluid potential energy -m g.r          */
    double internal;            /* sum m e(rho), e' = p/rho^2 (Tait)      */
    uint64_t step;              /* steps taken (member 0)                 */
    uint64_t pairs_total;       /* neighbour pairs evaluated, all calls   */
    uint64_t candidates_total;  /* 27-cell candidates tested, all calls   */
    uint64_t pairs_last;        /* pairs of the last interaction          */
    uint64_t candidates_last;
    uint64_t pairs_fluid_last;      /* of which with a fluid particle i     */
    uint64_t pairs_boundary_last;   /* of which with a boundary particle i  */
    uint64_t pairs_fluid_total;
    uint64_t pairs_boundary_total;
    uint32_t n_out;             /* excluded particles                     */
    uint32_t status;            /* SPH_STATUS_* bits                      */
    float amax, cmax, mumax;    /* CFL terms of the last step-setting
                                   evaluation (member 0)                */
} sph_diag;

typedef struct sph_ctx sph_ctx;

/* One member of an ensemble of independent simulations run in lockstep
 * (the batched configuration: many uneven dam breaks in one launch).  The
 * members share sph_params' dp, h, rho0, gamma, alpha, eta2_coef, gravity,
 * cfl, mass and dt_fixed; each has its own domain, c0 and end time.
 * Particle ids: member q owns the n_particles consecutive ids that follow
 * member q-1's, its first n_bound ids being boundary particles. */
typedef struct sph_instance {
    double dmin[3], dmax[3];    /* this member's cell-grid domain        */
    double c0;                  /* this member's reference sound speed   */
    double t_end;               /* the member stops once t >= t_end
                                   (its step size becomes 0)            */
    uint32_t n_particles;
    uint32_t n_bound;
} sph_instance;

/* Bytes of device workspace for n particles under params (no side
 * effects, no CUDA calls). */
int sph_query_sizes(const sph_params *params, uint32_t n_particles,
                    sph_sizes *out);

/* Create a context over a caller-owned device workspace.  d_workspace must
 * be 256-byte aligned and at least sizes.workspace_bytes long.  stream is a
 * cudaStream_t (NULL = legacy default stream).  Sync (zeroes a few
 * counters).  *out is owned by the caller and freed with sph_destroy. */
int sph_init(const sph_params *params, uint32_t n_particles,
             void *d_workspace, uint64_t workspace_bytes, void *stream,
             sph_ctx **out);

/* Ensemble versions of sph_query_sizes / sph_init: n_inst members, whose
 * particle counts add up to the context's n.  params supplies the shared
 * constants (its dmin, dmax, c0 and n_bound are ignored).  Per-member step
 * sizes, times and end flags live on the device; every other call works on
 * the whole ensemble at once (one sort, one interaction launch, one
 * integrator launch per stage).  sph_init is the ensemble of one with
 * t_end = infinity. */
int sph_query_sizes_batch(const sph_params *params, const sph_instance *inst,
                          uint32_t n_inst, sph_sizes *out);
int sph_init_batch(const sph_params *params, const sph_instance *inst,
                   uint32_t n_inst, void *d_workspace,
                   uint64_t workspace_bytes, void *stream, sph_ctx **out);

/* Per-member simulated time, current step size, end flag and step count,
 * copied into caller-owned host arrays of n_inst entries (any pointer may
 * be NULL).  Sync. */
int sph_instance_state(sph_ctx *ctx, double *t, double *dt, uint32_t *done,
                       uint64_t *steps);

/* Restore each member's simulated time and step count (host arrays of
 * n_inst entries; steps may be NULL to keep the counts), e.g. after
 * sph_upload of a checkpointed state (the saved state of Sec. 3, copied to
 * the host when saving, is what a run resumes from).  Times must be finite
 * and non-negative (SPH_ERR_INVALID_ARG otherwise).  A member whose t reaches its t_end is
 * marked done again, one below it runs again.  With the symplectic
 * scheme the next step size comes from the state alone, so a run resumed
 * from (state, t, steps) repeats the uninterrupted run bit for bit; the
 * Verlet scheme restarts with an Euler step (its earlier state is not part
 * of a checkpoint).  Sync. */
int sph_set_instance_state(sph_ctx *ctx, const double *t, const uint64_t *steps);

/* Copy a particle state from host or device memory (any order; the arrays
 * may live on either side, unified addressing decides): pos[3n] float64
 * (x,y,z interleaved), vel[3n] float32, rho[n] float32, ids[n] uint32 (a
 * permutation of 0..n-1 is not required, but ids must be distinct).  Sync.
 * The state needs sph_build_cells before sph_interact. */
int sph_upload(sph_ctx *ctx, const double *pos, const float *vel,
               const float *rho, const uint32_t *ids);

/* Sec. 3.1: cell label of every particle (FP64, x fastest), sort by
 * (label, id), first index per cell, and reorder of all state arrays.  The
 * sort is a radix sort with a single digit, the whole label (a counting
 * sort: the per-cell counts are its histogram, the first indices its scan,
 * one scatter places every particle in its cell); the reorder then ranks the
 * particles of each cell by id, the tie-break of the Sec. 4.3 example.
 * Async. */
int sph_build_cells(sph_ctx *ctx);

/* Sec. 3.2: pair sums of Eq. 7 (density rate, every in-domain particle)
 * and Eq. 9 (acceleration, gravity included, fluid particles; boundary
 * particles get gravity only since Sec. 2.3 never moves them), in FP32 on
 * cell-relative coordinates, plus the CFL reductions of Sec. 3.3 (sets the device-side
 * step size unless params.dt_fixed > 0, or a predictor step is pending:
 * the half-step evaluation keeps the step size of the step's first
 * evaluation).  Requires built cells.  Async.
 * flags: SPH_INTERACT_COUNTS also stores each particle's neighbour count
 * (readable as SPH_ARRAY_NNB). */
#define SPH_INTERACT_COUNTS 1u
int sph_interact(sph_ctx *ctx, uint32_t flags);

/* Predictor half step of the symplectic scheme from the current rates:
 * fluid r += dt/2 v, v += dt/2 a; every in-domain particle rho += dt/2
 * drho/dt (Sec. 2.3: boundary particles keep r and v).  Keeps the start
 * state for sph_correct and recomputes the cell labels.  Async. */
int sph_predict(sph_ctx *ctx);

/* Corrector of the symplectic scheme, from the start state kept by
 * sph_predict and the rates of the last sph_interact: fluid
 * v = v0 + dt a, r = r0 + dt/2 (v + v0); rho = rho0 (2 - e)/(2 + e) with
 * e = -dt (drho/dt) / rho_half.  Advances t and the step count.  Async. */
int sph_correct(sph_ctx *ctx);

/* Verlet step of Sec. 3.3 (contexts with SPH_SCHEME_VERLET; SPH_ERR_STATE
 * otherwise), from the rates of the last sph_interact and the state one step
 * earlier, in the SPHysics form the paper cites:
 *   fluid:          r1 = r + dt v + dt^2/2 a
 *                   v1 = v_prev + 2 dt a     (leapfrog step)
 *                   v1 = v + dt a            (Euler step)
 *   every in-domain particle: rho1 = rho_prev + 2 dt drho/dt (leapfrog),
 *                   rho + dt drho/dt (Euler)
 * Each member counts its steps from its last sph_upload (or sph_init, or
 * surrogate advance); step k is an Euler step when k is a multiple of
 * params.verlet_every, so the first step after new state arrives, which has
 * no earlier state, is one.  Boundary
 * particles keep r and v (Sec. 2.3).  Advances t and the step count and
 * recomputes the cell labels.  Async.  sph_predict / sph_correct return
 * SPH_ERR_STATE on these contexts. */
int sph_verlet(sph_ctx *ctx);

/* nsteps full steps.  Symplectic: interact, CFL step, predict, rebuild,
 * interact, correct, rebuild (two force evaluations per step).  Verlet:
 * interact, CFL step, sph_verlet, rebuild (one).  Builds the cells first if
 * needed.  Async. */
int sph_step(sph_ctx *ctx, uint32_t nsteps);

/* Run nsteps steps; after every save_every steps (and at the end) wait for
 * the stream, read the device status word and call cb(user, step, t), from
 * which the caller may call sph_download or sph_diagnostics (the paper's
 * "copy to the host only when saving", Sec. 3).  cb may be NULL.  A non-zero
 * return from cb stops the rollout early (still SPH_OK).  A status bit set
 * during a chunk (non-finite rates, a bounded wait that gave up, a capacity
 * overflow) ends the rollout at that save boundary, before cb, with the
 * code sph_check returns; the state is that of the end of the chunk.
 * Sync. */
typedef int (*sph_snapshot_fn)(void *user, uint64_t step, double t);
int sph_rollout(sph_ctx *ctx, uint32_t nsteps, uint32_t save_every,
                sph_snapshot_fn cb, void *user);

/* Copy the current state (sorted order) to host or device arrays laid out
 * as in sph_upload.  Any pointer may be NULL to skip it.  Sync. */
int sph_download(sph_ctx *ctx, double *pos, float *vel, float *rho,
                 uint32_t *ids);

/* As sph_download, with each array indexed by particle id instead of the
 * sorted order (row id holds particle id).  Needs every uploaded id below
 * n (SPH_ERR_STATE otherwise).  Sync. */
int sph_download_by_id(sph_ctx *ctx, double *pos, float *vel, float *rho);

/* Pipelined transfers.  Sec. 3 keeps the whole simulation on the GPU and
 * copies to the host only when saving; these calls let those copies (and
 * the uploads of new states) run on copy engines while the GPU keeps
 * stepping, instead of stalling the caller and the stream.
 *
 * sph_async_transfer_bytes: bytes of the device buffer the calls need: three
 * staging slots of 44 B per particle (two for uploads, one for downloads),
 * each rounded to 256 bytes.
 * sph_enable_async_transfers: attach that caller-owned buffer (device,
 * 256-byte aligned, at least the bytes above; SPH_ERR_WORKSPACE otherwise)
 * and create the context's two copy streams (one per direction) and their
 * events; they are destroyed by sph_destroy.  The library allocates no
 * device memory for them.  Calling it again with another buffer first waits
 * for every transfer.  Sync. */
uint64_t sph_async_transfer_bytes(const sph_ctx *ctx);
int sph_enable_async_transfers(sph_ctx *ctx, void *d_buf, uint64_t bytes);

/* As sph_upload, but only enqueued: the copies of the arrays into an upload
 * slot run on the host-to-device copy stream (after that slot's previous
 * upload was unpacked), and the unpack that replaces the state is ordered on
 * the context's stream after them, so the copies overlap whatever the stream
 * is still running.  The arrays must stay unchanged until
 * sph_sync_transfers.  The id check of sph_upload (every id below n, needed
 * by sph_download_by_id) is read at the next sph_sync_transfers.
 * SPH_ERR_STATE if sph_enable_async_transfers was not called.  Async. */
int sph_upload_async(sph_ctx *ctx, const double *pos, const float *vel,
                     const float *rho, const uint32_t *ids);

/* As sph_download, but only enqueued: the state is packed into the download
 * slot on the context's stream (after the previous download's copies left
 * the slot), and the copies to the arrays run on the device-to-host copy
 * stream, overlapping the work enqueued after this call.  The arrays hold
 * the state of this point of the stream after sph_sync_transfers.  Any
 * pointer may be NULL.  SPH_ERR_STATE without a state or without
 * sph_enable_async_transfers.  Async. */
int sph_download_async(sph_ctx *ctx, double *pos, float *vel, float *rho,
                       uint32_t *ids);

/* Wait for both copy streams and the context's stream, then read the id
 * check of the last pipelined upload.  Sync. */
int sph_sync_transfers(sph_ctx *ctx);

/* Copy an internal device array to host memory for inspection.  bytes must
 * equal the array's size (see sph_array_bytes).  Sync.
 *   SPH_ARRAY_KEY      uint32[n]  cell label of each particle, sorted order
 *   SPH_ARRAY_CELL_OFF uint32[ncells+2] first index of each cell (the last
 *                      two entries: in-domain count, n)
 *   SPH_ARRAY_ACE      float32[4n] (ax, ay, az, drho/dt) per particle
 *   SPH_ARRAY_NNB      uint32[n]  neighbour counts (SPH_INTERACT_COUNTS)
 *   SPH_ARRAY_NNB64    uint32[n]  neighbour counts with the FP64 predicate
 *                      (sph_neighbour_counts_fp64)
 *   SPH_ARRAY_POSC     float32[4n] cell-relative position and p/rho^2
 *   SPH_ARRAY_DT       float64[n_inst] current step size of each member
 *   SPH_ARRAY_PREV     float32[4n] (vx, vy, vz, rho) one step earlier, in the
 *                      order of the state (Verlet contexts after a step)
 *   SPH_ARRAY_UNITS    uint32[1 + 2 cap]: the number of interaction work units
 *                      m, then m (first sorted index, end) pairs, each a run
 *                      of particles of one row of cells (Sec. 3.2; cut for
 *                      the interaction variant in use); the words past 1 + 2m
 *                      are unspecified.  cap bounds m for the context.  Needs
 *                      built cells (SPH_ERR_STATE otherwise).  The list is
 *                      built in one launch when the grid has at most 8,192
 *                      rows of at most 1,023 cells, unless the environment
 *                      sets SPH_UNITS_FUSED=0 when the context is created;
 *                      the list is the same either way. */
#define SPH_ARRAY_KEY      0
#define SPH_ARRAY_CELL_OFF 1
#define SPH_ARRAY_ACE      2
#define SPH_ARRAY_NNB      3
#define SPH_ARRAY_NNB64    4
#define SPH_ARRAY_POSC     5
#define SPH_ARRAY_DT       6
#define SPH_ARRAY_PREV     7
#define SPH_ARRAY_UNITS    8
uint64_t sph_array_bytes(const sph_ctx *ctx, int which);
int sph_read_array(sph_ctx *ctx, int which, void *host, uint64_t bytes);

/* Sec. 4.2-4.3: the data a sub-domain of a one-dimensional decomposition
 * along x sends to its neighbours, selected on the GPU as the paper does it:
 * label every particle, order by (label, id) with the radix sort, copy the
 * labelled ones out.  The sub-domain is [xlo, xhi) and holds the context's
 * particles.  Labels (FP64 x, xlo + 2h and xhi - 2h each rounded once):
 *   SPH_SUBDOMAIN_EDGE     1 if xlo <= x < xlo + 2h (left edge), 2 if
 *                          xhi - 2h <= x < xhi (right edge), else 0: the
 *                          edge particles that build the neighbours' halos.
 *                          Needs xhi - xlo >= 4h (no particle in both edges)
 *   SPH_SUBDOMAIN_MIGRATE  1 if x < xlo (moved to the left neighbour), 2 if
 *                          x >= xhi (moved to the right one), else 0
 * Particles outside the cell-grid domain are not labelled.  counts[3]
 * receives the number of in-domain particles with label 0, 1 and 2.  The
 * m = counts[1] + counts[2] labelled particles are copied, label 1 first,
 * each label in ascending id (the order of the worked example of Sec. 4.3),
 * into pos[3m] (float64 x,y,z), vel[3m] (float32), rho[m], ids[m]: host or
 * device arrays owned by the caller, any of them NULL to skip it.
 * capacity < m returns SPH_ERR_CAPACITY with counts filled and nothing
 * copied.  The state itself is not reordered (the cell order stays).
 * Needs built cells and a single simulation (SPH_ERR_STATE otherwise).
 * Sync; a radix-sort look-back that gave up shows in sph_check. */
#define SPH_SUBDOMAIN_EDGE     0
#define SPH_SUBDOMAIN_MIGRATE  1
int sph_subdomain_select(sph_ctx *ctx, int mode, double xlo, double xhi,
                         uint32_t *counts, uint32_t capacity, double *pos,
                         float *vel, float *rho, uint32_t *ids);

/* Sec. 3.2 neighbour counts with the FP64 predicate |r_ij|^2 < (2h)^2,
 * |r|^2 = (dx*dx + dy*dy) + dz*dz without contraction, on the current
 * cells (for bit-exact comparison; not used by the time step).  Async. */
int sph_neighbour_counts_fp64(sph_ctx *ctx);

/* FP64 conservation sums, counters and status.  Sync. */
int sph_diagnostics(sph_ctx *ctx, sph_diag *out);

/* Free-surface front of the dam-break flow (the test case of Sec. 6, Fig. 1;
 * the paper plots it but does not define it): for each member, the largest
 * FP64 x of the in-domain fluid particles with z_lo <= z < z_hi -- for a
 * surge along +x over a floor at z_f, the band z_f <= z < z_f + 2 dp.
 * front[n_inst] is a caller-owned host array; a member with no particle in
 * the band gets -INFINITY.  Needs z_lo < z_hi (SPH_ERR_INVALID_ARG) and
 * built cells (SPH_ERR_STATE).  A maximum does not depend on the order of
 * the particles, so the value is exact (bit-identical to the same maximum
 * taken on the host).  Sync. */
int sph_front(sph_ctx *ctx, double z_lo, double z_hi, double *front);

/* Map the device status word to an error code (SPH_OK if clear).  Sync.
 * The word keeps its bits until sph_clear_status. */
int sph_check(sph_ctx *ctx);

/* Clear the device status word once the caller has handled what sph_check
 * reported.  Sync. */
int sph_clear_status(sph_ctx *ctx);

/* Self-test of the failure path; the paper has no counterpart.  Bounded
 * device waits must be testable without hanging a GPU: this runs the radix
 * sort's decoupled look-back (the same device code as the sort) against a
 * predecessor tile whose status nothing ever publishes, with a limit of
 * `polls` polls (1 to 2^20).  The wait gives up and sets SPH_STATUS_TIMEOUT
 * in the context's status word, as a stalled sort would, so sph_check
 * returns SPH_ERR_TIMEOUT.  The particle state and cells are untouched (the
 * look-back runs on status words reserved for this test).  Sync. */
int sph_selftest_timeout(sph_ctx *ctx, uint32_t polls);

/* The same for the one-launch unit list's row look-back (see
 * SPH_ARRAY_UNITS): one warp waits, with a limit of `polls` polls (1 to
 * 2^20), on the word of a preceding row that nothing publishes, gives up and
 * sets SPH_STATUS_TIMEOUT, so sph_check returns SPH_ERR_TIMEOUT.  The state,
 * cells and unit list are untouched.  Sync. */
int sph_units_selftest_timeout(sph_ctx *ctx, uint32_t polls);

/* Block shapes of the interaction kernel ("variants": particles per work
 * unit, staged candidates per unit, neighbour-list slots per lane) and the
 * autotuner that picks one.  Results do not depend on the variant beyond
 * FP32 summation order within a particle's own sum, which is the same for
 * every variant (each particle sums its neighbours in the sorted order).
 * sph_autotune times `reps` interaction launches of every variant on the
 * current cells (CUDA events on the context's stream), selects the fastest
 * and writes the per-variant milliseconds to ms_per_variant (NULL allowed,
 * else sph_num_variants() floats).  It leaves the state and step size
 * untouched.  Sync. */
uint32_t sph_num_variants(void);
int sph_set_variant(sph_ctx *ctx, uint32_t variant);
int sph_autotune(sph_ctx *ctx, uint32_t reps, float *ms_per_variant,
                 uint32_t *best);

/* Number of kernels one sph_step(ctx, 1) launches. */
uint32_t sph_kernels_per_step(const sph_ctx *ctx);

/* 1 when the step's kernels are launched with programmatic dependent launch
 * (each may be scheduled while its predecessor drains and waits for it on
 * the device before touching memory; results are the same either way), 0
 * when not.  Decided once per process by the first sph_init or
 * sph_init_batch: off when the environment sets SPH_PDL=0, or when the
 * driver refuses such launches inside a captured conditional node (checked
 * with a graph whose loop body never runs).  0 before the first context. */
int sph_pdl_enabled(void);

/* FP32 issue-rate probe (a measurement helper; the paper has no
 * counterpart): launches `blocks` blocks of 256 threads on stream, each
 * thread running `iters` iterations of 128 independent fused multiply-adds
 * (256 flop), and writes one float per thread to d_out (a caller-owned
 * device array of blocks * 256 floats).  Timing it with events gives the
 * measured FP32 peak used as the interaction's roofline denominator.
 * Async. */
int sph_fma_probe(float *d_out, uint32_t blocks, uint32_t iters, void *stream);

const char *sph_last_error(const sph_ctx *ctx);

/* Wait for the context's stream and its copy streams, then free the context
 * (its graphs, streams and events).  The workspace and the transfer buffer
 * may be freed once this returns.  Sync. */
void sph_destroy(sph_ctx *ctx);

/* Sec. 3.1 / Sec. 4.3: stable LSD radix sort of (key, value) pairs by the
 * low key_bits bits of the key (8 bits per pass, onesweep with decoupled
 * look-back).  Equal keys keep their input order, so sorting labels whose
 * values are ids in ascending order reproduces the (label, id) order of the
 * paper's example.  d_vals_in may be NULL: values are then the input
 * indices 0..n-1.  All arrays are device arrays of n uint32; outputs must
 * not alias inputs.  d_scratch must hold sph_radix_sort_scratch_bytes(n)
 * bytes (256-byte aligned).  Async on stream. */
uint64_t sph_radix_sort_scratch_bytes(uint32_t n);
int sph_radix_sort_pairs(const uint32_t *d_keys_in, const uint32_t *d_vals_in,
                         uint32_t *d_keys_out, uint32_t *d_vals_out,
                         uint32_t n, uint32_t key_bits, void *d_scratch,
                         uint64_t scratch_bytes, void *stream);

/* Outcome of the last sph_radix_sort_pairs call of n pairs on d_scratch:
 * waits for stream, then SPH_OK, or SPH_ERR_TIMEOUT if a decoupled look-back
 * wait gave up (its bounded spin ran out; the order is then not valid).
 * Each sort clears the flag before it starts.  Arguments as for the sort
 * (n >= 1).  Sync. */
int sph_radix_sort_status(const void *d_scratch, uint64_t scratch_bytes,
                          uint32_t n, void *stream);

/* Self-test of that failure path; the paper has no counterpart.  Runs the
 * sort's look-back on d_scratch (laid out for n pairs) against a
 * predecessor tile whose status nothing publishes, with a limit of `polls`
 * polls (1 to 2^20), so the wait gives up and the next
 * sph_radix_sort_status reports SPH_ERR_TIMEOUT.  Sync. */
int sph_radix_sort_selftest_timeout(void *d_scratch, uint64_t scratch_bytes,
                                    uint32_t n, uint32_t polls, void *stream);

/* The same stable radix sort without caller scratch.  The paper has no
 * counterpart: this is for callers that cannot give the library device
 * memory -- C code with no device allocator of its own, a process whose
 * device memory belongs to another allocator's pool, or a latency-critical
 * loop that must not call cudaMalloc/cudaFree (they can synchronise the
 * device).  The scratch lives in a fixed array inside libsph.so, about
 * 9.4 MB per device: it is reserved on every device whose context loads the
 * library's module, whether or not this entry point is ever called, and
 * held until the process exits; nothing is allocated per call.  Limits and
 * behaviour:
 *   - n <= SPH_RADIX_SORT_STATIC_MAX_N, else SPH_ERR_TOO_LARGE (no work done)
 *   - arrays as for sph_radix_sort_pairs (device, n uint32 each, outputs not
 *     aliasing inputs, d_vals_in may be NULL for values 0..n-1)
 *   - the first call with a given device current looks up the array's
 *     device address (a CUDA runtime query): make that first call before
 *     any stream capture.  The address is kept for the life of the process:
 *     after cudaDeviceReset (or any teardown of the device's primary
 *     context) it is stale, so do not use this entry point after one
 *   - a look-back wait that gave up is reported by
 *     sph_radix_sort_static_status, not by the return value
 *   - all calls on one device share the array and it keeps the last call's
 *     contents (each call clears what must start at zero); calls that overlap
 *     on the GPU race, so serialise them (e.g. one stream)
 * Async on stream. */
#define SPH_RADIX_SORT_STATIC_MAX_N (1u << 20)
int sph_radix_sort_pairs_static(const uint32_t *d_keys_in,
                                const uint32_t *d_vals_in,
                                uint32_t *d_keys_out, uint32_t *d_vals_out,
                                uint32_t n, uint32_t key_bits, void *stream);

/* Outcome of the last sph_radix_sort_pairs_static call on the current
 * device: waits for stream, then SPH_OK or SPH_ERR_TIMEOUT (a look-back
 * wait gave up; the order is then not valid).  Reads the fixed array; the
 * same first-call and overlap rules apply.  Sync. */
int sph_radix_sort_static_status(void *stream);

/* Self-test of that failure path on the fixed array (the paper has no
 * counterpart), as sph_radix_sort_selftest_timeout: afterwards
 * sph_radix_sort_static_status reports SPH_ERR_TIMEOUT until the next
 * sort.  polls 1 to 2^20.  Sync. */
int sph_radix_sort_static_selftest_timeout(uint32_t polls, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
