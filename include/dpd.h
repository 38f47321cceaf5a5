/*
 * dpd.h -- C ABI of the GB300 DPD pair-interaction engine (libdpd.so).
 *
 * The engine advances a periodic system of dissipative-particle-dynamics
 * (DPD) particles on one GPU: cell binning and reordering, a cutoff
 * neighbour list, the fused conservative + dissipative + random pair force
 * with a pair-symmetric counter-based Gaussian, harmonic bonds, a body force
 * and the lambda form of velocity Verlet.  Method: Tang & Karniadakis,
 * "Accelerating Dissipative Particle Dynamics Simulations on GPUs"
 * (arXiv:1311.0402); each entry point cites the passage that defines what it
 * computes.
 *
 * Conventions for every entry point:
 *   - Host arrays are owned by the caller; the library copies what it needs
 *     before returning and keeps no pointer to them.
 *   - The library owns all device memory of a handle (allocated by
 *     dpd_create / dpd_set_state, freed by dpd_destroy).
 *   - Calls are synchronous: results are complete when the call returns.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Particle arrays passed in are in the caller's order ("particle index"
 *     0..n-1); every array passed out uses that same order, whatever
 *     reordering the engine does internally.
 *   - Vectors are n x 3 row-major doubles (x0 y0 z0 x1 y1 z1 ...).
 *   - Status codes: DPD_OK on success.  DPD_ERR_ARG for invalid arguments
 *     (the handle's state is left unchanged).  A CUDA failure latches
 *     DPD_ERR_CUDA on the handle.  dpd_last_error() describes the last
 *     failure.
 */
#ifndef DPD_H
#define DPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpd_sim dpd_sim; /* opaque handle */

typedef enum {
    DPD_OK = 0,
    DPD_ERR_ARG = 1,          /* invalid argument; nothing changed */
    DPD_ERR_OOM = 2,          /* device or host allocation failed (a call that fails
                                 this way while staging its input changes no state;
                                 for tests, the environment variable
                                 DPD_TEST_FAIL_ALLOC=1 makes every device allocation
                                 of a handle fail this way) */
    DPD_ERR_CUDA = 3,         /* a CUDA call failed (latched) */
    DPD_ERR_NBR_OVERFLOW = 4, /* a group of 32 particles had more pairs than its list holds */
    DPD_ERR_NONFINITE = 5,    /* a force or position became NaN / Inf */
    DPD_ERR_TIMEOUT = 6,      /* the GPU did not finish within the wait limit */
    DPD_ERR_STATE = 7         /* call order: e.g. dpd_step before dpd_set_state */
} dpd_status;

/* Run options.  Fill with dpd_default_options() and override fields. */
typedef struct {
    double skin;              /* neighbour-list skin added to r_c (default 0.3) */
    int32_t rebuild_every;    /* 0 (default): rebuild when a particle has moved more
                                 than skin/2 since the last build; k > 0: also
                                 rebuild at least every k steps */
    int32_t body_force_mode;  /* 0 none, 1 uniform g, 2 +g for y < L_y/2 and -g above
                                 (reverse Poiseuille, Sec. 4.2 of the paper) */
    uint64_t seed;            /* global seed of the random force (default 42) */
    double lambda;            /* velocity-Verlet prediction factor (default 0.5) */
    double body_force[3];     /* g (force per particle, unit mass) */
    int32_t nbr_capacity;     /* list capacity per particle: particles are listed in
                                 groups of 32 consecutive ones, each group holding
                                 up to 32 x nbr_capacity pair entries; 0 = from the
                                 density, grown when a build overflows */
    int32_t graph_steps;      /* steps per captured CUDA graph (default 8; 0 = no graphs) */
    int32_t deterministic;    /* 0 (default): each pair is evaluated once and its force is
                                 added to the second particle with float atomics, so force
                                 sums are not bitwise reproducible run to run; 1: every
                                 pair is evaluated by both particles and each force is
                                 summed in a fixed order (bit-identical runs, about 1.5x
                                 the pair work).  Random numbers and neighbour sets are
                                 deterministic in both modes. */
    int32_t conditional_rebuild; /* 1 (default): inside the CUDA graphs, each step's rebuild
                                 chain sits under a conditional node that the device sets
                                 from the rebuild flag, so steps without a rebuild launch
                                 none of its kernels; 0: the chain is launched every step
                                 and its kernels return at once unless flagged */
    int32_t list_builder;     /* 0 (default): list entries placed by warp-ballot prefix
                                 sums (deterministic order, Sec. 3.3); 1: by an atomic add
                                 per entry -- the paper's Table 2 comparison; the list order
                                 (and so force summation order) then varies run to run */
    int32_t no_reorder;       /* 0 (default): at every rebuild the particles are reordered
                                 into cell order (Sec. 3.2); 1: they stay in load order and
                                 the list is built through the sort permutation -- the
                                 paper's reorder on/off comparison (Sec. 3.2); slower */
    int32_t list_layout;      /* 0 (default): packed lists per group of 32 particles (see
                                 nbr_capacity), consumed 32 entries at a time; 1: the
                                 paper's layout (Sec. 3.3): one row of nbr_capacity entries
                                 per particle, written row-major by the builder with the
                                 pairs inside r_c at build time from the front of the row
                                 and the skin pairs from its back (double insertion), the
                                 two parts joined by a second kernel, each 32 x 32 tile of
                                 the table transposed in place by a third, and the pair
                                 force evaluated by one thread per particle walking its row
                                 (every pair by both particles, fixed order).  Layout 1
                                 needs at least 3 cells along every axis. */
    double wait_timeout_s;    /* host wait limit per call (default 600 s) */
    void *stream;             /* cudaStream_t to run on; NULL = a stream of the handle */
} dpd_options;

/* Observables of the current full-step state (Alg. 1 "calculate statistics"). */
typedef struct {
    uint64_t step;
    int64_t n;
    double kinetic;      /* sum m v^2 / 2 (m = 1) */
    double temperature;  /* sum m v^2 / (3N - 3) */
    double virial;       /* sum_{i<j} r_ij . (F^C_ij + F^bond_ij) at the current positions */
    double pressure;     /* (sum m v^2 + virial) / (3V) */
    double momentum[3];  /* sum m v */
} dpd_obs;

/* Default options (skin 0.3, displacement-triggered rebuild, seed 42,
 * lambda 0.5, no body force, automatic capacity, 8-step graphs). */
void dpd_default_options(dpd_options *opt);

/* Create a simulation handle.
 * Defines the pair force of Eqs. 2-9 (Sec. 2): for |r_ij| < rc,
 *   F_ij = [a_{t_i t_j} w - gamma w^{2s} (e_ij . v_ij) + sigma w^s xi_ij dt^{-1/2}] e_ij,
 *   w = 1 - |r_ij| / rc, sigma = sqrt(2 gamma kT) (Eq. 9), r_ij = r_i - r_j.
 * box:       three box lengths (periodic in all directions), each > 2 (rc + skin).
 * n_species: 1..8; a_ij: n_species x n_species row-major, symmetric.
 * gamma >= 0, kT >= 0, rc > 0, s > 0, dt > 0.  opt may be NULL (defaults).
 * Returns DPD_ERR_ARG (and *out = NULL) on invalid parameters. */
dpd_status dpd_create(dpd_sim **out, const double box[3], int32_t n_species, const double *a_ij,
                      double gamma, double kT, double rc, double s, double dt,
                      const dpd_options *opt);

/* Load particles (Alg. 1 "CPU -> GPU").  1 <= n <= 2^27 (a list entry packs
 * a particle index into 27 bits).  x, v: n x 3; positions are wrapped
 * into [0, L) and rounded to FP32 on the device.  species: n entries in
 * [0, n_species) or NULL (all 0).  tag: n distinct identity tags keying the
 * random force, or NULL (tag = particle index).  step: the step number of
 * this state (keys the random force).  Builds the cell and neighbour lists
 * and computes the force at this state.  Replaces any previous state and
 * drops previously set bonds.  The arrays are the caller's and are copied.
 * DPD_ERR_ARG for n outside that range, x or v NULL, a non-finite value, a
 * species out of range or repeated tags; DPD_ERR_OOM when device memory runs
 * out.  On any error the previous state (if any) is kept and stays usable. */
dpd_status dpd_set_state(dpd_sim *h, int64_t n, const double *x, const double *v,
                         const int32_t *species, const uint32_t *tag, uint64_t step);

/* Harmonic bonds F = -K (r - r0) e_ij between particle indices (Sec. 4.5).
 * pairs: nb x 2 particle indices (the order of dpd_set_state); each particle
 * may appear in at most 6 bonds.  Bonded pairs also feel the pair force.
 * Recomputes the force of the current state.  nb = 0 removes all bonds.
 * pairs is the caller's and is copied.  DPD_ERR_STATE without a state;
 * DPD_ERR_ARG for nb < 0, a NULL pairs with nb > 0, a non-finite k or r0, an
 * index out of range, a bond of a particle with itself or a seventh bond on a
 * particle. */
dpd_status dpd_set_bonds(dpd_sim *h, int64_t nb, const uint32_t *pairs, double k, double r0);

/* Rebuild the cell list, particle order and neighbour list now (Secs. 3.2-3.3).
 * The list holds every pair with d^2 < (rc + skin)^2 under the FP32
 * minimum-image predicate d = x_j - x_i (per axis: d -= L if d > L/2, d += L
 * if d < -L/2), d^2 = (dx dx + dy dy) + dz dz, each operation rounded.  With
 * automatic capacity the list grows when it overflows; with a fixed
 * nbr_capacity an overflow returns DPD_ERR_NBR_OVERFLOW.  DPD_ERR_STATE
 * without a state. */
dpd_status dpd_build_neighbors(dpd_sim *h);

/* The cutoff neighbour list of Sec. 3.3 (every pair with d^2 < r_list^2,
 * r_list = r_c + skin, by the predicate above, as of the last build): copy
 * its pairs as caller particle indices (i < j, each pair once whatever the
 * force mode), at most cap pairs into pairs_out (cap x 2 uint32, owned by the
 * caller), and the number of distinct pairs into *n_out (which may exceed
 * cap).  pairs_out may be NULL with cap = 0 to query the count.  Waits for
 * the queued work.  DPD_ERR_STATE without a loaded state; DPD_ERR_ARG for
 * cap < 0, pairs_out NULL with cap > 0, or n_out NULL. */
dpd_status dpd_get_neighbors(dpd_sim *h, int64_t cap, uint32_t *pairs_out, int64_t *n_out);

/* Total force f_i = sum_j F_ij (Eq. 2) + bonds + body force at the current
 * positions, velocities and step key, into f_out (n x 3, nullable).  Does
 * not change the state.  Uses the current neighbour list, which every call
 * leaves valid for the current positions (no particle has moved more than
 * skin/2 since it was built).  f_out is the caller's.  Waits.  DPD_ERR_STATE
 * without a state; DPD_ERR_NONFINITE if a force is not finite. */
dpd_status dpd_forces(dpd_sim *h, double *f_out);

/* The force the integrator holds for the next step (n x 3 doubles in the
 * caller's order, owned by the caller): the pair force of Eqs. 2-9 plus bonds
 * and the body force at the current positions, the f of Algorithm 1's next
 * half kick.  Waits.  DPD_ERR_STATE without a state; DPD_ERR_ARG for NULL. */
dpd_status dpd_get_force(dpd_sim *h, double *f_out);

/* Replace the force the integrator holds (n x 3, caller's order, rounded to
 * FP32).  With dpd_get_state and dpd_get_force it completes a checkpoint:
 * the force held between steps was evaluated with the predicted velocity
 * v~ of the lambda scheme (Sec. 3.1), which dpd_set_state cannot recompute
 * from (x, v) alone.  f is the caller's and is copied.  DPD_ERR_STATE without
 * a state; DPD_ERR_ARG for NULL or a non-finite value. */
dpd_status dpd_set_force(dpd_sim *h, const double *f);

/* Advance nsteps steps (Alg. 1 main loop, Sec. 3.1): for each step
 *   x += dt v + dt^2/2 f;  v~ = v + lambda dt f;  rebuild lists if needed;
 *   f' = F(x, v~, step + 1);  v += dt/2 (f + f');  step += 1.
 * Returns DPD_ERR_NBR_OVERFLOW or DPD_ERR_NONFINITE if detected (the state
 * is then unreliable; reload it with dpd_set_state). */
dpd_status dpd_step(dpd_sim *h, int64_t nsteps);

/* dpd_step split in two, for overlapping several handles (each on its own
 * stream) from one host thread: dpd_step_async queues nsteps on the handle's
 * stream and returns at once; dpd_sync waits for everything queued and
 * reports a device error of any queued run (overflow, non-finite force,
 * staging timeout), as dpd_step does; dpd_query sets *idle = 1 when the
 * handle's stream has finished all queued work (no wait).  Other calls that
 * read the state wait for queued steps first (stream order). */
dpd_status dpd_step_async(dpd_sim *h, int64_t nsteps);
dpd_status dpd_sync(dpd_sim *h);
dpd_status dpd_query(dpd_sim *h, int32_t *idle);

/* Choose the neighbour-list skin by measurement.  The skin trades list
 * length (candidates per particle grow as (rc + skin)^3, Sec. 3.3) against
 * rebuild frequency (a rebuild each time a particle has moved skin/2).  For
 * each of the ncand candidate skins the system given by the dpd_create
 * arguments (opt may be NULL; its skin is replaced) and the state (x, v:
 * n x 3, species: n or NULL) runs on a temporary handle: a warm-up of
 * steps/4 steps, then `steps` steps timed as by dpd_step_profiled.
 * *best_skin receives the fastest candidate and ms_per_step (ncand entries,
 * nullable) the time per step of each (infinity for a candidate that failed,
 * e.g. a box too small for it).  Returns DPD_ERR_ARG for missing arguments,
 * else DPD_OK if any candidate ran, else the last candidate's error.  Uses
 * the current device; allocates and frees its own device memory. */
dpd_status dpd_tune_skin(const double box[3], int32_t n_species, const double *a_ij, double gamma, double kT,
                         double rc, double s, double dt, const dpd_options *opt, int64_t n, const double *x,
                         const double *v, const int32_t *species, const double *candidates, int32_t ncand,
                         int32_t steps, double *best_skin, double *ms_per_step);

/* Failure-detection self-test: runs the device's bounded wait (the one the
 * neighbour builder uses for its TMA-staged halos) on a transaction that
 * nothing delivers.  The wait gives up after `polls` polls (1..2^20), sets
 * the timeout bit of the device error word, and the call returns
 * DPD_ERR_TIMEOUT -- the status a real stalled copy produces.  The bit is
 * cleared afterwards; the handle and its state stay usable.  Needs a loaded
 * state (DPD_ERR_STATE otherwise). */
dpd_status dpd_wait_selftest(dpd_sim *h, uint32_t polls);

/* Per-phase device times of a run, measured with CUDA events recorded on
 * the handle's stream around every kernel group of every step. */
typedef struct {
    double total_ms;        /* first to last event */
    double integrate_ms;    /* the opening velocity-Verlet phase 1 of the call */
    double rebuild_ms;      /* binning / scan / reorder / neighbour-list chain */
    double force_ms;        /* the force phase: pair force, bonds, body force
                               and the integration into the next step (in
                               Newton-3 mode the pair kernel, then the settle
                               kernel that completes the sums and integrates) */
    double pair_ms;         /* the pair kernel alone (part of force_ms) */
    int64_t steps;
    int64_t force_launches;
    int64_t kernel_launches;
    int64_t rebuilds;       /* rebuilds that ran during the call */
} dpd_step_times;

/* dpd_step with CUDA events around each kernel group of each step (the
 * kernels and their order are those of dpd_step; the run is captured as a
 * single CUDA graph of nsteps steps when graph_steps > 0).  times may be
 * NULL. */
dpd_status dpd_step_profiled(dpd_sim *h, int64_t nsteps, dpd_step_times *times);

/* Observables of the current full-step state (Algorithm 1's "calculate
 * statistics"): T = sum m v^2 / (3N - 3), p = (sum m v^2 + virial) / (3V)
 * with the virial of the conservative force (Eq. 3) and the bonds, kinetic
 * energy and momentum, reduced on the device in a fixed order and summed in
 * FP64.  *out is the caller's.  Waits for the queued work.  DPD_ERR_STATE
 * without a state; DPD_ERR_ARG for NULL. */
dpd_status dpd_observables(dpd_sim *h, dpd_obs *out);

/* The same observables, delivered asynchronously: the reduction is queued on
 * the handle's stream behind the work already queued (e.g. dpd_step_async),
 * so it describes the state that work reaches, and the finished dpd_obs is
 * copied into *out.  out must be page-locked host memory (cudaHostAlloc,
 * cudaHostRegister or a pinned tensor) owned by the caller; its contents are
 * valid after the next dpd_sync (or any call that waits on the handle), and
 * bit-identical to what dpd_observables returns for the same state.  Returns
 * DPD_ERR_ARG if out is NULL or not page-locked; errors of the queued work
 * are reported by dpd_sync, and the values written then are not meaningful.
 * Lets a run read its statistics every step (Alg. 1 "calculate
 * statistics") without a host wait per step. */
dpd_status dpd_observables_async(dpd_sim *h, dpd_obs *out);

/* Binned velocity profile, as the flow validations of Sec. 4.2 measure it:
 * v[vel_axis] along bin_axis in nbins equal bins over the box,
 * sum_out[b] += sum of v, count_out[b] += number of particles.  Both arrays
 * (nbins doubles each, the caller's) are accumulated into, not cleared.
 * Waits.  DPD_ERR_ARG for an axis outside 0..2, nbins outside 1..100000 or a
 * NULL array; DPD_ERR_STATE without a state. */
dpd_status dpd_profile(dpd_sim *h, int32_t bin_axis, int32_t vel_axis, int32_t nbins,
                       double *sum_out, double *count_out);

/* The integrator's state at the current full step (Sec. 3.1, Algorithm 1) in
 * the caller's particle order: x, v (n x 3 doubles, owned by the caller, each
 * nullable) as stored on the device (FP32 values, x wrapped into [0, L)), and
 * the step (nullable).  Waits for the queued work.  DPD_ERR_STATE without a
 * state. */
dpd_status dpd_get_state(dpd_sim *h, double *x, double *v, uint64_t *step);

/* Number of particles, of neighbour-list rebuilds so far (the rebuild branch
 * of Algorithm 1) and the list capacity per particle; each output nullable.
 * Waits for the queued work; without a state n, rebuilds and the capacity
 * read 0. */
dpd_status dpd_info(dpd_sim *h, int64_t *n, int64_t *rebuilds, int32_t *nbr_capacity);

/* Issue-rate probe for the denominator of the ALU roofline the pair kernel
 * is measured against (152 SMs x 128 FP32/INT32 lanes x clock): kind 0 times
 * chains of FP32 fused multiply-adds (one lane-op each), kind 1 chains of
 * 32-bit integer xor-then-add (two lane-ops per link); every thread carries
 * eight independent chains, eight blocks of 256 threads per SM.  One warm-up
 * launch, then `reps` (1..1000) timed launches with CUDA events on a
 * temporary stream of the current device.  *lane_ops_per_s receives the
 * measured lane-operations per second, *ms_per_launch the mean launch time
 * (either may not be NULL).  DPD_ERR_ARG for another kind or reps out of
 * range, DPD_ERR_CUDA for a failed launch. */
dpd_status dpd_alu_peak(int32_t kind, int32_t reps, double *lane_ops_per_s, double *ms_per_launch);

/* The pair random numbers, computed by the device kernels (Sec. 3.5):
 * for each k, sig = TEA-16 signature of (bitrev(tag), step) under the key
 * of seed, (A, B) = TEA-4 of (min(sig_i, sig_j), max(sig_i, sig_j)),
 * out_hash[2k] = A, out_hash[2k+1] = B, out_xi[k] = the FP32 Gaussian
 * sign(B) sqrt(-2 ln u1) cos(pi u2).  Host arrays of m (tags) and 2m / m
 * entries; out_xi may be NULL.  Uses the current device; creates a
 * temporary stream. */
dpd_status dpd_pair_rng(uint64_t seed, uint64_t step, int64_t m, const uint32_t *tag_i,
                        const uint32_t *tag_j, uint32_t *out_hash, float *out_xi);

/* ---------------------------------------------------------------------------
 * Allocation-free pair force (this entry point has no counterpart in the
 * paper; it exists for callers that cannot allocate device memory: an
 * application that owns all GPU memory through its own pool or allocator, a
 * plug-in running inside another framework's memory budget, or code in a
 * context where cudaMalloc is not permitted).  The caller passes device
 * inputs and outputs it already owns; the library allocates nothing.
 * ------------------------------------------------------------------------- */

/* Parameters of dpd_forces_static (the same physics as dpd_create). */
typedef struct {
    double box[3];           /* periodic box, each length > 2 rc */
    int32_t n_species;       /* 1..8 */
    int32_t body_force_mode; /* 0 none, 1 uniform, 2 +g for y < L_y/2 and -g above */
    double a_ij[64];         /* n_species x n_species row-major, symmetric */
    double gamma, kT, rc, s, dt;
    uint64_t seed;           /* seed of the random force (TEA key) */
    double body_force[3];
} dpd_static_params;

/* The same total force as dpd_forces gives for this state (DPD pair forces
 * and the body force; no bonds) on n particles at one step, with no device
 * allocation.  All arrays are DEVICE pointers
 * owned by the caller, in the caller's order:
 *   pos:       n x 4 floats (x, y, z in [0, L), species as int bits)
 *   vel:       n x 4 floats (vx, vy, vz, unused)
 *   tag:       n identity tags keying the random force, or NULL (tag = index)
 *   force_out: n x 4 floats (fx, fy, fz, 0)
 * step keys the random force; stream is a cudaStream_t (NULL = default).
 * The work is enqueued on the stream and the call returns without waiting:
 * force_out is complete when the stream reaches that point.
 * Scratch: one static device array of fixed size inside the library, which
 * every GPU that loads the library holds until the process exits.  Limits:
 * n <= dpd_forces_static_max_particles() (131072) and at most 65536 cells of
 * side >= rc; larger inputs return DPD_ERR_ARG with a message and launch
 * nothing.  The array's device address is looked up on the first call made
 * on each device, so make that first call before any CUDA stream capture.
 * Every call reuses the same array (the cell counts are cleared at the start
 * of each call), so calls whose kernels overlap on the GPU -- on different
 * streams, or from different host threads without ordering -- race on it.
 * The force sums run in a fixed order, so repeated calls on the same input
 * give the same bits.  A species outside 0..n_species-1 is not read from
 * the parameter table: the force of that particle, and of every particle
 * within rc of it, is written as NaN (the call itself still returns
 * DPD_OK, since it does not wait for the kernels).
 * Errors: DPD_ERR_ARG for invalid or oversized input, DPD_ERR_CUDA for a
 * failed launch; dpd_forces_static_last_error() describes the failure. */
dpd_status dpd_forces_static(const dpd_static_params *params, int64_t n, const float *pos, const float *vel,
                             const uint32_t *tag, uint64_t step, float *force_out, void *stream);

/* Largest n dpd_forces_static accepts. */
int64_t dpd_forces_static_max_particles(void);

/* Description of the last dpd_forces_static failure on this host thread. */
const char *dpd_forces_static_last_error(void);

/* Description of the last failure on h (or of the last handle-less failure
 * when h is NULL).  Valid until the next call on h. */
const char *dpd_last_error(const dpd_sim *h);

/* Free the handle and all its device memory.  NULL is ignored. */
void dpd_destroy(dpd_sim *h);

#ifdef __cplusplus
}
#endif

#endif /* DPD_H */
