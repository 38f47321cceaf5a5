/* dpd_ensemble.h -- many small independent DPD boxes advanced together by
 * one persistent fused kernel.
 *
 * Each box is the periodic DPD system of dpd.h (pair force of Eqs. 2-9,
 * random force from the pair-symmetric TEA hash keyed on (step, i, j) of
 * Sec. 3.5 and Algorithm 4, the lambda form of velocity Verlet of Sec. 3.1 /
 * Algorithm 1), with its own size, parameters, seed and step.  A launch
 * advances every listed box a whole chunk of steps: each box is owned by a
 * thread-block cluster of C CTAs, every CTA keeps a replica of the box's
 * positions and velocities in shared memory, and each step bins the box into
 * cells of side >= r_c (the cell list of Sec. 3.2.3), evaluates the pair
 * forces of its share of the cells (the 27-cell stencil of Sec. 3.3.1, no
 * neighbour list, no skin), integrates the particles it owns and sends their
 * new state to the other replicas through distributed shared memory.
 * Nothing goes to device memory between the chunk's first and last step.
 *
 * Results: every force is summed in a fixed order (cells in a fixed stencil
 * order, particles of a cell by index, fixed-size batches), so a box's
 * trajectory is bit-identical whatever the other boxes, the cluster size C
 * and the block size are (unless the Newton-3 option is set).  They agree
 * with dpd.h's engine to FP32 rounding, not bit for bit (different
 * summation order).
 *
 * Limits: a box must fit in one CTA's shared memory (about 4,000 particles
 * with lambda = 1/2, about 3,200 otherwise; dpd_ensemble_fits tells), have at
 * least three cells of side r_c (1 + 1e-4) along each axis, and carries no
 * bonds.  Larger boxes belong on dpd.h's engine.
 *
 * All functions return dpd_status (dpd.h); on an error
 * dpd_ensemble_last_error() describes it.  Device memory is stream-ordered on
 * the ensemble's stream.  Not thread-safe per handle. */
#ifndef DPD_ENSEMBLE_H
#define DPD_ENSEMBLE_H

#include "dpd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpd_ensemble dpd_ensemble;

typedef struct {
    int32_t threads;       /* threads per CTA: 128, 256 or 512; 0 = per size class (512, and 256
                              for the smallest boxes; fewer when a box's footprint needs it) */
    int32_t cluster;       /* CTAs per box: 1, 2, 4 or 8; 0 = per size class (2) */
    double wait_timeout_s; /* deadline of every host wait (default 600) */
    void *stream;          /* cudaStream_t; NULL = a stream of the handle */
    int32_t newton3;       /* 1: each pair evaluated once (half stencil), the partner's share
                              added by an atomic in the shared memory of the CTA that owns
                              it; the last bits of a trajectory then vary run to run.
                              0 (default): every pair from both sides in a fixed order
                              (bit-reproducible). */
} dpd_ensemble_options;

/* Parameters of one box (the arguments of dpd_create plus the options that
 * apply here). */
typedef struct {
    double box[3];          /* box lengths, each >= 3 rc (1 + 1e-4) */
    int32_t n_species;      /* 1..8 */
    const double *a_ij;     /* n_species x n_species, row-major, symmetric */
    double gamma, kT, rc, s, dt;
    double lambda;          /* velocity-Verlet lambda (0.5: the paper's scheme) */
    uint64_t seed;          /* random-force key */
    int32_t body_force_mode;/* 0 none, 1 uniform, 2 reverse Poiseuille (sign by y half) */
    double body_force[3];
} dpd_box_params;

void dpd_ensemble_default_options(dpd_ensemble_options *opt);

/* Create an empty ensemble.  opt may be NULL.  DPD_ERR_CUDA without a GPU. */
dpd_status dpd_ensemble_create(dpd_ensemble **out, const dpd_ensemble_options *opt);

/* 1 if a box of these parameters and n particles fits the ensemble kernel,
 * else 0 (too many particles for shared memory, fewer than three cells
 * along an axis, or invalid parameters). */
int32_t dpd_ensemble_fits(const dpd_box_params *p, int64_t n);

/* Add a box: n particles, x and v (n x 3, FP64, caller order; positions are
 * wrapped into the box), species (n, nullable = all 0), at step `step`.
 * Particle i keeps index i (and random-force tag i) for the box's life.
 * The force at the initial state is computed before the box's first step.
 * *id receives the box's id (>= 0).  DPD_ERR_ARG if the box does not fit
 * (dpd_ensemble_fits) or an input is invalid (non-finite values, species out
 * of range); nothing is added then. */
dpd_status dpd_ensemble_add(dpd_ensemble *e, const dpd_box_params *p, int64_t n, const double *x, const double *v,
                            const int32_t *species, uint64_t step, int32_t *id);

/* Remove a box and free its memory (stream-ordered). */
dpd_status dpd_ensemble_remove(dpd_ensemble *e, int32_t id);

/* Advance box ids[k] by steps[k] steps (steps[k] >= 0) for k < m, all in
 * one launch per size class; ids == NULL with m == 0 advances every box by
 * steps[0].  The class launches (forked onto one stream per class and
 * joined back) are captured as a CUDA graph and the graph is replayed by
 * later calls with the same launch structure -- the same boxes per class,
 * whatever their step counts, which the launches read from device
 * descriptors uploaded before each replay; a new structure is captured
 * anew.  So the handle's stream must not itself be under capture.  Returns
 * after queueing (asynchronous); dpd_ensemble_sync waits and reports
 * device-side errors (a non-finite force: DPD_ERR_NONFINITE). */
dpd_status dpd_ensemble_step(dpd_ensemble *e, const int32_t *ids, const int32_t *steps, int32_t m);

/* How many step calls captured a new graph and how many replayed one. */
dpd_status dpd_ensemble_graph_stats(dpd_ensemble *e, int64_t *captures, int64_t *replays);

/* Wait for everything queued on the ensemble (deadline wait_timeout_s). */
dpd_status dpd_ensemble_sync(dpd_ensemble *e);

/* State of a box in caller order: x, v (n x 3, nullable), the step. Waits. */
dpd_status dpd_ensemble_get_state(dpd_ensemble *e, int32_t id, double *x, double *v, uint64_t *step);

/* Force on each particle at the box's current state (n x 3).  Waits. */
dpd_status dpd_ensemble_get_forces(dpd_ensemble *e, int32_t id, double *f);

/* Observables of a box (dpd_obs of dpd.h): kinetic sums, the conservative
 * virial of its current state, pressure, momentum.  Waits. */
dpd_status dpd_ensemble_observables(dpd_ensemble *e, int32_t id, dpd_obs *out);

/* Number of boxes and of particles over all boxes. */
dpd_status dpd_ensemble_info(dpd_ensemble *e, int32_t *nboxes, int64_t *nparticles);

/* Autotuner: for each size class present (boxes grouped by how many CTAs of
 * their shared-memory footprint fit on one SM), time `steps` steps of that
 * class's boxes, run on scratch copies of their current state, for every
 * feasible (threads per CTA, CTAs per box) in {128, 256, 512} x {1, 2, 4, 8}
 * and keep the fastest per class for later dpd_ensemble_step calls (the
 * boxes' own state does not change).  With table != NULL, table[k] receives
 * the ms per step of candidate k (threads index * 4 + cluster index; +inf if
 * infeasible) of the last class tuned.  Overrides the handle's fixed options. */
dpd_status dpd_ensemble_tune(dpd_ensemble *e, int32_t steps, double *table);

/* Per size class (0 = largest footprint .. 3), the threads per CTA and CTAs
 * per box the next launch uses (both 0 for a class without boxes). */
dpd_status dpd_ensemble_config(dpd_ensemble *e, int32_t threads[4], int32_t cluster[4]);

void dpd_ensemble_destroy(dpd_ensemble *e);

const char *dpd_ensemble_last_error(dpd_ensemble *e);

#ifdef __cplusplus
}
#endif

#endif
