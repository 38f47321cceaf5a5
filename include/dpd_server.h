/* dpd_server.h -- continuous batching of independent DPD boxes on one GPU.
 *
 * A serving loop over the engine of dpd.h for ensemble and parameter-sweep
 * runs: clients submit boxes of any size and parameters (each a complete
 * run: state, parameters, number of steps); the server admits them as device
 * memory and slots allow, keeps every admitted box's particle state resident
 * on the device, and advances all admitted boxes concurrently -- each on its
 * own CUDA stream, in chunks of steps replayed from that box's CUDA graphs --
 * so the work of boxes that arrive while others run overlaps on the GPU.  A
 * box's result (final state and observables) does not depend on what else
 * runs: every box is an independent handle with its own stream, buffers and
 * random-number key, and in deterministic mode (dpd_options.deterministic =
 * 1) its trajectory is bit-identical to the same run made alone.
 *
 * The method computed for each box is the one of dpd.h (Tang & Karniadakis,
 * arXiv:1311.0402, Eqs. 1-9, Algorithms 1-4); the server adds only
 * scheduling.  Time-to-completion (t_done - t_submit) is reported per box so
 * that callers can form p50 / p99 latencies next to throughput.
 *
 * Conventions: host arrays are copied at submission; the server owns all
 * device memory of the boxes it runs; every call returns a dpd_status and
 * dpd_server_last_error gives the message of the last failure.  All calls
 * are thread-safe: submit and wait may be called from any thread.
 */
#ifndef DPD_SERVER_H
#define DPD_SERVER_H

#include "dpd.h"
#include "dpd_ensemble.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dpd_server dpd_server; /* opaque */

typedef struct {
    int32_t max_active;        /* boxes resident and stepping at once (default 32) */
    int32_t workers;           /* host worker threads sharing the boxes (default 4): creating,
                                  loading, capturing and reading back boxes is host work */
    int32_t chunk_steps;       /* steps queued per box per scheduling pass (default 100) */
    double mem_budget_bytes;   /* device memory the boxes may take, by the server's estimate
                                  of each box; 0 (default) = 60 % of the free device memory
                                  when the server is created */
    dpd_options box_options;   /* run options of every box (the seed and the stream are
                                  taken per box: each box gets its own stream) */
    int32_t ensemble;          /* 1: boxes that fit the ensemble kernel (dpd_ensemble.h:
                                  about 4,000 particles or fewer, each side >= 3 rc) run
                                  there instead, all of them advanced together by one
                                  launch per size class and chunk, driven by one more
                                  worker thread; 2: a box that fits goes to the ensemble
                                  only when, at its admission, every one of the
                                  max_active handle slots is busy (otherwise it runs on a
                                  handle: the ensemble adds throughput under load without
                                  costing per-box latency when slots are free); 0
                                  (default): every box on its own handle */
    int32_t ensemble_slots;    /* boxes resident in the ensemble at once (default 1024) */
} dpd_server_options;

/* One box to run: the arguments of dpd_create + dpd_set_state + dpd_step.
 * a_ij: n_species x n_species, symmetric.  x, v: n x 3; species: n entries or
 * NULL.  Tags are the particle indices.  steps >= 1. */
typedef struct {
    double box[3];
    int32_t n_species;
    const double *a_ij;
    double gamma, kT, rc, s, dt;
    uint64_t seed;             /* random-force key of this box (Sec. 3.5) */
    int64_t n;
    const double *x, *v;
    const int32_t *species;
    uint64_t steps;
    double skin;               /* neighbour-list skin of this box; 0 = box_options.skin
                                  (dpd_tune_skin chooses one by measurement) */
} dpd_request;

typedef struct {
    uint64_t ticket;
    int32_t status;            /* dpd_status of the box's run */
    int64_t n;
    uint64_t steps;
    double t_submit;           /* seconds on the server clock (dpd_server_now) */
    double t_admit;            /* admitted: taken from the queue (device memory reserved) */
    double t_done;             /* final state read back */
    dpd_obs obs;               /* observables of the final state */
    int32_t engine;            /* 0: the box ran on its own handle (dpd.h); 1: in the
                                  ensemble kernel (dpd_ensemble.h) */
} dpd_result;

/* Results of boxes run by the ensemble kernel are bit-identical to the same box
 * run alone through dpd_ensemble.h in the same chunks of chunk_steps, and agree
 * with dpd.h's engine to FP32 rounding (a different summation order).
 *
 * Defaults: max_active 32, 4 workers, chunk_steps 100, budget 60 % of free memory,
 * dpd_default_options() for the boxes with conditional_rebuild = 0 (for
 * boxes of a few thousand particles the plain chain launches are cheaper).
 * For more than 8 boxes to run concurrently, set CUDA_DEVICE_MAX_CONNECTIONS
 * (e.g. to 32) in the environment before the first CUDA call. */
void dpd_server_default_options(dpd_server_options *o);

/* Start the serving loop (its worker threads) on the current device.
 * DPD_ERR_ARG for max_active < 1, workers < 1, chunk_steps < 1 or a negative
 * budget. */
dpd_status dpd_server_create(const dpd_server_options *o, dpd_server **out);

/* Queue a box; *ticket identifies it.  The request is validated here
 * (DPD_ERR_ARG, nothing queued) and its arrays copied.  A box whose
 * estimated memory exceeds the whole budget is refused with DPD_ERR_OOM. */
dpd_status dpd_server_submit(dpd_server *s, const dpd_request *r, uint64_t *ticket);

/* Wait up to timeout_s seconds for a box to finish; fills *res and, when
 * non-NULL, the final positions and velocities (n x 3, the request's particle
 * order).  DPD_ERR_TIMEOUT if it has not finished (it keeps running; wait
 * again); DPD_ERR_ARG for an unknown or already collected ticket.  The box's
 * own outcome is res->status. */
dpd_status dpd_server_wait(dpd_server *s, uint64_t ticket, double timeout_s, dpd_result *res, double *x_out,
                           double *v_out);

/* Seconds since the server started (the clock of t_submit / t_admit / t_done). */
double dpd_server_now(const dpd_server *s);

/* Boxes queued, running and finished-but-uncollected, and the estimated
 * device bytes held by running boxes. */
dpd_status dpd_server_counts(dpd_server *s, int64_t *queued, int64_t *running, int64_t *finished,
                             double *mem_bytes);

/* The last failure message (a submit, a wait or a box's run); the string
 * belongs to the calling thread and stays valid until its next call. */
const char *dpd_server_last_error(const dpd_server *s);

/* Stop the loop: queued boxes are dropped, running boxes are stopped after
 * their queued chunk, and all device memory of the boxes is freed.  No other
 * call on s may run during or after this one. */
void dpd_server_destroy(dpd_server *s);

#ifdef __cplusplus
}
#endif

#endif /* DPD_SERVER_H */
