// tune.cu -- choosing the neighbour-list skin by measurement.
//
// The skin trades the list's length (candidates per particle grow as
// (r_c + skin)^3, Sec. 3.3) against how often it is rebuilt (a particle may
// move skin/2 between builds).  Which side wins depends on the system size,
// density and temperature, so the choice is measured: every candidate runs the
// caller's system on a temporary handle, timed with the same CUDA events as
// dpd_step_profiled, and the fastest per step is kept.  Host code only; it
// drives the engine through its public entry points.
#include "dpd.h"

#include <cmath>
#include <cstring>
#include <limits>
#include <string>

extern "C" dpd_status dpd_tune_skin(const double box[3], int32_t n_species, const double *a_ij, double gamma,
                                    double kT, double rc, double s, double dt, const dpd_options *opt, int64_t n,
                                    const double *x, const double *v, const int32_t *species,
                                    const double *candidates, int32_t ncand, int32_t steps, double *best_skin,
                                    double *ms_per_step)
{
    if (!box || !a_ij || !x || !v || !candidates || ncand < 1 || steps < 1 || !best_skin) return DPD_ERR_ARG;
    dpd_options base;
    if (opt) base = *opt; else dpd_default_options(&base);
    double best = std::numeric_limits<double>::infinity();
    *best_skin = -1.0;
    dpd_status last = DPD_ERR_ARG;
    for (int32_t k = 0; k < ncand; ++k) {
        double ms = std::numeric_limits<double>::infinity();
        dpd_options o = base;
        o.skin = candidates[k];
        dpd_sim *h = nullptr;
        dpd_status st = dpd_create(&h, box, n_species, a_ij, gamma, kT, rc, s, dt, &o);
        if (st == DPD_OK) st = dpd_set_state(h, n, x, v, species, nullptr, 0);
        // warm-up (graph capture, first rebuilds), then the timed steps
        if (st == DPD_OK) st = dpd_step(h, (steps + 3) / 4);
        dpd_step_times t;
        std::memset(&t, 0, sizeof(t));
        if (st == DPD_OK) st = dpd_step_profiled(h, steps, &t);
        if (st == DPD_OK && t.total_ms > 0.0) ms = t.total_ms / steps;
        if (h) dpd_destroy(h);
        last = st;
        if (ms_per_step) ms_per_step[k] = ms;
        if (ms < best) {
            best = ms;
            *best_skin = candidates[k];
        }
    }
    return *best_skin >= 0.0 ? DPD_OK : last;
}
