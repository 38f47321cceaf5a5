// server.cu -- continuous batching of independent DPD boxes (dpd_server.h).
//
// Host code only: a worker thread drives handles of the engine (dpd.h)
// through its public entry points.  Each admitted box is one dpd_sim with
// its own stream; the worker queues a chunk of steps on every box whose
// stream is idle (dpd_step_async, replayed from the box's CUDA graphs),
// checks finished chunks (dpd_sync), and admits queued boxes first-fit by
// estimated device memory whenever a box finishes.  Device memory of the
// handles is stream-ordered, so creating or freeing one box never waits for
// the others.  With the ensemble option, boxes small enough for the ensemble
// kernel (dpd_ensemble.h) go to one more worker instead, which keeps them all
// in one dpd_ensemble and advances every one of them a chunk per launch.
#include "dpd_server.h"
#include "dpd_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket = 0;
    double box[3] = {0, 0, 0};
    int32_t n_species = 1;
    std::vector<double> a;
    double gamma = 0, kT = 0, rc = 1, s = 1, dt = 0.01;
    uint64_t seed = 0;
    int64_t n = 0;
    std::vector<double> x, v;
    std::vector<int32_t> species;
    uint64_t steps = 0;
    double skin = 0;        // 0: the server's box_options.skin
    double est_bytes = 0;
    double est_ens_bytes = 0;
    bool ens = false;       // routed to the ensemble kernel at submission (ensemble = 1)
    bool ens_fit = false;   // fits the ensemble kernel (ensemble = 2 decides at admission)
    double t_submit = 0;
    double t_admit = 0;     // stamped under the server's lock when taken from the queue
};

struct Done {
    dpd_result res;
    std::vector<double> x, v;
};

struct Slot {
    Job job;
    dpd_sim *sim = nullptr;
    uint64_t left = 0;      // steps not yet queued
    bool queued = false;    // a chunk is on the stream, not yet checked
    double t_admit = 0;
};

// Device bytes of one box, following the engine's allocations: the
// double-buffered particle arrays and scratch (about 300 B per particle), the
// list at the automatic capacity (32 entries per particle group slot), the
// cell tables, and a fixed allowance.
double estimate_bytes(const Job &j, const dpd_options &o)
{
    const double V = j.box[0] * j.box[1] * j.box[2];
    const double rl = j.rc + (j.skin > 0.0 ? j.skin : o.skin);
    const double mean = (double)j.n / V * 4.0 / 3.0 * M_PI * rl * rl * rl;
    double cap = std::max(std::ceil(1.6 * mean + 24.0), 32.0);
    cap = std::ceil(cap / 8.0) * 8.0;
    double ncell = 1.0;
    for (int a = 0; a < 3; ++a) ncell *= std::max(1.0, std::floor(j.box[a] / (rl * (1.0 + 1e-4))));
    const double groups = (double)j.n / 32.0 + ncell / 64.0 + 2.0;
    return (double)j.n * 320.0 + groups * 32.0 * cap * 4.0 + ncell * 160.0 + 4.0 * 1024 * 1024;
}

// Device bytes of a box in the ensemble: state, tags and indices (56 B per
// particle), its staging at upload (48 B per particle) and a small allowance.
double estimate_ensemble_bytes(const Job &j) { return (double)j.n * 104.0 + 64.0 * 1024; }

dpd_box_params box_params_of(const Job &j, const dpd_options &o)
{
    dpd_box_params p;
    std::memset(&p, 0, sizeof(p));
    for (int a = 0; a < 3; ++a) {
        p.box[a] = j.box[a];
        p.body_force[a] = o.body_force[a];
    }
    p.n_species = j.n_species;
    p.a_ij = j.a.data();
    p.gamma = j.gamma;
    p.kT = j.kT;
    p.rc = j.rc;
    p.s = j.s;
    p.dt = j.dt;
    p.lambda = o.lambda;
    p.seed = j.seed;
    p.body_force_mode = o.body_force_mode;
    return p;
}

}  // namespace

struct dpd_server {
    dpd_server_options opt;
    int device = 0;
    Clock::time_point t0;
    double budget = 0;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> pending;
    std::map<uint64_t, Done> done;
    std::map<uint64_t, bool> known;  // submitted and not yet collected
    int64_t running = 0;
    int64_t handle_active = 0;  // boxes admitted to their own handles and not finished
    double mem_used = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    std::thread ens_worker;
    std::string err;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

dpd_status fail_s(dpd_server *s, dpd_status st, const std::string &msg)
{
    if (s) {
        std::lock_guard<std::mutex> lk(s->m);
        s->err = msg;
    }
    return st;
}

void finish(dpd_server *S, Slot &sl, dpd_status st, const std::string &msg)
{
    Done d;
    std::memset(&d.res, 0, sizeof(d.res));
    d.res.ticket = sl.job.ticket;
    d.res.status = st;
    d.res.n = sl.job.n;
    d.res.steps = sl.job.steps;
    d.res.t_submit = sl.job.t_submit;
    d.res.t_admit = sl.t_admit;
    if (st == DPD_OK && sl.sim) {
        d.x.resize(3 * (size_t)sl.job.n);
        d.v.resize(3 * (size_t)sl.job.n);
        dpd_status s2 = dpd_observables(sl.sim, &d.res.obs);
        if (s2 == DPD_OK) s2 = dpd_get_state(sl.sim, d.x.data(), d.v.data(), nullptr);
        if (s2 != DPD_OK) d.res.status = s2;
    }
    std::string m2 = msg;
    if (d.res.status != DPD_OK && m2.empty() && sl.sim) m2 = dpd_last_error(sl.sim);
    if (sl.sim) dpd_destroy(sl.sim);
    sl.sim = nullptr;
    d.res.t_done = S->now();
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->done[sl.job.ticket] = std::move(d);
        S->running -= 1;
        S->handle_active -= 1;
        S->mem_used -= sl.job.est_bytes;
        if (!m2.empty()) S->err = "ticket " + std::to_string(sl.job.ticket) + ": " + m2;
    }
    S->cv_done.notify_all();
}

// Create the handle of an admitted box and upload its state.
dpd_status start(dpd_server *S, Slot &sl)
{
    dpd_options o = S->opt.box_options;
    o.seed = sl.job.seed;
    if (sl.job.skin > 0.0) o.skin = sl.job.skin;
    o.stream = nullptr;  // a stream of the box's own
    dpd_status st = dpd_create(&sl.sim, sl.job.box, sl.job.n_species, sl.job.a.data(), sl.job.gamma, sl.job.kT,
                               sl.job.rc, sl.job.s, sl.job.dt, &o);
    if (st != DPD_OK) {
        sl.sim = nullptr;
        return st;
    }
    st = dpd_set_state(sl.sim, sl.job.n, sl.job.x.data(), sl.job.v.data(),
                       sl.job.species.empty() ? nullptr : sl.job.species.data(), nullptr, 0);
    // the host copies are no longer needed
    std::vector<double>().swap(sl.job.x);
    std::vector<double>().swap(sl.job.v);
    std::vector<int32_t>().swap(sl.job.species);
    return st;
}

// One worker: its own set of at most `slots` running boxes; the queue, the
// memory budget and the results are shared under the server's lock.
void worker_loop(dpd_server *S, int slots)
{
    cudaSetDevice(S->device);
    std::vector<Slot> active;
    for (;;) {
        // ---- admission: first fit by estimated memory, in submission order
        std::vector<Job> admit;
        bool stopping = false;
        {
            std::unique_lock<std::mutex> lk(S->m);
            bool mine = false;  // a queued box this kind of worker runs
            for (const Job &j : S->pending) mine = mine || !j.ens;
            if (active.empty() && !mine && !S->stop) S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            stopping = S->stop;
            if (!stopping) {
                int looked = 0;
                for (auto it = S->pending.begin();
                     it != S->pending.end() && (int)(active.size() + admit.size()) < slots && looked < 16;) {
                    if (it->ens) {
                        ++it;
                        continue;
                    }
                    if (S->mem_used + it->est_bytes <= S->budget) {
                        S->mem_used += it->est_bytes;
                        S->running += 1;
                        S->handle_active += 1;
                        it->t_admit = S->now();
                        admit.push_back(std::move(*it));
                        it = S->pending.erase(it);
                    } else {
                        ++it;
                        ++looked;
                    }
                }
            }
        }
        if (stopping) break;
        for (Job &j : admit) {
            active.emplace_back();
            Slot &sl = active.back();
            sl.job = std::move(j);
            sl.left = sl.job.steps;
            sl.t_admit = sl.job.t_admit;
            dpd_status st = start(S, sl);
            if (st != DPD_OK) {
                std::string msg = sl.sim ? dpd_last_error(sl.sim) : dpd_last_error(nullptr);
                finish(S, sl, st, msg);
                active.pop_back();
            }
        }
        // ---- progress: every box whose stream is idle gets its next chunk
        bool progressed = !admit.empty();
        for (size_t k = 0; k < active.size();) {
            Slot &sl = active[k];
            int32_t idle = 0;
            dpd_status st = dpd_query(sl.sim, &idle);
            if (st == DPD_OK && !idle) {
                ++k;
                continue;
            }
            progressed = true;
            if (st == DPD_OK && sl.queued) {
                st = dpd_sync(sl.sim);
                sl.queued = false;
            }
            if (st == DPD_OK && sl.left > 0) {
                const uint64_t c = std::min<uint64_t>(sl.left, (uint64_t)S->opt.chunk_steps);
                st = dpd_step_async(sl.sim, (int64_t)c);
                if (st == DPD_OK) {
                    sl.left -= c;
                    sl.queued = true;
                    ++k;
                    continue;
                }
            }
            finish(S, sl, st, "");
            active.erase(active.begin() + (long)k);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // ---- shutdown: stop the running boxes after their queued chunk
    for (Slot &sl : active) finish(S, sl, DPD_ERR_STATE, "server stopped");
    std::lock_guard<std::mutex> lk(S->m);
    for (Job &j : S->pending) {
        Done d;
        std::memset(&d.res, 0, sizeof(d.res));
        d.res.ticket = j.ticket;
        d.res.status = DPD_ERR_STATE;
        d.res.n = j.n;
        d.res.steps = j.steps;
        d.res.t_submit = j.t_submit;
        d.res.t_done = S->now();
        S->done[j.ticket] = std::move(d);
    }
    S->pending.clear();
}

// The ensemble worker: admits the boxes routed to the ensemble kernel (first
// fit by memory, in submission order), advances all of them by one chunk per
// pass -- one launch per size class -- and reads back the finished ones.
void ensemble_loop(dpd_server *S)
{
    cudaSetDevice(S->device);
    struct EJob {
        Job job;
        int32_t id = -1;
        uint64_t left = 0;
    };
    dpd_ensemble *E = nullptr;
    dpd_status est = dpd_ensemble_create(&E, nullptr);
    std::string emsg = est == DPD_OK ? "" : std::string("ensemble: ") + dpd_ensemble_last_error(nullptr);
    std::vector<EJob> active;
    auto done_job = [&](EJob &ej, dpd_status st, const std::string &msg) {
        Done d;
        std::memset(&d.res, 0, sizeof(d.res));
        d.res.ticket = ej.job.ticket;
        d.res.status = st;
        d.res.n = ej.job.n;
        d.res.steps = ej.job.steps;
        d.res.t_submit = ej.job.t_submit;
        d.res.t_admit = ej.job.t_admit;
        d.res.engine = 1;
        std::string m2 = msg;
        if (st == DPD_OK && ej.id >= 0) {
            d.x.resize(3 * (size_t)ej.job.n);
            d.v.resize(3 * (size_t)ej.job.n);
            dpd_status s2 = dpd_ensemble_observables(E, ej.id, &d.res.obs);
            if (s2 == DPD_OK) s2 = dpd_ensemble_get_state(E, ej.id, d.x.data(), d.v.data(), nullptr);
            if (s2 != DPD_OK) {
                d.res.status = s2;
                m2 = dpd_ensemble_last_error(E);
            }
        }
        if (E && ej.id >= 0) dpd_ensemble_remove(E, ej.id);
        d.res.t_done = S->now();
        {
            std::lock_guard<std::mutex> lk(S->m);
            S->done[ej.job.ticket] = std::move(d);
            S->running -= 1;
            S->mem_used -= ej.job.est_bytes;
            if (!m2.empty()) S->err = "ticket " + std::to_string(ej.job.ticket) + ": " + m2;
        }
        S->cv_done.notify_all();
    };
    const int slots = S->opt.ensemble_slots;
    for (;;) {
        std::vector<Job> admit;
        bool stopping = false;
        {
            std::unique_lock<std::mutex> lk(S->m);
            // adaptive routing (ensemble = 2): a box that fits is taken here
            // only while every handle slot is busy, so under light load the
            // boxes keep the handles' per-box latency
            const bool handles_full = S->handle_active >= S->opt.max_active;
            auto mine = [&](const Job &j) { return j.ens || (S->opt.ensemble == 2 && j.ens_fit && handles_full); };
            bool any = false;
            for (const Job &j : S->pending) any = any || mine(j);
            if (active.empty() && !any && !S->stop) S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            stopping = S->stop;
            if (!stopping) {
                int looked = 0;
                for (auto it = S->pending.begin();
                     it != S->pending.end() && (int)(active.size() + admit.size()) < slots && looked < 16;) {
                    if (!mine(*it)) {
                        ++it;
                        continue;
                    }
                    if (!it->ens) it->est_bytes = it->est_ens_bytes;  // taken by adaptive routing
                    if (S->mem_used + it->est_bytes <= S->budget) {
                        S->mem_used += it->est_bytes;
                        S->running += 1;
                        it->t_admit = S->now();
                        admit.push_back(std::move(*it));
                        it = S->pending.erase(it);
                    } else {
                        ++it;
                        ++looked;
                    }
                }
            }
        }
        if (stopping) break;
        for (Job &j : admit) {
            EJob ej;
            ej.job = std::move(j);
            ej.left = ej.job.steps;
            dpd_status st = est;
            if (st == DPD_OK) {
                const dpd_box_params p = box_params_of(ej.job, S->opt.box_options);
                st = dpd_ensemble_add(E, &p, ej.job.n, ej.job.x.data(), ej.job.v.data(),
                                      ej.job.species.empty() ? nullptr : ej.job.species.data(), 0, &ej.id);
            }
            std::vector<double>().swap(ej.job.x);
            std::vector<double>().swap(ej.job.v);
            std::vector<int32_t>().swap(ej.job.species);
            if (st != DPD_OK) {
                ej.id = -1;
                done_job(ej, st, est == DPD_OK ? std::string(dpd_ensemble_last_error(E)) : emsg);
                continue;
            }
            active.push_back(std::move(ej));
        }
        if (active.empty()) continue;
        // one chunk for every resident box
        std::vector<int32_t> ids, steps;
        for (const EJob &ej : active) {
            ids.push_back(ej.id);
            steps.push_back((int32_t)std::min<uint64_t>(ej.left, (uint64_t)S->opt.chunk_steps));
        }
        dpd_status st = dpd_ensemble_step(E, ids.data(), steps.data(), (int32_t)ids.size());
        if (st == DPD_OK) st = dpd_ensemble_sync(E);
        if (st != DPD_OK) {
            // a failed chunk ends every box of it; a CUDA failure ends the ensemble
            const std::string msg = dpd_ensemble_last_error(E);
            for (EJob &ej : active) done_job(ej, st, msg);
            active.clear();
            if (st == DPD_ERR_CUDA || st == DPD_ERR_TIMEOUT) {
                dpd_ensemble_destroy(E);
                E = nullptr;
                est = dpd_ensemble_create(&E, nullptr);
                emsg = est == DPD_OK ? "" : std::string("ensemble: ") + dpd_ensemble_last_error(nullptr);
            }
            continue;
        }
        for (size_t k = 0; k < active.size();) {
            active[k].left -= (uint64_t)steps[k];
            if (active[k].left == 0) {
                done_job(active[k], DPD_OK, "");
                active.erase(active.begin() + (long)k);
                steps.erase(steps.begin() + (long)k);
            } else {
                ++k;
            }
        }
    }
    for (EJob &ej : active) done_job(ej, DPD_ERR_STATE, "server stopped");
    if (E) dpd_ensemble_destroy(E);
    std::lock_guard<std::mutex> lk(S->m);
    for (Job &j : S->pending) {
        Done d;
        std::memset(&d.res, 0, sizeof(d.res));
        d.res.ticket = j.ticket;
        d.res.status = DPD_ERR_STATE;
        d.res.n = j.n;
        d.res.steps = j.steps;
        d.res.t_submit = j.t_submit;
        d.res.t_done = S->now();
        S->done[j.ticket] = std::move(d);
    }
    S->pending.clear();
}

}  // namespace

extern "C" {

void dpd_server_default_options(dpd_server_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->max_active = 32;
    o->workers = 4;
    o->chunk_steps = 100;
    o->mem_budget_bytes = 0.0;
    dpd_default_options(&o->box_options);
    // small boxes: launching the rebuild chain's early-exit kernels costs
    // less than executing a conditional node's body (measured)
    o->box_options.conditional_rebuild = 0;
    o->ensemble = 0;
    o->ensemble_slots = 1024;
}

dpd_status dpd_server_create(const dpd_server_options *o, dpd_server **out)
{
    if (!out) return DPD_ERR_ARG;
    *out = nullptr;
    dpd_server_options opt;
    if (o) opt = *o; else dpd_server_default_options(&opt);
    if (opt.max_active < 1 || opt.workers < 1 || opt.chunk_steps < 1 || !(opt.mem_budget_bytes >= 0.0) ||
        opt.ensemble < 0 || opt.ensemble > 2 || (opt.ensemble && opt.ensemble_slots < 1))
        return DPD_ERR_ARG;
    dpd_server *S = new dpd_server();
    S->opt = opt;
    S->t0 = Clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return DPD_ERR_CUDA;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return DPD_ERR_CUDA;
    }
    S->budget = opt.mem_budget_bytes > 0.0 ? opt.mem_budget_bytes : 0.6 * (double)free_b;
    const int nw = std::min(opt.workers, opt.max_active);
    for (int w = 0; w < nw; ++w) {
        const int slots = opt.max_active / nw + (w < opt.max_active % nw ? 1 : 0);
        S->workers.emplace_back(worker_loop, S, slots);
    }
    if (opt.ensemble) S->ens_worker = std::thread(ensemble_loop, S);
    *out = S;
    return DPD_OK;
}

dpd_status dpd_server_submit(dpd_server *S, const dpd_request *r, uint64_t *ticket)
{
    if (!S) return DPD_ERR_ARG;
    if (!r || !ticket || !r->a_ij || !r->x || !r->v || r->n <= 0 || r->n > dpd::kMaxParticles || r->steps < 1 ||
        r->n_species < 1 || r->n_species > dpd::kMaxSpecies || !(r->skin >= 0.0))
        return fail_s(S, DPD_ERR_ARG, "invalid request");
    Job j;
    for (int a = 0; a < 3; ++a) j.box[a] = r->box[a];
    j.n_species = r->n_species;
    j.a.assign(r->a_ij, r->a_ij + (size_t)r->n_species * r->n_species);
    j.gamma = r->gamma;
    j.kT = r->kT;
    j.rc = r->rc;
    j.s = r->s;
    j.dt = r->dt;
    j.seed = r->seed;
    j.n = r->n;
    j.x.assign(r->x, r->x + 3 * (size_t)r->n);
    j.v.assign(r->v, r->v + 3 * (size_t)r->n);
    if (r->species) j.species.assign(r->species, r->species + (size_t)r->n);
    j.steps = r->steps;
    j.skin = r->skin;
    if (S->opt.ensemble) {
        const dpd_box_params p = box_params_of(j, S->opt.box_options);
        j.ens_fit = dpd_ensemble_fits(&p, j.n) != 0;
        j.ens = j.ens_fit && S->opt.ensemble == 1;
    }
    j.est_ens_bytes = estimate_ensemble_bytes(j);
    j.est_bytes = j.ens ? j.est_ens_bytes : estimate_bytes(j, S->opt.box_options);
    if (j.est_bytes > S->budget) return fail_s(S, DPD_ERR_OOM, "box needs more device memory than the budget");
    {
        std::lock_guard<std::mutex> lk(S->m);
        if (S->stop) {
            S->err = "server stopped";
            return DPD_ERR_STATE;
        }
        j.ticket = S->next_ticket++;
        j.t_submit = S->now();
        *ticket = j.ticket;
        S->known[j.ticket] = true;
        S->pending.push_back(std::move(j));
    }
    S->cv_work.notify_all();
    return DPD_OK;
}

dpd_status dpd_server_wait(dpd_server *S, uint64_t ticket, double timeout_s, dpd_result *res, double *x_out,
                           double *v_out)
{
    if (!S || !res) return DPD_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->m);
    if (!S->known.count(ticket)) {
        S->err = "unknown or collected ticket";
        return DPD_ERR_ARG;
    }
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(timeout_s, 0.0)));
    while (!S->done.count(ticket)) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !S->done.count(ticket)) {
            S->err = "box not finished";
            return DPD_ERR_TIMEOUT;
        }
    }
    Done &d = S->done[ticket];
    *res = d.res;
    if (x_out && !d.x.empty()) std::memcpy(x_out, d.x.data(), sizeof(double) * d.x.size());
    if (v_out && !d.v.empty()) std::memcpy(v_out, d.v.data(), sizeof(double) * d.v.size());
    S->done.erase(ticket);
    S->known.erase(ticket);
    return DPD_OK;
}

double dpd_server_now(const dpd_server *S) { return S ? S->now() : 0.0; }

dpd_status dpd_server_counts(dpd_server *S, int64_t *queued, int64_t *running, int64_t *finished, double *mem_bytes)
{
    if (!S) return DPD_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->m);
    if (queued) *queued = (int64_t)S->pending.size();
    if (running) *running = S->running;
    if (finished) *finished = (int64_t)S->done.size();
    if (mem_bytes) *mem_bytes = S->mem_used;
    return DPD_OK;
}

const char *dpd_server_last_error(const dpd_server *S)
{
    if (!S) return "null server";
    // workers may set the message at any time: hand out a copy owned by the
    // calling thread (valid until its next call)
    thread_local std::string copy;
    {
        std::lock_guard<std::mutex> lk(const_cast<dpd_server *>(S)->m);
        copy = S->err;
    }
    return copy.c_str();
}

void dpd_server_destroy(dpd_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &t : S->workers)
        if (t.joinable()) t.join();
    if (S->ens_worker.joinable()) S->ens_worker.join();
    delete S;
}

}  // extern "C"
