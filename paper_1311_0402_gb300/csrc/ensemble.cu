// ensemble.cu -- host side of the ensemble kernel (dpd_ensemble.h): boxes
// with their own device memory, the descriptors of each launch, size classes
// by shared-memory footprint (one launch each, on forked streams, so small
// boxes pack several CTAs per SM), and the autotuner over threads per CTA and
// CTAs per box.
#include "dpd_ensemble.h"
#include "ensemble.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

using namespace dpd;

namespace {

thread_local std::string g_ens_error;
constexpr int kClasses = 4;
const int kThreadChoices[3] = {128, 256, 512};
const int kClusterChoices[4] = {1, 2, 4, 8};

struct EBox {
    int32_t id = -1;
    int64_t n = 0;
    int cls = 0;
    bool need_init = true;
    uint64_t step = 0;
    double box[3] = {0, 0, 0};
    EnsBox desc;             // host copy; pointers into mem
    void *mem = nullptr;     // one device block: state, tags, caller indices, error word, descriptor, observables
    uint32_t *pid = nullptr;
    EnsBox *d_self = nullptr;  // the descriptor in device memory (observables)
    double *d_obs = nullptr;
};

}  // namespace

struct dpd_ensemble {
    dpd_ensemble_options opt;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cls_stream[kClasses] = {};
    cudaEvent_t fork = nullptr, join[kClasses] = {}, ev = nullptr, t0 = nullptr, t1 = nullptr;
    std::map<int32_t, EBox> boxes;
    int32_t next_id = 0;
    EnsBox *d_desc = nullptr;
    size_t desc_cap = 0;
    uint32_t *d_any_err = nullptr;
    int threads[kClasses] = {0, 0, 0, 0};
    int cluster[kClasses] = {0, 0, 0, 0};
    bool tuned = false;
    size_t limit = 0;
    bool failed = false;
    std::string err;
    // the fork / class launches / join sequence of the last step call,
    // captured as a CUDA graph and replayed while the launch structure (the
    // classes, box counts, descriptor offsets and launch shapes) repeats
    cudaGraphExec_t graph = nullptr;
    std::vector<uint64_t> graph_key;
    int64_t graph_replays = 0;
    int64_t graph_captures = 0;
};

namespace {

dpd_status efail(dpd_ensemble *e, dpd_status st, const std::string &msg)
{
    if (e) {
        e->err = msg;
        if (st == DPD_ERR_CUDA) e->failed = true;
    }
    g_ens_error = msg;
    return st;
}

#define ENS_TRY(e, call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return efail((e), DPD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

dpd_status ewait(dpd_ensemble *e)
{
    cudaError_t c = cudaEventRecord(e->ev, e->stream);
    if (c != cudaSuccess) return efail(e, DPD_ERR_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(c));
    auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        c = cudaEventQuery(e->ev);
        if (c == cudaSuccess) return DPD_OK;
        if (c != cudaErrorNotReady) return efail(e, DPD_ERR_CUDA, std::string("kernel failure: ") + cudaGetErrorString(c));
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > e->opt.wait_timeout_s)
            return efail(e, DPD_ERR_TIMEOUT, "GPU did not finish within " + std::to_string(e->opt.wait_timeout_s) + " s");
        if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int cells_along(double L, double rc) { return (int)std::floor(L / (rc * (1.0 + 1e-4))); }

// Parameter checks shared by fits and add; empty string = valid.
std::string check_params(const dpd_box_params *p, int64_t n, int nc[3])
{
    if (!p) return "null parameters";
    if (!(p->n_species >= 1 && p->n_species <= kMaxSpecies) || !p->a_ij) return "n_species in 1..8 and a_ij required";
    if (!(p->gamma >= 0) || !(p->kT >= 0) || !(p->rc > 0) || !(p->s > 0) || !(p->dt > 0) || !std::isfinite(p->gamma) ||
        !std::isfinite(p->kT) || !std::isfinite(p->rc) || !std::isfinite(p->s) || !std::isfinite(p->dt) ||
        !std::isfinite(p->lambda))
        return "gamma >= 0, kT >= 0, rc > 0, s > 0, dt > 0 and finite lambda required";
    for (int i = 0; i < p->n_species; ++i)
        for (int j = 0; j < p->n_species; ++j) {
            const double x = p->a_ij[i * p->n_species + j];
            if (!std::isfinite(x) || x != p->a_ij[j * p->n_species + i]) return "a_ij must be finite and symmetric";
        }
    if (p->body_force_mode < 0 || p->body_force_mode > 2) return "body_force_mode in 0..2";
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->body_force[a])) return "body force must be finite";
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(p->box[a]) || !(p->box[a] > 0)) return "box lengths must be positive";
        nc[a] = cells_along(p->box[a], p->rc);
        if (nc[a] < 3) return "each box length must be at least 3 rc (1 + 1e-4)";
    }
    if (n < 1 || n > kEnsMaxN) return "1 <= n <= 65535";
    if ((int64_t)nc[0] * nc[1] * nc[2] > (1 << 20)) return "too many cells";
    return "";
}

size_t footprint(int64_t n, int ncell, bool lhalf, int threads)
{
    return ens_layout((int)n, ncell, lhalf, threads).total;
}

// Size class: how many CTAs of the box's footprint (256 threads) fit on one
// SM -- 1 (class 0), 2, 3, or 4 and more (class 3).
int class_of(int64_t n, int ncell, bool lhalf, size_t limit)
{
    const size_t need = footprint(n, ncell, lhalf, 256);
    const size_t k = need ? limit / need : 4;
    return (int)std::min<size_t>(std::max<size_t>(k, 1), 4) - 1;
}

// Shapes the autotuner chose on seeded streams of boxes of L = 6..10 (512
// threads and 2 CTAs per box, 256 threads for the smallest class); a launch
// steps down from these when a box's footprint does not fit.
int default_threads(int cls) { return cls == 3 ? 256 : 512; }
int default_cluster(int) { return 2; }

void fill_desc(EnsBox &d, const dpd_box_params *p, int64_t n, const int nc[3])
{
    std::memset(&d, 0, sizeof(d));
    d.n = (int)n;
    d.ncell = nc[0] * nc[1] * nc[2];
    for (int a = 0; a < 3; ++a) {
        d.nc[a] = nc[a];
        d.L[a] = (float)p->box[a];
        d.halfL[a] = 0.5f * d.L[a];
        d.cpl[a] = (float)(nc[a] / p->box[a]);
        d.body[a] = (float)p->body_force[a];
    }
    const float rcf = (float)p->rc;
    d.rc2 = rcf * rcf;
    d.inv_rc = (float)(1.0 / p->rc);
    d.gamma = (float)p->gamma;
    d.sigma_isdt = (float)(std::sqrt(2.0 * p->gamma * p->kT) / std::sqrt(p->dt));
    d.s = (float)p->s;
    d.s_mode = p->s == 1.0 ? 1 : (p->s == 0.5 ? 2 : (p->s == 2.0 ? 3 : 0));
    d.dt = (float)p->dt;
    d.half_dt = (float)(0.5 * p->dt);
    d.lambda_dt = (float)(p->lambda * p->dt);
    d.lhalf = p->lambda == 0.5 ? 1 : 0;
    d.n_species = p->n_species;
    for (int k = 0; k < p->n_species * p->n_species; ++k) d.a[k] = (float)p->a_ij[k];
    d.body_mode = p->body_force_mode;
    d.key[0] = (uint32_t)(p->seed & 0xFFFFFFFFull);
    d.key[1] = (uint32_t)(p->seed >> 32);
    d.key[2] = 0x243F6A88u;
    d.key[3] = 0x85A308D3u;
}

dpd_status ensure_desc(dpd_ensemble *e, size_t count)
{
    if (count <= e->desc_cap) return DPD_OK;
    size_t cap = std::max<size_t>(count, 2 * e->desc_cap);
    if (e->d_desc) cudaFreeAsync(e->d_desc, e->stream);
    e->d_desc = nullptr;
    e->desc_cap = 0;
    cudaError_t c = cudaMallocAsync((void **)&e->d_desc, cap * sizeof(EnsBox), e->stream);
    if (c != cudaSuccess) {
        cudaGetLastError();
        return efail(e, DPD_ERR_OOM, "descriptor allocation failed");
    }
    e->desc_cap = cap;
    return DPD_OK;
}

// One launch of a class's boxes (descriptors at dev, count nb): threads and
// cluster reduced until the footprint and the cluster shape fit.
struct Shape {
    int threads, cluster;
    size_t smem;
};

bool shape_for(const std::vector<const EBox *> &bs, bool lhalf, int s_mode, bool n3, int threads, int cluster,
               size_t limit, Shape &out)
{
    size_t smem = 0;
    for (const EBox *b : bs) smem = std::max(smem, footprint(b->n, b->desc.ncell, lhalf, threads));
    if (smem > limit) return false;
    if (ensemble_max_clusters(lhalf, s_mode, n3, threads, cluster, smem) < 1) return false;
    out = {threads, cluster, smem};
    return true;
}

bool pick_shape(const std::vector<const EBox *> &bs, bool lhalf, int s_mode, bool n3, int threads, int cluster,
                size_t limit, Shape &out)
{
    for (int t = threads; t >= 128; t /= 2)
        for (int c = cluster; c >= 1; c /= 2)
            if (shape_for(bs, lhalf, s_mode, n3, t, c, limit, out)) return true;
    return false;
}

// Launch groups: boxes of one class that share the kernel variant.
struct Group {
    int cls;
    bool lhalf;
    int s_mode;
    std::vector<const EBox *> init, run;
    std::vector<int> run_steps;
};

}  // namespace

extern "C" {

void dpd_ensemble_default_options(dpd_ensemble_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->wait_timeout_s = 600.0;
}

dpd_status dpd_ensemble_create(dpd_ensemble **out, const dpd_ensemble_options *opt)
{
    if (!out) return efail(nullptr, DPD_ERR_ARG, "null output");
    *out = nullptr;
    dpd_ensemble_options o;
    if (opt) o = *opt; else dpd_ensemble_default_options(&o);
    if (o.threads != 0 && o.threads != 128 && o.threads != 256 && o.threads != 512)
        return efail(nullptr, DPD_ERR_ARG, "threads in {0, 128, 256, 512}");
    if (o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4 && o.cluster != 8)
        return efail(nullptr, DPD_ERR_ARG, "cluster in {0, 1, 2, 4, 8}");
    if (!(o.wait_timeout_s > 0)) return efail(nullptr, DPD_ERR_ARG, "wait_timeout_s > 0");
    if (o.newton3 != 0 && o.newton3 != 1) return efail(nullptr, DPD_ERR_ARG, "newton3 in {0, 1}");
    dpd_ensemble *e = new dpd_ensemble();
    e->opt = o;
    if (o.stream) {
        e->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete e;
            return efail(nullptr, DPD_ERR_CUDA, "cudaStreamCreate failed (no GPU?)");
        }
        e->own_stream = true;
    }
    bool ok = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&e->t0) == cudaSuccess && cudaEventCreate(&e->t1) == cudaSuccess;
    for (int c = 0; ok && c < kClasses; ++c)
        ok = cudaStreamCreateWithFlags(&e->cls_stream[c], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->join[c], cudaEventDisableTiming) == cudaSuccess;
    e->limit = ok ? ensemble_smem_limit() : 0;
    if (ok && e->limit > 0) ok = cudaMallocAsync((void **)&e->d_any_err, sizeof(uint32_t), e->stream) == cudaSuccess;
    if (ok && e->limit > 0) ok = cudaMemsetAsync(e->d_any_err, 0, sizeof(uint32_t), e->stream) == cudaSuccess;
    if (!ok || e->limit == 0) {
        cudaGetLastError();
        dpd_ensemble_destroy(e);
        return efail(nullptr, DPD_ERR_CUDA, "ensemble setup failed (no GPU, or kernel attributes refused)");
    }
    for (int c = 0; c < kClasses; ++c) {
        e->threads[c] = o.threads ? o.threads : default_threads(c);
        e->cluster[c] = o.cluster ? o.cluster : default_cluster(c);
    }
    *out = e;
    return DPD_OK;
}

int32_t dpd_ensemble_fits(const dpd_box_params *p, int64_t n)
{
    int nc[3];
    if (!check_params(p, n, nc).empty()) return 0;
    const size_t limit = ensemble_smem_limit();
    if (limit == 0) return 0;
    return footprint(n, nc[0] * nc[1] * nc[2], p->lambda == 0.5, 128) <= limit ? 1 : 0;
}

dpd_status dpd_ensemble_add(dpd_ensemble *e, const dpd_box_params *p, int64_t n, const double *x, const double *v,
                            const int32_t *species, uint64_t step, int32_t *id)
{
    if (!e || !x || !v || !id) return efail(e, DPD_ERR_ARG, "null argument");
    if (e->failed) return efail(e, DPD_ERR_CUDA, "ensemble is in a failed state: " + e->err);
    int nc[3];
    const std::string why = check_params(p, n, nc);
    if (!why.empty()) return efail(e, DPD_ERR_ARG, why);
    const int ncell = nc[0] * nc[1] * nc[2];
    const bool lhalf = p->lambda == 0.5;
    if (footprint(n, ncell, lhalf, 128) > e->limit)
        return efail(e, DPD_ERR_ARG, "box does not fit one CTA's shared memory (" + std::to_string(n) + " particles)");

    EBox b;
    b.id = e->next_id;
    b.n = n;
    b.step = step;
    std::memcpy(b.box, p->box, sizeof(b.box));
    fill_desc(b.desc, p, n, nc);
    b.cls = class_of(n, ncell, lhalf, e->limit);
    // one block: pos, vel, frc (float4), tag, pid (u32), err (16 B), descriptor, observables
    const size_t f4 = ens_align16((size_t)n * 16), u4 = ens_align16((size_t)n * 4);
    const size_t o_vel = f4, o_frc = 2 * f4, o_tag = 3 * f4, o_pid = o_tag + u4, o_err = o_pid + u4,
                 o_self = o_err + 16, o_obs = o_self + ens_align16(sizeof(EnsBox)), total = o_obs + 64;
    if (cudaMallocAsync(&b.mem, total, e->stream) != cudaSuccess) {
        cudaGetLastError();
        return efail(e, DPD_ERR_OOM, "device allocation of " + std::to_string(total) + " bytes failed");
    }
    char *m = (char *)b.mem;
    b.desc.pos = (float4 *)m;
    b.desc.vel = (float4 *)(m + o_vel);
    b.desc.frc = (float4 *)(m + o_frc);
    b.desc.tag = (const uint32_t *)(m + o_tag);
    b.pid = (uint32_t *)(m + o_pid);
    b.desc.err = (uint32_t *)(m + o_err);
    b.desc.any_err = e->d_any_err;
    b.d_self = (EnsBox *)(m + o_self);
    b.d_obs = (double *)(m + o_obs);

    // staged FP64 input, validated and converted on the device
    dpd_status st = DPD_OK;
    void *stage = nullptr;
    const size_t sx = (size_t)n * 3 * sizeof(double), ssp = species ? ens_align16((size_t)n * 4) : 0;
    auto cleanup = [&](dpd_status s, const std::string &msg) {
        if (stage) cudaFreeAsync(stage, e->stream);
        cudaFreeAsync(b.mem, e->stream);
        return efail(e, s, msg);
    };
    if (cudaMallocAsync(&stage, 2 * sx + ssp + 16, e->stream) != cudaSuccess) {
        cudaGetLastError();
        stage = nullptr;
        return cleanup(DPD_ERR_OOM, "staging allocation failed");
    }
    double *dx = (double *)stage, *dv = (double *)((char *)stage + sx);
    int32_t *dsp = species ? (int32_t *)((char *)stage + 2 * sx) : nullptr;
    uint32_t *bad = (uint32_t *)((char *)stage + 2 * sx + ssp);
    cudaError_t c = cudaMemcpyAsync(dx, x, sx, cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess) c = cudaMemcpyAsync(dv, v, sx, cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess && species) c = cudaMemcpyAsync(dsp, species, (size_t)n * 4, cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess) c = cudaMemsetAsync(bad, 0, 4, e->stream);
    if (c == cudaSuccess) c = launch_import_check(n, p->n_species, dx, dv, dsp, bad, e->stream);
    uint32_t hbad = 0;
    if (c == cudaSuccess) c = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, e->stream);
    if (c != cudaSuccess) {
        cudaGetLastError();
        return cleanup(DPD_ERR_CUDA, std::string("state upload: ") + cudaGetErrorString(c));
    }
    st = ewait(e);
    if (st) return cleanup(st, e->err);
    if (hbad & 1u) return cleanup(DPD_ERR_ARG, "non-finite position or velocity");
    if (hbad & 2u) return cleanup(DPD_ERR_ARG, "species out of range");
    SimParams P;
    std::memset(&P, 0, sizeof(P));
    for (int a = 0; a < 3; ++a) P.L[a] = (float)p->box[a];
    c = launch_import(P, p->box, n, dx, dv, dsp, nullptr, b.desc.pos, b.desc.vel, (uint32_t *)b.desc.tag, b.pid,
                      e->stream);
    if (c == cudaSuccess) c = cudaMemsetAsync(b.desc.frc, 0, f4, e->stream);
    if (c == cudaSuccess) c = cudaMemsetAsync(b.desc.err, 0, 16, e->stream);
    b.desc.step = step;
    if (c == cudaSuccess) c = cudaMemcpyAsync(b.d_self, &b.desc, sizeof(EnsBox), cudaMemcpyHostToDevice, e->stream);
    if (c != cudaSuccess) {
        cudaGetLastError();
        return cleanup(DPD_ERR_CUDA, std::string("state import: ") + cudaGetErrorString(c));
    }
    cudaFreeAsync(stage, e->stream);
    stage = nullptr;
    // the host copy in b.desc is read by cudaMemcpyAsync from pageable memory
    // (staged before the call returns), so b can move into the map
    *id = b.id;
    e->boxes[b.id] = b;
    e->next_id++;
    return DPD_OK;
}

dpd_status dpd_ensemble_remove(dpd_ensemble *e, int32_t id)
{
    if (!e) return efail(e, DPD_ERR_ARG, "null handle");
    auto it = e->boxes.find(id);
    if (it == e->boxes.end()) return efail(e, DPD_ERR_ARG, "unknown box id " + std::to_string(id));
    // ordered after every launch that reads the box: those were queued on the
    // class streams, which the handle's stream joined
    cudaFreeAsync(it->second.mem, e->stream);
    e->boxes.erase(it);
    return DPD_OK;
}

dpd_status dpd_ensemble_step(dpd_ensemble *e, const int32_t *ids, const int32_t *steps, int32_t m)
{
    if (!e || !steps || m < 0 || (m > 0 && !ids)) return efail(e, DPD_ERR_ARG, "bad arguments");
    if (e->failed) return efail(e, DPD_ERR_CUDA, "ensemble is in a failed state: " + e->err);
    // the requested steps per box
    std::map<int32_t, int> want;
    if (m == 0 && !ids) {
        if (steps[0] < 0) return efail(e, DPD_ERR_ARG, "steps must be >= 0");
        for (auto &kv : e->boxes) want[kv.first] = steps[0];
    } else {
        for (int32_t k = 0; k < m; ++k) {
            if (steps[k] < 0) return efail(e, DPD_ERR_ARG, "steps must be >= 0");
            if (!e->boxes.count(ids[k])) return efail(e, DPD_ERR_ARG, "unknown box id " + std::to_string(ids[k]));
            want[ids[k]] += steps[k];
        }
    }
    // groups by (class, kernel variant); init launches for new boxes first
    std::map<std::tuple<int, int, int>, Group> groups;
    for (auto &kv : want) {
        EBox &b = e->boxes[kv.first];
        if (kv.second == 0 && !b.need_init) continue;
        auto key = std::make_tuple(b.cls, b.desc.lhalf, b.desc.s_mode);
        Group &g = groups[key];
        g.cls = b.cls;
        g.lhalf = b.desc.lhalf != 0;
        g.s_mode = b.desc.s_mode;
        if (b.need_init) g.init.push_back(&b);
        if (kv.second > 0) {
            g.run.push_back(&b);
            g.run_steps.push_back(kv.second);
        }
    }
    if (groups.empty()) return DPD_OK;
    // descriptors: per group, the init boxes then the run boxes (largest first)
    std::vector<EnsBox> descs;
    struct Launch {
        int cls;
        bool lhalf;
        int s_mode;
        size_t off;
        int nb;
        Shape shape;
    };
    std::vector<Launch> launches;
    for (auto &kv : groups) {
        Group &g = kv.second;
        std::vector<size_t> order(g.run.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return g.run[a]->n > g.run[b]->n; });
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<const EBox *> bs;
            const size_t off = descs.size();
            if (pass == 0) {
                for (const EBox *b : g.init) {
                    EnsBox d = b->desc;
                    d.step = b->step;
                    d.steps = 0;
                    descs.push_back(d);
                    bs.push_back(b);
                }
            } else {
                for (size_t k : order) {
                    EnsBox d = g.run[k]->desc;
                    d.step = g.run[k]->step;
                    d.steps = g.run_steps[k];
                    descs.push_back(d);
                    bs.push_back(g.run[k]);
                }
            }
            if (bs.empty()) continue;
            Shape sh;
            if (!pick_shape(bs, g.lhalf, g.s_mode, e->opt.newton3 != 0, e->threads[g.cls], e->cluster[g.cls], e->limit,
                            sh))
                return efail(e, DPD_ERR_ARG, "no launch shape fits these boxes");
            launches.push_back({g.cls, g.lhalf, g.s_mode, off, (int)bs.size(), sh});
        }
    }
    dpd_status st = ensure_desc(e, descs.size());
    if (st) return st;
    ENS_TRY(e, cudaMemcpyAsync(e->d_desc, descs.data(), descs.size() * sizeof(EnsBox), cudaMemcpyHostToDevice, e->stream));
    // the launches read their descriptors (steps, step numbers) from d_desc,
    // so one captured graph serves every call with the same structure
    std::vector<uint64_t> key = {(uint64_t)(uintptr_t)e->d_desc, (uint64_t)descs.size(), (uint64_t)e->opt.newton3};
    for (const Launch &L : launches) {
        key.push_back((uint64_t)L.cls | ((uint64_t)L.lhalf << 8) | ((uint64_t)L.s_mode << 16) |
                      ((uint64_t)L.shape.cluster << 24) | ((uint64_t)L.shape.threads << 32));
        key.push_back((uint64_t)L.off | ((uint64_t)L.nb << 32));
        key.push_back((uint64_t)L.shape.smem);
    }
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t err = cudaEventRecord(e->fork, e->stream);
        bool used[kClasses] = {false, false, false, false};
        for (const Launch &L : launches) {
            if (err != cudaSuccess) break;
            cudaStream_t s = e->cls_stream[L.cls];
            if (!used[L.cls]) {
                err = cudaStreamWaitEvent(s, e->fork, 0);
                used[L.cls] = true;
            }
            if (err == cudaSuccess)
                err = launch_ensemble(e->d_desc + L.off, L.nb, L.lhalf, L.s_mode, e->opt.newton3 != 0,
                                      L.shape.threads, L.shape.cluster, L.shape.smem, s);
        }
        for (int c = 0; c < kClasses && err == cudaSuccess; ++c)
            if (used[c]) {
                err = cudaEventRecord(e->join[c], e->cls_stream[c]);
                if (err == cudaSuccess) err = cudaStreamWaitEvent(e->stream, e->join[c], 0);
            }
        return err;
    };
    if (!(e->graph && key == e->graph_key)) {
        if (e->graph) cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
        e->graph_key.clear();
        cudaGraph_t g = nullptr;
        ENS_TRY(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ce = enqueue();
        const cudaError_t ee = cudaStreamEndCapture(e->stream, &g);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return efail(e, DPD_ERR_CUDA, std::string("graph capture of the ensemble launches: ") +
                                              cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        const cudaError_t ie = cudaGraphInstantiate(&e->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            e->graph = nullptr;
            return efail(e, DPD_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        }
        e->graph_key = key;
        e->graph_captures += 1;
    } else {
        e->graph_replays += 1;
    }
    ENS_TRY(e, cudaGraphLaunch(e->graph, e->stream));
    for (auto &kv : groups) {
        Group &g = kv.second;
        for (const EBox *b : g.init) const_cast<EBox *>(b)->need_init = false;
        for (size_t k = 0; k < g.run.size(); ++k) const_cast<EBox *>(g.run[k])->step += (uint64_t)g.run_steps[k];
    }
    return DPD_OK;
}

dpd_status dpd_ensemble_sync(dpd_ensemble *e)
{
    if (!e) return efail(e, DPD_ERR_ARG, "null handle");
    if (e->failed) return efail(e, DPD_ERR_CUDA, "ensemble is in a failed state: " + e->err);
    uint32_t any = 0;
    ENS_TRY(e, cudaMemcpyAsync(&any, e->d_any_err, 4, cudaMemcpyDeviceToHost, e->stream));
    dpd_status st = ewait(e);
    if (st) return st;
    if (!any) return DPD_OK;
    std::string which;
    for (auto &kv : e->boxes) {
        uint32_t w = 0;
        ENS_TRY(e, cudaMemcpyAsync(&w, kv.second.desc.err, 4, cudaMemcpyDeviceToHost, e->stream));
        st = ewait(e);
        if (st) return st;
        if (w) which += (which.empty() ? "" : ", ") + std::to_string(kv.first);
    }
    ENS_TRY(e, cudaMemsetAsync(e->d_any_err, 0, 4, e->stream));
    if (any & kErrBadIndex)
        return efail(e, DPD_ERR_STATE, "internal error: a pair index out of range in box(es) " + which);
    return efail(e, DPD_ERR_NONFINITE, "non-finite force in box(es) " + which);
}

dpd_status dpd_ensemble_get_state(dpd_ensemble *e, int32_t id, double *x, double *v, uint64_t *step)
{
    if (!e) return efail(e, DPD_ERR_ARG, "null handle");
    auto it = e->boxes.find(id);
    if (it == e->boxes.end()) return efail(e, DPD_ERR_ARG, "unknown box id " + std::to_string(id));
    const EBox &b = it->second;
    if (x || v) {
        // a box never stepped since its addition still needs its initial force
        // only for stepping; its state is the loaded one
        const size_t bytes = (size_t)b.n * 3 * sizeof(double);
        void *stage = nullptr;
        if (cudaMallocAsync(&stage, 2 * bytes, e->stream) != cudaSuccess) {
            cudaGetLastError();
            return efail(e, DPD_ERR_OOM, "staging allocation failed");
        }
        double *dx = (double *)stage, *dv = (double *)((char *)stage + bytes);
        cudaError_t c = cudaSuccess;
        if (x) c = launch_export(b.n, b.desc.pos, b.pid, dx, e->stream);
        if (c == cudaSuccess && v) c = launch_export(b.n, b.desc.vel, b.pid, dv, e->stream);
        if (c == cudaSuccess && x) c = cudaMemcpyAsync(x, dx, bytes, cudaMemcpyDeviceToHost, e->stream);
        if (c == cudaSuccess && v) c = cudaMemcpyAsync(v, dv, bytes, cudaMemcpyDeviceToHost, e->stream);
        cudaFreeAsync(stage, e->stream);
        if (c != cudaSuccess) {
            cudaGetLastError();
            return efail(e, DPD_ERR_CUDA, std::string("state download: ") + cudaGetErrorString(c));
        }
        dpd_status st = ewait(e);
        if (st) return st;
    }
    if (step) *step = b.step;
    return DPD_OK;
}

dpd_status dpd_ensemble_get_forces(dpd_ensemble *e, int32_t id, double *f)
{
    if (!e || !f) return efail(e, DPD_ERR_ARG, "null argument");
    auto it = e->boxes.find(id);
    if (it == e->boxes.end()) return efail(e, DPD_ERR_ARG, "unknown box id " + std::to_string(id));
    if (it->second.need_init) {
        const int32_t zero = 0;
        dpd_status st = dpd_ensemble_step(e, &id, &zero, 1);
        if (st) return st;
    }
    const EBox &b = it->second;
    const size_t bytes = (size_t)b.n * 3 * sizeof(double);
    void *stage = nullptr;
    if (cudaMallocAsync(&stage, bytes, e->stream) != cudaSuccess) {
        cudaGetLastError();
        return efail(e, DPD_ERR_OOM, "staging allocation failed");
    }
    cudaError_t c = launch_export(b.n, b.desc.frc, b.pid, (double *)stage, e->stream);
    if (c == cudaSuccess) c = cudaMemcpyAsync(f, stage, bytes, cudaMemcpyDeviceToHost, e->stream);
    cudaFreeAsync(stage, e->stream);
    if (c != cudaSuccess) {
        cudaGetLastError();
        return efail(e, DPD_ERR_CUDA, std::string("force download: ") + cudaGetErrorString(c));
    }
    return ewait(e);
}

dpd_status dpd_ensemble_observables(dpd_ensemble *e, int32_t id, dpd_obs *out)
{
    if (!e || !out) return efail(e, DPD_ERR_ARG, "null argument");
    auto it = e->boxes.find(id);
    if (it == e->boxes.end()) return efail(e, DPD_ERR_ARG, "unknown box id " + std::to_string(id));
    if (it->second.need_init) {  // the virial comes from the force evaluation
        const int32_t zero = 0;
        dpd_status st = dpd_ensemble_step(e, &id, &zero, 1);
        if (st) return st;
    }
    const EBox &b = it->second;
    double h[8];
    ENS_TRY(e, launch_ensemble_observe(b.d_self, 1, b.d_obs, e->stream));
    ENS_TRY(e, cudaMemcpyAsync(h, b.d_obs, sizeof(h), cudaMemcpyDeviceToHost, e->stream));
    dpd_status st = ewait(e);
    if (st) return st;
    const double V = b.box[0] * b.box[1] * b.box[2];
    out->step = b.step;
    out->n = b.n;
    out->kinetic = 0.5 * h[0];
    out->temperature = b.n > 1 ? h[0] / (3.0 * b.n - 3.0) : 0.0;
    out->virial = h[1];
    out->pressure = (h[0] + h[1]) / (3.0 * V);
    out->momentum[0] = h[2];
    out->momentum[1] = h[3];
    out->momentum[2] = h[4];
    return DPD_OK;
}

dpd_status dpd_ensemble_graph_stats(dpd_ensemble *e, int64_t *captures, int64_t *replays)
{
    if (!e) return efail(e, DPD_ERR_ARG, "null handle");
    if (captures) *captures = e->graph_captures;
    if (replays) *replays = e->graph_replays;
    return DPD_OK;
}

dpd_status dpd_ensemble_info(dpd_ensemble *e, int32_t *nboxes, int64_t *nparticles)
{
    if (!e) return efail(e, DPD_ERR_ARG, "null handle");
    int64_t np = 0;
    for (auto &kv : e->boxes) np += kv.second.n;
    if (nboxes) *nboxes = (int32_t)e->boxes.size();
    if (nparticles) *nparticles = np;
    return DPD_OK;
}

dpd_status dpd_ensemble_tune(dpd_ensemble *e, int32_t steps, double *table)
{
    if (!e || steps < 1) return efail(e, DPD_ERR_ARG, "bad arguments");
    if (e->failed) return efail(e, DPD_ERR_CUDA, "ensemble is in a failed state: " + e->err);
    // initial forces first, so every scratch copy starts from a complete state
    {
        std::vector<int32_t> ids;
        for (auto &kv : e->boxes)
            if (kv.second.need_init) ids.push_back(kv.first);
        if (!ids.empty()) {
            std::vector<int32_t> zeros(ids.size(), 0);
            dpd_status st = dpd_ensemble_step(e, ids.data(), zeros.data(), (int32_t)ids.size());
            if (st) return st;
        }
    }
    dpd_status st = ewait(e);
    if (st) return st;
    for (int cls = 0; cls < kClasses; ++cls) {
        // this class's boxes, grouped by kernel variant; scratch state for each
        std::map<std::pair<int, int>, std::vector<const EBox *>> vars;
        for (auto &kv : e->boxes)
            if (kv.second.cls == cls) vars[{kv.second.desc.lhalf, kv.second.desc.s_mode}].push_back(&kv.second);
        if (vars.empty()) continue;
        std::vector<EnsBox> descs;
        std::vector<std::pair<size_t, int>> spans;  // (offset, count) per variant
        std::vector<void *> scratch;
        bool ok = true;
        for (auto &kv : vars) {
            spans.push_back({descs.size(), (int)kv.second.size()});
            for (const EBox *b : kv.second) {
                void *mem = nullptr;
                const size_t f4 = ens_align16((size_t)b->n * 16);
                if (cudaMallocAsync(&mem, 3 * f4 + 16, e->stream) != cudaSuccess) {
                    cudaGetLastError();
                    ok = false;
                    break;
                }
                scratch.push_back(mem);
                EnsBox d = b->desc;
                d.pos = (float4 *)mem;
                d.vel = (float4 *)((char *)mem + f4);
                d.frc = (float4 *)((char *)mem + 2 * f4);
                d.err = (uint32_t *)((char *)mem + 3 * f4);
                d.any_err = d.err;  // scratch runs report nothing to the ensemble
                d.step = b->step;
                d.steps = steps;
                descs.push_back(d);
            }
            if (!ok) break;
        }
        auto release = [&]() {
            for (void *p : scratch) cudaFreeAsync(p, e->stream);
            scratch.clear();
        };
        // a CUDA failure inside the timing loop: scratch back to the pool, then report
#define TUNE_TRY(call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            release();                                                                                 \
            return efail(e, DPD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
        }                                                                                              \
    } while (0)
        if (!ok) {
            release();
            return efail(e, DPD_ERR_OOM, "tuner scratch allocation failed");
        }
        st = ensure_desc(e, descs.size());
        if (st) {
            release();
            return st;
        }
        TUNE_TRY(cudaMemcpyAsync(e->d_desc, descs.data(), descs.size() * sizeof(EnsBox), cudaMemcpyHostToDevice,
                                   e->stream));
        double best = std::numeric_limits<double>::infinity();
        int best_t = e->threads[cls], best_c = e->cluster[cls];
        double tab[12];
        for (int ti = 0; ti < 3; ++ti)
            for (int ci = 0; ci < 4; ++ci) {
                const int T = kThreadChoices[ti], C = kClusterChoices[ci];
                tab[ti * 4 + ci] = std::numeric_limits<double>::infinity();
                std::vector<Shape> shapes;
                size_t k = 0;
                bool feasible = true;
                for (auto &kv : vars) {
                    Shape sh;
                    if (!shape_for(kv.second, kv.first.first != 0, kv.first.second, e->opt.newton3 != 0, T, C, e->limit,
                                   sh))
                        feasible = false;
                    shapes.push_back(sh);
                    ++k;
                }
                if (!feasible) continue;
                // fresh copies of the current state, then one warm-up and one timed chunk
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {
                    size_t j = 0;
                    for (auto &kv : vars)
                        for (const EBox *b : kv.second) {
                            const size_t f4 = ens_align16((size_t)b->n * 16);
                            TUNE_TRY(cudaMemcpyAsync(scratch[j], b->desc.pos, f4, cudaMemcpyDeviceToDevice, e->stream));
                            TUNE_TRY(cudaMemcpyAsync((char *)scratch[j] + f4, b->desc.vel, f4, cudaMemcpyDeviceToDevice,
                                                       e->stream));
                            TUNE_TRY(cudaMemcpyAsync((char *)scratch[j] + 2 * f4, b->desc.frc, f4,
                                                       cudaMemcpyDeviceToDevice, e->stream));
                            ++j;
                        }
                    TUNE_TRY(cudaEventRecord(e->t0, e->stream));
                    size_t v = 0;
                    for (auto &kv : vars) {
                        TUNE_TRY(launch_ensemble(e->d_desc + spans[v].first, spans[v].second, kv.first.first != 0,
                                                   kv.first.second, e->opt.newton3 != 0, shapes[v].threads,
                                                   shapes[v].cluster, shapes[v].smem, e->stream));
                        ++v;
                    }
                    TUNE_TRY(cudaEventRecord(e->t1, e->stream));
                    st = ewait(e);
                    if (st) {
                        release();
                        return st;
                    }
                    TUNE_TRY(cudaEventElapsedTime(&ms, e->t0, e->t1));
                }
                tab[ti * 4 + ci] = (double)ms / steps;
                if (tab[ti * 4 + ci] < best) {
                    best = tab[ti * 4 + ci];
                    best_t = T;
                    best_c = C;
                }
            }
        release();
#undef TUNE_TRY
        if (table) std::memcpy(table, tab, sizeof(tab));
        e->threads[cls] = best_t;
        e->cluster[cls] = best_c;
    }
    e->tuned = true;
    return ewait(e);
}

dpd_status dpd_ensemble_config(dpd_ensemble *e, int32_t threads[4], int32_t cluster[4])
{
    if (!e || !threads || !cluster) return efail(e, DPD_ERR_ARG, "null argument");
    bool present[kClasses] = {false, false, false, false};
    for (auto &kv : e->boxes) present[kv.second.cls] = true;
    for (int c = 0; c < kClasses; ++c) {
        threads[c] = present[c] ? e->threads[c] : 0;
        cluster[c] = present[c] ? e->cluster[c] : 0;
    }
    return DPD_OK;
}

void dpd_ensemble_destroy(dpd_ensemble *e)
{
    if (!e) return;
    // a step that failed after forking may have left launches on the class
    // streams that the handle's stream never joined: let them finish first
    for (int c = 0; c < kClasses; ++c)
        if (e->cls_stream[c]) cudaStreamSynchronize(e->cls_stream[c]);
    if (e->stream) {
        for (auto &kv : e->boxes) cudaFreeAsync(kv.second.mem, e->stream);
        if (e->d_desc) cudaFreeAsync(e->d_desc, e->stream);
        if (e->d_any_err) cudaFreeAsync(e->d_any_err, e->stream);
        cudaStreamSynchronize(e->stream);
    }
    for (int c = 0; c < kClasses; ++c) {
        if (e->cls_stream[c]) cudaStreamDestroy(e->cls_stream[c]);
        if (e->join[c]) cudaEventDestroy(e->join[c]);
    }
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->ev) cudaEventDestroy(e->ev);
    if (e->t0) cudaEventDestroy(e->t0);
    if (e->t1) cudaEventDestroy(e->t1);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    cudaGetLastError();
    delete e;
}

const char *dpd_ensemble_last_error(dpd_ensemble *e)
{
    return e ? e->err.c_str() : g_ens_error.c_str();
}

}  // extern "C"
