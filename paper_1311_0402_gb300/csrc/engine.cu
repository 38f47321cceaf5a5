// engine.cu -- host engine and C ABI of libdpd.so (declared in dpd.h).
//
// Owns the device memory of a simulation, builds the cell geometry (Morton
// ranks of the cells and the ascending 27-cell stencils, built once, as the
// coarse stencil of Sec. 3.3.1), uploads and downloads particle state in the
// caller's order, and drives the per-step kernel sequence of Algorithm 1:
//   phase 1 (+ signature, displacement check) -> rebuild chain (runs only
//   when flagged on the device) -> pair force -> phase 2,
// captured into CUDA graphs of several steps that are replayed, so a step
// costs no host round trip.  Host waits poll an event with a deadline.
#include "dpd.h"
#include "dpd_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

using namespace dpd;

namespace {

thread_local std::string g_last_error;

struct Geometry {
    int nc[3];
    int ncell;
    std::vector<uint32_t> rank_of_cell;  // linear (cz, cy, cx) -> rank
    std::vector<uint32_t> stencil;       // [ncell][27]
    int nb[3] = {0, 0, 0};               // bricks per axis
    std::vector<uint32_t> brick_lo, brick_hi;  // first / last Morton rank of each brick
    std::vector<uint32_t> brick_ord;           // position of each brick in ascending rank order
};

uint32_t spread3(uint32_t v)  // 10 bits -> every third bit
{
    uint32_t x = v & 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

void build_geometry(const int nc[3], Geometry &g)
{
    g.nc[0] = nc[0]; g.nc[1] = nc[1]; g.nc[2] = nc[2];
    g.ncell = nc[0] * nc[1] * nc[2];
    std::vector<std::pair<uint64_t, uint32_t>> order(g.ncell);
    for (int z = 0; z < nc[2]; ++z)
        for (int y = 0; y < nc[1]; ++y)
            for (int x = 0; x < nc[0]; ++x) {
                uint32_t lin = (uint32_t)((z * nc[1] + y) * nc[0] + x);
                uint64_t code = (uint64_t)spread3((uint32_t)x) | ((uint64_t)spread3((uint32_t)y) << 1) |
                                ((uint64_t)spread3((uint32_t)z) << 2);
                order[lin] = {code, lin};
            }
    std::sort(order.begin(), order.end());
    g.rank_of_cell.assign(g.ncell, 0);
    std::vector<uint32_t> lin_of_rank(g.ncell);
    for (int r = 0; r < g.ncell; ++r) {
        g.rank_of_cell[order[r].second] = (uint32_t)r;
        lin_of_rank[r] = order[r].second;
    }
    // distinct neighbour offsets per axis ({-1,0,1}, or fewer when an axis
    // has fewer than three cells so no cell is listed twice)
    std::vector<int> off[3];
    for (int a = 0; a < 3; ++a) {
        if (nc[a] >= 3) off[a] = {-1, 0, 1};
        else if (nc[a] == 2) off[a] = {0, 1};
        else off[a] = {0};
    }
    g.stencil.assign((size_t)g.ncell * kStencil, kNone);
    std::vector<uint32_t> tmp;
    for (int r = 0; r < g.ncell; ++r) {
        uint32_t lin = lin_of_rank[r];
        int x = lin % nc[0], y = (lin / nc[0]) % nc[1], z = lin / (nc[0] * nc[1]);
        tmp.clear();
        for (int oz : off[2])
            for (int oy : off[1])
                for (int ox : off[0]) {
                    int cx = (x + ox + nc[0]) % nc[0], cy = (y + oy + nc[1]) % nc[1], cz = (z + oz + nc[2]) % nc[2];
                    tmp.push_back(g.rank_of_cell[(cz * nc[1] + cy) * nc[0] + cx]);
                }
        std::sort(tmp.begin(), tmp.end());
        std::copy(tmp.begin(), tmp.end(), g.stencil.begin() + (size_t)r * kStencil);
    }
    // aligned kBrick^3 blocks of cells: consecutive Morton ranks
    for (int a = 0; a < 3; ++a) g.nb[a] = (nc[a] + kBrick - 1) / kBrick;
    const int nbricks = g.nb[0] * g.nb[1] * g.nb[2];
    g.brick_lo.assign(nbricks, 0xFFFFFFFFu);
    g.brick_hi.assign(nbricks, 0u);
    for (int z = 0; z < nc[2]; ++z)
        for (int y = 0; y < nc[1]; ++y)
            for (int x = 0; x < nc[0]; ++x) {
                const int b = ((z / kBrick) * g.nb[1] + y / kBrick) * g.nb[0] + x / kBrick;
                const uint32_t r = g.rank_of_cell[(z * nc[1] + y) * nc[0] + x];
                g.brick_lo[b] = std::min(g.brick_lo[b], r);
                g.brick_hi[b] = std::max(g.brick_hi[b], r);
            }
    // the bricks partition the rank range into consecutive intervals; their
    // order along it numbers the group lists
    std::vector<std::pair<uint32_t, int>> by_rank(nbricks);
    for (int b = 0; b < nbricks; ++b) by_rank[b] = {g.brick_lo[b], b};
    std::sort(by_rank.begin(), by_rank.end());
    g.brick_ord.assign(nbricks, 0u);
    for (int k = 0; k < nbricks; ++k) g.brick_ord[by_rank[k].second] = (uint32_t)k;
}

}  // namespace

struct dpd_sim {
    // parameters
    double box[3];
    int n_species;
    std::vector<double> a;
    double gamma, kT, rc, s, dt;
    dpd_options opt;
    SimParams P;
    Ptrs D;
    Geometry geo;
    int n_scan_blocks = 0;
    // device memory
    std::vector<void *> allocs;        // per-n allocations
    std::vector<void *> static_allocs; // geometry + control
    int64_t n = 0;
    int64_t cap_alloc_n = -1;
    size_t red_doubles = 0;
    bool has_state = false;
    bool failed = false;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;             // captures the bodies of conditional graph nodes
    bool own_stream = false;
    cudaEvent_t ev = nullptr;
    std::map<int, cudaGraphExec_t> graphs;  // steps per graph -> executable
    std::map<int64_t, cudaGraphExec_t> timed_graphs;  // profiled runs, by steps
    std::vector<cudaEvent_t> tev;           // timing events
    uint64_t step = 0;                       // host mirror of the device step
    bool pending = false;                    // steps queued by dpd_step_async not yet checked by dpd_sync
    std::string err;
    std::vector<uint32_t> bond_partner_host;
    bool bonds_set = false;
};

namespace {

// An NVTX range over one API call, for profilers that record NVTX (the
// kernels of the call appear inside it on the timeline).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

dpd_status fail(dpd_sim *h, dpd_status st, const std::string &msg)
{
    if (h) {
        h->err = msg;
        if (st == DPD_ERR_CUDA) h->failed = true;
    }
    g_last_error = msg;
    return st;
}

#define CUDA_TRY(h, call)                                                                             \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail((h), DPD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// handle's stream, from the device's default pool): creating and destroying a
// handle never synchronises the whole device, so handles on other streams
// keep running (the serving loop relies on this).
// Keep freed stream-ordered memory in this process's pool of the current
// device instead of returning it at every synchronisation, so that handles
// created after others were destroyed reuse it without new mappings.
void keep_pool_memory()
{
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    uint64_t threshold = UINT64_MAX;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold) != cudaSuccess) cudaGetLastError();
}

// Host-side allocation-failure injection for the failure tests: while the
// environment variable DPD_TEST_FAIL_ALLOC is "1", every device allocation a
// handle asks for reports failure without reaching the allocator, so the
// out-of-memory paths run with no GPU fault and no real memory pressure.
bool alloc_refused()
{
    const char *e = std::getenv("DPD_TEST_FAIL_ALLOC");
    return e && e[0] == '1' && e[1] == '\0';
}

dpd_status dev_alloc(dpd_sim *h, void **p, size_t bytes, std::vector<void *> &list)
{
    if (bytes == 0) bytes = 16;
    if (alloc_refused())
        return fail(h, DPD_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes refused (DPD_TEST_FAIL_ALLOC)");
    cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, DPD_ERR_OOM, std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    list.push_back(*p);
    return DPD_OK;
}

void dev_free(dpd_sim *h, void *p, std::vector<void *> &list)
{
    auto it = std::find(list.begin(), list.end(), p);
    if (it != list.end()) list.erase(it);
    cudaFreeAsync(p, h->stream);
}

// Scratch device memory for one call, stream-ordered, freed (back to the
// pool) when the call returns.
struct Staging {
    dpd_sim *h;
    std::vector<void *> blocks;
    cudaError_t err = cudaSuccess;
    explicit Staging(dpd_sim *hh) : h(hh) {}
    void *get(size_t bytes)
    {
        void *p = nullptr;
        if (err == cudaSuccess && alloc_refused()) err = cudaErrorMemoryAllocation;
        if (err == cudaSuccess) err = cudaMallocAsync(&p, bytes ? bytes : 16, h->stream);
        if (err != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        blocks.push_back(p);
        return p;
    }
    bool ok() const { return err == cudaSuccess; }
    std::string error() const { return cudaGetErrorString(err); }
    ~Staging()
    {
        for (void *p : blocks) cudaFreeAsync(p, h->stream);
    }
};

void free_list(dpd_sim *h, std::vector<void *> &list)
{
    for (void *p : list) cudaFreeAsync(p, h->stream);
    list.clear();
}

// Wait for the stream with a deadline (no unbounded host spin).
dpd_status wait(dpd_sim *h)
{
    cudaError_t e = cudaEventRecord(h->ev, h->stream);
    if (e != cudaSuccess) return fail(h, DPD_ERR_CUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
    auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        e = cudaEventQuery(h->ev);
        if (e == cudaSuccess) return DPD_OK;
        if (e != cudaErrorNotReady) return fail(h, DPD_ERR_CUDA, std::string("kernel failure: ") + cudaGetErrorString(e));
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > h->opt.wait_timeout_s)
            return fail(h, DPD_ERR_TIMEOUT, "GPU did not finish within " + std::to_string(h->opt.wait_timeout_s) + " s");
        if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

dpd_status read_ctl(dpd_sim *h, DevCtl &c)
{
    CUDA_TRY(h, cudaMemcpyAsync(&c, h->D.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
    return wait(h);
}

dpd_status check_err(dpd_sim *h, DevCtl &c)
{
    dpd_status st = read_ctl(h, c);
    if (st) return st;
    if (c.err & kErrNbrOverflow)
        return fail(h, DPD_ERR_NBR_OVERFLOW,
                    "neighbour list overflow: a group list of " + std::to_string(c.max_nnb) + " entries > capacity " +
                        std::to_string(h->P.gcap));
    if (c.err & kErrNonFinite) return fail(h, DPD_ERR_NONFINITE, "non-finite force");
    if (c.err & kErrTimeout) return fail(h, DPD_ERR_TIMEOUT, "a device-side wait for staged data ran out");
    if (c.err & kErrBadIndex)
        return fail(h, DPD_ERR_STATE, "a kernel met a list entry outside the particle range (the access was skipped)");
    return DPD_OK;
}

void drop_graphs(dpd_sim *h)
{
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    for (auto &kv : h->timed_graphs) cudaGraphExecDestroy(kv.second);
    h->timed_graphs.clear();
}

constexpr int kRebuildKernels = 9;  // bin, 3 scan, scatter, rank, gather, commit, nbuild

// Timing event on the stream; inside a graph capture it becomes an event
// record node whose timestamp stays readable after the graph runs.
// event record flags: external during stream capture (so the graph keeps
// the records as timing nodes), plain otherwise
unsigned int rec_flags(dpd_sim *h)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return 0u;
    return cs == cudaStreamCaptureStatusActive ? (unsigned int)cudaEventRecordExternal : 0u;
}

cudaError_t rec(dpd_sim *h, cudaEvent_t e) { return cudaEventRecordWithFlags(e, h->stream, rec_flags(h)); }

// Rebuild chains inside captured graphs.  Each step's chain sits in the
// body of a conditional IF node whose handle the preceding advance kernel
// sets from the device rebuild flag, so a step without a rebuild launches
// none of the chain's kernels (outside graphs the chain is launched and its
// kernels return at once when the flag is clear).  The handles default to 1
// at every launch of the graph: an unset handle runs the chain, which still
// checks the flag itself.
struct CondCapture {
    bool active = false;
    std::vector<cudaGraphConditionalHandle> handles;  // one per step
    std::vector<cudaGraph_t> bodies;                  // IF bodies, filled after the capture
};

cudaError_t cond_begin(dpd_sim *h, int64_t k, CondCapture &cc)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cc.handles.assign((size_t)k, 0);
    for (int64_t s = 0; s < k && e == cudaSuccess; ++s)
        e = cudaGraphConditionalHandleCreate(&cc.handles[(size_t)s], g, 1u, cudaGraphCondAssignDefault);
    cc.active = e == cudaSuccess;
    return e;
}

NextCond next_cond(const CondCapture &cc, int64_t s)
{
    if (!cc.active || s >= (int64_t)cc.handles.size()) return NextCond{0, 0};
    return NextCond{cc.handles[(size_t)s], 1};
}

// The rebuild chain of step s: an IF node under capture, the chain otherwise.
cudaError_t rebuild_step(dpd_sim *h, CondCapture &cc, int64_t s)
{
    if (!cc.active) return launch_rebuild(h->P, h->D, h->stream, h->n_scan_blocks);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, &edata, &ndeps);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = cc.handles[(size_t)s];
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, edata, ndeps, &np);
    if (e != cudaSuccess) return e;
    cc.bodies.push_back(np.conditional.phGraph_out[0]);
    return cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// After the capture: each IF body gets the rebuild chain, captured on the
// handle's side stream.
cudaError_t cond_fill(dpd_sim *h, CondCapture &cc)
{
    for (cudaGraph_t body : cc.bodies) {
        cudaError_t e = cudaStreamBeginCaptureToGraph(h->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        e = launch_rebuild(h->P, h->D, h->side, h->n_scan_blocks);
        cudaGraph_t out = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->side, &out);
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
    }
    return cudaSuccess;
}

// The kernel sequence of enqueue_steps with timing events between the
// groups: ev[0] | phase 1 | ev[1] | rebuild | ev[2] | pair kernel | ev[3] |
// settle + advance | ev[4] | rebuild | ev[5] ...  (3 events per step)
cudaError_t enqueue_steps_timed(dpd_sim *h, int64_t k, CondCapture &cc)
{
    cudaError_t e = rec(h, h->tev[0]);
    if (e == cudaSuccess) e = launch_phase1(h->P, h->D, h->stream, next_cond(cc, 0));
    if (e == cudaSuccess) e = rec(h, h->tev[1]);
    const unsigned int fl = rec_flags(h);
    for (int64_t s = 0; s < k && e == cudaSuccess; ++s) {
        e = rebuild_step(h, cc, s);
        if (e == cudaSuccess) e = rec(h, h->tev[3 * s + 2]);
        if (e == cudaSuccess)
            e = launch_force(h->P, h->D, s + 1 < k ? kForceStep : kForceFinish, false, h->stream, h->tev[3 * s + 3], fl,
                             next_cond(cc, s + 1));
        if (e == cudaSuccess) e = rec(h, h->tev[3 * s + 4]);
    }
    return e;
}

// Kernel sequence of k steps (starting and ending at a full-step state):
// phase 1, then per step the rebuild chain (runs only when flagged), the
// pair kernel and the integration into the next step (or the finish of the
// last).
cudaError_t enqueue_steps(dpd_sim *h, int64_t k, CondCapture &cc)
{
    cudaError_t e = launch_phase1(h->P, h->D, h->stream, next_cond(cc, 0));
    for (int64_t s = 0; s < k && e == cudaSuccess; ++s) {
        e = rebuild_step(h, cc, s);
        if (e == cudaSuccess)
            e = launch_force(h->P, h->D, s + 1 < k ? kForceStep : kForceFinish, false, h->stream, nullptr, 0,
                             next_cond(cc, s + 1));
    }
    return e;
}

// Capture k steps (timed: with the events of enqueue_steps_timed) into an
// executable graph.
dpd_status capture_steps(dpd_sim *h, int64_t k, bool timed, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    CondCapture cc;
    cudaError_t e = h->opt.conditional_rebuild ? cond_begin(h, k, cc) : cudaSuccess;
    if (e == cudaSuccess) e = timed ? enqueue_steps_timed(h, k, cc) : enqueue_steps(h, k, cc);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) e = cond_fill(h, cc);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(h, DPD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, DPD_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    *out = ex;
    return DPD_OK;
}

dpd_status get_graph(dpd_sim *h, int k, cudaGraphExec_t *out)
{
    auto it = h->graphs.find(k);
    if (it != h->graphs.end()) {
        *out = it->second;
        return DPD_OK;
    }
    cudaGraphExec_t ex = nullptr;
    dpd_status st = capture_steps(h, k, false, &ex);
    if (st) return st;
    h->graphs[k] = ex;
    *out = ex;
    return DPD_OK;
}

// Group lists: with bricks, brick b's groups take ids from lo_b / 32 +
// ord(b), so n / 32 + nbricks ids cover every brick; otherwise 32-aligned
// tiles.
int group_count(const dpd_sim *h, int64_t n)
{
    return h->P.use_bricks ? (int)(n / kGroup) + h->P.nbricks : (int)((n + kGroup - 1) / kGroup);
}

// per-particle capacity from the largest group total of a build
int capacity_for_total(uint32_t max_total)
{
    int cap = (int)(((uint64_t)max_total * 5 / 4 + 64 + kGroup - 1) / kGroup);
    return std::max((cap + 7) / 8 * 8, 32);
}

int auto_capacity(const dpd_sim *h, int64_t n)
{
    double V = h->box[0] * h->box[1] * h->box[2];
    double rl = h->rc + h->opt.skin;
    double mean = (double)n / V * 4.0 / 3.0 * M_PI * rl * rl * rl;
    int cap = (int)std::ceil(1.6 * mean + 24.0);
    cap = (cap + 7) / 8 * 8;
    return std::max(cap, 32);
}

dpd_status alloc_particles(dpd_sim *h, int64_t n, int cap)
{
    drop_graphs(h);
    free_list(h, h->allocs);
    Ptrs &D = h->D;
    const size_t f4 = sizeof(float4) * (size_t)n, u4 = sizeof(uint32_t) * (size_t)n;
    dpd_status st = DPD_OK;
    auto A = [&](void **p, size_t b) { if (st == DPD_OK) st = dev_alloc(h, p, b, h->allocs); };
    for (int b = 0; b < 2; ++b) {
        A((void **)&D.pos[b], f4);
        A((void **)&D.vel[b], f4);
        A((void **)&D.force[b], f4);
        A((void **)&D.tag[b], u4);
        A((void **)&D.pid[b], u4);
        if (!h->P.lambda_half) A((void **)&D.vkick[b], f4);
        else D.vkick[b] = nullptr;
    }
    A((void **)&D.xref, f4);
    A((void **)&D.fout, f4);
    A((void **)&D.facc[0], f4);
    A((void **)&D.facc[1], f4);
    A((void **)&D.key, u4);
    A((void **)&D.slot, u4);
    A((void **)&D.tmp_idx, u4);
    A((void **)&D.skey, sizeof(unsigned long long) * (size_t)n);
    A((void **)&D.perm, u4);
    A((void **)&D.idx_of_pid, u4);
    h->P.ngroups = group_count(h, n);
    A((void **)&D.gdesc, sizeof(uint2) * (size_t)h->P.ngroups);
    A((void **)&D.rowcnt, u4);
    A((void **)&D.nbr, (size_t)h->P.ngroups * kGroup * (size_t)cap * sizeof(uint32_t));
    h->red_doubles = std::max<size_t>((size_t)observe_blocks_for((int)n) * 8 + 8, 4096);
    A((void **)&D.vir_part, sizeof(double) * (size_t)((h->P.ngroups + kForceWarps - 1) / kForceWarps));
    A((void **)&D.red, h->red_doubles * sizeof(double));
    A((void **)&D.bond_partner, sizeof(uint32_t) * (size_t)n * kMaxBonds);
    if (st) return st;
    CUDA_TRY(h, cudaMemsetAsync((void *)D.bond_partner, 0xFF, sizeof(uint32_t) * (size_t)n * kMaxBonds, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(D.gdesc, 0, sizeof(uint2) * (size_t)h->P.ngroups, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(D.rowcnt, 0, u4, h->stream));
    // partials of a pair kernel launched with fewer blocks than the largest count stay zero
    CUDA_TRY(h, cudaMemsetAsync(D.vir_part, 0, sizeof(double) * (size_t)((h->P.ngroups + kForceWarps - 1) / kForceWarps),
                                h->stream));
    for (int b = 0; b < 2; ++b) CUDA_TRY(h, cudaMemsetAsync(D.facc[b], 0, f4, h->stream));
    h->P.cap = cap;
    h->P.gcap = kGroup * cap;
    h->cap_alloc_n = n;
    return DPD_OK;
}

// Force a rebuild and a force evaluation at the current state (no step).
dpd_status rebuild_and_force(dpd_sim *h, bool grow_on_overflow)
{
    for (int attempt = 0; attempt < 4; ++attempt) {
        uint32_t one = 1u;
        CUDA_TRY(h, cudaMemcpyAsync(&h->D.ctl->rebuild, &one, sizeof(one), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaMemsetAsync(&h->D.ctl->err, 0, sizeof(uint32_t), h->stream));
        CUDA_TRY(h, launch_rebuild(h->P, h->D, h->stream, h->n_scan_blocks));
        CUDA_TRY(h, launch_force(h->P, h->D, kForceEval, false, h->stream));
        DevCtl c;
        dpd_status st = check_err(h, c);
        if (st != DPD_ERR_NBR_OVERFLOW || !grow_on_overflow) return st;
        // grow the list: keep the particle arrays, reallocate the table (the
        // row layout reports its longest row, the packed one its largest group)
        const int cap = h->P.list_layout == 1 ? ((int)((uint64_t)c.max_nnb * 5 / 4 + 8) + 31) / 32 * 32
                                              : capacity_for_total(c.max_nnb);
        if ((int64_t)cap * kGroup >= (int64_t(1) << 26))
            return fail(h, DPD_ERR_NBR_OVERFLOW, "neighbour list overflow: group list beyond 2^26 entries");
        dev_free(h, h->D.nbr, h->allocs);
        st = dev_alloc(h, (void **)&h->D.nbr, (size_t)h->P.ngroups * kGroup * (size_t)cap * sizeof(uint32_t),
                       h->allocs);
        if (st) return st;
        h->P.cap = cap;
        h->P.gcap = kGroup * cap;
        drop_graphs(h);
    }
    return fail(h, DPD_ERR_NBR_OVERFLOW, "neighbour list overflow after regrowing");
}

dpd_status guard(dpd_sim *h, bool need_state)
{
    if (!h) return fail(nullptr, DPD_ERR_ARG, "null handle");
    if (h->failed) return fail(h, DPD_ERR_CUDA, "handle has a latched CUDA failure: " + h->err);
    if (need_state && !h->has_state) return fail(h, DPD_ERR_STATE, "no particle state: call dpd_set_state first");
    return DPD_OK;
}

// Download a float4 array and its caller indices; scatter xyz into out (n x 3).
dpd_status download_xyz(dpd_sim *h, const float4 *dev, double *out)
{
    DevCtl c;
    dpd_status st = read_ctl(h, c);
    if (st) return st;
    // scattered to caller order and widened on the device, one copy out
    Staging o(h);
    double *od = (double *)o.get(sizeof(double) * 3 * (size_t)h->n);
    if (!o.ok()) return fail(h, DPD_ERR_OOM, "device staging for the state: " + o.error());
    CUDA_TRY(h, launch_export(h->n, dev, h->D.pid[c.oparity], od, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(out, od, sizeof(double) * 3 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream));
    return wait(h);
}

}  // namespace

extern "C" {

void dpd_default_options(dpd_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->skin = 0.3;
    o->rebuild_every = 0;
    o->body_force_mode = 0;
    o->seed = 42;
    o->lambda = 0.5;
    o->nbr_capacity = 0;
    o->graph_steps = 8;
    o->deterministic = 0;
    o->conditional_rebuild = 1;
    o->list_builder = 0;
    o->no_reorder = 0;
    o->wait_timeout_s = 600.0;
    o->stream = nullptr;
}

dpd_status dpd_create(dpd_sim **out, const double box[3], int32_t n_species, const double *a_ij, double gamma,
                      double kT, double rc, double s, double dt, const dpd_options *opt)
{
    if (!out) return fail(nullptr, DPD_ERR_ARG, "out is NULL");
    *out = nullptr;
    dpd_options o;
    dpd_default_options(&o);
    if (opt) o = *opt;
    if (!box || !a_ij) return fail(nullptr, DPD_ERR_ARG, "box and a_ij are required");
    if (!(rc > 0) || !(dt > 0) || !(kT >= 0) || !(gamma >= 0) || !(s > 0) || !(o.skin >= 0) || !std::isfinite(rc) ||
        !std::isfinite(dt) || !std::isfinite(kT) || !std::isfinite(gamma) || !std::isfinite(s))
        return fail(nullptr, DPD_ERR_ARG, "need rc > 0, dt > 0, kT >= 0, gamma >= 0, s > 0, skin >= 0");
    if (n_species < 1 || n_species > kMaxSpecies) return fail(nullptr, DPD_ERR_ARG, "n_species must be in 1..8");
    for (int i = 0; i < n_species; ++i)
        for (int j = 0; j < n_species; ++j) {
            double x = a_ij[i * n_species + j];
            if (!std::isfinite(x) || x != a_ij[j * n_species + i])
                return fail(nullptr, DPD_ERR_ARG, "a_ij must be finite and symmetric");
        }
    if (o.body_force_mode < 0 || o.body_force_mode > 2) return fail(nullptr, DPD_ERR_ARG, "body_force_mode in 0..2");
    if (o.list_builder < 0 || o.list_builder > 1) return fail(nullptr, DPD_ERR_ARG, "list_builder in 0..1");
    if (o.no_reorder < 0 || o.no_reorder > 1) return fail(nullptr, DPD_ERR_ARG, "no_reorder in 0..1");
    if (o.list_layout < 0 || o.list_layout > 1) return fail(nullptr, DPD_ERR_ARG, "list_layout in 0..1");
    if (o.rebuild_every < 0 || o.graph_steps < 0 || o.nbr_capacity < 0 || !(o.wait_timeout_s > 0))
        return fail(nullptr, DPD_ERR_ARG, "rebuild_every, graph_steps, nbr_capacity >= 0; wait_timeout_s > 0");
    const double rl = rc + o.skin;
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 2.0 * rl) || !std::isfinite(box[a]))
            return fail(nullptr, DPD_ERR_ARG, "each box length must exceed 2 (rc + skin)");
        // cell side >= r_list (1 + 1e-4): the margin covers the FP32
        // rounding of the cell index and of the pair predicate
        nc[a] = std::max(1, (int)std::floor(box[a] / (rl * (1.0 + 1e-4))));
        if (nc[a] > 1024) return fail(nullptr, DPD_ERR_ARG, "more than 1024 cells along an axis");
    }
    if ((int64_t)nc[0] * nc[1] * nc[2] >= (1 << 26)) return fail(nullptr, DPD_ERR_ARG, "too many cells");

    dpd_sim *h = new dpd_sim();
    std::memcpy(h->box, box, sizeof(h->box));
    h->n_species = n_species;
    h->a.assign(a_ij, a_ij + n_species * n_species);
    h->gamma = gamma; h->kT = kT; h->rc = rc; h->s = s; h->dt = dt;
    h->opt = o;
    SimParams &P = h->P;
    std::memset(&P, 0, sizeof(P));
    for (int a = 0; a < 3; ++a) {
        P.nc[a] = nc[a];
        P.L[a] = (float)box[a];
        P.halfL[a] = 0.5f * P.L[a];
        P.cells_per_len[a] = (float)(nc[a] / box[a]);
        P.body[a] = (float)o.body_force[a];
    }
    P.ncell = nc[0] * nc[1] * nc[2];
    const float rcf = (float)rc, rlf = (float)rl;
    P.rc = rcf;
    P.rc2 = rcf * rcf;
    P.inv_rc = (float)(1.0 / rc);
    P.rlist2 = rlf * rlf;
    P.gamma = (float)gamma;
    P.sigma_isdt = (float)(std::sqrt(2.0 * gamma * kT) / std::sqrt(dt));
    P.s = (float)s;
    P.s_mode = s == 1.0 ? 1 : (s == 0.5 ? 2 : (s == 2.0 ? 3 : 0));
    P.dt = (float)dt;
    P.half_dt = (float)(0.5 * dt);
    P.lambda_dt = (float)(o.lambda * dt);
    P.lambda_half = o.lambda == 0.5 ? 1 : 0;
    const double hs = 0.5 * o.skin * 0.98;  // 2 % margin against FP32 rounding
    P.disp2 = (float)(hs * hs);
    // a particle this far from every face has all its list neighbours on the
    // same side of the periodic boundary (list radius + the most both ends
    // can move before a rebuild + a rounding margin)
    const double wm = rl + o.skin + 0.01;
    P.wrap_margin = (2.0 * wm < box[0] && 2.0 * wm < box[1] && 2.0 * wm < box[2]) ? (float)wm : 0.0f;
    P.n_species = n_species;
    for (int k = 0; k < n_species * n_species; ++k) P.a[k] = (float)a_ij[k];
    P.body_mode = o.body_force_mode;
    P.rebuild_every = o.rebuild_every;
    P.newton3 = o.deterministic ? 0 : 1;
    P.key[0] = (uint32_t)(o.seed & 0xFFFFFFFFull);
    P.key[1] = (uint32_t)(o.seed >> 32);
    P.key[2] = 0x243F6A88u;
    P.key[3] = 0x85A308D3u;

    // stream and control block
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(nullptr, DPD_ERR_CUDA, "cudaStreamCreate failed (no GPU?)");
        }
        h->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->side = nullptr;
        dpd_destroy(h);
        return fail(nullptr, DPD_ERR_CUDA, "cudaStreamCreate failed");
    }
    if (cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        dpd_destroy(h);
        return fail(nullptr, DPD_ERR_CUDA, "cudaEventCreate failed");
    }
    keep_pool_memory();
    build_geometry(nc, h->geo);
    h->n_scan_blocks = scan_blocks_for(P.ncell);
    P.no_reorder = o.no_reorder;
    P.use_bricks = (!o.no_reorder && nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3) ? 1 : 0;
    // the paper's row layout: full lists built brick by brick, one thread per
    // particle in the pair force
    P.list_layout = o.list_layout;
    if (o.list_layout == 1) {
        if (!P.use_bricks) {
            dpd_destroy(h);
            return fail(nullptr, DPD_ERR_ARG, "list_layout 1 needs at least 3 cells along every axis and no_reorder 0");
        }
        P.newton3 = 0;
    }
    P.list_builder = o.list_builder;
    for (int a = 0; a < 3; ++a) P.nb[a] = h->geo.nb[a];
    P.nbricks = h->geo.nb[0] * h->geo.nb[1] * h->geo.nb[2];
    if (cudaError_t ea = init_kernel_attributes(); ea != cudaSuccess) {
        cudaGetLastError();
        dpd_destroy(h);
        return fail(nullptr, DPD_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(ea));
    }
    dpd_status st = DPD_OK;
    auto A = [&](void **p, size_t b) { if (st == DPD_OK) st = dev_alloc(h, p, b, h->static_allocs); };
    A((void **)&h->D.ctl, sizeof(DevCtl));
    A((void **)&h->D.obs, sizeof(dpd_obs));
    A((void **)&h->D.rank_of_cell, sizeof(uint32_t) * P.ncell);
    A((void **)&h->D.stencil, sizeof(uint32_t) * (size_t)P.ncell * kStencil);
    A((void **)&h->D.cell_count, sizeof(uint32_t) * P.ncell);
    A((void **)&h->D.cell_start, sizeof(uint32_t) * (P.ncell + 1));
    A((void **)&h->D.scan_part, sizeof(uint32_t) * (h->n_scan_blocks + 1));
    A((void **)&h->D.brick_rank_lo, sizeof(uint32_t) * P.nbricks);
    A((void **)&h->D.brick_rank_hi, sizeof(uint32_t) * P.nbricks);
    A((void **)&h->D.brick_ord, sizeof(uint32_t) * P.nbricks);

    if (st) {
        std::string m = h->err;
        dpd_destroy(h);
        return fail(nullptr, st, m);
    }
    cudaError_t e = cudaMemcpyAsync((void *)h->D.rank_of_cell, h->geo.rank_of_cell.data(), sizeof(uint32_t) * P.ncell,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)h->D.stencil, h->geo.stencil.data(), sizeof(uint32_t) * (size_t)P.ncell * kStencil,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)h->D.brick_rank_lo, h->geo.brick_lo.data(), sizeof(uint32_t) * P.nbricks,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)h->D.brick_rank_hi, h->geo.brick_hi.data(), sizeof(uint32_t) * P.nbricks,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)h->D.brick_ord, h->geo.brick_ord.data(), sizeof(uint32_t) * P.nbricks,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->D.cell_count, 0, sizeof(uint32_t) * P.ncell, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->D.ctl, 0, sizeof(DevCtl), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        dpd_destroy(h);
        return fail(nullptr, DPD_ERR_CUDA, std::string("upload of cell tables: ") + cudaGetErrorString(e));
    }
    *out = h;
    return DPD_OK;
}

dpd_status dpd_set_state(dpd_sim *h, int64_t n, const double *x, const double *v, const int32_t *species,
                         const uint32_t *tag, uint64_t step)
{
    NvtxRange nvtx_("dpd_set_state");
    dpd_status st = guard(h, false);
    if (st) return st;
    if (n <= 0 || n > kMaxParticles || !x || !v) return fail(h, DPD_ERR_ARG, "need 0 < n <= 2^27 and x, v");
    if (tag) {
        std::vector<uint32_t> sorted(tag, tag + n);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return fail(h, DPD_ERR_ARG, "tags must be distinct");
    }
    // the caller's arrays go to device staging as they are; the checks and
    // the conversion to the device layout run there (kernels_io.cu), and the
    // live state is touched only once the checks pass
    Staging in(h);
    double *xd = (double *)in.get(sizeof(double) * 3 * (size_t)n);
    double *vd = (double *)in.get(sizeof(double) * 3 * (size_t)n);
    int32_t *spd = species ? (int32_t *)in.get(sizeof(int32_t) * (size_t)n) : nullptr;
    uint32_t *tgd = tag ? (uint32_t *)in.get(sizeof(uint32_t) * (size_t)n) : nullptr;
    uint32_t *bad = (uint32_t *)in.get(sizeof(uint32_t));
    if (!in.ok()) return fail(h, DPD_ERR_OOM, "device staging for the state: " + in.error());
    CUDA_TRY(h, cudaMemcpyAsync(xd, x, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(vd, v, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    if (spd) CUDA_TRY(h, cudaMemcpyAsync(spd, species, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    if (tgd) CUDA_TRY(h, cudaMemcpyAsync(tgd, tag, sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(bad, 0, sizeof(uint32_t), h->stream));
    CUDA_TRY(h, launch_import_check(n, h->n_species, xd, vd, spd, bad, h->stream));
    uint32_t bad_h = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&bad_h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    st = wait(h);
    if (st) return st;
    if (bad_h & 1u) return fail(h, DPD_ERR_ARG, "non-finite x or v");
    if (bad_h & 2u) return fail(h, DPD_ERR_ARG, "species out of range");
    int cap = h->opt.nbr_capacity > 0 ? h->opt.nbr_capacity : auto_capacity(h, n);
    if (h->P.list_layout == 1) cap = (cap + 31) / 32 * 32;  // whole 32 x 32 tiles per row
    if (h->P.use_bricks) {
        // staging buffer of the brick builder: the expected halo population
        // with a wide margin; a brick beyond it reads global memory
        const double cellvol = (h->box[0] / h->P.nc[0]) * (h->box[1] / h->P.nc[1]) * (h->box[2] / h->P.nc[2]);
        const double mean = (double)n / (h->box[0] * h->box[1] * h->box[2]) * cellvol * kHaloCells;
        int bc = (int)std::ceil(1.1 * mean + 6.0 * std::sqrt(mean) + 64.0);
        bc = (bc + 31) / 32 * 32;
        h->P.brick_cap = std::min(std::max(bc, 256), std::min(max_brick_cap(), 65535));
    }
    if (n != h->n || cap != h->P.cap || h->cap_alloc_n != n) {
        h->n = n;
        h->P.n = (int)n;
        st = alloc_particles(h, n, cap);
        if (st) {
            h->has_state = false;
            return st;
        }
    }
    h->has_state = false;
    h->pending = false;
    h->bonds_set = false;
    h->P.has_bonds = 0;
    drop_graphs(h);
    Ptrs &D = h->D;
    CUDA_TRY(h, launch_import(h->P, h->box, n, xd, vd, spd, tgd, D.pos[0], D.vel[0], D.tag[0], D.pid[0], h->stream));
    CUDA_TRY(h, cudaMemsetAsync(D.force[0], 0, sizeof(float4) * n, h->stream));
    if (!h->P.lambda_half) CUDA_TRY(h, cudaMemsetAsync(D.vkick[0], 0, sizeof(float4) * n, h->stream));
    CUDA_TRY(h, cudaMemsetAsync((void *)D.bond_partner, 0xFF, sizeof(uint32_t) * (size_t)n * kMaxBonds, h->stream));
    for (int b = 0; b < 2; ++b) CUDA_TRY(h, cudaMemsetAsync(D.facc[b], 0, sizeof(float4) * n, h->stream));
    DevCtl c;
    std::memset(&c, 0, sizeof(c));
    c.step = step;
    CUDA_TRY(h, cudaMemcpyAsync(D.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, launch_signature(h->P, D, h->stream));
    h->step = step;
    st = rebuild_and_force(h, h->opt.nbr_capacity == 0);
    if (st) return st;
    h->has_state = true;
    return DPD_OK;
}

dpd_status dpd_set_bonds(dpd_sim *h, int64_t nb, const uint32_t *pairs, double k, double r0)
{
    dpd_status st = guard(h, true);
    if (st) return st;
    if (nb < 0 || (nb > 0 && !pairs) || !std::isfinite(k) || !std::isfinite(r0))
        return fail(h, DPD_ERR_ARG, "invalid bond arguments");
    std::vector<uint32_t> bp((size_t)h->n * kMaxBonds, kNone);
    std::vector<int> deg(h->n, 0);
    for (int64_t b = 0; b < nb; ++b) {
        uint32_t i = pairs[2 * b], j = pairs[2 * b + 1];
        if (i >= (uint64_t)h->n || j >= (uint64_t)h->n || i == j) return fail(h, DPD_ERR_ARG, "bond index out of range");
        if (deg[i] >= kMaxBonds || deg[j] >= kMaxBonds) return fail(h, DPD_ERR_ARG, "more than 6 bonds on a particle");
        bp[(size_t)i * kMaxBonds + deg[i]++] = j;
        bp[(size_t)j * kMaxBonds + deg[j]++] = i;
    }
    CUDA_TRY(h, cudaMemcpyAsync((void *)h->D.bond_partner, bp.data(), sizeof(uint32_t) * bp.size(),
                                cudaMemcpyHostToDevice, h->stream));
    h->P.has_bonds = nb > 0 ? 1 : 0;
    h->P.k_bond = (float)k;
    h->P.r0_bond = (float)r0;
    h->bonds_set = nb > 0;
    drop_graphs(h);
    CUDA_TRY(h, launch_index(h->P, h->D, h->stream));
    CUDA_TRY(h, launch_force(h->P, h->D, kForceEval, false, h->stream));
    DevCtl c;
    return check_err(h, c);
}

dpd_status dpd_build_neighbors(dpd_sim *h)
{
    NvtxRange nvtx_("dpd_build_neighbors");
    dpd_status st = guard(h, true);
    if (st) return st;
    if (h->pending && (st = dpd_sync(h)) != DPD_OK) return st;  // report a queued run's error first
    return rebuild_and_force(h, h->opt.nbr_capacity == 0);
}

dpd_status dpd_get_neighbors(dpd_sim *h, int64_t cap, uint32_t *pairs_out, int64_t *n_out)
{
    dpd_status st = guard(h, true);
    if (st) return st;
    if (cap < 0 || (cap > 0 && !pairs_out) || !n_out) return fail(h, DPD_ERR_ARG, "invalid output arguments");
    DevCtl c;
    st = read_ctl(h, c);
    if (st) return st;
    const int64_t n = h->n;
    int G = h->P.ngroups;
    std::vector<uint32_t> nbr((size_t)G * h->P.gcap), pid(n);
    std::vector<uint2> desc(G);
    CUDA_TRY(h, cudaMemcpyAsync(nbr.data(), h->D.nbr, sizeof(uint32_t) * nbr.size(), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(desc.data(), h->D.gdesc, sizeof(uint2) * G, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(pid.data(), h->D.pid[c.oparity], sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, h->stream));
    st = wait(h);
    if (st) return st;
    std::vector<uint64_t> pr;
    if (h->P.list_layout == 1) {
        // rows of the transposed table: entry k of particle i at row
        // 32 (i / 32) + k % 32, entry 32 (k / 32) + i % 32
        std::vector<uint32_t> rc(n);
        CUDA_TRY(h, cudaMemcpyAsync(rc.data(), h->D.rowcnt, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, h->stream));
        st = wait(h);
        if (st) return st;
        const size_t cap = (size_t)h->P.cap;
        for (int64_t i = 0; i < n; ++i) {
            if (rc[i] > cap) return fail(h, DPD_ERR_STATE, "row longer than its capacity");
            for (uint32_t k = 0; k < rc[i]; ++k) {
                const size_t at = ((size_t)(i / 32) * 32 + k % 32) * cap + (k / 32) * 32 + (size_t)(i % 32);
                const uint32_t j = nbr[at];
                if (j >= (uint32_t)n) return fail(h, DPD_ERR_STATE, "neighbour entry out of range");
                const uint32_t a = std::min(pid[i], pid[j]), b2 = std::max(pid[i], pid[j]);
                if (a != b2) pr.push_back(((uint64_t)a << 32) | b2);
            }
        }
        G = 0;  // no group lists
    }
    for (int g = 0; g < G; ++g) {
        const uint32_t first = desc[g].x, owners = desc[g].y & 63u, ne = desc[g].y >> 6;
        if (owners > (uint32_t)kGroup || ne > (uint32_t)h->P.gcap || (owners && first + owners > (uint64_t)n))
            return fail(h, DPD_ERR_STATE, "corrupt group descriptor");
        const uint32_t *list = nbr.data() + (size_t)g * h->P.gcap;
        for (uint32_t k = 0; k < ne; ++k) {
            const uint32_t own = list[k] >> kOwnerShift, j = list[k] & kIndexMask;
            if (own >= owners || j >= (uint32_t)n) return fail(h, DPD_ERR_STATE, "neighbour entry out of range");
            const uint32_t i = first + own;
            const uint32_t a = std::min(pid[i], pid[j]), b2 = std::max(pid[i], pid[j]);
            if (a != b2) pr.push_back(((uint64_t)a << 32) | b2);
        }
    }
    std::sort(pr.begin(), pr.end());
    pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
    *n_out = (int64_t)pr.size();
    for (int64_t k = 0; k < cap && k < (int64_t)pr.size(); ++k) {
        pairs_out[2 * k] = (uint32_t)(pr[k] >> 32);
        pairs_out[2 * k + 1] = (uint32_t)(pr[k] & 0xFFFFFFFFu);
    }
    return DPD_OK;
}

dpd_status dpd_forces(dpd_sim *h, double *f_out)
{
    NvtxRange nvtx_("dpd_forces");
    dpd_status st = guard(h, true);
    if (st) return st;
    if (h->pending && (st = dpd_sync(h)) != DPD_OK) return st;  // report a queued run's error first
    CUDA_TRY(h, cudaMemsetAsync(&h->D.ctl->err, 0, sizeof(uint32_t), h->stream));
    CUDA_TRY(h, launch_force(h->P, h->D, kForceEval, true, h->stream));
    DevCtl c;
    st = check_err(h, c);
    if (st) return st;
    if (!f_out) return DPD_OK;
    return download_xyz(h, h->D.fout, f_out);
}

dpd_status dpd_get_force(dpd_sim *h, double *f_out)
{
    dpd_status st = guard(h, true);
    if (st) return st;
    if (!f_out) return fail(h, DPD_ERR_ARG, "f_out is NULL");
    DevCtl c;
    st = read_ctl(h, c);
    if (st) return st;
    return download_xyz(h, h->D.force[c.parity], f_out);
}

dpd_status dpd_set_force(dpd_sim *h, const double *f)
{
    dpd_status st = guard(h, true);
    if (st) return st;
    if (!f) return fail(h, DPD_ERR_ARG, "f is NULL");
    DevCtl c;
    st = read_ctl(h, c);
    if (st) return st;
    std::vector<uint32_t> pid(h->n);
    CUDA_TRY(h, cudaMemcpyAsync(pid.data(), h->D.pid[c.oparity], sizeof(uint32_t) * h->n, cudaMemcpyDeviceToHost,
                                h->stream));
    st = wait(h);
    if (st) return st;
    std::vector<float4> buf(h->n);
    for (int64_t p = 0; p < h->n; ++p) {
        const uint32_t i = pid[p];
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(f[3 * (size_t)i + a])) return fail(h, DPD_ERR_ARG, "non-finite force");
        buf[p] = make_float4((float)f[3 * (size_t)i], (float)f[3 * (size_t)i + 1], (float)f[3 * (size_t)i + 2], 0.0f);
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->D.force[c.parity], buf.data(), sizeof(float4) * h->n, cudaMemcpyHostToDevice,
                                h->stream));
    return wait(h);
}

dpd_status dpd_step_async(dpd_sim *h, int64_t nsteps)
{
    NvtxRange nvtx_("dpd_step_async");
    dpd_status st = guard(h, true);
    if (st) return st;
    if (nsteps < 0) return fail(h, DPD_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return DPD_OK;
    // the error word is cleared only when no unchecked run is queued, so an
    // error of an earlier chunk survives until dpd_sync reads it
    if (!h->pending) CUDA_TRY(h, cudaMemsetAsync(&h->D.ctl->err, 0, sizeof(uint32_t), h->stream));
    h->pending = true;
    const int K = h->opt.graph_steps;
    int64_t left = nsteps;
    if (K > 0) {
        cudaGraphExec_t gx;
        st = get_graph(h, K, &gx);
        if (st) return st;
        while (left >= K) {
            CUDA_TRY(h, cudaGraphLaunch(gx, h->stream));
            left -= K;
        }
        if (left > 0) {
            st = get_graph(h, (int)left, &gx);
            if (st) return st;
            CUDA_TRY(h, cudaGraphLaunch(gx, h->stream));
            left = 0;
        }
    } else {
        CondCapture none;
        CUDA_TRY(h, enqueue_steps(h, left, none));
    }
    h->step += (uint64_t)nsteps;
    return DPD_OK;
}

dpd_status dpd_sync(dpd_sim *h)
{
    NvtxRange nvtx_("dpd_sync");
    dpd_status st = guard(h, true);
    if (st) return st;
    DevCtl c;
    st = check_err(h, c);
    if (st == DPD_ERR_TIMEOUT) return st;  // still running: the run stays pending
    h->pending = false;
    if (st) h->has_state = false;
    return st;
}

dpd_status dpd_query(dpd_sim *h, int32_t *idle)
{
    if (!h || !idle) return fail(h, DPD_ERR_ARG, "null argument");
    const cudaError_t e = cudaStreamQuery(h->stream);
    if (e == cudaSuccess) {
        *idle = 1;
        return DPD_OK;
    }
    if (e == cudaErrorNotReady) {
        *idle = 0;
        return DPD_OK;
    }
    cudaGetLastError();
    return fail(h, DPD_ERR_CUDA, std::string("kernel failure: ") + cudaGetErrorString(e));
}

dpd_status dpd_wait_selftest(dpd_sim *h, uint32_t polls)
{
    dpd_status st = guard(h, true);
    if (st) return st;
    if (polls < 1 || polls > (1u << 20)) return fail(h, DPD_ERR_ARG, "polls must be in 1..2^20");
    if (h->pending && (st = dpd_sync(h)) != DPD_OK) return st;
    CUDA_TRY(h, cudaMemsetAsync(&h->D.ctl->err, 0, sizeof(uint32_t), h->stream));
    CUDA_TRY(h, launch_wait_probe(h->D, polls, h->stream));
    DevCtl c;
    st = check_err(h, c);
    // the probe's error bit must not leak into the next call
    CUDA_TRY(h, cudaMemsetAsync(&h->D.ctl->err, 0, sizeof(uint32_t), h->stream));
    dpd_status st2 = wait(h);
    return st != DPD_OK ? st : st2;
}

dpd_status dpd_step(dpd_sim *h, int64_t nsteps)
{
    dpd_status st = dpd_step_async(h, nsteps);
    if (st || nsteps == 0) return st;
    return dpd_sync(h);
}

dpd_status dpd_step_profiled(dpd_sim *h, int64_t nsteps, dpd_step_times *out)
{
    NvtxRange nvtx_("dpd_step_profiled");
    dpd_status st = guard(h, true);
    if (st) return st;
    if (nsteps < 1 || nsteps > 100000) return fail(h, DPD_ERR_ARG, "nsteps must be in 1..100000");
    if (h->pending && (st = dpd_sync(h)) != DPD_OK) return st;  // report a queued run's error first
    const size_t nev = (size_t)(3 * nsteps + 2);
    while (h->tev.size() < nev) {
        cudaEvent_t e;
        CUDA_TRY(h, cudaEventCreate(&e));
        h->tev.push_back(e);
    }
    DevCtl c0;
    st = read_ctl(h, c0);
    if (st) return st;
    CUDA_TRY(h, cudaMemsetAsync(&h->D.ctl->err, 0, sizeof(uint32_t), h->stream));
    if (h->opt.graph_steps > 0) {
        cudaGraphExec_t ex = nullptr;
        auto it = h->timed_graphs.find(nsteps);
        if (it != h->timed_graphs.end()) {
            ex = it->second;
        } else {
            st = capture_steps(h, nsteps, true, &ex);
            if (st) return st;
            h->timed_graphs[nsteps] = ex;
        }
        CUDA_TRY(h, cudaGraphLaunch(ex, h->stream));
    } else {
        CondCapture none;
        CUDA_TRY(h, enqueue_steps_timed(h, nsteps, none));
    }
    h->step += (uint64_t)nsteps;
    DevCtl c;
    st = check_err(h, c);
    if (st) {
        h->has_state = false;
        return st;
    }
    if (out) {
        std::memset(out, 0, sizeof(*out));
        cudaError_t eerr = cudaSuccess;
        auto el = [&](size_t a, size_t b) {
            float t = 0.f;
            cudaError_t e = cudaEventElapsedTime(&t, h->tev[a], h->tev[b]);
            if (e != cudaSuccess && eerr == cudaSuccess) eerr = e;
            return (double)t;
        };
        out->integrate_ms = el(0, 1);
        for (int64_t s = 0; s < nsteps; ++s) {
            out->rebuild_ms += el(s == 0 ? 1 : 3 * s + 1, 3 * s + 2);
            out->pair_ms += el(3 * s + 2, 3 * s + 3);
            out->force_ms += el(3 * s + 2, 3 * s + 4);
        }
        out->total_ms = el(0, 3 * nsteps + 1);
        if (eerr != cudaSuccess) {
            cudaGetLastError();
            return fail(h, DPD_ERR_STATE, std::string("event timing unavailable: ") + cudaGetErrorString(eerr));
        }
        out->steps = nsteps;
        out->force_launches = nsteps;
        // per step: pair kernel (+ settle), advance; the rebuild chain on every
        // step outside graphs, only on rebuild steps inside them (conditional
        // nodes); plus the opening phase 1 + advance
        out->rebuilds = (int64_t)(c.nrebuild - c0.nrebuild);
        const int64_t chains = h->opt.graph_steps > 0 && h->opt.conditional_rebuild ? out->rebuilds : nsteps;
        out->kernel_launches = nsteps * (2 + (h->P.newton3 ? 1 : 0)) + 2 + chains * kRebuildKernels;
    }
    return DPD_OK;
}

dpd_status dpd_observables(dpd_sim *h, dpd_obs *out)
{
    NvtxRange nvtx_("dpd_observables");
    dpd_status st = guard(h, true);
    if (st) return st;
    if (!out) return fail(h, DPD_ERR_ARG, "out is NULL");
    const int nb = observe_blocks_for((int)h->n);
    CUDA_TRY(h, launch_observe(h->P, h->D, nb, h->stream));
    double acc[8];
    CUDA_TRY(h, cudaMemcpyAsync(acc, h->D.red + (size_t)nb * 8, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    DevCtl c;
    CUDA_TRY(h, cudaMemcpyAsync(&c, h->D.ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    st = wait(h);
    if (st) return st;
    const double V = h->box[0] * h->box[1] * h->box[2];
    out->step = c.step;
    out->n = h->n;
    out->kinetic = 0.5 * acc[0];
    out->temperature = h->n > 1 ? acc[0] / (3.0 * h->n - 3.0) : 0.0;
    out->virial = acc[4];
    out->pressure = (acc[0] + acc[4]) / (3.0 * V);
    out->momentum[0] = acc[1];
    out->momentum[1] = acc[2];
    out->momentum[2] = acc[3];
    return DPD_OK;
}

static_assert(sizeof(dpd_obs) == 9 * 8 && offsetof(dpd_obs, step) == 0 && offsetof(dpd_obs, n) == 8 &&
                  offsetof(dpd_obs, kinetic) == 16 && offsetof(dpd_obs, temperature) == 24 &&
                  offsetof(dpd_obs, virial) == 32 && offsetof(dpd_obs, pressure) == 40 &&
                  offsetof(dpd_obs, momentum) == 48,
              "k_obs_finish writes dpd_obs as nine 8-byte words");

dpd_status dpd_observables_async(dpd_sim *h, dpd_obs *out)
{
    NvtxRange nvtx_("dpd_observables_async");
    dpd_status st = guard(h, true);
    if (st) return st;
    if (!out) return fail(h, DPD_ERR_ARG, "out is NULL");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, out) != cudaSuccess || a.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return fail(h, DPD_ERR_ARG, "out must be page-locked host memory");
    }
    const int nb = observe_blocks_for((int)h->n);
    const double V = h->box[0] * h->box[1] * h->box[2];
    CUDA_TRY(h, launch_observe(h->P, h->D, nb, h->stream));
    CUDA_TRY(h, launch_observe_finish(h->D, nb, h->n, h->n > 1 ? 3.0 * h->n - 3.0 : 0.0, 3.0 * V, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(out, h->D.obs, sizeof(dpd_obs), cudaMemcpyDeviceToHost, h->stream));
    return DPD_OK;
}

dpd_status dpd_profile(dpd_sim *h, int32_t bin_axis, int32_t vel_axis, int32_t nbins, double *sum_out,
                       double *count_out)
{
    dpd_status st = guard(h, true);
    if (st) return st;
    if (bin_axis < 0 || bin_axis > 2 || vel_axis < 0 || vel_axis > 2 || nbins < 1 || nbins > 100000 || !sum_out ||
        !count_out)
        return fail(h, DPD_ERR_ARG, "invalid profile arguments");
    int nblocks = (int)std::min<int64_t>(std::max<int64_t>(1, h->n / 1024), 1024);
    size_t need = (size_t)nblocks * 2 * nbins;
    if (need > h->red_doubles) {
        double *nr = nullptr;
        st = dev_alloc(h, (void **)&nr, need * sizeof(double), h->allocs);
        if (st) return st;
        dev_free(h, h->D.red, h->allocs);
        h->D.red = nr;
        h->red_doubles = need;
        drop_graphs(h);
    }
    CUDA_TRY(h, launch_profile(h->P, h->D, bin_axis, vel_axis, nbins, nblocks, h->stream));
    std::vector<double> part(need);
    CUDA_TRY(h, cudaMemcpyAsync(part.data(), h->D.red, sizeof(double) * need, cudaMemcpyDeviceToHost, h->stream));
    st = wait(h);
    if (st) return st;
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < nbins; ++k) {
            sum_out[k] += part[((size_t)b * nbins + k) * 2];
            count_out[k] += part[((size_t)b * nbins + k) * 2 + 1];
        }
    return DPD_OK;
}

dpd_status dpd_get_state(dpd_sim *h, double *x, double *v, uint64_t *step)
{
    NvtxRange nvtx_("dpd_get_state");
    dpd_status st = guard(h, true);
    if (st) return st;
    DevCtl c;
    st = read_ctl(h, c);
    if (st) return st;
    if (x) {
        st = download_xyz(h, h->D.pos[c.parity], x);
        if (st) return st;
    }
    if (v) {
        st = download_xyz(h, h->D.vel[c.parity], v);
        if (st) return st;
    }
    if (step) *step = c.step;
    return DPD_OK;
}

dpd_status dpd_info(dpd_sim *h, int64_t *n, int64_t *rebuilds, int32_t *nbr_capacity)
{
    dpd_status st = guard(h, false);
    if (st) return st;
    DevCtl c;
    std::memset(&c, 0, sizeof(c));
    if (h->has_state) {
        st = read_ctl(h, c);
        if (st) return st;
    }
    if (n) *n = h->n;
    if (rebuilds) *rebuilds = (int64_t)c.nrebuild;
    if (nbr_capacity) *nbr_capacity = h->P.cap;
    return DPD_OK;
}

dpd_status dpd_pair_rng(uint64_t seed, uint64_t step, int64_t m, const uint32_t *tag_i, const uint32_t *tag_j,
                        uint32_t *out_hash, float *out_xi)
{
    if (m < 0 || (m > 0 && (!tag_i || !tag_j || !out_hash))) return fail(nullptr, DPD_ERR_ARG, "invalid arguments");
    if (m == 0) return DPD_OK;
    cudaStream_t s = nullptr;
    uint32_t *dti = nullptr, *dtj = nullptr, *dh = nullptr;
    float *dx = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dti, sizeof(uint32_t) * m);
    if (e == cudaSuccess) e = cudaMalloc(&dtj, sizeof(uint32_t) * m);
    if (e == cudaSuccess) e = cudaMalloc(&dh, sizeof(uint32_t) * 2 * m);
    if (e == cudaSuccess && out_xi) e = cudaMalloc(&dx, sizeof(float) * m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dti, tag_i, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dtj, tag_j, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_pair_rng(seed, step, m, dti, dtj, dh, dx, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_hash, dh, sizeof(uint32_t) * 2 * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && out_xi) e = cudaMemcpyAsync(out_xi, dx, sizeof(float) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dti); cudaFree(dtj); cudaFree(dh); cudaFree(dx);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, DPD_ERR_CUDA, std::string("dpd_pair_rng: ") + cudaGetErrorString(e));
    }
    return DPD_OK;
}

dpd_status dpd_alu_peak(int32_t kind, int32_t reps, double *lane_ops_per_s, double *ms_per_launch)
{
    if ((kind != 0 && kind != 1) || reps < 1 || reps > 1000 || !lane_ops_per_s || !ms_per_launch)
        return fail(nullptr, DPD_ERR_ARG, "dpd_alu_peak: kind must be 0 or 1, reps 1..1000, outputs non-NULL");
    const cudaError_t e = time_alu_peak(kind, reps, lane_ops_per_s, ms_per_launch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, DPD_ERR_CUDA, std::string("dpd_alu_peak: ") + cudaGetErrorString(e));
    }
    return DPD_OK;
}

const char *dpd_last_error(const dpd_sim *h)
{
    if (h) return h->err.c_str();
    return g_last_error.c_str();
}

void dpd_destroy(dpd_sim *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    free_list(h, h->allocs);
    free_list(h, h->static_allocs);
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    if (h->ev) cudaEventDestroy(h->ev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->side) cudaStreamDestroy(h->side);
    delete h;
}

}  // extern "C"
