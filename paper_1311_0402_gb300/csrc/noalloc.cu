// noalloc.cu -- dpd_forces_static: the pair force of a small system computed
// without any device allocation, for callers that cannot allocate device
// memory themselves (a host application that hands the library memory it
// manages in its own pool, code running inside another framework's memory
// budget, or a caller in a context where cudaMalloc is not allowed).
//
// Every call uses one file-scope scratch array in device global memory
// (kScratchBytes, fixed at compile time; every GPU that loads the library
// holds it until the process exits).  Its device address is looked up once
// per device with cudaGetSymbolAddress, on the first call made on that
// device (so that first call must come before any stream capture), and is
// passed to the kernels.  Calls share the array: two calls whose kernels
// overlap on the GPU (different streams, or different host threads on the
// same device without ordering) race on it and give wrong results.
#include "dpd.h"
#include "dpd_internal.cuh"
#include "dpd_math.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace {

using namespace dpd;

constexpr int kNAMaxParticles = 131072;
constexpr int kNAMaxCells = 65536;
constexpr int kNAThreads = 256;

// scratch layout (byte offsets, 256-aligned)
constexpr size_t kOffKey = 0;                                          // u32 [max particles]
constexpr size_t kOffIdx = kOffKey + 4 * (size_t)kNAMaxParticles;     // u32 [max particles]
constexpr size_t kOffFill = kOffIdx + 4 * (size_t)kNAMaxParticles;    // u32 [max particles]
constexpr size_t kOffSig = kOffFill + 4 * (size_t)kNAMaxParticles;    // u32 [max particles]
constexpr size_t kOffCount = kOffSig + 4 * (size_t)kNAMaxParticles;   // u32 [max cells]
constexpr size_t kOffStart = kOffCount + 4 * (size_t)kNAMaxCells;     // u32 [max cells + 1]
constexpr size_t kScratchBytes = kOffStart + 4 * ((size_t)kNAMaxCells + 64);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct NAParams {
    int n;
    int nc[3];
    int ncell;
    float L[3], halfL[3], cells_per_len[3];
    float rc2, inv_rc, gamma, sigma_isdt, s;
    int s_mode;
    int n_species;
    float a[kMaxSpecies * kMaxSpecies];
    int body_mode;
    float body[3];
    uint32_t key[4];
    uint32_t step;
};

struct NAScratch {
    uint32_t *key;    // cell of each particle
    uint32_t *fill;   // cell members in the order the atomics placed them
    uint32_t *idx;    // cell members in index order
    uint32_t *sig, *count, *start;
};

__device__ __forceinline__ int na_cell_axis(float x, float cpl, int nc)
{
    int c = (int)(x * cpl);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_na_clear(NAParams P, NAScratch S)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += gridDim.x * blockDim.x) S.count[c] = 0u;
}

__global__ void k_na_bin(NAParams P, NAScratch S, const float4 *pos, const uint32_t *tag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        float4 p = pos[i];
        int cx = na_cell_axis(p.x, P.cells_per_len[0], P.nc[0]);
        int cy = na_cell_axis(p.y, P.cells_per_len[1], P.nc[1]);
        int cz = na_cell_axis(p.z, P.cells_per_len[2], P.nc[2]);
        uint32_t c = (uint32_t)((cz * P.nc[1] + cy) * P.nc[0] + cx);
        S.key[i] = c;
        atomicAdd(&S.count[c], 1u);
        S.sig[i] = signature(tag ? tag[i] : (uint32_t)i, P.step, P.key);
    }
}

// One block: exclusive scan of the counts into start[], counts reset to 0
// (they are reused as fill cursors).
__global__ void __launch_bounds__(1024) k_na_scan(NAParams P, NAScratch S)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < P.ncell; base += blockDim.x) {
        int c = base + threadIdx.x;
        uint32_t v = c < P.ncell ? S.count[c] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_tot[lane];
            uint32_t wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_tot[lane] = wi - w;
        }
        __syncthreads();
        uint32_t excl = carry + warp_tot[warp] + incl - v;
        if (c < P.ncell) {
            S.start[c] = excl;
            S.count[c] = 0u;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) S.start[P.ncell] = (uint32_t)P.n;
}

__global__ void k_na_fill(NAParams P, NAScratch S)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        uint32_t c = S.key[i];
        S.fill[S.start[c] + atomicAdd(&S.count[c], 1u)] = (uint32_t)i;
    }
}

// Each particle's place in its cell is the number of members with a smaller
// index, so idx[] holds every cell in index order whatever order the atomics
// filled it in, and the force sums run in a fixed order.  One thread per
// particle reads its own cell once: no thread does more than the cell's
// occupancy in work.
__global__ void k_na_rank(NAParams P, NAScratch S)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const uint32_t c = S.key[i];
        const uint32_t b = S.start[c], e = S.start[c + 1];
        uint32_t r = 0;
        for (uint32_t q = b; q < e; ++q) r += S.fill[q] < (uint32_t)i ? 1u : 0u;
        S.idx[b + r] = (uint32_t)i;
    }
}

// Pair force of Eqs. 2-9 for particle i over the particles of its 27
// surrounding cells (cells of side >= r_c), FP32 predicate d^2 < r_c^2.
template <int SMODE>
__global__ void k_na_force(NAParams P, NAScratch S, const float4 *pos, const float4 *vel, float4 *fout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float4 pi = pos[i];
    const float4 vi = vel[i];
    const uint32_t si = S.sig[i];
    const int ti = __float_as_int(pi.w);
    // a species outside 0..n_species-1 (in this particle or a partner within
    // r_c) makes the force NaN; the parameter table is never read with it
    bool bad = (unsigned)ti >= (unsigned)P.n_species;
    const int cx = na_cell_axis(pi.x, P.cells_per_len[0], P.nc[0]);
    const int cy = na_cell_axis(pi.y, P.cells_per_len[1], P.nc[1]);
    const int cz = na_cell_axis(pi.z, P.cells_per_len[2], P.nc[2]);
    int lo[3], cnt[3];
    const int c3[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a) {
        // distinct neighbour cells per axis: {-1, 0, 1}, {0, 1} or {0}
        if (P.nc[a] >= 3) { lo[a] = -1; cnt[a] = 3; }
        else if (P.nc[a] == 2) { lo[a] = 0; cnt[a] = 2; }
        else { lo[a] = 0; cnt[a] = 1; }
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int oz = 0; oz < cnt[2]; ++oz)
        for (int oy = 0; oy < cnt[1]; ++oy)
            for (int ox = 0; ox < cnt[0]; ++ox) {
                int nx = (c3[0] + lo[0] + ox + P.nc[0]) % P.nc[0];
                int ny = (c3[1] + lo[1] + oy + P.nc[1]) % P.nc[1];
                int nz = (c3[2] + lo[2] + oz + P.nc[2]) % P.nc[2];
                uint32_t c = (uint32_t)((nz * P.nc[1] + ny) * P.nc[0] + nx);
                for (uint32_t q = S.start[c]; q < S.start[c + 1]; ++q) {
                    const uint32_t j = S.idx[q];
                    if (j == (uint32_t)i) continue;
                    const float4 pj = pos[j];
                    const float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
                    const float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
                    const float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
                    const float d2 = dist2_rn(dx, dy, dz);
                    if (!(d2 < P.rc2 && d2 > 0.0f)) continue;
                    const float4 vj = vel[j];
                    const float inv_r = rsqrtf(d2);
                    const float r = d2 * inv_r;
                    const float w = fmaxf(fmaf(-r, P.inv_rc, 1.0f), 0.0f);
                    const float wR = weight_R<SMODE>(w, P.s);
                    const float ev = -((dx * (vi.x - vj.x) + dy * (vi.y - vj.y)) + dz * (vi.z - vj.z)) * inv_r;
                    uint32_t A, B;
                    pair_hash(si, S.sig[j], P.key, A, B);
                    const float xi = gauss_from_hash(A, B);
                    const int tj = __float_as_int(pj.w);
                    if (bad || (unsigned)tj >= (unsigned)P.n_species) {
                        bad = true;
                        continue;
                    }
                    const float a = P.a[ti * P.n_species + tj];
                    const float F = fmaf(a, w, fmaf(-P.gamma * wR * wR, ev, P.sigma_isdt * wR * xi));
                    const float sc = -F * inv_r;
                    fx = fmaf(sc, dx, fx);
                    fy = fmaf(sc, dy, fy);
                    fz = fmaf(sc, dz, fz);
                }
            }
    if (P.body_mode == 1) {
        fx += P.body[0]; fy += P.body[1]; fz += P.body[2];
    } else if (P.body_mode == 2) {
        const float sg = pi.y < P.halfL[1] ? 1.0f : -1.0f;
        fx = fmaf(sg, P.body[0], fx); fy = fmaf(sg, P.body[1], fy); fz = fmaf(sg, P.body[2], fz);
    }
    if (bad) fx = fy = fz = __int_as_float(0x7FC00000);  // quiet NaN
    fout[i] = make_float4(fx, fy, fz, 0.0f);
}

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
void *g_na_addr[kMaxDevices] = {};
thread_local std::string g_na_err;

dpd_status na_fail(dpd_status st, const std::string &m)
{
    g_na_err = m;
    return st;
}

}  // namespace

extern "C" {

const char *dpd_forces_static_last_error(void) { return g_na_err.c_str(); }

int64_t dpd_forces_static_max_particles(void) { return kNAMaxParticles; }

dpd_status dpd_forces_static(const dpd_static_params *prm, int64_t n, const float *pos, const float *vel,
                             const uint32_t *tag, uint64_t step, float *force_out, void *stream)
{
    if (!prm || !pos || !vel || !force_out) return na_fail(DPD_ERR_ARG, "params, pos, vel and force_out are required");
    if (n < 1 || n > kNAMaxParticles)
        return na_fail(DPD_ERR_ARG, "n = " + std::to_string(n) + " is outside 1.." + std::to_string(kNAMaxParticles) +
                                        " (the size of the static scratch of dpd_forces_static)");
    if (prm->n_species < 1 || prm->n_species > kMaxSpecies) return na_fail(DPD_ERR_ARG, "n_species must be in 1..8");
    if (!(prm->rc > 0) || !(prm->dt > 0) || !(prm->gamma >= 0) || !(prm->kT >= 0) || !(prm->s > 0))
        return na_fail(DPD_ERR_ARG, "need rc > 0, dt > 0, gamma >= 0, kT >= 0, s > 0");
    if (prm->body_force_mode < 0 || prm->body_force_mode > 2) return na_fail(DPD_ERR_ARG, "body_force_mode in 0..2");
    NAParams P;
    std::memset(&P, 0, sizeof(P));
    P.n = (int)n;
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        double L = prm->box[a];
        if (!(L > 2.0 * prm->rc) || !std::isfinite(L)) return na_fail(DPD_ERR_ARG, "each box length must exceed 2 rc");
        int nc = (int)std::floor(L / (prm->rc * (1.0 + 1e-4)));
        P.nc[a] = nc < 1 ? 1 : nc;
        ncell *= P.nc[a];
        P.L[a] = (float)L;
        P.halfL[a] = 0.5f * P.L[a];
        P.cells_per_len[a] = (float)(P.nc[a] / L);
        P.body[a] = (float)prm->body_force[a];
    }
    if (ncell > kNAMaxCells)
        return na_fail(DPD_ERR_ARG, "the box needs " + std::to_string(ncell) + " cells, more than the " +
                                        std::to_string(kNAMaxCells) + " of the static scratch");
    for (int i = 0; i < prm->n_species; ++i)
        for (int j = 0; j < prm->n_species; ++j) {
            double x = prm->a_ij[i * prm->n_species + j];
            if (!std::isfinite(x) || x != prm->a_ij[j * prm->n_species + i])
                return na_fail(DPD_ERR_ARG, "a_ij must be finite and symmetric");
            P.a[i * prm->n_species + j] = (float)x;
        }
    P.ncell = (int)ncell;
    const float rcf = (float)prm->rc;
    P.rc2 = rcf * rcf;
    P.inv_rc = (float)(1.0 / prm->rc);
    P.gamma = (float)prm->gamma;
    P.sigma_isdt = (float)(std::sqrt(2.0 * prm->gamma * prm->kT) / std::sqrt(prm->dt));
    P.s = (float)prm->s;
    P.s_mode = prm->s == 1.0 ? 1 : (prm->s == 0.5 ? 2 : (prm->s == 2.0 ? 3 : 0));
    P.n_species = prm->n_species;
    P.body_mode = prm->body_force_mode;
    P.key[0] = (uint32_t)(prm->seed & 0xFFFFFFFFull);
    P.key[1] = (uint32_t)(prm->seed >> 32);
    P.key[2] = 0x243F6A88u;
    P.key[3] = 0x85A308D3u;
    P.step = (uint32_t)step;

    // device address of the scratch array, looked up once per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(DPD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(DPD_ERR_ARG, "device ordinal beyond 64");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(DPD_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            g_na_addr[dev] = p;
        }
        base = g_na_addr[dev];
    }
    unsigned char *b = (unsigned char *)base;
    NAScratch S;
    S.key = (uint32_t *)(b + kOffKey);
    S.idx = (uint32_t *)(b + kOffIdx);
    S.fill = (uint32_t *)(b + kOffFill);
    S.sig = (uint32_t *)(b + kOffSig);
    S.count = (uint32_t *)(b + kOffCount);
    S.start = (uint32_t *)(b + kOffStart);

    cudaStream_t s = (cudaStream_t)stream;
    const float4 *p4 = (const float4 *)pos;
    const float4 *v4 = (const float4 *)vel;
    float4 *f4 = (float4 *)force_out;
    int gn = (int)((n + kNAThreads - 1) / kNAThreads);
    int gc = (P.ncell + kNAThreads - 1) / kNAThreads;
    k_na_clear<<<gc, kNAThreads, 0, s>>>(P, S);
    k_na_bin<<<gn, kNAThreads, 0, s>>>(P, S, p4, tag);
    k_na_scan<<<1, 1024, 0, s>>>(P, S);
    k_na_fill<<<gn, kNAThreads, 0, s>>>(P, S);
    k_na_rank<<<gn, kNAThreads, 0, s>>>(P, S);
    switch (P.s_mode) {
    case 1: k_na_force<1><<<gn, kNAThreads, 0, s>>>(P, S, p4, v4, f4); break;
    case 2: k_na_force<2><<<gn, kNAThreads, 0, s>>>(P, S, p4, v4, f4); break;
    case 3: k_na_force<3><<<gn, kNAThreads, 0, s>>>(P, S, p4, v4, f4); break;
    default: k_na_force<0><<<gn, kNAThreads, 0, s>>>(P, S, p4, v4, f4); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DPD_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return DPD_OK;
}

}  // extern "C"
