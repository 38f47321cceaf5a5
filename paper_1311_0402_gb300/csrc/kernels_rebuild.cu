// kernels_rebuild.cu -- binning, scan, deterministic reorder and neighbour
// list construction (Secs. 3.2-3.3 of Tang & Karniadakis).
//
// The chain runs inside captured CUDA graphs every step; each kernel first
// reads the device rebuild flag set by the integrator's displacement check
// and returns at once when no rebuild is due, so the graph never changes.
//
//   k_bin      cell of each particle (cells ranked along a Morton curve, the
//              first level of the paper's two-level Morton order) + an
//              arrival slot from a per-cell counter, and a 6-bit Morton key
//              of the particle's sub-cell (the second level)
//   k_scan_*   exclusive scan of the cell counts -> cell_start
//   k_scatter  provisional position = cell_start + slot
//   k_rank     final position = cell_start + rank of (sub-cell key, caller
//              index) inside the cell: independent of the atomics' order,
//              so the particle order and the lists are deterministic
//   k_gather   permute the particle arrays into the other buffer set
//   k_commit   flip the live buffer set
//   k_nbuild   one thread per particle walks the 27 stencil cells in
//              ascending rank order, so every list is strictly increasing
//              (the property of the paper's builder, obtained here without
//              warp votes because each thread owns its particle's row)
#include "dpd_internal.cuh"
#include "dpd_math.cuh"
#include "brick.cuh"

namespace dpd {

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 512;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;  // 2048 cells per block
constexpr uint32_t kCellMask = (1u << 26) - 1u;

int grid_for(int n)
{
    int g = (n + kThreads - 1) / kThreads;
    return g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
}

__device__ __forceinline__ int cell_axis(float x, float cpl, int nc, float *frac)
{
    float f = x * cpl;
    int c = (int)f;  // x >= 0; NaN converts to 0
    c = c < 0 ? 0 : (c >= nc ? nc - 1 : c);
    *frac = f - (float)c;
    return c;
}

__device__ __forceinline__ uint32_t sub_axis(float frac)
{
    int s = (int)(frac * 4.0f);
    return (uint32_t)(s < 0 ? 0 : (s > 3 ? 3 : s));
}

// Morton interleave of three 2-bit coordinates (x in the lowest bit).
__device__ __forceinline__ uint32_t morton2bit(uint32_t x, uint32_t y, uint32_t z)
{
    return (x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2) | ((x & 2u) << 2) | ((y & 2u) << 3) | ((z & 2u) << 4);
}

__device__ __forceinline__ uint32_t cell_rank_of(const SimParams &P, const uint32_t *rank_of_cell, float4 p,
                                                 uint32_t *sub)
{
    float fx, fy, fz;
    int cx = cell_axis(p.x, P.cells_per_len[0], P.nc[0], &fx);
    int cy = cell_axis(p.y, P.cells_per_len[1], P.nc[1], &fy);
    int cz = cell_axis(p.z, P.cells_per_len[2], P.nc[2], &fz);
    if (sub) *sub = morton2bit(sub_axis(fx), sub_axis(fy), sub_axis(fz));
    return rank_of_cell[(cz * P.nc[1] + cy) * P.nc[0] + cx];
}

__global__ void k_bin(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t par = D.ctl->parity;
    const float4 *pos = D.pos[par];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        uint32_t sub;
        uint32_t c = cell_rank_of(P, D.rank_of_cell, pos[i], &sub);
        D.key[i] = (sub << 26) | c;
        D.slot[i] = atomicAdd(&D.cell_count[c], 1u);
    }
}

// Block-level exclusive scan of up to kScanTile values; returns the total.
__device__ uint32_t block_exclusive_scan(uint32_t (&v)[kScanPerThread], uint32_t *warp_sums)
{
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        uint32_t x = v[k];
        v[k] = t;
        t += x;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (kScanThreads / 32) ? warp_sums[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (kScanThreads / 32)) warp_sums[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31) warp_sums[32] = wi;                        // block total
    }
    __syncthreads();
    uint32_t off = warp_sums[warp] + incl - t;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) v[k] += off;
    uint32_t total = warp_sums[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    __shared__ uint32_t ws[33];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
    uint32_t v[kScanPerThread];
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) v[k] = (base + k < P.ncell) ? D.cell_count[base + k] : 0u;
    uint32_t total = block_exclusive_scan(v, ws);
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
        if (base + k < P.ncell) D.cell_start[base + k] = v[k];
    if (threadIdx.x == 0) D.scan_part[blockIdx.x] = total;
}

// Scans the block totals (one block, loops over tiles of kScanTile).
__global__ void __launch_bounds__(kScanThreads) k_scan_top(int nblocks, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    __shared__ uint32_t ws[33];
    uint32_t carry = 0;
    for (int tile = 0; tile < nblocks; tile += kScanTile) {
        const int base = tile + threadIdx.x * kScanPerThread;
        uint32_t v[kScanPerThread];
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k) v[k] = (base + k < nblocks) ? D.scan_part[base + k] : 0u;
        uint32_t total = block_exclusive_scan(v, ws);
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k)
            if (base + k < nblocks) D.scan_part[base + k] = v[k] + carry;
        carry += total;
    }
}

__global__ void k_scan_add(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= P.ncell; c += gridDim.x * blockDim.x) {
        if (c == P.ncell)
            D.cell_start[c] = (uint32_t)P.n;
        else
            D.cell_start[c] += D.scan_part[c / kScanTile];
    }
}

__global__ void k_scatter(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t *pid = D.pid[D.ctl->oparity];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        uint32_t k = D.key[i];
        uint32_t dst = D.cell_start[k & kCellMask] + D.slot[i];
        D.tmp_idx[dst] = (uint32_t)i;
        D.skey[dst] = ((unsigned long long)(k >> 26) << 32) | pid[i];
    }
}

__global__ void k_rank(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n; p += gridDim.x * blockDim.x) {
        uint32_t i = D.tmp_idx[p];
        uint32_t c = D.key[i] & kCellMask;
        uint32_t b = D.cell_start[c], e = D.cell_start[c + 1];
        unsigned long long my = D.skey[p];
        uint32_t r = 0;
        for (uint32_t q = b; q < e; ++q) r += (D.skey[q] < my) ? 1u : 0u;
        D.perm[b + r] = i;
    }
}

template <bool LHALF>
__global__ void k_gather(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t s = D.ctl->parity, t = s ^ 1u;
    const uint32_t os = D.ctl->oparity, ot = os ^ 1u;
    const int lim = P.n > P.ncell ? P.n : P.ncell;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < lim; p += gridDim.x * blockDim.x) {
        if (p < P.n) {
            uint32_t i = D.perm[p];
            float4 x = D.pos[s][i];
            D.pos[t][p] = x;
            D.xref[p] = x;
            D.vel[t][p] = D.vel[s][i];
            if (!LHALF) D.vkick[t][p] = D.vkick[s][i];
            D.force[t][p] = D.force[s][i];
            D.tag[ot][p] = D.tag[os][i];
            uint32_t id = D.pid[os][i];
            D.pid[ot][p] = id;
            D.idx_of_pid[id] = (uint32_t)p;
        }
        if (p < P.ncell) D.cell_count[p] = 0u;
    }
}

__global__ void k_commit(Ptrs D)
{
    DevCtl *c = D.ctl;
    if (!c->rebuild) return;
    c->parity ^= 1u;
    c->oparity ^= 1u;
    c->since_rebuild = 0u;
    c->nrebuild += 1ull;
    c->max_nnb = 0u;
}

__global__ void k_nbuild(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t par = D.ctl->parity;
    const float4 *pos = D.pos[par];
    uint32_t local_max = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        float4 pi = pos[i];
        uint32_t c = cell_rank_of(P, D.rank_of_cell, pi, nullptr);
        const uint32_t *st = D.stencil + (size_t)c * kStencil;
        uint32_t *row = D.nbr + (size_t)(i >> 5) * P.cap * 32 + (i & 31);
        uint32_t cnt = 0;
        for (int s = 0; s < kStencil; ++s) {
            uint32_t cc = st[s];
            if (cc == kNone) break;
            uint32_t b = D.cell_start[cc], e = D.cell_start[cc + 1];
            for (uint32_t j = b; j < e; ++j) {
                if (P.newton3 ? j <= (uint32_t)i : j == (uint32_t)i) continue;
                float4 pj = pos[j];
                float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
                float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
                float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
                if (dist2_rn(dx, dy, dz) < P.rlist2) {
                    if (cnt < (uint32_t)P.cap) row[(size_t)cnt * 32] = j;
                    ++cnt;
                }
            }
        }
        if (cnt > (uint32_t)P.cap) atomicOr(&D.ctl->err, kErrNbrOverflow);
        D.nnb[i] = cnt < (uint32_t)P.cap ? cnt : (uint32_t)P.cap;
        local_max = cnt > local_max ? cnt : local_max;
    }
    // warp max, then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, local_max, o);
        local_max = y > local_max ? y : local_max;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&D.ctl->max_nnb, local_max);
}

// Neighbour build, one CTA per brick (see brick.cuh).  In Newton-3 mode the
// rows keep only partners j > i (half rows), and stencil cells whose
// particles all precede i are skipped outright.  The CTA stages the
// positions of the brick's halo in shared memory with bulk (TMA) copies; each
// thread owns one particle of the brick and tests the particles of its 27
// surrounding cells, read from shared memory, with the FP32 predicate,
// appending hits to its own row in the fixed stencil order (dz, dy, dx =
// -1..1, each cell in index order): deterministic rows with no votes or
// atomics.  Stencil cells whose nearest point lies beyond r_list are skipped.
// A brick whose halo exceeds the staging buffer reads positions from global
// memory.
constexpr int kBuildThreads = 256;

template <bool WRAP>
__device__ __forceinline__ bool within_list(const SimParams &P, float4 pj, float4 pi)
{
    float dx, dy, dz;
    if (WRAP) {
        dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
        dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
        dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
    } else {
        dx = __fsub_rn(pj.x, pi.x);
        dy = __fsub_rn(pj.y, pi.y);
        dz = __fsub_rn(pj.z, pi.z);
    }
    return dist2_rn(dx, dy, dz) < P.rlist2;
}

// Squared distance from a particle at fractional position f (in units of the
// cell side, per axis) in its cell to the neighbour cell at offset o, along
// the axis: 0 for the same slab, f for the slab below, 1 - f for the slab
// above; times the squared side.  A cell whose nearest point is farther than
// r_list (with a margin far above FP32 rounding of positions and cell
// indices) holds no particle the predicate can admit and is skipped.
__device__ __forceinline__ float slab_gap(float f, int o, float side)
{
    const float g = o < 0 ? f : (o > 0 ? 1.0f - f : 0.0f);
    const float d = fmaxf(g * side - 1e-4f, 0.0f);
    return d * d;
}

// Row of one particle: the particles of its 27 surrounding cells (stencil
// order dz, dy, dx = -1..1, each cell in index order) that pass the FP32
// predicate, as 32-bit global indices in the particle's row of its 32-wide
// tile (entry k at k * 32).  Candidate positions come from the staged halo
// (STAGED) or from global memory.
template <bool WRAP, bool STAGED, bool HALF>
__device__ __forceinline__ uint32_t build_row(const SimParams &P, const float4 *pos, const float4 *s_pos,
                                              const uint32_t *s_off, const uint32_t *s_gstart,
                                              const uint32_t *s_cnt, int hx, int hy, int hz, const float *frac,
                                              uint32_t i, float4 pi, uint32_t *row, uint32_t cap)
{
    const float side[3] = {P.L[0] / (float)P.nc[0], P.L[1] / (float)P.nc[1], P.L[2] / (float)P.nc[2]};
    uint32_t cnt = 0;
    for (int oz = -1; oz <= 1; ++oz) {
        const float gz = slab_gap(frac[2], oz, side[2]);
        for (int oy = -1; oy <= 1; ++oy) {
            const float gyz = gz + slab_gap(frac[1], oy, side[1]);
            for (int ox = -1; ox <= 1; ++ox) {
                if (gyz + slab_gap(frac[0], ox, side[0]) >= P.rlist2) continue;
                const int t = brick_halo_slot(hx + ox, hy + oy, hz + oz);
                const uint32_t o = s_off[t], g = s_gstart[t], n = s_cnt[t];
                if (HALF && g + n <= i + 1u) continue;  // every particle of the cell precedes i
                for (uint32_t e = 0; e < n; ++e) {
                    const uint32_t j = g + e;
                    const float4 pj = STAGED ? s_pos[o + e] : pos[j];
                    const bool hit = within_list<WRAP>(P, pj, pi) & (HALF ? (j > i) : (j != i));
                    if (hit & (cnt < cap)) row[(size_t)cnt * 32] = j;
                    cnt += hit ? 1u : 0u;
                }
            }
        }
    }
    return cnt;
}

__global__ void __launch_bounds__(kBuildThreads) k_nbuild_brick(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    extern __shared__ float4 s_pos[];  // [P.brick_cap] staged halo positions
    __shared__ uint32_t s_off[kHaloCells + 1];
    __shared__ uint32_t s_gstart[kHaloCells];
    __shared__ uint32_t s_cnt[kHaloCells];
    __shared__ uint32_t s_wsum[kBuildThreads / 32];
    __shared__ __align__(8) uint64_t s_bar;
    const uint32_t par = D.ctl->parity;
    const float4 *pos = D.pos[par];
    const int b = blockIdx.x;
    const BrickRange br = brick_halo(P, D, b, s_off, s_gstart, s_cnt, s_wsum);
    const bool local = s_off[kHaloCells] <= (uint32_t)P.brick_cap;  // halo fits the staging buffer
    bool staged = true;
    if (local) staged = brick_stage_bulk(D, &s_bar, s_pos, pos, nullptr, nullptr, s_off, s_gstart, s_cnt);
    if (!staged) {  // the error word is set; leave no rows behind for the force kernel
        for (uint32_t i = br.lo + threadIdx.x; i < br.hi; i += blockDim.x) D.nnb[i] = 0u;
        return;
    }
    const int bx = b % P.nb[0], by = (b / P.nb[0]) % P.nb[1], bz = b / (P.nb[0] * P.nb[1]);
    const uint32_t cap = (uint32_t)P.cap;
    const bool grid5 = P.nc[0] >= 5 && P.nc[1] >= 5 && P.nc[2] >= 5;
    uint32_t local_max = 0;
    const uint32_t nloc = br.hi - br.lo;
    for (uint32_t p0 = 0; p0 < nloc; p0 += blockDim.x) {
        const uint32_t p = p0 + threadIdx.x;
        const bool valid = p < nloc;
        const uint32_t i = br.lo + p;
        float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
        int cx = 1, cy = 1, cz = 1;
        float fx_ = 0.f, fy_ = 0.f, fz_ = 0.f;
        if (valid) {
            pi = pos[i];
            cx = cell_axis(pi.x, P.cells_per_len[0], P.nc[0], &fx_);
            cy = cell_axis(pi.y, P.cells_per_len[1], P.nc[1], &fy_);
            cz = cell_axis(pi.z, P.cells_per_len[2], P.nc[2], &fz_);
        }
        const int hx = cx - bx * kBrick + 1, hy = cy - by * kBrick + 1, hz = cz - bz * kBrick + 1;  // 1..kBrick
        // a cell one layer or more inside a grid of >= 5 cells per axis never
        // sees a periodic image in its stencil: the whole warp can skip the
        // minimum image when all its particles sit in such cells
        const bool inner = grid5 && cx >= 1 && cx <= P.nc[0] - 2 && cy >= 1 && cy <= P.nc[1] - 2 && cz >= 1 &&
                           cz <= P.nc[2] - 2;
        const bool warp_inner = __all_sync(0xFFFFFFFFu, inner || !valid);
        if (!valid) continue;
        uint32_t *row = D.nbr + (size_t)(i >> 5) * cap * 32 + (i & 31u);
        const float frac[3] = {fx_, fy_, fz_};
        uint32_t cnt;
        if (P.newton3) {
            if (local)
                cnt = warp_inner
                          ? build_row<false, true, true>(P, pos, s_pos, s_off, s_gstart, s_cnt, hx, hy, hz, frac, i, pi, row, cap)
                          : build_row<true, true, true>(P, pos, s_pos, s_off, s_gstart, s_cnt, hx, hy, hz, frac, i, pi, row, cap);
            else
                cnt = build_row<true, false, true>(P, pos, s_pos, s_off, s_gstart, s_cnt, hx, hy, hz, frac, i, pi, row, cap);
        } else {
            if (local)
                cnt = warp_inner
                          ? build_row<false, true, false>(P, pos, s_pos, s_off, s_gstart, s_cnt, hx, hy, hz, frac, i, pi, row, cap)
                          : build_row<true, true, false>(P, pos, s_pos, s_off, s_gstart, s_cnt, hx, hy, hz, frac, i, pi, row, cap);
            else
                cnt = build_row<true, false, false>(P, pos, s_pos, s_off, s_gstart, s_cnt, hx, hy, hz, frac, i, pi, row, cap);
        }
        if (cnt > cap) atomicOr(&D.ctl->err, kErrNbrOverflow);
        D.nnb[i] = min(cnt, cap);
        local_max = max(local_max, cnt);
    }
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xFFFFFFFFu, local_max, o));
    if ((threadIdx.x & 31) == 0 && local_max) atomicMax(&D.ctl->max_nnb, local_max);
}

}  // namespace

int scan_blocks_for(int ncell) { return (ncell + kScanTile - 1) / kScanTile; }

cudaError_t init_build_attributes(int max_dyn_smem)
{
    return cudaFuncSetAttribute(k_nbuild_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
}

cudaError_t launch_rebuild(const SimParams &P, const Ptrs &D, cudaStream_t s, int n_scan_blocks)
{
    const int g = grid_for(P.n);
    k_bin<<<g, kThreads, 0, s>>>(P, D);
    k_scan_blocks<<<n_scan_blocks, kScanThreads, 0, s>>>(P, D);
    k_scan_top<<<1, kScanThreads, 0, s>>>(n_scan_blocks, D);
    k_scan_add<<<grid_for(P.ncell + 1), kThreads, 0, s>>>(P, D);
    k_scatter<<<g, kThreads, 0, s>>>(P, D);
    k_rank<<<g, kThreads, 0, s>>>(P, D);
    const int gg = grid_for(P.n > P.ncell ? P.n : P.ncell);
    if (P.lambda_half)
        k_gather<true><<<gg, kThreads, 0, s>>>(P, D);
    else
        k_gather<false><<<gg, kThreads, 0, s>>>(P, D);
    k_commit<<<1, 1, 0, s>>>(D);
    if (P.use_bricks) {
        k_nbuild_brick<<<P.nbricks, kBuildThreads, sizeof(float4) * (size_t)P.brick_cap, s>>>(P, D);
    } else {
        k_nbuild<<<g, kThreads, 0, s>>>(P, D);
    }
    return cudaGetLastError();
}

}  // namespace dpd
