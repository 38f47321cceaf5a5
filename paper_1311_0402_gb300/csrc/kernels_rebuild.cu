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
//   k_nbuild_brick / k_nbuild
//              packed neighbour lists of groups of 32 particles, hits
//              compacted by warp ballots as in the paper's builder (Sec. 3.3);
//              the list order depends only on the positions
#include "dpd_internal.cuh"

#include <type_traits>
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
    return g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);  // grid-stride beyond 8 blocks per SM (measured faster)
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

// IDENT (reorder ablation): the arrays keep their order; the copy into the
// other buffer set is the identity.
template <bool LHALF, bool IDENT>
__global__ void k_gather(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t s = D.ctl->parity, t = s ^ 1u;
    const uint32_t os = D.ctl->oparity, ot = os ^ 1u;
    const int lim = P.n > P.ncell ? P.n : P.ncell;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < lim; p += gridDim.x * blockDim.x) {
        if (p < P.n) {
            uint32_t i = IDENT ? (uint32_t)p : D.perm[p];
            if (kChecked && i >= (uint32_t)P.n) {
                atomicOr(&D.ctl->err, kErrBadIndex);
                i = (uint32_t)p;
            }
            float4 x = D.pos[s][i];
            D.pos[t][p] = x;
            D.xref[p] = x;
            D.vel[t][p] = D.vel[s][i];
            if (!LHALF) D.vkick[t][p] = D.vkick[s][i];
            // force[] is not carried: every reader finds it rewritten first
            // (a force evaluation, or the last step of a run)
            D.tag[ot][p] = D.tag[os][i];
            uint32_t id = D.pid[os][i];
            D.pid[ot][p] = id;
            if (P.has_bonds) D.idx_of_pid[id] = (uint32_t)p;  // bond partners are found by caller index
        }
        if (p < P.ncell) D.cell_count[p] = 0u;
    }
}

// idx_of_pid of the live order (when bonds are first set)
__global__ void k_index(SimParams P, Ptrs D)
{
    const uint32_t *pid = D.pid[D.ctl->oparity];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n; p += gridDim.x * blockDim.x) D.idx_of_pid[pid[p]] = (uint32_t)p;
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

// ---------------------------------------------------------------------------
// Neighbour build into packed group lists.  A warp builds one group: lane l
// owns particle first + l and walks its own candidate sequence (the
// particles of its surrounding cells, cell by cell, each cell in index
// order); all lanes take one candidate per iteration in lockstep, and the
// hits of an iteration are compacted with a ballot and appended to the
// group's list in lane order.  The list content and order depend only on the
// positions: deterministic, with no atomics.  In Newton-3 mode a particle
// keeps only partners j > i, and a cell's walk starts past i.

// Append the hits of one lockstep iteration to a group list; returns the
// group's new running total (entries past gcap are counted, not written).
__device__ __forceinline__ uint32_t append_hits(bool hit, uint32_t lane, uint32_t j, uint32_t total,
                                                uint32_t *list, uint32_t gcap)
{
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
    if (hit) {
        const uint32_t k = total + (uint32_t)__popc(m & ((1u << lane) - 1u));
        if (k < gcap) list[k] = (lane << kOwnerShift) | j;
    }
    return total + (uint32_t)__popc(m);
}

// Group descriptor and overflow flag, written by lane 0.
__device__ __forceinline__ void write_group(const Ptrs &D, const SimParams &P, uint32_t g, uint32_t first,
                                            uint32_t owners, uint32_t total)
{
    const uint32_t ne = total < (uint32_t)P.gcap ? total : (uint32_t)P.gcap;
    D.gdesc[g] = make_uint2(first, owners | (ne << 6));
    if (total > (uint32_t)P.gcap) atomicOr(&D.ctl->err, kErrNbrOverflow);
}

// Builder for grids with fewer than three cells along some axis (no
// bricks): groups are the 32-aligned tiles, candidates come from the
// deduplicated cell stencil in global memory.  NOREORDER (reorder ablation):
// the particles stay in load order, so a cell's members are found through
// the sort permutation and the half-list rule is tested per candidate.
template <bool NOREORDER>
__global__ void k_nbuild(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t par = D.ctl->parity;
    const float4 *__restrict__ pos = D.pos[par];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nwarps = gridDim.x * blockDim.x / 32u;
    uint32_t local_max = 0;
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / 32u; g < (uint32_t)P.ngroups; g += nwarps) {
        const uint32_t i = g * kGroup + lane;
        const bool valid = i < (uint32_t)P.n;
        const float4 pi = valid ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t *st = D.stencil + (size_t)(valid ? cell_rank_of(P, D.rank_of_cell, pi, nullptr) : 0u) * kStencil;
        uint32_t s = valid ? 0u : (uint32_t)kStencil, b = 0, n = 0, e = 0;
        auto next_cell = [&]() {
            while (e >= n && s < (uint32_t)kStencil) {
                const uint32_t cc = st[s++];
                if (cc == kNone) {
                    s = kStencil;
                    break;
                }
                b = D.cell_start[cc];
                n = D.cell_start[cc + 1] - b;
                e = (!NOREORDER && P.newton3 && i >= b) ? i + 1u - b : 0u;
            }
        };
        next_cell();
        uint32_t *list = D.nbr + (size_t)g * P.gcap;
        uint32_t total = 0;
        for (;;) {
            const bool act = e < n;
            if (!__any_sync(0xFFFFFFFFu, act)) break;
            bool hit = false;
            uint32_t j = 0;
            if (act) {
                j = NOREORDER ? D.perm[b + e] : b + e;
                const float4 pj = pos[j];
                const float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
                const float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
                const float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
                hit = (dist2_rn(dx, dy, dz) < P.rlist2) & (P.newton3 ? (!NOREORDER || j > i) : j != i);
                ++e;
                if (e >= n) next_cell();
            }
            total = append_hits(hit, lane, j, total, list, (uint32_t)P.gcap);
        }
        if (lane == 0) {
            const uint32_t owners = (uint32_t)P.n - g * kGroup < 32u ? (uint32_t)P.n - g * kGroup : 32u;
            write_group(D, P, g, g * kGroup, owners, total);
        }
        local_max = total > local_max ? total : local_max;
    }
    if (lane == 0 && local_max) atomicMax(&D.ctl->max_nnb, local_max);
}

// Brick builder: one CTA per brick (see brick.cuh).  The CTA stages the
// positions of the brick's halo in shared memory with bulk (TMA) copies;
// its warps take the brick's particles in groups of 32 and build each
// group cell by cell.  For a cell C the warp lays out one candidate
// sequence: C's own particles (index order), then the particles of the
// stencil cells it needs -- in Newton-3 mode those of higher rank than C,
// otherwise all 26 -- and copies it, in chunks, to a per-warp buffer
// (position, index).  The candidates j > i of an owner i at place p of C are
// then exactly the suffix from p + 1 on, because cells are index ranges in
// rank order; full lists take the whole sequence minus i.  For each owner of
// the group in C, all 32 lanes test 32 consecutive candidates per
// iteration, the owner's position broadcast from shared memory, and append
// the hits with a ballot.  No lane diverges and the list order is fixed by
// the positions.  The groups of brick b get the ids lo/32 + ord(b) onwards,
// where ord is the brick's position in rank order: unique ids with no count
// pass; the ids a brick leaves unused (at most one or two) get empty
// descriptors.  A brick whose halo exceeds the staging buffer reads
// positions from global memory.
constexpr int kBuildThreads = 256;
constexpr int kBuildWarps = kBuildThreads / 32;
constexpr int kSlots = 3;               // candidates per lane and chunk, held in registers
constexpr int kChunk = 32 * kSlots;     // chunk of the candidate sequence
// Three candidates per lane and four resident blocks per SM (64 registers,
// no spill): 0.809 against 0.848 ms per rebuild on the 3M fluid with four
// candidates and three blocks (80 registers).  A cell whose sequence needs a
// second chunk interleaves its owners' entries chunk by chunk, which costs the
// pair kernel 1 % (0.311 against 0.308 ms); two candidates per lane cost it
// 2.5 % for a smaller builder gain.
constexpr int kBuildMinBlocks = 4;

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

template <bool WRAP>
__device__ __forceinline__ float pair_d2(const SimParams &P, float4 pj, float4 pi)
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
    return dist2_rn(dx, dy, dz);
}

// fn(std::integral_constant<int, m>) with m = ns clamped to [1, M]: the pass
// instantiated for the chunk's number of live slots (never more than the
// candidate registers hold).
template <int M, typename F>
__device__ __forceinline__ void with_slots(uint32_t ns, F &&fn)
{
    if constexpr (M > 1) {
        if (ns < (uint32_t)M) {
            with_slots<M - 1>(ns, fn);
            return;
        }
    }
    fn(std::integral_constant<int, M>{});
}

// Per-warp table of one slot of the candidate sequence: head[l] is the
// sequence entry (cell) whose first candidate falls on lane l.
struct CellSeq {
    uint8_t head[32];
    uint32_t count;    // atomic-append variant: the group's running total
    uint32_t rows[32]; // row layout: each owner's counts, core | skin << 16
};

// Row layout (list_layout 1, the paper's Sec. 3.3): owner io has the row
// nbr[io * cap, io * cap + cap).  A warp works on one owner at a time; the
// pairs inside r_c at build time (core) are appended at the front of the row
// in sequence order, the other pairs inside r_list (skin) at its back in
// reverse order -- the double insertion, one table and two counters -- and
// k_rows_join later moves the skin part behind the core part.  Full lists:
// every pair is listed by both of its particles.
template <bool WRAP, bool STAGED, int NS>
__device__ __forceinline__ void owner_pass_rows(const SimParams &P, const float4 *__restrict__ pos,
                                                const float4 *s_pos, const uint32_t *s_off,
                                                const float4 (&cand)[kSlots], int t, uint32_t g_own, uint32_t p_lo,
                                                uint32_t p_hi, uint32_t c0, uint32_t c1, uint32_t first, uint32_t lane,
                                                uint32_t *nbr, uint32_t cap, uint32_t *rows)
{
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t p = p_lo; p < p_hi; ++p) {
        const uint32_t io = g_own + p;
        const float4 pio = STAGED ? s_pos[s_off[t] + p] : pos[io];
        const uint32_t o = io - first;
        uint32_t core = rows[o] & 0xFFFFu, skin = rows[o] >> 16;
        uint32_t *row = nbr + (size_t)io * cap;
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) {
            const uint32_t k = c0 + 32u * sl + lane;
            const uint32_t j = __float_as_uint(cand[sl].w);
            const float d2 = pair_d2<WRAP>(P, cand[sl], pio);
            const bool cand_ok = (k < c1) & (j != io);
            const uint32_t m_core = __ballot_sync(0xFFFFFFFFu, cand_ok & (d2 < P.rc2));
            const uint32_t m_skin = __ballot_sync(0xFFFFFFFFu, cand_ok & (d2 < P.rlist2) & !(d2 < P.rc2));
            if ((m_core >> lane) & 1u) {
                const uint32_t q = core + (uint32_t)__popc(m_core & lt);
                if (q < cap) row[q] = j;
            }
            if ((m_skin >> lane) & 1u) {
                const uint32_t q = skin + (uint32_t)__popc(m_skin & lt);
                if (q < cap) row[cap - 1u - q] = j;
            }
            core += (uint32_t)__popc(m_core);
            skin += (uint32_t)__popc(m_skin);
        }
        __syncwarp();
        if (lane == 0) rows[o] = min(core, 0xFFFFu) | (min(skin, 0xFFFFu) << 16);
        __syncwarp();
    }
}

// One chunk against the owners [p_lo, p_hi) of cell slot t, kOwnersPerPass
// owners at a time: every ballot of the pass over the NS live slots first
// (no branches between them, so the tests overlap), then each owner's hits
// are appended in turn, so an owner's entries stay contiguous in the list.
constexpr int kOwnersPerPass = 1;

// ATOMIC (an ablation of the paper's Table 2, ballot against atomic
// insertion): every hit takes its slot with an atomic add on the group's
// shared counter instead of a ballot prefix; the list order then varies run
// to run.
template <bool WRAP, bool STAGED, bool HALF, int NS, bool ATOMIC>
__device__ __forceinline__ uint32_t owner_pass(const SimParams &P, const float4 *__restrict__ pos,
                                               const float4 *s_pos, const uint32_t *s_off, const float4 (&cand)[kSlots],
                                               int t, uint32_t g_own, uint32_t p_lo, uint32_t p_hi, uint32_t c0,
                                               uint32_t c1, uint32_t first, uint32_t lane, uint32_t *list,
                                               uint32_t gcap, uint32_t total, uint32_t *count)
{
    constexpr int NO = kOwnersPerPass;
    const uint32_t lt = (1u << lane) - 1u;
    if constexpr (ATOMIC) {
        for (uint32_t p = p_lo; p < p_hi; ++p) {
            const uint32_t io = g_own + p;
            const float4 pio = STAGED ? s_pos[s_off[t] + p] : pos[io];
            const uint32_t k0 = HALF ? max(p + 1u, c0) : c0;
            const uint32_t entry_owner = (io - first) << kOwnerShift;
#pragma unroll
            for (int sl = 0; sl < NS; ++sl) {
                const uint32_t k = c0 + 32u * sl + lane;
                const uint32_t j = __float_as_uint(cand[sl].w);
                if ((k < c1) & (k >= k0) & within_list<WRAP>(P, cand[sl], pio) & (HALF || j != io)) {
                    const uint32_t q = atomicAdd(count, 1u);
                    if (q < gcap) list[q] = entry_owner | j;
                }
            }
        }
        return total;
    } else {
        for (uint32_t p = p_lo; p < p_hi; p += (uint32_t)NO) {
            uint32_t m[NO][NS];
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                const bool live = p + (uint32_t)o < p_hi;
                const uint32_t po = live ? p + (uint32_t)o : p;
                const uint32_t io = g_own + po;
                const float4 pio = STAGED ? s_pos[s_off[t] + po] : pos[io];
                const uint32_t k0 = HALF ? max(po + 1u, c0) : c0;
#pragma unroll
                for (int sl = 0; sl < NS; ++sl) {
                    const uint32_t k = c0 + 32u * sl + lane;
                    const uint32_t j = __float_as_uint(cand[sl].w);
                    m[o][sl] = __ballot_sync(0xFFFFFFFFu, live & (k < c1) & (k >= k0) & within_list<WRAP>(P, cand[sl], pio) &
                                                              (HALF || j != io));
                }
            }
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                const uint32_t entry_owner = (g_own + p + (uint32_t)o - first) << kOwnerShift;
#pragma unroll
                for (int sl = 0; sl < NS; ++sl) {
                    if ((m[o][sl] >> lane) & 1u) {
                        const uint32_t q = total + (uint32_t)__popc(m[o][sl] & lt);
                        if (q < gcap) list[q] = entry_owner | __float_as_uint(cand[sl].w);
                    }
                    total += (uint32_t)__popc(m[o][sl]);
                }
            }
        }
        return total;
    }
}

// The owners [p_lo, p_hi) (places in cell slot t) of a group whose first
// particle is `first`: their pairs with the candidate sequence, appended to
// the group list; returns the new running total.  A chunk of kChunk
// candidates is held in registers, lane l holding entries c0 + 32 s + l;
// every owner of the cell tests against the same registers (owner_pass).
template <bool WRAP, bool STAGED, bool HALF, bool ATOMIC, bool ROWS = false>
__device__ __forceinline__ uint32_t build_cell(const SimParams &P, const float4 *__restrict__ pos,
                                               const float4 *s_pos, const uint32_t *s_off, const uint32_t *s_gstart,
                                               const uint32_t *s_cnt, CellSeq &w, int t, uint32_t p_lo, uint32_t p_hi,
                                               uint32_t first, uint32_t lane, uint32_t *list, uint32_t gcap,
                                               uint32_t total)
{
    const uint32_t g_own = s_gstart[t], n_own = s_cnt[t];
    // lanes 0..26: stencil cell (dz, dy, dx) = (l / 9, l / 3 % 3, l % 3) - 1;
    // lane 13 is the cell itself
    uint32_t n_use = 0;
    int ts = t;
    if (lane < (uint32_t)kStencil) {
        ts = t + ((int)(lane / 9u) - 1) * (kHalo * kHalo) + ((int)(lane / 3u % 3u) - 1) * kHalo + ((int)(lane % 3u) - 1);
        const uint32_t n = s_cnt[ts];
        const bool use = lane != 13u && (!HALF || s_gstart[ts] > g_own);
        n_use = use ? n : 0u;
    }
    uint32_t incl = n_use;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    const uint32_t total_seq = n_own + __shfl_sync(0xFFFFFFFFu, incl, 31);
    // this lane's sequence entry (lanes 0..26): own cell first (lane 13),
    // then the used stencil cells in lane order
    const uint32_t my_start = lane == 13u ? 0u : n_own + incl - n_use;
    const uint32_t my_n = lane == 13u ? n_own : n_use;
    const uint32_t my_g = lane < (uint32_t)kStencil ? s_gstart[ts] : 0u;
    const uint32_t my_o = lane < (uint32_t)kStencil ? s_off[ts] : 0u;
    for (uint32_t c0 = 0; c0 < total_seq; c0 += (uint32_t)kChunk) {
        const uint32_t c1 = min(total_seq, c0 + (uint32_t)kChunk);
        float4 cand[kSlots];
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
            const uint32_t kb = c0 + 32u * sl;
            cand[sl] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kb < c1) {
                // the cell of candidate kb + lane: the last cell starting at or
                // below it in this slot, else the cell covering kb
                const bool covers = my_n > 0u && my_start <= kb && kb < my_start + my_n;
                const bool starts = my_n > 0u && my_start > kb && my_start < kb + 32u;
                if (covers) w.head[0] = (uint8_t)lane;
                if (starts) w.head[my_start - kb] = (uint8_t)lane;
                const uint32_t hmask = __reduce_or_sync(0xFFFFFFFFu, starts ? 1u << (my_start - kb) : 0u) | 1u;
                __syncwarp();
                const int h = 31 - __clz(hmask & (0xFFFFFFFFu >> (31u - lane)));
                const int c = w.head[h];
                __syncwarp();
                const uint32_t cs = __shfl_sync(0xFFFFFFFFu, my_start, c);
                const uint32_t cg = __shfl_sync(0xFFFFFFFFu, my_g, c);
                const uint32_t co = __shfl_sync(0xFFFFFFFFu, my_o, c);
                const uint32_t k = kb + lane;
                if (k < c1) {
                    const uint32_t e = k - cs;
                    const uint32_t j = cg + e;
                    float4 pj = STAGED ? s_pos[co + e] : pos[j];
                    pj.w = __uint_as_float(j);
                    cand[sl] = pj;
                }
            }
        }
        const uint32_t ns = (c1 - c0 + 31u) / 32u;  // live slots of this chunk
        if (ROWS) {
            // list = the whole table, gcap = the row capacity
            with_slots<kSlots>(ns, [&](auto m) {
                owner_pass_rows<WRAP, STAGED, decltype(m)::value>(P, pos, s_pos, s_off, cand, t, g_own, p_lo, p_hi, c0,
                                                                  c1, first, lane, list, gcap, w.rows);
            });
            continue;
        }
        with_slots<kSlots>(ns, [&](auto m) {
            total = owner_pass<WRAP, STAGED, HALF, decltype(m)::value, ATOMIC>(P, pos, s_pos, s_off, cand, t, g_own,
                                                                           p_lo, p_hi, c0, c1, first, lane, list, gcap,
                                                                           total, &w.count);
        });
    }
    return total;
}

template <bool ATOMIC, bool ROWS>
__global__ void __launch_bounds__(kBuildThreads, kBuildMinBlocks) k_nbuild_brick(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    extern __shared__ float4 s_pos[];  // [P.brick_cap] staged halo positions
    __shared__ uint32_t s_off[kHaloCells + 1];
    __shared__ uint32_t s_gstart[kHaloCells];
    __shared__ uint32_t s_cnt[kHaloCells];
    __shared__ uint32_t s_wsum[kBuildWarps];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ CellSeq s_seq[kBuildWarps];
    const uint32_t par = D.ctl->parity;
    const float4 *pos = D.pos[par];
    const int b = blockIdx.x;
    const BrickRange br = brick_halo(P, D, b, s_off, s_gstart, s_cnt, s_wsum);
    const uint32_t ord = D.brick_ord[b];
    const uint32_t gbase = br.lo / kGroup + ord, gnext = br.hi / kGroup + ord + 1u;
    const uint32_t nloc = br.hi - br.lo, ngrp = (nloc + kGroup - 1) / kGroup;
    const bool local = s_off[kHaloCells] <= (uint32_t)P.brick_cap;  // halo fits the staging buffer
    bool staged = true;
    if (local) staged = brick_stage_bulk(D, &s_bar, s_pos, pos, nullptr, nullptr, s_off, s_gstart, s_cnt);
    if (!staged) {  // the error word is set; leave no lists behind for the force kernel
        for (uint32_t g = gbase + threadIdx.x; g < gnext; g += blockDim.x) D.gdesc[g] = make_uint2(0u, 0u);
        return;
    }
    const int bx = b % P.nb[0], by = (b / P.nb[0]) % P.nb[1], bz = b / (P.nb[0] * P.nb[1]);
    const uint32_t gcap = (uint32_t)P.gcap;
    const bool grid5 = P.nc[0] >= 5 && P.nc[1] >= 5 && P.nc[2] >= 5;
    const uint32_t lane = threadIdx.x & 31u;
    CellSeq &w = s_seq[threadIdx.x / 32u];
    uint32_t local_max = 0;
    for (uint32_t q = threadIdx.x / 32u; q < ngrp; q += kBuildWarps) {
        const uint32_t first = br.lo + q * kGroup;
        const uint32_t owners = nloc - q * kGroup < (uint32_t)kGroup ? nloc - q * kGroup : (uint32_t)kGroup;
        // halo slot of each lane's cell (the own cells of the brick are at 1..kBrick per axis)
        int t_lane = -1, inner_lane = 1;
        if (lane < owners) {
            const float4 pi = pos[first + lane];
            float f;
            const int cx = cell_axis(pi.x, P.cells_per_len[0], P.nc[0], &f);
            const int cy = cell_axis(pi.y, P.cells_per_len[1], P.nc[1], &f);
            const int cz = cell_axis(pi.z, P.cells_per_len[2], P.nc[2], &f);
            t_lane = brick_halo_slot(cx - bx * kBrick + 1, cy - by * kBrick + 1, cz - bz * kBrick + 1);
            // a cell one layer or more inside a grid of >= 5 cells per axis
            // never sees a periodic image in its stencil
            inner_lane = grid5 && cx >= 1 && cx <= P.nc[0] - 2 && cy >= 1 && cy <= P.nc[1] - 2 && cz >= 1 &&
                         cz <= P.nc[2] - 2;
        }
        uint32_t *list = ROWS ? D.nbr : D.nbr + (size_t)(gbase + q) * gcap;
        uint32_t total = 0;
        if (ATOMIC) {
            if (lane == 0) w.count = 0u;
            __syncwarp();
        }
        if (ROWS) {
            w.rows[lane] = 0u;
            __syncwarp();
        }
        // the group's particles are sorted by cell: take the cells in turn
        for (uint32_t l0 = 0; l0 < owners;) {
            const int t = __shfl_sync(0xFFFFFFFFu, t_lane, (int)l0);
            const uint32_t same = __ballot_sync(0xFFFFFFFFu, t_lane == t);
            const uint32_t run = (uint32_t)__popc(same);  // lanes of this cell (consecutive)
            const bool inner = __shfl_sync(0xFFFFFFFFu, inner_lane, (int)l0) != 0;
            const uint32_t p_lo = first + l0 - s_gstart[t];
            const uint32_t p_hi = p_lo + run;
            if (ROWS) {
                const uint32_t rcap = (uint32_t)P.cap;
                if (!local)
                    build_cell<true, false, false, false, true>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, rcap, 0u);
                else if (inner)
                    build_cell<false, true, false, false, true>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, rcap, 0u);
                else
                    build_cell<true, true, false, false, true>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, rcap, 0u);
            } else if (P.newton3) {
                if (!local)
                    total = build_cell<true, false, true, ATOMIC>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, gcap, total);
                else if (inner)
                    total = build_cell<false, true, true, ATOMIC>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, gcap, total);
                else
                    total = build_cell<true, true, true, ATOMIC>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, gcap, total);
            } else {
                if (!local)
                    total = build_cell<true, false, false, ATOMIC>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, gcap, total);
                else if (inner)
                    total = build_cell<false, true, false, ATOMIC>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, gcap, total);
                else
                    total = build_cell<true, true, false, ATOMIC>(P, pos, s_pos, s_off, s_gstart, s_cnt, w, t, p_lo, p_hi, first, lane, list, gcap, total);
            }
            l0 += run;
        }
        if (ATOMIC) {
            __syncwarp();
            total = w.count;
        }
        if (ROWS) {
            // each owner's counts; a row whose two parts do not fit its
            // capacity reports an overflow (the list is rebuilt larger)
            __syncwarp();
            const uint32_t rc = w.rows[lane];
            const uint32_t len = (rc & 0xFFFFu) + (rc >> 16);
            if (lane < owners) {
                D.rowcnt[first + lane] = rc;
                if (len > (uint32_t)P.cap) atomicOr(&D.ctl->err, kErrNbrOverflow);
            }
            total = __reduce_max_sync(0xFFFFFFFFu, lane < owners ? len : 0u);
            __syncwarp();
        } else if (lane == 0) {
            write_group(D, P, gbase + q, first, owners, total);
        }
        local_max = total > local_max ? total : local_max;
    }
    // ids of this brick's range that no group took
    for (uint32_t g = gbase + ngrp + threadIdx.x; g < gnext; g += blockDim.x) D.gdesc[g] = make_uint2(0u, 0u);
    if (lane == 0 && local_max) atomicMax(&D.ctl->max_nnb, local_max);
}

// Row layout: join the two parts of every row (the paper's NeighborListJoin):
// the skin entries, stored from the row's end backwards, are moved behind the
// core entries in their insertion order, so a row reads core pairs first and
// skin pairs after them.  One thread per row: reverse the skin block in
// place, then copy it down to the end of the core block (copying towards
// lower addresses in increasing order never overwrites an unread entry).
__global__ void k_rows_join(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    const uint32_t cap = (uint32_t)P.cap;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const uint32_t rc = D.rowcnt[i];
        uint32_t core = rc & 0xFFFFu, skin = rc >> 16;
        if (core > cap) core = cap;
        if (skin > cap - core) skin = cap - core;  // overflowed: reported by the builder
        uint32_t *row = D.nbr + (size_t)i * cap;
        for (uint32_t a = cap - skin, b = cap - 1u; a < b; ++a, --b) {
            const uint32_t x = row[a];
            row[a] = row[b];
            row[b] = x;
        }
        for (uint32_t k = 0; k < skin; ++k) row[core + k] = row[cap - skin + k];
        D.rowcnt[i] = core + skin;
    }
}

// Row layout: transpose every 32 x 32 tile of the table in place (the paper's
// local transposition, NeighborListTranspose): rows 32 g .. 32 g + 31 and
// entries 32 c .. 32 c + 31 swap their roles, so that entry k of particle
// 32 g + l ends up at row 32 g + (k mod 32), entry 32 (k div 32) + l, and a
// warp whose lane l walks particle 32 g + l reads each entry index with one
// coalesced load.  One warp per group of 32 rows, over the tiles its
// longest row reaches.
__global__ void k_rows_transpose(SimParams P, Ptrs D)
{
    if (!D.ctl->rebuild) return;
    __shared__ uint32_t tile[kBuildWarps][32][33];
    const uint32_t cap = (uint32_t)P.cap, lane = threadIdx.x & 31u, wl = threadIdx.x / 32u;
    const uint32_t ngroups = ((uint32_t)P.n + 31u) / 32u;
    const uint32_t nwarps = gridDim.x * blockDim.x / 32u;
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / 32u; g < ngroups; g += nwarps) {
        const uint32_t i = g * 32u + lane;
        const uint32_t len = i < (uint32_t)P.n ? D.rowcnt[i] : 0u;
        const uint32_t ntiles = (__reduce_max_sync(0xFFFFFFFFu, len) + 31u) / 32u;
        uint32_t *base = D.nbr + (size_t)g * 32u * cap;
        for (uint32_t c = 0; c < ntiles; ++c) {
#pragma unroll 8
            for (uint32_t r = 0; r < 32u; ++r) tile[wl][r][lane] = base[(size_t)r * cap + 32u * c + lane];
            __syncwarp();
#pragma unroll 8
            for (uint32_t r = 0; r < 32u; ++r) base[(size_t)r * cap + 32u * c + lane] = tile[wl][lane][r];
            __syncwarp();
        }
    }
}

// Failure-detection probe: the bounded mbarrier wait of the brick staging,
// on a transaction that nothing delivers (expect_tx with no copy issued).
// The wait gives up after `polls` polls and the timeout bit is set; no
// asynchronous copy is in flight, so the block exits cleanly.
__global__ void k_wait_probe(Ptrs D, uint32_t polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect_tx(&bar, 16u);
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, polls);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(&D.ctl->err, kErrTimeout);
}

}  // namespace

cudaError_t launch_wait_probe(const Ptrs &D, uint32_t polls, cudaStream_t s)
{
    k_wait_probe<<<1, 32, 0, s>>>(D, polls);
    return cudaGetLastError();
}

int scan_blocks_for(int ncell) { return (ncell + kScanTile - 1) / kScanTile; }

cudaError_t init_build_attributes(int max_dyn_smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_nbuild_brick<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_nbuild_brick<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_nbuild_brick<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
    return e;
}

cudaError_t launch_index(const SimParams &P, const Ptrs &D, cudaStream_t s)
{
    k_index<<<grid_for(P.n), kThreads, 0, s>>>(P, D);
    return cudaGetLastError();
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
    if (P.no_reorder) {
        if (P.lambda_half) k_gather<true, true><<<gg, kThreads, 0, s>>>(P, D);
        else k_gather<false, true><<<gg, kThreads, 0, s>>>(P, D);
    } else {
        if (P.lambda_half) k_gather<true, false><<<gg, kThreads, 0, s>>>(P, D);
        else k_gather<false, false><<<gg, kThreads, 0, s>>>(P, D);
    }
    k_commit<<<1, 1, 0, s>>>(D);
    if (P.use_bricks) {
        const size_t smem = sizeof(float4) * (size_t)P.brick_cap;
        if (P.list_layout == 1) {
            k_nbuild_brick<false, true><<<P.nbricks, kBuildThreads, smem, s>>>(P, D);
            k_rows_join<<<g, kThreads, 0, s>>>(P, D);
            k_rows_transpose<<<grid_for((P.n + 31) / 32 * 32), kBuildThreads, 0, s>>>(P, D);
        } else if (P.list_builder == 1) {
            k_nbuild_brick<true, false><<<P.nbricks, kBuildThreads, smem, s>>>(P, D);
        } else {
            k_nbuild_brick<false, false><<<P.nbricks, kBuildThreads, smem, s>>>(P, D);
        }
    } else if (P.no_reorder) {
        k_nbuild<true><<<g, kThreads, 0, s>>>(P, D);
    } else {
        k_nbuild<false><<<g, kThreads, 0, s>>>(P, D);
    }
    return cudaGetLastError();
}

}  // namespace dpd
