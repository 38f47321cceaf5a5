// kernels_ensemble.cu -- the ensemble kernel: many small boxes, each owned by
// a thread-block cluster, advanced a whole chunk of steps per launch with the
// box resident in shared memory.
//
// Every CTA of a box's cluster holds a replica of the box (positions, the
// velocity the pair force reads with the particle's signature, the
// half-kicked velocity when lambda != 1/2) and, each step:
//   1. bins the box into cells of side >= r_c (the cell list of Sec. 3.2.3):
//      a counting sort by shared-memory atomics, then each cell's members put
//      in index order, so every replica holds the same cell lists;
//   2. evaluates the pair forces of its share of the cells: work units of
//      consecutive cells go round-robin to the cluster's CTAs and their warps.
//      A warp takes a unit cell by cell; a cell's 27-cell stencil (Sec.
//      3.3.1) is gathered in rounds of 128 candidates, each lane holding 4 in
//      registers, and every owner of the cell tests them 32 at a time.  Lane
//      l < 27 keeps neighbour cell l's periodic shift s; a slot holding a
//      shifted candidate fetches it by shuffle and forms (x_j - x_i) + s, the
//      rounding of the other kernels' FP32 predicate.  Hits inside r_c go to
//      a per-warp ring in shared memory, evaluated 32 pairs at a time by the
//      whole warp (Eqs. 2-9, the TEA hash and Box-Muller Gaussian of Sec.
//      3.5), and summed per owner by a segmented shuffle scan (each pair is
//      seen from both sides).
//      Within a candidate round every owner's hits are one run of the ring;
//      the ring is emptied between rounds, so a batch never holds two runs of
//      one owner.  In the optional Newton-3 mode the stencil is halved (the
//      own cell's later members and the 13 forward cells) and the partner's
//      share goes by an atomic to the shared memory of the CTA that
//      integrates it;
//   3. integrates the particles of its cells (the lambda form of velocity
//      Verlet, Sec. 3.1 / Algorithm 1) and stores their new state into every
//      replica of the cluster through distributed shared memory.
// Two cluster barriers per step separate the reads of a step from the
// writes of the next (a third, in Newton-3 mode with more than one CTA per
// box, orders the zeroing of every replica's accumulators before any remote
// add).  The last step writes positions, full-step velocities and forces
// (w = the particle's virial share) to device memory.
//
// Fixed summation order (the default mode): units never span a queue flush, a
// cell's members are in index order and the stencil order is fixed, so a force
// does not depend on the cluster size, the block size or the other boxes of
// the launch.
#include "dpd_math.cuh"
#include "ensemble.cuh"

#include <algorithm>
#include <cooperative_groups.h>
#include <mutex>

namespace cg = cooperative_groups;

namespace dpd {

namespace {

constexpr int kEnsMaxThreads = 512;
constexpr int kObsThreads = 256;

// x wrapped into [0, L) (the same arithmetic as the other integrators).
__device__ __forceinline__ float ens_wrap(float x, float L, float invL)
{
    x = x - L * floorf(x * invL);
    if (x >= L) x -= L;
    if (x < 0.0f) x += L;
    if (x >= L) x = 0.0f;
    return x;
}

__device__ __forceinline__ int ens_axis(float x, float cpl, int nc)
{
    const int c = (int)(x * cpl);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__device__ __forceinline__ int ens_cell(const EnsBox &B, float4 p)
{
    return (ens_axis(p.z, B.cpl[2], B.nc[2]) * B.nc[1] + ens_axis(p.y, B.cpl[1], B.nc[1])) * B.nc[0] +
           ens_axis(p.x, B.cpl[0], B.nc[0]);
}

struct EnsPtrs {
    float4 *pos, *u, *vh, *f;
    uint32_t *start, *cnt;
    uint16_t *idx, *slot;
    uint8_t *own;  // Newton-3 mode: the cluster rank that integrates each particle this step
    int C, rank;   // CTAs per box, this CTA's rank
};

// Exclusive scan of cnt[0, ncell) into start[0, ncell], start[ncell] = total.
__device__ void ens_scan(const uint32_t *cnt, uint32_t *start, int ncell, uint32_t *wsum)
{
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = T >> 5;
    const int per = (ncell + T - 1) / T;
    const int lo = min(ncell, t * per), hi = min(ncell, lo + per);
    uint32_t sum = 0;
    for (int c = lo; c < hi; ++c) sum += cnt[c];
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? wsum[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) wsum[lane] = wi - w;
        if (lane == 31) wsum[32] = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - sum;
    for (int c = lo; c < hi; ++c) {
        start[c] = run;
        run += cnt[c];
    }
    if (t == 0) start[ncell] = wsum[32];
    __syncthreads();
}

// Evaluate ring entries [head, head + nb) (nb <= 32), one pair per lane, and
// add the sums of each run of equal owners to the owner's accumulator.
template <int SMODE, bool VIR, bool N3>
__device__ __forceinline__ void ens_batch(const EnsBox &B, const EnsPtrs &S, const float4 *q, const uint32_t (&key)[4],
                                          uint32_t head, int nb, int lane)
{
    __syncwarp();
    float fx = 0.f, fy = 0.f, fz = 0.f, fw = 0.f;
    uint32_t owner = 0x10000u + (uint32_t)lane;  // distinct dummy owners for idle lanes
    const float4 e = q[(head + (uint32_t)lane) & (kEnsQueue - 1)];
    const uint32_t pk = __float_as_uint(e.w);
    const uint32_t i = pk >> 16, j = pk & 0xFFFFu;
    // an entry naming a particle outside the box would be a bookkeeping fault:
    // it is reported and skipped, never dereferenced
    const bool bad = lane < nb && (i >= (uint32_t)B.n || j >= (uint32_t)B.n);
    if (bad) {
        atomicOr(B.err, kErrBadIndex);
        atomicOr(B.any_err, kErrBadIndex);
    }
    if (lane < nb && !bad) {
        owner = i;
        const float4 wi = S.u[i], vj = S.u[j];
        const float dx = e.x, dy = e.y, dz = e.z;
        const float d2 = dist2_rn(dx, dy, dz);
        const float inv_r = rsqrtf(d2);
        const float r = d2 * inv_r;
        const float wgt = fmaxf(fmaf(-r, B.inv_rc, 1.0f), 0.0f);
        const float wR = weight_R<SMODE>(wgt, B.s);
        // e_ij = -d / r; e . v_ij = -(d . (v_i - v_j)) / r
        const float ev = -((dx * (wi.x - vj.x) + dy * (wi.y - vj.y)) + dz * (wi.z - vj.z)) * inv_r;
        uint32_t A, Bw;
        pair_hash(__float_as_uint(wi.w), __float_as_uint(vj.w), key, A, Bw);
        const float xi = gauss_from_hash(A, Bw);
        float a = B.a[0];
        if (B.n_species > 1) a = B.a[__float_as_int(S.pos[i].w) * B.n_species + __float_as_int(S.pos[j].w)];
        const float F = fmaf(a, wgt, fmaf(-B.gamma * wR * wR, ev, B.sigma_isdt * wR * xi));
        if (VIR) fw = N3 ? a * wgt * r : 0.5f * (a * wgt * r);  // once per pair, or from both ends
        const float sc = -F * inv_r;
        fx = sc * dx;
        fy = sc * dy;
        fz = sc * dz;
        if (N3) {  // Newton's third law: the partner gets -F e_ij, in its owner's shared memory
            float4 *fj = S.f;
            if (S.C > 1 && (int)S.own[j] != S.rank) fj = cg::this_cluster().map_shared_rank(S.f, (int)S.own[j]);
            atomicAdd(&fj[j].x, -fx);
            atomicAdd(&fj[j].y, -fy);
            atomicAdd(&fj[j].z, -fz);
        }
    }
    // segmented inclusive scan over runs of equal owners (fixed order)
    const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, owner, 1);
    const uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != owner);
    const int first = 31 - __clz(heads & (0xFFFFFFFFu >> (31 - lane)));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float ax = __shfl_up_sync(0xFFFFFFFFu, fx, d);
        const float ay = __shfl_up_sync(0xFFFFFFFFu, fy, d);
        const float az = __shfl_up_sync(0xFFFFFFFFu, fz, d);
        float aw = 0.f;
        if (VIR) aw = __shfl_up_sync(0xFFFFFFFFu, fw, d);
        if (lane - first >= d) {
            fx += ax;
            fy += ay;
            fz += az;
            if (VIR) fw += aw;
        }
    }
    const uint32_t next = __shfl_down_sync(0xFFFFFFFFu, owner, 1);
    if (lane < nb && (lane == 31 || next != owner)) {
        if (N3) {  // other warps add partner shares to the same accumulator
            atomicAdd(&S.f[owner].x, fx);
            atomicAdd(&S.f[owner].y, fy);
            atomicAdd(&S.f[owner].z, fz);
            if (VIR) atomicAdd(&S.f[owner].w, fw);
        } else {
            float4 acc = S.f[owner];
            acc.x += fx;
            acc.y += fy;
            acc.z += fz;
            if (VIR) acc.w += fw;
            S.f[owner] = acc;
        }
    }
    __syncwarp();
}

// Pair forces of the owners in work unit u (cells [u K, u K + K)) into S.f.
// N3: half stencil (the own cell's later members and the 13 forward cells),
// the partner's share added by a shared-memory atomic.
template <int SMODE, bool VIR, bool N3>
__device__ void ens_unit(const EnsBox &B, const EnsPtrs &S, float4 *q, uint32_t *cand, int u, int lane)
{
    const uint32_t key[4] = {B.key[0], B.key[1], B.key[2], B.key[3]};
    const uint32_t lt = (1u << lane) - 1u;
    const int c0 = u * kEnsUnitCells, c1 = min(c0 + kEnsUnitCells, B.ncell);
    const int ncx = B.nc[0], ncy = B.nc[1], ncz = B.nc[2];
    uint32_t head = 0u, tail = 0u;
    for (int c = c0; c < c1; ++c) {
        const int ob = (int)S.start[c], oe = (int)S.start[c + 1];
        if (ob == oe) continue;
        if (!N3)
            for (int k = ob + lane; k < oe; k += 32) S.f[S.idx[k]] = make_float4(0.f, 0.f, 0.f, 0.f);
        // lane l < 27: neighbour cell l of the stencil, its member range and shift
        const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
        // (the shift stays in the lane's registers; a candidate fetches it by shuffle)
        int len = 0, sbeg = 0;
        float shx = 0.f, shy = 0.f, shz = 0.f;
        if (lane < (N3 ? 14 : 27)) {
            int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
            if (N3) {  // lane 0: the own cell; lanes 1..13: the forward offsets
                const int k = lane - 1;
                ox = lane == 0 ? 0 : (k < 9 ? k % 3 - 1 : (k < 12 ? k - 10 : 1));
                oy = lane == 0 ? 0 : (k < 9 ? k / 3 - 1 : (k < 12 ? 1 : 0));
                oz = lane == 0 ? 0 : (k < 9 ? 1 : 0);
            }
            int x = cx + ox, y = cy + oy, z = cz + oz;
            if (x < 0) { x += ncx; shx = -B.L[0]; } else if (x >= ncx) { x -= ncx; shx = B.L[0]; }
            if (y < 0) { y += ncy; shy = -B.L[1]; } else if (y >= ncy) { y -= ncy; shy = B.L[1]; }
            if (z < 0) { z += ncz; shz = -B.L[2]; } else if (z >= ncz) { z -= ncz; shz = B.L[2]; }
            const int cc = (z * ncy + y) * ncx + x;
            sbeg = (int)S.start[cc];
            len = (int)S.start[cc + 1] - sbeg;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const int pre = incl - len;
        const int ncand = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const int len0 = __shfl_sync(0xFFFFFFFFu, len, 0);  // N3: the own cell leads the candidates
        for (int base = 0; base < ncand; base += kEnsCand) {
            __syncwarp();
            if (lane < (N3 ? 14 : 27)) {
                const int lo = max(pre, base), hi = min(pre + len, base + kEnsCand);
                for (int p = lo; p < hi; ++p) cand[p - base] = (uint32_t)S.idx[sbeg + p - pre] | ((uint32_t)lane << 16);
            }
            __syncwarp();
            const int nch = min(kEnsCand, ncand - base);
            // this lane's candidates of the round in registers: base + 32 r + lane.
            // A slot with a periodic image anywhere in the warp is marked; its
            // tests add the shift after the difference, (x_j - x_i) + s, the
            // rounding of the pinned FP32 predicate.
            float px[kEnsSlots], py[kEnsSlots], pz[kEnsSlots];
            uint32_t pe[kEnsSlots];  // j | stencil cell << 16
            uint32_t shifted = 0u;   // warp-uniform: bit r = slot r holds a shifted candidate
#pragma unroll
            for (int r = 0; r < kEnsSlots; ++r) {
                const int t = 32 * r + lane;
                const bool act = t < nch;
                const uint32_t e = act ? cand[t] : 0u;
                const int sl = (int)(e >> 16);
                // every lane takes part in each shuffle and the ballot
                const float sx = __shfl_sync(0xFFFFFFFFu, shx, sl);
                const float sy = __shfl_sync(0xFFFFFFFFu, shy, sl);
                const float sz = __shfl_sync(0xFFFFFFFFu, shz, sl);
                const bool sh = act & ((sx != 0.0f) | (sy != 0.0f) | (sz != 0.0f));
                if (__ballot_sync(0xFFFFFFFFu, sh)) shifted |= 1u << r;
                pe[r] = e;
                px[r] = py[r] = pz[r] = 1.0e30f;  // never inside r_c
                if (act) {
                    const float4 pj = S.pos[e & 0xFFFFu];
                    px[r] = pj.x;
                    py[r] = pj.y;
                    pz[r] = pj.z;
                }
            }
            const int nslots = (nch + 31) >> 5;
            for (int o = ob; o < oe; ++o) {
                const uint32_t i = S.idx[o];
                const float4 pi = S.pos[i];
#pragma unroll
                for (int r = 0; r < kEnsSlots; ++r) {
                    if (r < nslots) {
                        float dx = __fsub_rn(px[r], pi.x);
                        float dy = __fsub_rn(py[r], pi.y);
                        float dz = __fsub_rn(pz[r], pi.z);
                        if ((shifted >> r) & 1u) {
                            const int sl = (int)(pe[r] >> 16);
                            dx = __fadd_rn(dx, __shfl_sync(0xFFFFFFFFu, shx, sl));
                            dy = __fadd_rn(dy, __shfl_sync(0xFFFFFFFFu, shy, sl));
                            dz = __fadd_rn(dz, __shfl_sync(0xFFFFFFFFu, shz, sl));
                        }
                        const float d2 = dist2_rn(dx, dy, dz);
                        // N3: of the own cell only the members after the owner
                        const int tg = base + 32 * r + lane;
                        const bool fwd = !N3 || tg >= len0 || tg > o - ob;
                        const bool hit = (d2 < B.rc2) & (d2 > 0.0f) & fwd;
                        const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
                        if (hit)
                            q[(tail + __popc(m & lt)) & (kEnsQueue - 1)] =
                                make_float4(dx, dy, dz, __uint_as_float((i << 16) | (pe[r] & 0xFFFFu)));
                        tail += (uint32_t)__popc(m);
                        if (tail - head >= 32u) {
                            ens_batch<SMODE, VIR, N3>(B, S, q, key, head, 32, lane);
                            head += 32u;
                        }
                    }
                }
            }
            // another round visits the same owners again: empty the ring first,
            // so no batch holds two runs of one owner (their adds would race)
            if (base + kEnsCand < ncand) {
                while (tail != head) {
                    const int nb = (int)min(32u, tail - head);
                    ens_batch<SMODE, VIR, N3>(B, S, q, key, head, nb, lane);
                    head += (uint32_t)nb;
                }
            }
        }
    }
    while (tail != head) {
        const int nb = (int)min(32u, tail - head);
        ens_batch<SMODE, VIR, N3>(B, S, q, key, head, nb, lane);
        head += (uint32_t)nb;
    }
}

template <bool LHALF, int SMODE, bool N3>
__global__ void __launch_bounds__(kEnsMaxThreads, 1) k_ens_run(const EnsBox *__restrict__ boxes, int C)
{
    __shared__ EnsBox B;
    __shared__ uint32_t wsum[33];
    extern __shared__ __align__(16) unsigned char smem[];

    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(boxes + blockIdx.x / C);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&B);
        for (int k = threadIdx.x; k < (int)(sizeof(EnsBox) / 4); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = C > 1 ? (int)cl.block_rank() : 0;
    const int n = B.n, ncell = B.ncell, T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = T >> 5;
    const EnsLayout lay = ens_layout(n, ncell, LHALF, T);
    EnsPtrs S;
    S.pos = reinterpret_cast<float4 *>(smem + lay.pos);
    S.u = reinterpret_cast<float4 *>(smem + lay.u);
    S.vh = reinterpret_cast<float4 *>(smem + lay.vh);
    S.f = reinterpret_cast<float4 *>(smem + lay.f);
    S.start = reinterpret_cast<uint32_t *>(smem + lay.start);
    S.cnt = reinterpret_cast<uint32_t *>(smem + lay.cnt);
    S.idx = reinterpret_cast<uint16_t *>(smem + lay.idx);
    S.slot = reinterpret_cast<uint16_t *>(smem + lay.slot);
    S.own = reinterpret_cast<uint8_t *>(smem + lay.own);
    S.C = C;
    S.rank = rank;
    float4 *q = reinterpret_cast<float4 *>(smem + lay.q) + warp * kEnsQueue;
    uint32_t *cand = reinterpret_cast<uint32_t *>(smem + lay.cand) + warp * kEnsCand;
    const int steps = B.steps;
    const unsigned long long step0 = B.step;
    const float invL[3] = {1.0f / B.L[0], 1.0f / B.L[1], 1.0f / B.L[2]};

    // replica of the box; with steps > 0, phase 1 of the first step:
    //   u = v + dt/2 f,  x += dt u,  v~ = v + lambda dt f (= u when lambda = 1/2)
    for (int i = threadIdx.x; i < n; i += T) {
        float4 x = B.pos[i];
        const float4 v = B.vel[i];
        const uint32_t tg = __ldg(B.tag + i);
        if (steps == 0) {
            S.pos[i] = x;
            S.u[i] = make_float4(v.x, v.y, v.z, __uint_as_float(signature(tg, (uint32_t)step0, B.key)));
        } else {
            const float4 f = B.frc[i];
            const float ux = fmaf(B.half_dt, f.x, v.x), uy = fmaf(B.half_dt, f.y, v.y), uz = fmaf(B.half_dt, f.z, v.z);
            x.x = ens_wrap(fmaf(B.dt, ux, x.x), B.L[0], invL[0]);
            x.y = ens_wrap(fmaf(B.dt, uy, x.y), B.L[1], invL[1]);
            x.z = ens_wrap(fmaf(B.dt, uz, x.z), B.L[2], invL[2]);
            S.pos[i] = x;
            const float sig = __uint_as_float(signature(tg, (uint32_t)(step0 + 1ull), B.key));
            if (LHALF) {
                S.u[i] = make_float4(ux, uy, uz, sig);
            } else {
                S.u[i] = make_float4(fmaf(B.lambda_dt, f.x, v.x), fmaf(B.lambda_dt, f.y, v.y),
                                     fmaf(B.lambda_dt, f.z, v.z), sig);
                S.vh[i] = make_float4(ux, uy, uz, 0.0f);
            }
        }
    }
    for (int c = threadIdx.x; c < ncell; c += T) S.cnt[c] = 0u;
    __syncthreads();

    const int nunits = (ncell + kEnsUnitCells - 1) / kEnsUnitCells;
    const int nforce = steps == 0 ? 1 : steps;
    for (int s = 1; s <= nforce; ++s) {
        const bool last = s == nforce;
        // 1. cell lists
        for (int i = threadIdx.x; i < n; i += T) S.slot[i] = (uint16_t)atomicAdd(&S.cnt[ens_cell(B, S.pos[i])], 1u);
        __syncthreads();
        ens_scan(S.cnt, S.start, ncell, wsum);
        for (int i = threadIdx.x; i < n; i += T) {
            const int c = ens_cell(B, S.pos[i]);
            S.idx[S.start[c] + S.slot[i]] = (uint16_t)i;
            if (N3) {  // partner shares may come from any warp of the cluster
                S.f[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                S.own[i] = (uint8_t)((c / kEnsUnitCells) % C);
            }
        }
        for (int c = threadIdx.x; c < ncell; c += T) S.cnt[c] = 0u;
        __syncthreads();
        for (int c = threadIdx.x; c < ncell; c += T) {  // members of a cell in index order
            const int lo = (int)S.start[c], hi = (int)S.start[c + 1];
            for (int k = lo + 1; k < hi; ++k) {
                const uint16_t v = S.idx[k];
                int m = k - 1;
                while (m >= lo && S.idx[m] > v) {
                    S.idx[m + 1] = S.idx[m];
                    --m;
                }
                S.idx[m + 1] = v;
            }
        }
        __syncthreads();
        if (N3 && C > 1) cl.sync();  // every replica's accumulators are zero before any remote add
        // 2. pair forces of this CTA's units
        for (int u = rank + C * warp; u < nunits; u += C * nwarps) {
            if (last) ens_unit<SMODE, true, N3>(B, S, q, cand, u, lane);
            else ens_unit<SMODE, false, N3>(B, S, q, cand, u, lane);
        }
        __syncthreads();
        if (C > 1) cl.sync();  // every replica has been read for this step
        // 3. integrate the particles of this CTA's units
        const unsigned long long stepn = step0 + (unsigned long long)s + 1ull;  // step of the next force
        for (int u = rank + C * warp; u < nunits; u += C * nwarps) {
            const int k0 = (int)S.start[u * kEnsUnitCells];
            const int k1 = (int)S.start[min((u + 1) * kEnsUnitCells, ncell)];
            for (int k = k0 + lane; k < k1; k += 32) {
                const int i = S.idx[k];
                float4 f = S.f[i];
                const float4 x = S.pos[i];
                if (B.body_mode == 1) {
                    f.x += B.body[0]; f.y += B.body[1]; f.z += B.body[2];
                } else if (B.body_mode == 2) {
                    const float sg = x.y < B.halfL[1] ? 1.0f : -1.0f;
                    f.x = fmaf(sg, B.body[0], f.x); f.y = fmaf(sg, B.body[1], f.y); f.z = fmaf(sg, B.body[2], f.z);
                }
                if (!isfinite(f.x) || !isfinite(f.y) || !isfinite(f.z)) {
                    atomicOr(B.err, kErrNonFinite);
                    atomicOr(B.any_err, kErrNonFinite);
                }
                if (steps == 0) {
                    B.frc[i] = f;
                } else if (last) {
                    // phase 2 only: the full-step velocity
                    const float4 uo = LHALF ? S.u[i] : S.vh[i];
                    B.pos[i] = x;
                    B.vel[i] = make_float4(fmaf(B.half_dt, f.x, uo.x), fmaf(B.half_dt, f.y, uo.y),
                                           fmaf(B.half_dt, f.z, uo.z), 0.0f);
                    B.frc[i] = f;
                } else {
                    // phase 2 of this step and phase 1 of the next:
                    //   v = u + dt/2 f;  u' = v + dt/2 f;  v~ = v + lambda dt f;  x' = x + dt u'
                    const float4 uo = LHALF ? S.u[i] : S.vh[i];
                    const float sig = __uint_as_float(signature(__ldg(B.tag + i), (uint32_t)stepn, B.key));
                    float ux, uy, uz, tx, ty, tz;
                    if (LHALF) {
                        ux = fmaf(B.dt, f.x, uo.x); uy = fmaf(B.dt, f.y, uo.y); uz = fmaf(B.dt, f.z, uo.z);
                        tx = ux; ty = uy; tz = uz;
                    } else {
                        const float vx = fmaf(B.half_dt, f.x, uo.x), vy = fmaf(B.half_dt, f.y, uo.y),
                                    vz = fmaf(B.half_dt, f.z, uo.z);
                        ux = fmaf(B.half_dt, f.x, vx); uy = fmaf(B.half_dt, f.y, vy); uz = fmaf(B.half_dt, f.z, vz);
                        tx = fmaf(B.lambda_dt, f.x, vx); ty = fmaf(B.lambda_dt, f.y, vy);
                        tz = fmaf(B.lambda_dt, f.z, vz);
                    }
                    float4 xn = x;
                    xn.x = ens_wrap(fmaf(B.dt, ux, x.x), B.L[0], invL[0]);
                    xn.y = ens_wrap(fmaf(B.dt, uy, x.y), B.L[1], invL[1]);
                    xn.z = ens_wrap(fmaf(B.dt, uz, x.z), B.L[2], invL[2]);
                    const float4 un = make_float4(tx, ty, tz, sig);
                    const float4 vhn = make_float4(ux, uy, uz, 0.0f);
                    for (int r = 0; r < C; ++r) {
                        float4 *pp = C > 1 ? cl.map_shared_rank(S.pos, r) : S.pos;
                        float4 *up = C > 1 ? cl.map_shared_rank(S.u, r) : S.u;
                        pp[i] = xn;
                        up[i] = un;
                        if (!LHALF) {
                            float4 *hp = C > 1 ? cl.map_shared_rank(S.vh, r) : S.vh;
                            hp[i] = vhn;
                        }
                    }
                }
            }
        }
        if (!last) {
            if (C > 1) cl.sync();  // every replica holds the new state
            else __syncthreads();
        }
    }
    // no CTA leaves while another may still address its shared memory
    if (C > 1) cl.sync();
}

// Per box: sum v^2, virial (the w of the forces), momentum; FP64, fixed order.
__global__ void __launch_bounds__(kObsThreads) k_ens_observe(const EnsBox *__restrict__ boxes, double *out)
{
    __shared__ double sh[5][kObsThreads / 32];
    const EnsBox &B = boxes[blockIdx.x];
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < B.n; i += kObsThreads) {
        const float4 v = B.vel[i], f = B.frc[i];
        a[0] += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z;
        a[1] += (double)f.w;
        a[2] += v.x;
        a[3] += v.y;
        a[4] += v.z;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double x = a[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < kObsThreads / 32; ++w) s += sh[threadIdx.x][w];
        out[8 * blockIdx.x + threadIdx.x] = s;
    }
}

using EnsKernel = void (*)(const EnsBox *, int);

template <bool N3>
EnsKernel pick_n3(bool lhalf, int s_mode)
{
    switch (s_mode) {
    case 1: return lhalf ? k_ens_run<true, 1, N3> : k_ens_run<false, 1, N3>;
    case 2: return lhalf ? k_ens_run<true, 2, N3> : k_ens_run<false, 2, N3>;
    case 3: return lhalf ? k_ens_run<true, 3, N3> : k_ens_run<false, 3, N3>;
    default: return lhalf ? k_ens_run<true, 0, N3> : k_ens_run<false, 0, N3>;
    }
}

EnsKernel pick(bool lhalf, int s_mode, bool n3) { return n3 ? pick_n3<true>(lhalf, s_mode) : pick_n3<false>(lhalf, s_mode); }

size_t g_limit = 0;
std::once_flag g_once;

void init_attributes()
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    size_t limit = (size_t)optin;
    for (int v = 0; v < 16; ++v) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, pick(v & 1, (v >> 1) & 3, v >> 3)) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        limit = std::min(limit, (size_t)optin - fa.sharedSizeBytes);
    }
    for (int v = 0; v < 16; ++v)
        if (cudaFuncSetAttribute(pick(v & 1, (v >> 1) & 3, v >> 3), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)limit) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    g_limit = limit;
}

cudaLaunchConfig_t config_for(int nb, int threads, int cluster, size_t smem, cudaStream_t s, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nb * cluster), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

size_t ensemble_smem_limit()
{
    std::call_once(g_once, init_attributes);
    return g_limit;
}

int ensemble_max_clusters(bool lhalf, int s_mode, bool n3, int threads, int cluster, size_t smem)
{
    if (ensemble_smem_limit() == 0 || smem > g_limit) return 0;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = config_for(cluster, threads, cluster, smem, nullptr, at);
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, pick(lhalf, s_mode, n3), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return num;
}

cudaError_t launch_ensemble(const EnsBox *boxes, int nb, bool lhalf, int s_mode, bool n3, int threads, int cluster,
                            size_t smem, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    if (ensemble_smem_limit() == 0 || smem > g_limit || threads < 32 || threads > kEnsMaxThreads ||
        threads % 32 != 0 || cluster < 1 || cluster > kEnsMaxCluster)
        return cudaErrorInvalidValue;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = config_for(nb, threads, cluster, smem, s, at);
    return cudaLaunchKernelEx(&cfg, pick(lhalf, s_mode, n3), boxes, cluster);
}

cudaError_t launch_ensemble_observe(const EnsBox *boxes, int nb, double *out, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    k_ens_observe<<<nb, kObsThreads, 0, s>>>(boxes, out);
    return cudaGetLastError();
}

}  // namespace dpd
