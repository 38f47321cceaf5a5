// kernels_force.cu -- fused DPD pair force (Eqs. 2-9 with the in-situ
// Gaussian of Sec. 3.5), harmonic bonds (Sec. 4.5), body force (Sec. 4.2),
// and the velocity-Verlet phases (Sec. 3.1, Algorithm 1): k_force (pairs),
// k_settle (Newton-3 sums + integration), k_phase1, k_advance (rebuild
// flag, buffer flip, conditional graph node).
#include "dpd_internal.cuh"
#include "dpd_math.cuh"

namespace dpd {

namespace {

constexpr int kThreads = 256;
constexpr int kForceThreads = 32 * kForceWarps;

__device__ __forceinline__ float wrap_pos(float x, float L, float invL)
{
    x = x - L * floorf(x * invL);
    if (x >= L) x -= L;
    if (x < 0.0f) x += L;
    if (x >= L) x = 0.0f;  // -tiny + L rounded up to L
    return x;
}

// End of a kernel that moves particles: a block any of whose particles
// crossed the displacement threshold raises rebuild_next (a plain store of
// the same value from every such block).  k_advance, launched right after,
// publishes it and flips the buffer set; no block counts the others.
__device__ __forceinline__ void finish_block(DevCtl *ctl, bool moved)
{
    if (__syncthreads_or(moved) && threadIdx.x == 0) ctl->rebuild_next = 1u;
}

// One thread, after a moving kernel: the rebuild flag for the chain that
// follows (also raised when rebuild_every steps have passed), and, when the
// kernel integrated into the other buffer set, that set becomes the live one
// and the step advances.  Inside a CUDA graph the flag also sets the
// conditional node around the next rebuild chain, so a step without a
// rebuild launches none of the chain's kernels.
template <bool ADVANCE, bool CHECK_EVERY>
__global__ void k_advance(SimParams P, Ptrs D, NextCond nc)
{
    DevCtl *c = D.ctl;
    uint32_t next = c->rebuild_next;
    if (CHECK_EVERY && P.rebuild_every > 0 && c->since_rebuild + 1u >= (uint32_t)P.rebuild_every) next = 1u;
    c->rebuild = next;
    if (nc.use) cudaGraphSetConditional(nc.handle, next ? 1u : 0u);
    c->rebuild_next = 0u;
    if (ADVANCE) {
        c->parity ^= 1u;
        c->step += 1ull;
        c->since_rebuild += 1u;
    }
}

__device__ __forceinline__ bool moved_beyond(const SimParams &P, float4 x, float4 r)
{
    const float dx = min_image_rn(x.x, r.x, P.L[0], P.halfL[0]);
    const float dy = min_image_rn(x.y, r.y, P.L[1], P.halfL[1]);
    const float dz = min_image_rn(x.z, r.z, P.L[2], P.halfL[2]);
    return dist2_rn(dx, dy, dz) > P.disp2;
}

// Phase 1 of the step k -> k+1 from the full-step velocity v (in place):
//   u = v + dt/2 f,  x += dt u  (= x + dt v + dt^2/2 f),  v~ = v + lambda dt f
// (v~ = u when lambda = 1/2), signature for step k+1, displacement check.
template <bool LHALF>
__global__ void k_phase1(SimParams P, Ptrs D)
{
    DevCtl *ctl = D.ctl;
    const uint32_t par = ctl->parity;
    const uint32_t step1 = (uint32_t)(ctl->step + 1ull);
    float4 *pos = D.pos[par];
    float4 *vel = D.vel[par];
    const float4 *frc = D.force[par];
    const uint32_t *tag = D.tag[ctl->oparity];
    bool moved = false;
    const float invL[3] = {1.0f / P.L[0], 1.0f / P.L[1], 1.0f / P.L[2]};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float4 f = frc[i];
        const float4 v = vel[i];
        const uint32_t tg = tag[i];
        const float4 xr = D.xref[i];
        const float ux = fmaf(P.half_dt, f.x, v.x), uy = fmaf(P.half_dt, f.y, v.y), uz = fmaf(P.half_dt, f.z, v.z);
        float4 x = pos[i];
        x.x = wrap_pos(fmaf(P.dt, ux, x.x), P.L[0], invL[0]);
        x.y = wrap_pos(fmaf(P.dt, uy, x.y), P.L[1], invL[1]);
        x.z = wrap_pos(fmaf(P.dt, uz, x.z), P.L[2], invL[2]);
        pos[i] = x;
        const float sig = __uint_as_float(signature(tg, step1, P.key));
        if (LHALF) {
            vel[i] = make_float4(ux, uy, uz, sig);
        } else {
            vel[i] = make_float4(fmaf(P.lambda_dt, f.x, v.x), fmaf(P.lambda_dt, f.y, v.y), fmaf(P.lambda_dt, f.z, v.z), sig);
            D.vkick[par][i] = make_float4(ux, uy, uz, 0.0f);
        }
        moved |= moved_beyond(P, x, xr);
    }
    finish_block(ctl, moved);
}

__global__ void k_signature(SimParams P, Ptrs D)
{
    const uint32_t par = D.ctl->parity;
    const uint32_t step = (uint32_t)D.ctl->step;
    float4 *vel = D.vel[par];
    const uint32_t *tag = D.tag[D.ctl->oparity];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        float4 v = vel[i];
        v.w = __uint_as_float(signature(tag[i], step, P.key));
        vel[i] = v;
    }
}

// Bonds (Sec. 4.5) and the body force (Sec. 4.2) on particle i, added to f.
// With bvir, the bonds' virial share r_ij . F_ij is added to *bvir (half per
// end: each bond is seen from both of its particles).
__device__ __forceinline__ void add_bonds_body(const SimParams &P, const Ptrs &D, int i, float4 pi,
                                               const float4 *__restrict__ pos, uint32_t opar, float &fx,
                                               float &fy, float &fz, float *bvir = nullptr)
{
    if (P.has_bonds) {
        const uint32_t id = D.pid[opar][i];
        const uint32_t *bp = D.bond_partner + (size_t)id * kMaxBonds;
        for (int b = 0; b < kMaxBonds; ++b) {
            const uint32_t other = bp[b];
            if (other == kNone) break;
            const uint32_t jb = kChecked && other >= (uint32_t)P.n ? kNone : D.idx_of_pid[other];
            if (kChecked && jb >= (uint32_t)P.n) {
                atomicOr(&D.ctl->err, kErrBadIndex);
                break;
            }
            const float4 pj = pos[jb];
            const float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
            const float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
            const float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 > 0.0f) {
                const float inv_r = rsqrtf(d2);
                const float r = d2 * inv_r;
                // F_i = -K (r - r0) e_ij, e_ij = -d / r
                const float sc = P.k_bond * (r - P.r0_bond) * inv_r;
                fx = fmaf(sc, dx, fx);
                fy = fmaf(sc, dy, fy);
                fz = fmaf(sc, dz, fz);
                if (bvir) *bvir += 0.5f * (-P.k_bond * (r - P.r0_bond) * r);
            }
        }
    }
    if (P.body_mode == 1) {
        fx += P.body[0]; fy += P.body[1]; fz += P.body[2];
    } else if (P.body_mode == 2) {
        const float sg = pi.y < P.halfL[1] ? 1.0f : -1.0f;
        fx = fmaf(sg, P.body[0], fx); fy = fmaf(sg, P.body[1], fy); fz = fmaf(sg, P.body[2], fz);
    }
}

// Final stage of a force evaluation for particle i with total force f: per
// MODE the force is stored, or the step is integrated into the other buffer
// set.  Returns whether the particle moved past the rebuild threshold.
template <int MODE, bool LHALF>
__device__ __forceinline__ bool integrate_particle(const SimParams &P, const Ptrs &D, DevCtl *ctl, int i, float4 pi,
                                                   float4 vi, float fx, float fy, float fz, uint32_t par,
                                                   uint32_t opar, unsigned long long step0, int out_fout)
{
    bool moved = false;
    // every input is read before the first store: as far as the compiler
    // knows the stores may alias them, and reads issued after a store would
    // wait for another round trip to memory
    float4 u = vi, xr = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t tg = 0;
    if (MODE != kForceEval && !LHALF) u = D.vkick[par][i];
    if (MODE == kForceStep) {
        tg = D.tag[opar][i];
        xr = D.xref[i];
    }
    if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(&ctl->err, kErrNonFinite);
    const uint32_t nx = par ^ 1u;
    if (MODE == kForceEval) {
        float4 *out = out_fout ? D.fout : D.force[par];
        out[i] = make_float4(fx, fy, fz, 0.0f);
    } else if (MODE == kForceFinish) {
        // phase 2: v = u + dt/2 f; the state at the full step goes to the other set
        D.vel[nx][i] = make_float4(fmaf(P.half_dt, fx, u.x), fmaf(P.half_dt, fy, u.y), fmaf(P.half_dt, fz, u.z), vi.w);
        D.pos[nx][i] = pi;
        D.force[nx][i] = make_float4(fx, fy, fz, 0.0f);
        if (!LHALF) D.vkick[nx][i] = u;
    } else {
        // phase 2 of this step and phase 1 of the next:
        //   v = u + dt/2 f;  u' = v + dt/2 f;  v~ = v + lambda dt f;  x' = x + dt u'
        float ux, uy, uz, tx, ty, tz;
        if (LHALF) {
            ux = fmaf(P.dt, fx, u.x); uy = fmaf(P.dt, fy, u.y); uz = fmaf(P.dt, fz, u.z);
            tx = ux; ty = uy; tz = uz;
        } else {
            const float vx = fmaf(P.half_dt, fx, u.x), vy = fmaf(P.half_dt, fy, u.y), vz = fmaf(P.half_dt, fz, u.z);
            ux = fmaf(P.half_dt, fx, vx); uy = fmaf(P.half_dt, fy, vy); uz = fmaf(P.half_dt, fz, vz);
            tx = fmaf(P.lambda_dt, fx, vx); ty = fmaf(P.lambda_dt, fy, vy); tz = fmaf(P.lambda_dt, fz, vz);
            D.vkick[nx][i] = make_float4(ux, uy, uz, 0.0f);
        }
        float4 x = pi;
        x.x = wrap_pos(fmaf(P.dt, ux, x.x), P.L[0], 1.0f / P.L[0]);
        x.y = wrap_pos(fmaf(P.dt, uy, x.y), P.L[1], 1.0f / P.L[1]);
        x.z = wrap_pos(fmaf(P.dt, uz, x.z), P.L[2], 1.0f / P.L[2]);
        D.pos[nx][i] = x;
        const uint32_t sig = signature(tg, (uint32_t)(step0 + 2ull), P.key);
        D.vel[nx][i] = make_float4(tx, ty, tz, __uint_as_float(sig));
        moved = moved_beyond(P, x, xr);
    }
    return moved;
}

// Epilogue of the force kernels for particle i: bonds, body force, then the
// final stage (integrate_particle).
template <int MODE, bool LHALF>
__device__ __forceinline__ bool force_epilogue(const SimParams &P, const Ptrs &D, DevCtl *ctl, int i, float4 pi,
                                               float4 vi, float fx, float fy, float fz, uint32_t par, uint32_t opar,
                                               unsigned long long step0, int out_fout, float *bvir)
{
    add_bonds_body(P, D, i, pi, D.pos[par], opar, fx, fy, fz, bvir);
    return integrate_particle<MODE, LHALF>(P, D, ctl, i, pi, vi, fx, fy, fz, par, opar, step0, out_fout);
}

// ---------------------------------------------------------------------------
// Fused pair force.  Each warp owns one group (at most 32 consecutive
// particles in cell order, lane = owner) and walks the group's packed list
// 32 entries at a time: one coalesced load, every lane a candidate pair
// (owner, j).  Pairs inside r_c (the FP32 predicate) are appended to a
// per-warp ring queue in shared memory in list order (a ballot gives each
// hit its slot, as the paper's builder does for list entries); every time 32
// are queued the whole warp evaluates them together, one pair per lane, so
// the hash / Box-Muller / force arithmetic runs with full warps whatever the
// hit pattern.
//   F = a_{t_i t_j} w - gamma w_R^2 (e . v_ij) + sigma/sqrt(dt) w_R xi_ij,
//   f_i += F e_ij,  e_ij = (x_i - x_j) / r.
// The 32 results of a batch are summed per owner by a segmented scan and
// added to the owners' shared accumulators.  Deterministic mode (full lists,
// each pair seen from both sides): the adds run in lane order, so every
// force is summed in a fixed order.  Newton-3 mode (half lists): the adds
// are shared-memory atomics, and the partner's share, -F e_ij, goes to
// facc[j] by a global vector reduction.
// The epilogue adds bonds and the body force and, per MODE, writes the force
// or integrates (see launch_force).
constexpr int kQueue = 64;  // ring slots per warp (< 32 pending + 32 new)

// The candidate walk of a warp, templated on whether the minimum image can
// be needed: a warp whose 32 particles all lie at least (r_list + skin) from
// every face has no neighbour across the periodic boundary, so d = x_j - x_i
// is already the minimum image and the pinned predicate reduces to it.
template <bool WRAP>
__device__ __forceinline__ float3 pair_delta(const SimParams &P, float4 pj, float4 pi)
{
    if (WRAP)
        return make_float3(min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]), min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]),
                           min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]));
    return make_float3(__fsub_rn(pj.x, pi.x), __fsub_rn(pj.y, pi.y), __fsub_rn(pj.z, pi.z));
}

// Vector reduction into global memory (sm_90+): adds (x, y, z, 0) to *p.
__device__ __forceinline__ void red_add_f4(float4 *p, float x, float y, float z)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(0.0f)
                 : "memory");
}

// Shared state of a warp: owners' positions and velocities, the queue and
// the owners' force accumulators.
struct WarpSmem {
    float4 pi[32];
    float4 vi[32];
    float4 q[kQueue];      // (d, list entry: owner lane << kOwnerShift | j)
    uint8_t qo[kQueue];    // partner species (several species only)
    float acc[3][32];
};

template <bool ONE_SPECIES, int SMODE, bool WRAP, bool N3, bool VIR>
__device__ __forceinline__ void warp_pairs(const SimParams &P, const float4 *__restrict__ pos,
                                           const float4 *__restrict__ vel, const uint32_t *__restrict__ list,
                                           uint32_t nent, int lane, WarpSmem &w, const float *a_tab, float4 *facc,
                                           float &vir, uint32_t owners, bool &bad)
{
    const uint32_t key[4] = {P.key[0], P.key[1], P.key[2], P.key[3]};
    const uint32_t lt_mask = (1u << lane) - 1u;

    // Evaluate queue entries [head, head + nb) (nb <= 32), one per lane, and
    // add each result to its owner's accumulator.
    auto run_batch = [&](uint32_t head, int nb) {
        float fx = 0.f, fy = 0.f, fz = 0.f;
        const bool act = lane < nb;
        uint32_t owner = 32u + (uint32_t)lane;  // distinct dummy owners for idle lanes
        if (act) {
            const uint32_t slot = (head + (uint32_t)lane) & (kQueue - 1);
            const float4 q = w.q[slot];  // (d, list entry)
            const uint32_t ent = __float_as_uint(q.w);
            const uint32_t qo = ONE_SPECIES ? 0u : w.qo[slot];
            owner = ent >> kOwnerShift;
            const uint32_t j = ent & kIndexMask;
            const float4 wi = w.vi[owner];
            const float4 vj = __ldg(vel + j);
            const float dx = q.x, dy = q.y, dz = q.z;
            const float d2 = dist2_rn(dx, dy, dz);
            const float inv_r = rsqrtf(d2);
            const float r = d2 * inv_r;
            const float wgt = fmaxf(fmaf(-r, P.inv_rc, 1.0f), 0.0f);
            const float wR = weight_R<SMODE>(wgt, P.s);
            // e_ij = -d / r; e . v_ij = -(d . (v_i - v_j)) / r
            const float ev = -((dx * (wi.x - vj.x) + dy * (wi.y - vj.y)) + dz * (wi.z - vj.z)) * inv_r;
            uint32_t A, B;
            pair_hash(__float_as_uint(wi.w), __float_as_uint(vj.w), key, A, B);
            const float xi = gauss_from_hash(A, B);
            const float a = ONE_SPECIES ? P.a[0] : a_tab[__float_as_int(w.pi[owner].w) * P.n_species + (int)qo];
            const float F = fmaf(a, wgt, fmaf(-P.gamma * wR * wR, ev, P.sigma_isdt * wR * xi));
            // conservative virial r_ij . F^C_ij (each pair once in Newton-3
            // mode, from both ends otherwise)
            if (VIR) vir = fmaf(N3 ? 1.0f : 0.5f, a * wgt * r, vir);
            const float sc = -F * inv_r;
            fx = sc * dx;
            fy = sc * dy;
            fz = sc * dz;
            // Newton's third law: the partner gets -F once
            if (N3) red_add_f4(facc + j, -fx, -fy, -fz);
        }
        // Per-owner sums: the queue follows the list, whose entries come
        // owner by owner, so a batch holds a few runs of equal owners.  A
        // segmented inclusive scan (fixed order) leaves each run's sum on its
        // last lane, which adds it to the owner's accumulator.
        const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, owner, 1);
        const uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || prev != owner);
        const int start = 31 - __clz(heads & (0xFFFFFFFFu >> (31 - lane)));  // first lane of the run
        float sx = fx, sy = fy, sz = fz;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float ax = __shfl_up_sync(0xFFFFFFFFu, sx, d);
            const float ay = __shfl_up_sync(0xFFFFFFFFu, sy, d);
            const float az = __shfl_up_sync(0xFFFFFFFFu, sz, d);
            if (lane - start >= d) {
                sx += ax;
                sy += ay;
                sz += az;
            }
        }
        const bool tail_lane = owner < 32u && (lane == 31 || ((heads >> lane) & 2u) != 0u);
        if (N3) {
            // an owner can recur in a later run of the batch: atomics
            if (tail_lane) {
                atomicAdd(&w.acc[0][owner], sx);
                atomicAdd(&w.acc[1][owner], sy);
                atomicAdd(&w.acc[2][owner], sz);
            }
        } else {
            // fixed order: the runs add in lane order
            uint32_t tails = __ballot_sync(0xFFFFFFFFu, tail_lane);
            while (tails) {
                const int src = __ffs(tails) - 1;
                if (lane == src) {
                    w.acc[0][owner] += sx;
                    w.acc[1][owner] += sy;
                    w.acc[2][owner] += sz;
                }
                tails &= tails - 1u;
                __syncwarp();
            }
        }
        __syncwarp();
    };

    uint32_t head = 0u, tail = 0u;
    // one candidate (entry e, partner position pj): test it, queue it if
    // inside r_c, evaluate a full batch
    auto candidate = [&](bool act, uint32_t e, float4 pj) {
        const uint32_t own = e >> kOwnerShift;
        if (kChecked && act && ((e & kIndexMask) >= (uint32_t)P.n || own >= owners)) {
            bad = true;
            act = false;
        }
        const float3 d = pair_delta<WRAP>(P, pj, w.pi[own]);
        const float d2 = dist2_rn(d.x, d.y, d.z);
        // bitwise & keeps the test branch-free (no short-circuit evaluation)
        const bool hit = act & (d2 < P.rc2) & (d2 > 0.0f);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
        if (hit) {
            const uint32_t slot = (tail + (uint32_t)__popc(m & lt_mask)) & (kQueue - 1);
            // the entry keeps its owner bits; one species needs nothing else
            w.q[slot] = make_float4(d.x, d.y, d.z, __uint_as_float(e));
            if (!ONE_SPECIES) w.qo[slot] = (uint8_t)((uint32_t)__float_as_int(pj.w));
        }
        tail += (uint32_t)__popc(m);
        __syncwarp();
        if (tail - head >= 32u) {
            run_batch(head, 32);
            head += 32u;
        }
    };
    // Entries are loaded four iterations ahead through a register rotation
    // (the loop stays rolled: the batch evaluation inside it is large), and
    // each candidate's position one ahead.  Past the end a lane reads entry 0
    // (owner 0, particle 0), a valid address that the act flag discards.
    auto entry = [&](uint32_t k) -> uint32_t { return k < nent ? __ldg(list + k) : 0u; };
    // (the checked build clamps the prefetch index into range; the candidate
    // test then rejects the entry)
    auto at = [&](uint32_t e) -> uint32_t {
        const uint32_t j = e & kIndexMask;
        return (kChecked && j >= (uint32_t)P.n) ? 0u : j;
    };
    const uint32_t l = (uint32_t)lane;
    uint32_t e0 = entry(l), e1 = entry(32u + l), e2 = entry(64u + l), e3 = entry(96u + l);
    float4 pc = __ldg(pos + at(e0));
    for (uint32_t base = 0; base < nent; base += 32u) {
        const uint32_t e4 = entry(base + 128u + l);
        const float4 pn = __ldg(pos + at(e1));
        candidate(base + l < nent, e0, pc);
        e0 = e1;
        e1 = e2;
        e2 = e3;
        e3 = e4;
        pc = pn;
    }
    while (tail != head) {
        const int nb = (int)min(32u, tail - head);
        run_batch(head, nb);
        head += (uint32_t)nb;
    }
}

// Fixed-order block sum of one value per thread into *out (thread 0).
__device__ __forceinline__ void block_sum_double(float x, double *out)
{
    __shared__ double sh[kForceWarps];
    double v = x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kForceWarps; ++k) t += sh[k];
        *out = t;
    }
}

// VIR: also the virial of this evaluation (conservative pairs + bonds), one
// partial per block into D.vir_part -- for the evaluations that close a call,
// whose positions are the state the observables describe.
// 12 resident blocks per SM (48 warps) caps the kernel at 40 registers: the
// walk's scattered gathers need the extra warps to hide their latency
// (measured on the 3M fluid: 0.311 ms per launch against 0.338 ms at the
// compiler's 47 registers and 10 blocks; 32 registers spill and take 0.474).
constexpr int kForceMinBlocks = 12;
template <bool ONE_SPECIES, int SMODE, int MODE, bool LHALF, bool N3, bool VIR>
__global__ void __launch_bounds__(kForceThreads, kForceMinBlocks) k_force(SimParams P, Ptrs D, int out_fout)
{
    constexpr int W = kForceThreads / 32;
    __shared__ WarpSmem s_w[W];
    __shared__ float a_tab[kMaxSpecies * kMaxSpecies];
    if (!ONE_SPECIES) {
        for (int k = threadIdx.x; k < P.n_species * P.n_species; k += blockDim.x) a_tab[k] = P.a[k];
        __syncthreads();
    }
    DevCtl *ctl = D.ctl;
    const uint32_t par = ctl->parity;
    const uint32_t opar = ctl->oparity;
    const unsigned long long step0 = ctl->step;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &w = s_w[warp];
    const uint32_t gid = blockIdx.x * W + (uint32_t)warp;
    const uint2 desc = gid < (uint32_t)P.ngroups ? D.gdesc[gid] : make_uint2(0u, 0u);
    const uint32_t owners = desc.y & 63u, nent = desc.y >> 6;
    const int i = (int)desc.x + lane;
    const bool valid = (uint32_t)lane < owners;
    const float4 *__restrict__ pos = D.pos[par];
    const float4 *__restrict__ vel = D.vel[par];
    const float4 pi = valid ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 vi = valid ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    w.pi[lane] = pi;
    w.vi[lane] = vi;
    w.acc[0][lane] = 0.f;
    w.acc[1][lane] = 0.f;
    w.acc[2][lane] = 0.f;
    // the warp may skip the minimum image when all its particles are far from the faces
    const bool interior = !valid || (pi.x >= P.wrap_margin && pi.x <= P.L[0] - P.wrap_margin &&
                                     pi.y >= P.wrap_margin && pi.y <= P.L[1] - P.wrap_margin &&
                                     pi.z >= P.wrap_margin && pi.z <= P.L[2] - P.wrap_margin);
    const bool all_interior = __all_sync(0xFFFFFFFFu, interior) && P.wrap_margin > 0.0f;
    __syncwarp();
    const uint32_t *__restrict__ list = D.nbr + (size_t)gid * P.gcap;
    float vir = 0.0f;
    bool bad = false;
    // Newton-3 sums of this step go to facc[step & 1]; the other buffer,
    // read by the previous step's settle kernel, is cleared here for the next
    float4 *facc = D.facc[(uint32_t)step0 & 1u];
    if (N3 && valid) D.facc[((uint32_t)step0 & 1u) ^ 1u][i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (all_interior)
        warp_pairs<ONE_SPECIES, SMODE, false, N3, VIR>(P, pos, vel, list, nent, lane, w, a_tab, facc, vir, owners, bad);
    else
        warp_pairs<ONE_SPECIES, SMODE, true, N3, VIR>(P, pos, vel, list, nent, lane, w, a_tab, facc, vir, owners, bad);
    if (kChecked && __any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicOr(&ctl->err, kErrBadIndex);
    float fx = w.acc[0][lane], fy = w.acc[1][lane], fz = w.acc[2][lane];

    if (N3) {
        // this group's share of particle i's force joins the shares other
        // groups pushed into facc; the settle kernel completes the mode
        if (valid) {
            add_bonds_body(P, D, i, pi, pos, opar, fx, fy, fz, VIR ? &vir : nullptr);
            red_add_f4(facc + i, fx, fy, fz);
        }
        if (VIR) block_sum_double(vir, D.vir_part + blockIdx.x);
        return;
    }
    bool moved = false;
    if (valid)
        moved = force_epilogue<MODE, LHALF>(P, D, ctl, i, pi, vi, fx, fy, fz, par, opar, step0, out_fout,
                                            VIR ? &vir : nullptr);
    if (VIR) block_sum_double(vir, D.vir_part + blockIdx.x);
    if (MODE != kForceEval) finish_block(ctl, moved);
}

// Row layout (list_layout 1): the paper's force evaluation.  One thread per
// particle walks its row of the transposed table -- entry k of particle
// 32 g + l sits at row 32 g + (k mod 32), entry 32 (k div 32) + l, so the
// warp reads each entry index with one coalesced load -- and evaluates every
// pair inside r_c in its own branch, summing its force in registers in row
// order (full lists: every pair by both particles, no atomics).  The joined
// rows list each particle's core pairs first, the ones most likely to be
// inside r_c, so the warp's threads tend to take the branch together early
// in the walk.  The epilogue is the deterministic mode's.
template <bool ONE_SPECIES, int SMODE, bool WRAP, bool VIR>
__device__ __forceinline__ void row_pairs(const SimParams &P, const Ptrs &D, const float4 *__restrict__ pos,
                                          const float4 *__restrict__ vel, float4 pi, float4 vi, uint32_t len,
                                          uint32_t maxlen, size_t row0, int lane, const float *a_tab, float &fx,
                                          float &fy, float &fz, float &vir, bool &bad)
{
    const uint32_t key[4] = {P.key[0], P.key[1], P.key[2], P.key[3]};
    const size_t cap = (size_t)P.cap;
    const uint32_t *__restrict__ nbr = D.nbr;
    for (uint32_t k = 0; k < maxlen; ++k) {
        if (k < len) {
            const uint32_t j = __ldg(nbr + (row0 + (k & 31u)) * cap + (k & ~31u) + (uint32_t)lane);
            if (j >= (uint32_t)P.n) {  // reported, the access skipped
                bad = true;
                continue;
            }
            const float4 pj = __ldg(pos + j);
            const float3 d = pair_delta<WRAP>(P, pj, pi);
            const float d2 = dist2_rn(d.x, d.y, d.z);
            if (d2 < P.rc2 && d2 > 0.0f) {
                const float4 vj = __ldg(vel + j);
                const float inv_r = rsqrtf(d2);
                const float r = d2 * inv_r;
                const float wgt = fmaxf(fmaf(-r, P.inv_rc, 1.0f), 0.0f);
                const float wR = weight_R<SMODE>(wgt, P.s);
                const float ev = -((d.x * (vi.x - vj.x) + d.y * (vi.y - vj.y)) + d.z * (vi.z - vj.z)) * inv_r;
                uint32_t A, B;
                pair_hash(__float_as_uint(vi.w), __float_as_uint(vj.w), key, A, B);
                const float xi = gauss_from_hash(A, B);
                const float a = ONE_SPECIES ? P.a[0] : a_tab[__float_as_int(pi.w) * P.n_species + __float_as_int(pj.w)];
                const float F = fmaf(a, wgt, fmaf(-P.gamma * wR * wR, ev, P.sigma_isdt * wR * xi));
                if (VIR) vir = fmaf(0.5f, a * wgt * r, vir);
                const float sc = -F * inv_r;
                fx = fmaf(sc, d.x, fx);
                fy = fmaf(sc, d.y, fy);
                fz = fmaf(sc, d.z, fz);
            }
        }
    }
}

template <bool ONE_SPECIES, int SMODE, int MODE, bool LHALF, bool VIR>
__global__ void __launch_bounds__(kForceThreads) k_force_rows(SimParams P, Ptrs D, int out_fout)
{
    __shared__ float a_tab[kMaxSpecies * kMaxSpecies];
    if (!ONE_SPECIES) {
        for (int k = threadIdx.x; k < P.n_species * P.n_species; k += blockDim.x) a_tab[k] = P.a[k];
        __syncthreads();
    }
    DevCtl *ctl = D.ctl;
    const uint32_t par = ctl->parity;
    const uint32_t opar = ctl->oparity;
    const unsigned long long step0 = ctl->step;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < P.n;
    const float4 *__restrict__ pos = D.pos[par];
    const float4 *__restrict__ vel = D.vel[par];
    const float4 pi = valid ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 vi = valid ? vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t len = valid ? min(D.rowcnt[i], (uint32_t)P.cap) : 0u;
    const uint32_t maxlen = __reduce_max_sync(0xFFFFFFFFu, len);
    const size_t row0 = (size_t)(i - lane);
    const bool interior = !valid || (pi.x >= P.wrap_margin && pi.x <= P.L[0] - P.wrap_margin &&
                                     pi.y >= P.wrap_margin && pi.y <= P.L[1] - P.wrap_margin &&
                                     pi.z >= P.wrap_margin && pi.z <= P.L[2] - P.wrap_margin);
    const bool all_interior = __all_sync(0xFFFFFFFFu, interior) && P.wrap_margin > 0.0f;
    float fx = 0.f, fy = 0.f, fz = 0.f, vir = 0.f;
    bool bad = false;
    if (all_interior)
        row_pairs<ONE_SPECIES, SMODE, false, VIR>(P, D, pos, vel, pi, vi, len, maxlen, row0, lane, a_tab, fx, fy, fz,
                                                  vir, bad);
    else
        row_pairs<ONE_SPECIES, SMODE, true, VIR>(P, D, pos, vel, pi, vi, len, maxlen, row0, lane, a_tab, fx, fy, fz,
                                                 vir, bad);
    if (bad) atomicOr(&ctl->err, kErrBadIndex);
    bool moved = false;
    if (valid)
        moved = force_epilogue<MODE, LHALF>(P, D, ctl, i, pi, vi, fx, fy, fz, par, opar, step0, out_fout,
                                            VIR ? &vir : nullptr);
    if (VIR) block_sum_double(vir, D.vir_part + blockIdx.x);
    if (MODE != kForceEval) finish_block(ctl, moved);
}

// Newton-3 mode: f_i = facc[step & 1][i], the sum of the particle's own-group
// share and the partner shares the pair kernel's reductions added, then the
// force mode's final stage (store, or integrate into the other set).  A step
// leaves the buffer to the next step's pair kernel, which clears it; a plain
// evaluation (the step does not advance) clears it here.
template <int MODE, bool LHALF>
__global__ void __launch_bounds__(kThreads) k_settle(SimParams P, Ptrs D, int out_fout)
{
    DevCtl *ctl = D.ctl;
    const uint32_t par = ctl->parity;
    const uint32_t opar = ctl->oparity;
    const unsigned long long step0 = ctl->step;
    bool moved = false;
    float4 *facc = D.facc[(uint32_t)step0 & 1u];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float4 f = facc[i];
        const float4 pi = D.pos[par][i];
        const float4 vi = D.vel[par][i];
        moved |= integrate_particle<MODE, LHALF>(P, D, ctl, i, pi, vi, f.x, f.y, f.z, par, opar, step0, out_fout);
        if (MODE == kForceEval) facc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (MODE != kForceEval) finish_block(ctl, moved);
}


int grid_for(int n)
{
    int g = (n + kThreads - 1) / kThreads;
    return g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
}

constexpr int kMaxDynSmem = 160 * 1024;  // largest staging buffer the brick builder accepts

template <bool ONE, int MODE, bool LH, bool N3, bool VIR>
cudaError_t launch_force_v(const SimParams &P, const Ptrs &D, int of, cudaStream_t s)
{
    if (!N3 && P.list_layout == 1) {
        const int gr = (P.n + kForceThreads - 1) / kForceThreads;
        switch (P.s_mode) {
        case 1: k_force_rows<ONE, 1, MODE, LH, VIR><<<gr, kForceThreads, 0, s>>>(P, D, of); break;
        case 2: k_force_rows<ONE, 2, MODE, LH, VIR><<<gr, kForceThreads, 0, s>>>(P, D, of); break;
        case 3: k_force_rows<ONE, 3, MODE, LH, VIR><<<gr, kForceThreads, 0, s>>>(P, D, of); break;
        default: k_force_rows<ONE, 0, MODE, LH, VIR><<<gr, kForceThreads, 0, s>>>(P, D, of); break;
        }
        return cudaGetLastError();
    }
    const int g = (P.ngroups + kForceWarps - 1) / kForceWarps;
    switch (P.s_mode) {
    case 1: k_force<ONE, 1, MODE, LH, N3, VIR><<<g, kForceThreads, 0, s>>>(P, D, of); break;
    case 2: k_force<ONE, 2, MODE, LH, N3, VIR><<<g, kForceThreads, 0, s>>>(P, D, of); break;
    case 3: k_force<ONE, 3, MODE, LH, N3, VIR><<<g, kForceThreads, 0, s>>>(P, D, of); break;
    default: k_force<ONE, 0, MODE, LH, N3, VIR><<<g, kForceThreads, 0, s>>>(P, D, of); break;
    }
    return cudaGetLastError();
}

// The virial is taken by every evaluation except the inner steps of a run.
template <bool ONE, int MODE, bool LH, bool N3>
cudaError_t launch_force_m(const SimParams &P, const Ptrs &D, int of, cudaStream_t s, bool vir)
{
    return vir ? launch_force_v<ONE, MODE, LH, N3, true>(P, D, of, s) : launch_force_v<ONE, MODE, LH, N3, false>(P, D, of, s);
}

template <bool ONE>
cudaError_t launch_force_s(const SimParams &P, const Ptrs &D, int mode, int of, cudaStream_t s, cudaEvent_t after_pair,
                           unsigned int ev_flags, NextCond nc)
{
    if (P.newton3) {
        // pair kernel (accumulation only), then the settle kernel of the mode
        cudaError_t e = launch_force_m<ONE, kForceEval, true, true>(P, D, of, s, mode != kForceStep);
        if (e == cudaSuccess && after_pair) e = cudaEventRecordWithFlags(after_pair, s, ev_flags);
        if (e != cudaSuccess) return e;
        // one thread per particle: the kernel streams memory and needs every
        // load in flight at once
        const int g = (P.n + kThreads - 1) / kThreads;
        if (mode == kForceEval) k_settle<kForceEval, true><<<g, kThreads, 0, s>>>(P, D, of);
        else if (P.lambda_half) {
            if (mode == kForceStep) k_settle<kForceStep, true><<<g, kThreads, 0, s>>>(P, D, of);
            else k_settle<kForceFinish, true><<<g, kThreads, 0, s>>>(P, D, of);
        } else {
            if (mode == kForceStep) k_settle<kForceStep, false><<<g, kThreads, 0, s>>>(P, D, of);
            else k_settle<kForceFinish, false><<<g, kThreads, 0, s>>>(P, D, of);
        }
    } else {
        cudaError_t e;
        if (mode == kForceEval) e = launch_force_m<ONE, kForceEval, true, false>(P, D, of, s, true);
        else if (P.lambda_half)
            e = mode == kForceStep ? launch_force_m<ONE, kForceStep, true, false>(P, D, of, s, false)
                                   : launch_force_m<ONE, kForceFinish, true, false>(P, D, of, s, true);
        else
            e = mode == kForceStep ? launch_force_m<ONE, kForceStep, false, false>(P, D, of, s, false)
                                   : launch_force_m<ONE, kForceFinish, false, false>(P, D, of, s, true);
        if (e == cudaSuccess && after_pair) e = cudaEventRecordWithFlags(after_pair, s, ev_flags);
        if (e != cudaSuccess) return e;
    }
    if (mode == kForceStep) k_advance<true, true><<<1, 1, 0, s>>>(P, D, nc);
    else if (mode == kForceFinish) k_advance<true, false><<<1, 1, 0, s>>>(P, D, nc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t init_build_attributes(int max_dyn_smem);

int max_brick_cap() { return kMaxDynSmem / (int)sizeof(float4); }  // staged positions only

cudaError_t init_kernel_attributes() { return init_build_attributes(kMaxDynSmem); }

cudaError_t launch_signature(const SimParams &P, const Ptrs &D, cudaStream_t s)
{
    k_signature<<<grid_for(P.n), kThreads, 0, s>>>(P, D);
    return cudaGetLastError();
}

cudaError_t launch_phase1(const SimParams &P, const Ptrs &D, cudaStream_t s, NextCond nc)
{
    const int g = (P.n + kThreads - 1) / kThreads;
    if (P.lambda_half)
        k_phase1<true><<<g, kThreads, 0, s>>>(P, D);
    else
        k_phase1<false><<<g, kThreads, 0, s>>>(P, D);
    k_advance<false, true><<<1, 1, 0, s>>>(P, D, nc);
    return cudaGetLastError();
}

cudaError_t launch_force(const SimParams &P, const Ptrs &D, int mode, bool out_fout, cudaStream_t s,
                         cudaEvent_t after_pair, unsigned int ev_flags, NextCond nc)
{
    if (P.n_species == 1) return launch_force_s<true>(P, D, mode, out_fout ? 1 : 0, s, after_pair, ev_flags, nc);
    return launch_force_s<false>(P, D, mode, out_fout ? 1 : 0, s, after_pair, ev_flags, nc);
}

}  // namespace dpd
