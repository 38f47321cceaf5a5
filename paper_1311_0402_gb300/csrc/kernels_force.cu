// kernels_force.cu -- fused DPD pair force (Eqs. 2-9 with the in-situ
// Gaussian of Sec. 3.5), harmonic bonds (Sec. 4.5), body force (Sec. 4.2),
// the velocity-Verlet phases (Sec. 3.1, Algorithm 1) and the reductions of
// the per-step statistics.
#include "dpd_internal.cuh"
#include "dpd_math.cuh"

namespace dpd {

namespace {

constexpr int kThreads = 256;
constexpr int kForceThreads = 128;

__device__ __forceinline__ float wrap_pos(float x, float L, float invL)
{
    x = x - L * floorf(x * invL);
    if (x >= L) x -= L;
    if (x < 0.0f) x += L;
    if (x >= L) x = 0.0f;  // -tiny + L rounded up to L
    return x;
}

// Phase 1 of the step k -> k+1 from the full-step velocity, fused phase 2 of
// step k + phase 1 of step k+1, or phase 2 alone (MODE 0 / 1 / 2):
//   u = v + dt/2 f      (velocity at the half step)
//   x += dt u           (= x + dt v + dt^2/2 f)
//   v~ = v + lambda dt f  (the velocity the pair force sees; = u when
//                          lambda = 1/2)
//   v = u + dt/2 f'     (phase 2, after the new force f')
// Phases 1 also compute the particle's signature for step k+1 and flag a
// rebuild when the particle has moved more than skin/2 since the lists were
// built.
template <int MODE, bool LHALF>
__global__ void k_integrate(SimParams P, Ptrs D)
{
    const DevCtl *ctl = D.ctl;
    const uint32_t par = ctl->parity;
    const uint32_t step1 = (uint32_t)(ctl->step + 1ull);
    float4 *pos = D.pos[par];
    float4 *vel = D.vel[par];
    float4 *vk = D.vkick[par];
    const float4 *frc = D.force[par];
    const uint32_t *tag = D.tag[par];
    bool moved = false;
    const float invL[3] = {1.0f / P.L[0], 1.0f / P.L[1], 1.0f / P.L[2]};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        float4 f = frc[i];
        float4 v = vel[i];
        if (MODE == 2) {
            float4 u = LHALF ? v : vk[i];
            v.x = fmaf(P.half_dt, f.x, u.x);
            v.y = fmaf(P.half_dt, f.y, u.y);
            v.z = fmaf(P.half_dt, f.z, u.z);
            vel[i] = v;  // signature word unchanged
            continue;
        }
        float ux, uy, uz;   // new half-step velocity
        float tx, ty, tz;   // v~
        if (MODE == 0) {
            ux = fmaf(P.half_dt, f.x, v.x);
            uy = fmaf(P.half_dt, f.y, v.y);
            uz = fmaf(P.half_dt, f.z, v.z);
            tx = LHALF ? ux : fmaf(P.lambda_dt, f.x, v.x);
            ty = LHALF ? uy : fmaf(P.lambda_dt, f.y, v.y);
            tz = LHALF ? uz : fmaf(P.lambda_dt, f.z, v.z);
        } else if (LHALF) {
            // u' = u + dt f (phase 2 kick then phase 1 kick)
            ux = fmaf(P.dt, f.x, v.x);
            uy = fmaf(P.dt, f.y, v.y);
            uz = fmaf(P.dt, f.z, v.z);
            tx = ux; ty = uy; tz = uz;
        } else {
            float4 u = vk[i];
            float vx = fmaf(P.half_dt, f.x, u.x), vy = fmaf(P.half_dt, f.y, u.y), vz = fmaf(P.half_dt, f.z, u.z);
            ux = fmaf(P.half_dt, f.x, vx);
            uy = fmaf(P.half_dt, f.y, vy);
            uz = fmaf(P.half_dt, f.z, vz);
            tx = fmaf(P.lambda_dt, f.x, vx);
            ty = fmaf(P.lambda_dt, f.y, vy);
            tz = fmaf(P.lambda_dt, f.z, vz);
        }
        float4 x = pos[i];
        x.x = wrap_pos(fmaf(P.dt, ux, x.x), P.L[0], invL[0]);
        x.y = wrap_pos(fmaf(P.dt, uy, x.y), P.L[1], invL[1]);
        x.z = wrap_pos(fmaf(P.dt, uz, x.z), P.L[2], invL[2]);
        pos[i] = x;
        uint32_t sig = signature(tag[i], step1, P.key);
        vel[i] = make_float4(tx, ty, tz, __uint_as_float(sig));
        if (!LHALF) vk[i] = make_float4(ux, uy, uz, 0.0f);
        float4 r = D.xref[i];
        float dx = min_image_rn(x.x, r.x, P.L[0], P.halfL[0]);
        float dy = min_image_rn(x.y, r.y, P.L[1], P.halfL[1]);
        float dz = min_image_rn(x.z, r.z, P.L[2], P.halfL[2]);
        moved |= dist2_rn(dx, dy, dz) > P.disp2;
    }
    if (MODE != 2) {
        bool any = __syncthreads_or(moved);
        bool due = P.rebuild_every > 0 && ctl->since_rebuild + 1u >= (uint32_t)P.rebuild_every;
        if (threadIdx.x == 0 && (any || (due && blockIdx.x == 0))) atomicOr(&D.ctl->rebuild, 1u);
    }
}

__global__ void k_signature(SimParams P, Ptrs D)
{
    const uint32_t par = D.ctl->parity;
    const uint32_t step = (uint32_t)D.ctl->step;
    float4 *vel = D.vel[par];
    const uint32_t *tag = D.tag[par];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        float4 v = vel[i];
        v.w = __uint_as_float(signature(tag[i], step, P.key));
        vel[i] = v;
    }
}

// Pair force on particle i, one thread per particle over its full neighbour
// row (every pair is evaluated by both of its particles, so no atomics and a
// deterministic sum).  For each neighbour inside r_c (the FP32 predicate):
//   F = a_{t_i t_j} w - gamma w_R^2 (e . v_ij) + sigma/sqrt(dt) w_R xi_ij,
//   f_i += F e_ij,  e_ij = (x_i - x_j) / r.
template <bool ONE_SPECIES, int SMODE>
__global__ void __launch_bounds__(kForceThreads) k_force(SimParams P, Ptrs D, int out_fout, int inc_step)
{
    __shared__ float a_tab[kMaxSpecies * kMaxSpecies];
    if (!ONE_SPECIES) {
        for (int k = threadIdx.x; k < P.n_species * P.n_species; k += blockDim.x) a_tab[k] = P.a[k];
        __syncthreads();
    }
    DevCtl *ctl = D.ctl;
    const uint32_t par = ctl->parity;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->rebuild = 0u;
        if (inc_step) {
            ctl->step += 1ull;
            ctl->since_rebuild += 1u;
        }
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float4 *__restrict__ pos = D.pos[par];
    const float4 *__restrict__ vel = D.vel[par];
    const float4 pi = pos[i];
    const float4 vi = vel[i];
    const uint32_t si = __float_as_uint(vi.w);
    const int ti = __float_as_int(pi.w);
    const uint32_t key[4] = {P.key[0], P.key[1], P.key[2], P.key[3]};
    const float a0 = P.a[0];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int cnt = (int)D.nnb[i];
    const uint32_t *__restrict__ row = D.nbr + (size_t)(i >> 5) * P.cap * 32 + (i & 31);
    for (int k = 0; k < cnt; ++k) {
        const uint32_t j = __ldg(row + (size_t)k * 32);
        const float4 pj = __ldg(pos + j);
        const float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
        const float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
        const float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
        const float d2 = dist2_rn(dx, dy, dz);
        if (d2 < P.rc2 && d2 > 0.0f) {
            const float4 vj = __ldg(vel + j);
            const float inv_r = rsqrtf(d2);
            const float r = d2 * inv_r;
            const float w = fmaxf(fmaf(-r, P.inv_rc, 1.0f), 0.0f);
            const float wR = weight_R<SMODE>(w, P.s);
            // e_ij = -d / r; e . v_ij = -(d . (v_i - v_j)) / r
            const float ev = -((dx * (vi.x - vj.x) + dy * (vi.y - vj.y)) + dz * (vi.z - vj.z)) * inv_r;
            uint32_t A, B;
            pair_hash(si, __float_as_uint(vj.w), key, A, B);
            const float xi = gauss_from_hash(A, B);
            const float a = ONE_SPECIES ? a0 : a_tab[ti * P.n_species + __float_as_int(pj.w)];
            const float F = fmaf(a, w, fmaf(-P.gamma * wR * wR, ev, P.sigma_isdt * wR * xi));
            const float sc = -F * inv_r;
            fx = fmaf(sc, dx, fx);
            fy = fmaf(sc, dy, fy);
            fz = fmaf(sc, dz, fz);
        }
    }
    if (P.has_bonds) {
        const uint32_t id = D.pid[par][i];
        const uint32_t *bp = D.bond_partner + (size_t)id * kMaxBonds;
        for (int b = 0; b < kMaxBonds; ++b) {
            const uint32_t other = bp[b];
            if (other == kNone) break;
            const float4 pj = pos[D.idx_of_pid[other]];
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
            }
        }
    }
    if (P.body_mode == 1) {
        fx += P.body[0]; fy += P.body[1]; fz += P.body[2];
    } else if (P.body_mode == 2) {
        const float sg = pi.y < P.halfL[1] ? 1.0f : -1.0f;
        fx = fmaf(sg, P.body[0], fx); fy = fmaf(sg, P.body[1], fy); fz = fmaf(sg, P.body[2], fz);
    }
    if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(&ctl->err, kErrNonFinite);
    float4 *out = out_fout ? D.fout : D.force[par];
    out[i] = make_float4(fx, fy, fz, 0.0f);
}

// Deterministic block reduction of 8 doubles (fixed shuffle tree, then a
// fixed order over the warps); thread 0 writes the block's partials.
__device__ void block_reduce8(double (&v)[8], double *out)
{
    __shared__ double sh[8][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
}

// Per-block partial sums of: sum v^2, sum v (3), and the conservative +
// bond virial sum_{i<j} r_ij . F_ij (each pair seen from both ends, halved).
template <bool ONE_SPECIES>
__global__ void __launch_bounds__(kThreads) k_observe(SimParams P, Ptrs D)
{
    const uint32_t par = D.ctl->parity;
    const float4 *pos = D.pos[par];
    const float4 *vel = D.vel[par];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) {
        float4 v = vel[i];
        acc[0] = (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z;
        acc[1] = v.x; acc[2] = v.y; acc[3] = v.z;
        float4 pi = pos[i];
        const int ti = __float_as_int(pi.w);
        const int cnt = (int)D.nnb[i];
        const uint32_t *row = D.nbr + (size_t)(i >> 5) * P.cap * 32 + (i & 31);
        double vir = 0.0;
        for (int k = 0; k < cnt; ++k) {
            float4 pj = pos[row[(size_t)k * 32]];
            float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
            float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
            float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
            float d2 = dist2_rn(dx, dy, dz);
            if (d2 < P.rc2 && d2 > 0.0f) {
                float r = sqrtf(d2);
                float w = fmaxf(1.0f - r * P.inv_rc, 0.0f);
                float a = ONE_SPECIES ? P.a[0] : P.a[ti * P.n_species + __float_as_int(pj.w)];
                vir += 0.5 * (double)(a * w * r);
            }
        }
        if (P.has_bonds) {
            const uint32_t *bp = D.bond_partner + (size_t)D.pid[par][i] * kMaxBonds;
            for (int b = 0; b < kMaxBonds && bp[b] != kNone; ++b) {
                float4 pj = pos[D.idx_of_pid[bp[b]]];
                float dx = min_image_rn(pj.x, pi.x, P.L[0], P.halfL[0]);
                float dy = min_image_rn(pj.y, pi.y, P.L[1], P.halfL[1]);
                float dz = min_image_rn(pj.z, pi.z, P.L[2], P.halfL[2]);
                float r = sqrtf(dx * dx + dy * dy + dz * dz);
                vir += 0.5 * (double)(-P.k_bond * (r - P.r0_bond) * r);
            }
        }
        acc[4] = vir;
    }
    block_reduce8(acc, D.red + (size_t)blockIdx.x * 8);
}

// Binned profile: block b handles particles [b*chunk, (b+1)*chunk); thread t
// owns bins t, t + blockDim, ... and scans the chunk in order, so every
// partial is summed in a fixed order.  Partials: red[b][2*nbins].
__global__ void __launch_bounds__(kThreads) k_profile(SimParams P, Ptrs D, int bin_axis, int vel_axis, int nbins,
                                                     int chunk)
{
    const uint32_t par = D.ctl->parity;
    const float4 *pos = D.pos[par];
    const float4 *vel = D.vel[par];
    const int b0 = blockIdx.x * chunk;
    const int b1 = min(P.n, b0 + chunk);
    const float scale = (float)nbins / P.L[bin_axis];
    double *out = D.red + (size_t)blockIdx.x * 2 * nbins;
    for (int bin = threadIdx.x; bin < nbins; bin += blockDim.x) {
        double s = 0.0, c = 0.0;
        for (int p = b0; p < b1; ++p) {
            float4 x = pos[p];
            float xc = bin_axis == 0 ? x.x : (bin_axis == 1 ? x.y : x.z);
            int bb = (int)(xc * scale);
            bb = bb < 0 ? 0 : (bb >= nbins ? nbins - 1 : bb);
            if (bb == bin) {
                float4 v = vel[p];
                s += vel_axis == 0 ? v.x : (vel_axis == 1 ? v.y : v.z);
                c += 1.0;
            }
        }
        out[2 * bin] = s;
        out[2 * bin + 1] = c;
    }
}

__global__ void k_pair_rng(uint64_t seed, uint32_t step, int64_t m, const uint32_t *ti, const uint32_t *tj,
                           uint32_t *out_hash, float *out_xi)
{
    const uint32_t key[4] = {(uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), 0x243F6A88u, 0x85A308D3u};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t si = signature(ti[k], step, key);
        uint32_t sj = signature(tj[k], step, key);
        uint32_t A, B;
        pair_hash(si, sj, key, A, B);
        out_hash[2 * k] = A;
        out_hash[2 * k + 1] = B;
        if (out_xi) out_xi[k] = gauss_from_hash(A, B);
    }
}

int grid_for(int n)
{
    int g = (n + kThreads - 1) / kThreads;
    return g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
}

template <bool ONE>
cudaError_t launch_force_s(const SimParams &P, const Ptrs &D, int of, int inc, cudaStream_t s)
{
    const int g = (P.n + kForceThreads - 1) / kForceThreads;
    switch (P.s_mode) {
    case 1: k_force<ONE, 1><<<g, kForceThreads, 0, s>>>(P, D, of, inc); break;
    case 2: k_force<ONE, 2><<<g, kForceThreads, 0, s>>>(P, D, of, inc); break;
    case 3: k_force<ONE, 3><<<g, kForceThreads, 0, s>>>(P, D, of, inc); break;
    default: k_force<ONE, 0><<<g, kForceThreads, 0, s>>>(P, D, of, inc); break;
    }
    return cudaGetLastError();
}

}  // namespace

int observe_blocks_for(int n) { return (n + kThreads - 1) / kThreads; }

cudaError_t launch_signature(const SimParams &P, const Ptrs &D, cudaStream_t s)
{
    k_signature<<<grid_for(P.n), kThreads, 0, s>>>(P, D);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const SimParams &P, const Ptrs &D, int mode, cudaStream_t s)
{
    const int g = grid_for(P.n);
    if (P.lambda_half) {
        if (mode == 0) k_integrate<0, true><<<g, kThreads, 0, s>>>(P, D);
        else if (mode == 1) k_integrate<1, true><<<g, kThreads, 0, s>>>(P, D);
        else k_integrate<2, true><<<g, kThreads, 0, s>>>(P, D);
    } else {
        if (mode == 0) k_integrate<0, false><<<g, kThreads, 0, s>>>(P, D);
        else if (mode == 1) k_integrate<1, false><<<g, kThreads, 0, s>>>(P, D);
        else k_integrate<2, false><<<g, kThreads, 0, s>>>(P, D);
    }
    return cudaGetLastError();
}

cudaError_t launch_force(const SimParams &P, const Ptrs &D, bool out_fout, bool inc_step, cudaStream_t s)
{
    if (P.n_species == 1) return launch_force_s<true>(P, D, out_fout ? 1 : 0, inc_step ? 1 : 0, s);
    return launch_force_s<false>(P, D, out_fout ? 1 : 0, inc_step ? 1 : 0, s);
}

cudaError_t launch_observe(const SimParams &P, const Ptrs &D, int nblocks, cudaStream_t s)
{
    if (P.n_species == 1)
        k_observe<true><<<nblocks, kThreads, 0, s>>>(P, D);
    else
        k_observe<false><<<nblocks, kThreads, 0, s>>>(P, D);
    return cudaGetLastError();
}

cudaError_t launch_profile(const SimParams &P, const Ptrs &D, int bin_axis, int vel_axis, int nbins, int nblocks,
                           cudaStream_t s)
{
    const int chunk = (P.n + nblocks - 1) / nblocks;
    k_profile<<<nblocks, kThreads, 0, s>>>(P, D, bin_axis, vel_axis, nbins, chunk);
    return cudaGetLastError();
}

cudaError_t launch_pair_rng(uint64_t seed, uint64_t step, int64_t m, const uint32_t *ti, const uint32_t *tj,
                            uint32_t *out_hash, float *out_xi, cudaStream_t s)
{
    int64_t g = (m + kThreads - 1) / kThreads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    k_pair_rng<<<(int)g, kThreads, 0, s>>>(seed, (uint32_t)step, m, ti, tj, out_hash, out_xi);
    return cudaGetLastError();
}

}  // namespace dpd
