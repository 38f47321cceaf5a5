// kernels_observe.cu -- observables of the live state: kinetic sums and
// the virial (Eq. 3 pressure), binned velocity profiles (Sec. 4.2), and the
// pair random numbers exported for checking (Sec. 3.5).  None of these runs
// inside the stepping graphs.
#include "dpd_internal.cuh"
#include "dpd_math.cuh"

namespace dpd {

namespace {

constexpr int kThreads = 256;

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

// Observables, per-block partials of: sum v^2, sum v (3) over the
// particles, and the virial sum over pairs inside r_c of r_ij . F^C_ij plus
// the bonds' share (Eq. 3 and Sec. 4.5).  The virial comes from the force
// evaluation that closed the last call (a force evaluation, or the last step
// of a run): its positions are the current ones, and the pair kernel left one
// partial per block in vir_part, summed here in a fixed order.  The kinetic
// sums are exact to about 2^-48 per thread (Sum2), then FP64.
// Error-free FP32 accumulation (FP64 arithmetic is scarce on this part):
// s + c carries the exact running sum of a few dozen terms to about 2^-48
// relative (Knuth's TwoSum for each addition; a square enters as its exact
// two-term split hi + lo, hi = v v rounded, lo = fma(v, v, -hi)).
struct Sum2 {
    float s = 0.0f, c = 0.0f;
    // every operation rounded on its own: a contracted multiply-add would
    // break the error-free transformations
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        s = t;
    }
    __device__ __forceinline__ void add_square(float v)
    {
        const float hi = __fmul_rn(v, v);
        add(hi);
        c = __fadd_rn(c, fmaf(v, v, -hi));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__global__ void __launch_bounds__(kThreads) k_observe(SimParams P, Ptrs D)
{
    const float4 *__restrict__ vel = D.vel[D.ctl->parity];
    Sum2 v2, px, py, pz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.n; i += stride) {
        const float4 v = vel[i];
        v2.add_square(v.x);
        v2.add_square(v.y);
        v2.add_square(v.z);
        px.add(v.x);
        py.add(v.y);
        pz.add(v.z);
    }
    double acc[8] = {v2.value(), px.value(), py.value(), pz.value(), 0, 0, 0, 0};
    const int64_t nvir = (P.ngroups + kForceWarps - 1) / kForceWarps;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nvir; k += stride) acc[4] += D.vir_part[k];
    block_reduce8(acc, D.red + (size_t)blockIdx.x * 8);
}

// Sum of nb per-block partials (8 each) in a fixed order into out[0..7].
__global__ void __launch_bounds__(kThreads) k_reduce8(const double *part, int nb, double *out)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += part[(size_t)b * 8 + k];
    block_reduce8(acc, out);
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

// One thread: the derived observables of the sums k_reduce8 left (v^2,
// momentum, virial), by the same expressions as the host side of
// dpd_observables with its divisors passed in (3N - 3 and 3V), stored as the
// nine 8-byte words of a dpd_obs: step, n, kinetic, temperature, virial,
// pressure, momentum[3].
__global__ void k_obs_finish(const double *sums, const DevCtl *ctl, long long n, double dof, double three_v,
                             unsigned long long *out)
{
    const double s0 = sums[0], vir = sums[4];
    out[0] = ctl->step;
    out[1] = (unsigned long long)n;
    out[2] = (unsigned long long)__double_as_longlong(0.5 * s0);
    out[3] = (unsigned long long)__double_as_longlong(dof > 0.0 ? s0 / dof : 0.0);
    out[4] = (unsigned long long)__double_as_longlong(vir);
    out[5] = (unsigned long long)__double_as_longlong((s0 + vir) / three_v);
    for (int k = 0; k < 3; ++k) out[6 + k] = (unsigned long long)__double_as_longlong(sums[1 + k]);
}

}  // namespace

int observe_blocks_for(int n)
{
    const int g = (n + kThreads - 1) / kThreads;
    return g < 1 ? 1 : (g > 152 * 4 ? 152 * 4 : g);  // grid-stride beyond 4 blocks per SM
}

cudaError_t launch_observe(const SimParams &P, const Ptrs &D, int nblocks, cudaStream_t s)
{
    k_observe<<<nblocks, kThreads, 0, s>>>(P, D);
    k_reduce8<<<1, kThreads, 0, s>>>(D.red, nblocks, D.red + (size_t)nblocks * 8);
    return cudaGetLastError();
}

cudaError_t launch_observe_finish(const Ptrs &D, int nblocks, int64_t n, double dof, double three_v, cudaStream_t s)
{
    k_obs_finish<<<1, 1, 0, s>>>(D.red + (size_t)nblocks * 8, D.ctl, (long long)n, dof, three_v, D.obs);
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
