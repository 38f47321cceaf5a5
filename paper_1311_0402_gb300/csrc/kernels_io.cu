// kernels_io.cu -- moving particle state between the caller's layout (FP64
// x, y, z triples in the caller's particle order) and the device layout
// (FP32 float4 in cell order), on the device.  The load path of Algorithm 1
// ("CPU -> GPU") wraps positions into the box and rounds to FP32; the read
// path scatters by caller index and widens to FP64.
#include "dpd_internal.cuh"

#include <cmath>

namespace dpd {

namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n)
{
    const int64_t g = (n + kThreads - 1) / kThreads;
    return g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : (int)g);
}

// Position component wrapped into [0, L): w = x - L floor(x / L), every
// operation rounded on its own, then rounded to FP32; a value that rounds up
// to L is the same point as 0.
__device__ __forceinline__ float wrap_to_f32(double x, double L, float Lf)
{
    // inside the box already (the usual case): x itself, no FP64 division
    const double w = (x >= 0.0 && x < L) ? x : __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    float f = __double2float_rn(w);
    if (!(f < Lf)) f = 0.0f;
    if (f < 0.0f) f = 0.0f;
    return f;
}

// Validation only: bit 0 of *bad for a non-finite x or v, bit 1 for a
// species outside [0, n_species).
__global__ void k_import_check(int64_t n, int n_species, const double *__restrict__ x, const double *__restrict__ v,
                               const int32_t *__restrict__ sp, uint32_t *bad)
{
    uint32_t b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (!isfinite(x[3 * i + a]) || !isfinite(v[3 * i + a])) b |= 1u;
        if (sp && (sp[i] < 0 || sp[i] >= n_species)) b |= 2u;
    }
    if (__any_sync(0xFFFFFFFFu, b != 0u)) {
        const uint32_t w = __reduce_or_sync(0xFFFFFFFFu, b);
        if ((threadIdx.x & 31) == 0) atomicOr(bad, w);
    }
}

__global__ void k_import(int64_t n, double Lx, double Ly, double Lz, float Lxf, float Lyf, float Lzf,
                         const double *__restrict__ x, const double *__restrict__ v, const int32_t *__restrict__ sp,
                         const uint32_t *__restrict__ tag, float4 *pos, float4 *vel, uint32_t *tag_out,
                         uint32_t *pid_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = sp ? sp[i] : 0;
        pos[i] = make_float4(wrap_to_f32(x[3 * i], Lx, Lxf), wrap_to_f32(x[3 * i + 1], Ly, Lyf),
                             wrap_to_f32(x[3 * i + 2], Lz, Lzf), __int_as_float(s));
        vel[i] = make_float4(__double2float_rn(v[3 * i]), __double2float_rn(v[3 * i + 1]),
                             __double2float_rn(v[3 * i + 2]), 0.0f);
        tag_out[i] = tag ? tag[i] : (uint32_t)i;
        pid_out[i] = (uint32_t)i;
    }
}

// out[3 pid[p] + a] = src[p].a, widened to FP64.
__global__ void k_export(int64_t n, const float4 *__restrict__ src, const uint32_t *__restrict__ pid, double *out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = src[p];
        const size_t i = pid[p];
        out[3 * i] = q.x;
        out[3 * i + 1] = q.y;
        out[3 * i + 2] = q.z;
    }
}

}  // namespace

cudaError_t launch_import_check(int64_t n, int n_species, const double *x, const double *v, const int32_t *sp,
                                uint32_t *bad, cudaStream_t s)
{
    k_import_check<<<grid_for(n), kThreads, 0, s>>>(n, n_species, x, v, sp, bad);
    return cudaGetLastError();
}

cudaError_t launch_import(const SimParams &P, const double box[3], int64_t n, const double *x, const double *v,
                          const int32_t *sp, const uint32_t *tag, float4 *pos, float4 *vel, uint32_t *tag_out,
                          uint32_t *pid_out, cudaStream_t s)
{
    k_import<<<grid_for(n), kThreads, 0, s>>>(n, box[0], box[1], box[2], P.L[0], P.L[1], P.L[2], x, v, sp, tag, pos,
                                              vel, tag_out, pid_out);
    return cudaGetLastError();
}

cudaError_t launch_export(int64_t n, const float4 *src, const uint32_t *pid, double *out, cudaStream_t s)
{
    k_export<<<grid_for(n), kThreads, 0, s>>>(n, src, pid, out);
    return cudaGetLastError();
}

}  // namespace dpd
