// kernels_peak.cu -- issue-rate probes for the denominator of the pair
// kernel's ALU roofline: chains of FP32 fused multiply-adds, and chains of
// 32-bit integer xor-then-add, with eight independent chains per thread and
// eight blocks of 256 threads per SM, so that every scheduler always has an
// independent instruction to issue.  Fixed iteration counts, one output word
// per thread (the chains' results, so the compiler keeps the work).
#include "dpd_internal.cuh"

namespace dpd {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;
constexpr int kPeakChains = 8;
constexpr int kPeakIters = 4096;

// a <- a m + c on each chain (one FP32 lane-op per link); m and c are kernel
// arguments, so the chain cannot be folded at compile time.
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float m, float c, float *out)
{
    float a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = (float)(threadIdx.x + 37 * k) * 1e-3f;
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// a <- (a xor x) + y on each chain (one logic and one add lane-op per link;
// the mix of xor and add has no closed form the compiler could substitute).
__global__ void __launch_bounds__(kPeakThreads) k_peak_int(uint32_t x, uint32_t y, uint32_t *out)
{
    uint32_t a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = threadIdx.x * 2654435761u + (uint32_t)k;
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = (a[k] ^ x) + y;
    }
    uint32_t s = 0u;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t time_alu_peak(int kind, int reps, double *lane_ops_per_s, double *ms_per_launch)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = nsm * kPeakBlocksPerSM;
    const size_t nthreads = (size_t)blocks * kPeakThreads;
    void *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, nthreads * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto launch = [&]() {
        if (kind == 0)
            k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>(0.9999999f, 1.0e-7f, (float *)out);
        else
            k_peak_int<<<blocks, kPeakThreads, 0, s>>>(0x9E3779B9u, 0x7F4A7C15u, (uint32_t *)out);
        return cudaGetLastError();
    };
    if (e == cudaSuccess) e = launch();  // warm-up (clocks, instruction cache)
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
        const double ops_per_link = kind == 0 ? 1.0 : 2.0;
        const double ops = (double)nthreads * kPeakIters * kPeakChains * ops_per_link * reps;
        *lane_ops_per_s = ops / (ms * 1e-3);
        *ms_per_launch = ms / reps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    return e;
}

}  // namespace dpd
