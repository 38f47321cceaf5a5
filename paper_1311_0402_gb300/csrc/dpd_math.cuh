// dpd_math.cuh -- device arithmetic of the method: the FP32 pair predicate,
// the TEA hash and signature (Algorithm 4), the Box-Muller Gaussian
// (Sec. 3.5) and the DPD weight functions (Eqs. 7-8).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpd {

// Minimum-image component of d = x_j - x_i along one axis, every operation
// rounded on its own (no contraction), so the host and device predicates
// agree bit for bit: d -= L if d > L/2, d += L if d < -L/2.
__device__ __forceinline__ float min_image_rn(float xj, float xi, float L, float h)
{
    const float t = __fsub_rn(xj, xi);
    const float tm = __fsub_rn(t, L);
    const float tp = __fadd_rn(t, L);
    return t > h ? tm : (t < -h ? tp : t);  // selects, no branches
}

// d^2 = (dx dx + dy dy) + dz dz, each product and sum rounded on its own.
__device__ __forceinline__ float dist2_rn(float dx, float dy, float dz)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ROUNDS rounds of the Tiny Encryption Algorithm (Algorithm 4): the running
// sum grows by delta each round; v0 is updated from v1, then v1 from the new
// v0, each with the XOR of ((v << 4) + k), (v + sum) and ((v >> 5) + k').
template <int ROUNDS>
__device__ __forceinline__ void tea(uint32_t &v0, uint32_t &v1, uint32_t k0, uint32_t k1, uint32_t k2,
                                    uint32_t k3)
{
    uint32_t sum = 0u;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        sum += 0x9E3779B9u;
        v0 += ((v1 << 4) + k0) ^ (v1 + sum) ^ ((v1 >> 5) + k1);
        v1 += ((v0 << 4) + k2) ^ (v0 + sum) ^ ((v0 >> 5) + k3);
    }
}

// Per-particle signature of Algorithm 4 "Preprocess", keyed on the
// identity tag and the step: TEA-16 on (bitreverse(tag), step), v0 ^ v1.
__device__ __forceinline__ uint32_t signature(uint32_t tag, uint32_t step, const uint32_t key[4])
{
    uint32_t v0 = __brev(tag), v1 = step;
    tea<16>(v0, v1, key[0], key[1], key[2], key[3]);
    return v0 ^ v1;
}

// Pair hash: TEA-4 on (min, max) of the two signatures, so the result does
// not depend on which particle of the pair asks (Sec. 3.5: the same number
// must be reproduced for i-j and j-i without communication).
__device__ __forceinline__ void pair_hash(uint32_t si, uint32_t sj, const uint32_t key[4], uint32_t &A,
                                          uint32_t &B)
{
    A = min(si, sj);
    B = max(si, sj);
    tea<4>(A, B, key[0], key[1], key[2], key[3]);
}

// Gaussian from the two hash words by the basic Box-Muller transform
// (Sec. 3.5): radius sqrt(-2 ln u1) with u1 = (A + 1) 2^-32, phase
// cos(pi u2) with u2 = (B & 0x7fffffff) 2^-31 and the top bit of B as the
// sign of the cosine.
//
// -ln u1 is evaluated in FP32 without cancellation near u1 = 1:
// with q = 1 - u1 = (~A) 2^-32 (exact integer, one rounding on conversion),
//   q < 1/16:  -ln(1 - q) = q (1 + q/2 + q^2/3 + q^3/4 + q^4/5 + q^5/6) + R,
//              the Mercator (Taylor) series, |R| < q^7 / (7 (1 - q))
//              (relative to q below 1e-8);
//   otherwise: -ln u1 = -log2(u1) ln 2 with the hardware base-2 logarithm,
//              whose absolute error on [1/2, 1) and relative error below it
//              keep the result within a few 1e-7 relative (u1 <= 15/16).
__device__ __forceinline__ float gauss_from_hash(uint32_t A, uint32_t B)
{
    const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
    const float two_m31 = 4.6566128730773926e-10f;  // 2^-31
    float q = __uint2float_rn(~A) * two_m32;
    float series = fmaf(q, fmaf(q, fmaf(q, fmaf(q, fmaf(q, 1.0f / 6.0f, 0.2f), 0.25f), 1.0f / 3.0f), 0.5f), 1.0f);
    float nl_small = q * series;
    float u1 = fmaf(__uint2float_rn(A), two_m32, two_m32);
    float nl_big = -__log2f(u1) * 0.69314718055994531f;
    float nl = q < 0.0625f ? nl_small : nl_big;
    float rad = sqrtf(2.0f * nl);
    float u2 = __uint2float_rn(B & 0x7FFFFFFFu) * two_m31;
    float c = __cosf(3.14159265358979323846f * u2);
    float g = rad * c;
    return (B >> 31) ? -g : g;
}

// w_R = w^s (Eq. 8) for the exponent modes of SimParams::s_mode.
template <int SMODE>
__device__ __forceinline__ float weight_R(float w, float s)
{
    if (SMODE == 1) return w;
    if (SMODE == 2) return sqrtf(w);
    if (SMODE == 3) return w * w;
    return w > 0.0f ? exp2f(s * __log2f(w)) : 0.0f;
}

}  // namespace dpd
