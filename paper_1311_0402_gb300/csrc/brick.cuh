// brick.cuh -- the cell neighbourhood of a brick, staged in shared memory.
//
// A brick is an aligned kBrick^3 block of cells.  Because cells are ranked
// along a Morton curve, the cells of an aligned power-of-two block are
// consecutive ranks, so the brick's particles are one contiguous range of
// the cell-ordered arrays.  Its halo is the (kBrick+2)^3 block of cells
// around it (periodic), enumerated in (hz, hy, hx) order; the halo's
// particles are staged in that order, each cell's particles in index order,
// so a particle's "brick-local index" (its slot in the staged arrays) is
// fixed between rebuilds and the same in every kernel that stages the halo.
#pragma once

#include "dpd_internal.cuh"

namespace dpd {

struct BrickRange {
    uint32_t lo, hi;  // the brick's own particles [lo, hi)
};

__device__ __forceinline__ int brick_halo_slot(int hx, int hy, int hz) { return (hz * kHalo + hy) * kHalo + hx; }

// Fill the halo tables of brick b: s_cnt[t] particles of halo cell t start
// at global index s_gstart[t] and at staged slot s_off[t]; s_off[kHaloCells]
// is the halo's particle count.  Called by every thread of a block of at
// least kHaloCells threads (multiple of 32); s_wsum has blockDim/32 entries.
__device__ __forceinline__ BrickRange brick_halo(const SimParams &P, const Ptrs &D, int b, uint32_t *s_off,
                                                 uint32_t *s_gstart, uint32_t *s_cnt, uint32_t *s_wsum)
{
    const int bx = b % P.nb[0], by = (b / P.nb[0]) % P.nb[1], bz = b / (P.nb[0] * P.nb[1]);
    const int x0 = bx * kBrick, y0 = by * kBrick, z0 = bz * kBrick;
    uint32_t cnt = 0;
    if (threadIdx.x < kHaloCells) {
        const int t = threadIdx.x;
        const int hx = t % kHalo, hy = (t / kHalo) % kHalo, hz = t / (kHalo * kHalo);
        const int cx = (x0 + hx - 1 + P.nc[0]) % P.nc[0];
        const int cy = (y0 + hy - 1 + P.nc[1]) % P.nc[1];
        const int cz = (z0 + hz - 1 + P.nc[2]) % P.nc[2];
        const uint32_t r = D.rank_of_cell[(cz * P.nc[1] + cy) * P.nc[0] + cx];
        const uint32_t st = D.cell_start[r];
        cnt = D.cell_start[r + 1] - st;
        s_gstart[t] = st;
        s_cnt[t] = cnt;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_wsum[w];
    if (threadIdx.x < kHaloCells) s_off[threadIdx.x] = before + incl - cnt;
    if (threadIdx.x == kHaloCells - 1) s_off[kHaloCells] = before + incl;
    __syncthreads();
    BrickRange br;
    br.lo = D.cell_start[D.brick_rank_lo[b]];
    br.hi = D.cell_start[D.brick_rank_hi[b] + 1];
    return br;
}

// ---------------------------------------------------------------------------
// Bulk (TMA) staging: every halo cell is one contiguous range of the
// cell-ordered arrays, so it is copied into shared memory by one 1-D bulk
// copy (cp.async.bulk, global -> shared, 16-byte aligned, a multiple of 16
// bytes), whose completion is counted in bytes on an mbarrier.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Wait for phase `parity` of the mbarrier, at most `limit` polls; returns
// false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

constexpr uint32_t kStageWaitLimit = 1u << 22;  // polls (each try_wait also blocks for a while)

// Stage the halo of a brick (s_off / s_gstart / s_cnt from brick_halo) from
// up to two float4 arrays into dst0 / dst1 with bulk copies, one per cell
// and array; the caller guarantees s_off[kHaloCells] <= the buffers' size.
// Every thread of the block calls it; returns false (after setting the error
// word) if the copies did not complete within the poll limit.
__device__ __forceinline__ bool brick_stage_bulk(const Ptrs &D, uint64_t *bar, float4 *dst0,
                                                 const float4 *__restrict__ src0, float4 *dst1,
                                                 const float4 *__restrict__ src1, const uint32_t *s_off,
                                                 const uint32_t *s_gstart, const uint32_t *s_cnt)
{
    const uint32_t total = s_off[kHaloCells];
    const uint32_t narr = dst1 ? 2u : 1u;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, total * (uint32_t)sizeof(float4) * narr);
    }
    __syncthreads();
    if (threadIdx.x < kHaloCells) {
        const uint32_t t = threadIdx.x, n = s_cnt[t];
        if (n) {
            bulk_g2s(dst0 + s_off[t], src0 + s_gstart[t], n * (uint32_t)sizeof(float4), bar);
            if (dst1) bulk_g2s(dst1 + s_off[t], src1 + s_gstart[t], n * (uint32_t)sizeof(float4), bar);
        }
    }
    bool ok = mbar_wait(bar, 0u, kStageWaitLimit);
    if (!ok) {
        atomicOr(&D.ctl->err, kErrTimeout);
        mbar_wait(bar, 0u, kStageWaitLimit);  // let copies still in flight land before leaving
    }
    return __syncthreads_and(ok);
}

}  // namespace dpd
