// ensemble.cuh -- device descriptor, shared-memory layout and launchers of
// the ensemble kernel (many small boxes, one cluster of CTAs per box, the
// box resident in shared memory for a whole chunk of steps).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dpd_internal.cuh"

namespace dpd {

constexpr int kEnsQueue = 64;      // hit ring per warp (< 32 pending + 32 new)
constexpr int kEnsSlots = 4;       // candidates per lane per round, held in registers
constexpr int kEnsCand = 32 * kEnsSlots;  // candidate buffer per warp (a cell's 27-cell stencil, in rounds)
constexpr int kEnsUnitCells = 8;   // consecutive cells per work unit (one warp, queue flushed at the end)
constexpr int kEnsMaxCluster = 8;  // portable cluster size
constexpr int kEnsMaxN = 65535;    // particle indices are 16-bit

// One box of a launch (filled by the host, read once per CTA).
struct EnsBox {
    float4 *pos;            // [n] (x, y, z, species bits) at the box's step
    float4 *vel;            // [n] full-step velocity
    float4 *frc;            // [n] force at the step (w: the particle's conservative virial share)
    const uint32_t *tag;    // [n] random-force tags
    uint32_t *err;          // error bits of the box
    uint32_t *any_err;      // error bits of the whole ensemble (one read tells whether to look further)
    unsigned long long step;
    int n, ncell, steps;    // steps == 0: force only (initial force)
    int nc[3];
    int n_species, s_mode, body_mode, lhalf;
    float L[3], halfL[3], cpl[3];  // cpl = nc / L
    float rc2, inv_rc, gamma, sigma_isdt, s;
    float dt, half_dt, lambda_dt;
    float body[3];
    uint32_t key[4];
    float a[kMaxSpecies * kMaxSpecies];
};

__host__ __device__ inline size_t ens_align16(size_t b) { return (b + 15) & ~size_t(15); }

// Dynamic shared memory of one CTA, in this order: pos, u (the velocity the
// pair force reads, + signature), vh (lambda != 1/2 only), f, cell starts
// [ncell + 1], cell counts [ncell], sorted indices [n], arrival slots [n],
// owning CTA of each particle this step [n] (Newton-3 mode), then per warp
// the hit ring and the candidate buffer.
struct EnsLayout {
    size_t pos, u, vh, f, start, cnt, idx, slot, own, q, cand, total;
};

__host__ __device__ inline EnsLayout ens_layout(int n, int ncell, bool lhalf, int threads)
{
    EnsLayout l;
    size_t o = 0;
    l.pos = o; o += ens_align16((size_t)n * 16);
    l.u = o; o += ens_align16((size_t)n * 16);
    l.vh = o; if (!lhalf) o += ens_align16((size_t)n * 16);
    l.f = o; o += ens_align16((size_t)n * 16);
    l.start = o; o += ens_align16((size_t)(ncell + 1) * 4);
    l.cnt = o; o += ens_align16((size_t)ncell * 4);
    l.idx = o; o += ens_align16((size_t)n * 2);
    l.slot = o; o += ens_align16((size_t)n * 2);
    l.own = o; o += ens_align16((size_t)n);
    const int warps = threads / 32;
    l.q = o; o += (size_t)warps * kEnsQueue * 16;
    l.cand = o; o += (size_t)warps * kEnsCand * 4;
    l.total = o;
    return l;
}

// Launch the chunk kernel over nb boxes (descriptors in device memory),
// `cluster` CTAs per box, `threads` per CTA, `smem` dynamic bytes.
// n3: half stencil, the partner's share added by an atomic to the shared
// memory of the CTA that owns it; otherwise full stencil, fixed order.
cudaError_t launch_ensemble(const EnsBox *boxes, int nb, bool lhalf, int s_mode, bool n3, int threads, int cluster,
                            size_t smem, cudaStream_t s);
// Observables of nb boxes: out[8 b + (0..4)] = sum v^2, virial, momentum.
cudaError_t launch_ensemble_observe(const EnsBox *boxes, int nb, double *out, cudaStream_t s);
// Largest dynamic shared memory per CTA the kernels were set up for (0 if
// the attributes could not be set).
size_t ensemble_smem_limit();
// Active clusters of this shape the device can hold at once (0: cannot run).
int ensemble_max_clusters(bool lhalf, int s_mode, bool n3, int threads, int cluster, size_t smem);

}  // namespace dpd
