// dpd_internal.cuh -- device data layout, parameter blocks and kernel
// launchers shared by the translation units of libdpd.so.
//
// Layout (all particle arrays in cell order after a rebuild, double-buffered
// so a rebuild can gather into the other set; a device word selects the
// live set, so captured CUDA graphs never see a pointer change):
//   pos[p]   float4 (x, y, z, species as int bits)      16 B
//   vel[p]   float4 (vx, vy, vz, signature as u32 bits)  16 B  -- the velocity
//            the pair force reads (v~ of the lambda scheme) and the
//            particle's TEA signature for the current step (Sec. 3.5)
//   vkick[p] float4 (v + dt/2 f) when lambda != 1/2      16 B
//   force[p] float4 (fx, fy, fz, 0)                       16 B
//   tag[p]   u32 identity tag (keys the random force)
//   pid[p]   u32 caller's particle index
// Neighbour list, packed per group: a group is a run of at most 32
// consecutive particles (the particles of one brick in 32s, or 32-aligned
// tiles when there are no bricks).  Group g's pairs are one dense run of
// 32-bit entries at nbr[g * gcap], entry = (owner lane << 27) | j for the
// pair of particle first + lane with particle j; gdesc[g] = (first,
// owners | entries << 6).  A warp reads 32 consecutive entries in one
// 128-byte transaction (the coalesced, transposed access of Sec. 3.3), and
// the work of a group follows its total pair count rather than its longest
// row.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpd {

constexpr int kMaxSpecies = 8;
constexpr int kMaxBonds = 6;          // bonds per particle
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kOwnerShift = 27;                       // list entry: owner lane above bit 27
constexpr uint32_t kIndexMask = (1u << kOwnerShift) - 1u;
constexpr int64_t kMaxParticles = int64_t(1) << kOwnerShift;
constexpr int kGroup = 32;                            // particles per group (one warp)
constexpr int kForceWarps = 4;                        // groups per block of the pair kernel
constexpr int kStencil = 27;
// bricks: aligned kBrick^3 blocks of cells (contiguous ranges of the Morton
// cell order) with a one-cell halo, staged in shared memory by the builder
constexpr int kBrick = 4;
constexpr int kHalo = kBrick + 2;
constexpr int kHaloCells = kHalo * kHalo * kHalo;  // 216

// The checked build (compiled with DPD_CHECKED): kernels test the indices
// they read from device memory (list entries, permutations, bond partners)
// against the particle count before using them, skip a bad one and set
// kErrBadIndex, which the host reports.  The production build trusts them.
#ifdef DPD_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// device error bits
constexpr uint32_t kErrNbrOverflow = 1u;
constexpr uint32_t kErrNonFinite = 2u;
constexpr uint32_t kErrTimeout = 4u;  // a bounded device-side wait ran out
constexpr uint32_t kErrBadIndex = 8u; // an internal index out of range (reported, the access skipped)

struct DevCtl {
    uint32_t parity;         // live set of the state arrays (pos, vel, vkick, force)
    uint32_t rebuild;        // 1: the rebuild chain runs at its next launch
    uint32_t err;            // error bits
    uint32_t since_rebuild;  // steps since the last rebuild
    unsigned long long step; // step number of the live state
    unsigned long long nrebuild;
    uint32_t max_nnb;        // largest group list total (pair entries) of the last build
    uint32_t rebuild_next;   // displacement flag raised by the kernel running now
    uint32_t pad0;
    uint32_t oparity;        // live set of the order arrays (tag, pid): flips only at a rebuild
};

struct SimParams {
    int n;
    int ncell;
    int nc[3];
    int cap;                  // neighbour capacity per particle (a group holds 32 x cap entries)
    int gcap;                 // entries per group list = 32 * cap
    int ngroups;              // group descriptors (lists) in use
    float L[3];
    float halfL[3];
    float cells_per_len[3];   // nc / L
    float rc2, rc, inv_rc;    // FP32 cutoff for the force decision
    float rlist2;             // FP32 (rc + skin)^2 for the list
    float gamma;
    float sigma_isdt;         // sigma / sqrt(dt)
    float s;
    int s_mode;               // 1: s = 1, 2: s = 1/2, 3: s = 2, 0: general
    float dt, half_dt, lambda_dt;
    float disp2;              // (skin/2)^2 * 0.98^2: rebuild trigger
    float wrap_margin;        // r_list + skin + 0.01 if 2 x that < every L, else 0
    int lambda_half;          // lambda == 1/2 (vel holds v + dt/2 f)
    int n_species;
    int body_mode;
    float body[3];
    int rebuild_every;        // 0 = displacement only
    uint32_t key[4];          // TEA key
    float a[kMaxSpecies * kMaxSpecies];
    float k_bond, r0_bond;
    int has_bonds;
    int newton3;              // half lists (j > i): each pair once, forces summed by vector reductions
    int use_bricks;           // every axis has >= 3 cells: the brick-staged builder
    int list_builder;         // 0: ballot insertion; 1: atomic insertion (ablation)
    int no_reorder;           // 1: particles stay in load order (ablation; tile builder, no bricks)
    int list_layout;          // 0: packed group lists; 1: rows per particle (double insertion, join,
                              // 32x32 tile transpose; full lists, one thread per particle in the force)
    int brick_cap;            // halo particles the brick builder stages in shared memory
    int nb[3];                // bricks per axis
    int nbricks;
};

struct Ptrs {
    float4 *pos[2], *vel[2], *vkick[2], *force[2];
    uint32_t *tag[2], *pid[2];
    float4 *xref;             // positions at the last rebuild
    float4 *facc[2];          // Newton-3 mode: the force of each particle, summed by vector reductions;
                              // buffer (step & 1) takes step `step`'s sums while the pair kernel
                              // clears the other one for the next step
    float4 *fout;             // output of a standalone force evaluation
    DevCtl *ctl;
    unsigned long long *obs;  // the 9 words of a dpd_obs, written by k_obs_finish
    // cells
    const uint32_t *rank_of_cell;  // (cz * nc_y + cy) * nc_x + cx -> Morton rank
    const uint32_t *stencil;       // [ncell][27] neighbour ranks, ascending, kNone pad
    uint32_t *cell_count;          // [ncell]
    uint32_t *cell_start;          // [ncell + 1]
    uint32_t *scan_part;           // block sums of the scan
    uint32_t *key;                 // [n] cell rank per particle
    uint32_t *slot;                // [n] arrival slot inside the cell
    uint32_t *tmp_idx;             // [n] particle index in scatter order
    unsigned long long *skey;      // [n] in-cell sort key in scatter order
    uint32_t *perm;                // [n] new position -> old position
    uint32_t *idx_of_pid;          // [n] caller index -> current position (maintained while bonds are set)
    // neighbours
    uint32_t *nbr;                 // packed group lists, [ngroups][gcap]
    uint2 *gdesc;                  // [ngroups] (first particle, owners | entries << 6)
    uint32_t *rowcnt;              // list_layout 1: [n] row length (core | skin << 16 until the join)
    // bricks
    const uint32_t *brick_rank_lo; // [nbricks] first Morton rank of the brick's cells
    const uint32_t *brick_rank_hi; // [nbricks] last Morton rank (inclusive)
    const uint32_t *brick_ord;     // [nbricks] position of the brick in ascending rank order
    // bonds
    const uint32_t *bond_partner;  // [n][kMaxBonds] partner caller indices
    // reductions
    double *red;                   // per-block partials
    double *vir_part;              // [pair-kernel blocks] virial partials of the last force evaluation
                                   // that closed a call (force evaluation or a run's last step)
};

// ----------------------------------------------------------------- helpers
__host__ __device__ inline uint32_t ceil_div_u(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

// The conditional-graph node guarding the next step's rebuild chain: the
// advance kernel sets it to the rebuild flag (use = 0 outside graphs).
struct NextCond {
    cudaGraphConditionalHandle handle;
    int use;
};

// launchers (each returns the launch status)
cudaError_t launch_signature(const SimParams &P, const Ptrs &D, cudaStream_t s);
// velocity-Verlet phase 1 from the full-step velocity, in place
cudaError_t launch_phase1(const SimParams &P, const Ptrs &D, cudaStream_t s, NextCond next);
cudaError_t launch_rebuild(const SimParams &P, const Ptrs &D, cudaStream_t s, int n_scan_blocks);
// idx_of_pid for the live order (kept up to date by rebuilds only while bonds are set)
cudaError_t launch_index(const SimParams &P, const Ptrs &D, cudaStream_t s);
// Pair force.  kForceEval: the force of the live state into D.fout (out_fout)
// or force[parity], nothing else changes.  kForceStep: force at the live
// state, then phase 2 of this step and phase 1 of the next into the other
// buffer set (flips the live set, advances the step).  kForceFinish: force,
// then phase 2 only (full-step velocity and force into the other set).
enum ForceMode { kForceEval = 0, kForceStep = 1, kForceFinish = 2 };
// In Newton-3 mode the pair kernel only accumulates (facc) and a
// settle kernel completes the same mode afterwards; launch_force runs both.
// after_pair (optional) is recorded with ev_flags right after the pair kernel;
// next: the conditional node of the following step's rebuild chain.
cudaError_t launch_force(const SimParams &P, const Ptrs &D, int mode, bool out_fout, cudaStream_t s,
                         cudaEvent_t after_pair = nullptr, unsigned int ev_flags = 0, NextCond next = NextCond{0, 0});
// observables: nblocks per-block partials in D.red, then their fixed-order
// sum in D.red[nblocks * 8 .. + 8)
cudaError_t launch_observe(const SimParams &P, const Ptrs &D, int nblocks, cudaStream_t s);
cudaError_t launch_observe_finish(const Ptrs &D, int nblocks, int64_t n, double dof, double three_v, cudaStream_t s);
// state transfer in the caller's layout (kernels_io.cu): validation of FP64
// x, v and species (bits into *bad), conversion into the device layout, and
// the scatter of a float4 array to FP64 triples in caller order
cudaError_t launch_import_check(int64_t n, int n_species, const double *x, const double *v, const int32_t *sp,
                                uint32_t *bad, cudaStream_t s);
cudaError_t launch_import(const SimParams &P, const double box[3], int64_t n, const double *x, const double *v,
                          const int32_t *sp, const uint32_t *tag, float4 *pos, float4 *vel, uint32_t *tag_out,
                          uint32_t *pid_out, cudaStream_t s);
cudaError_t launch_export(int64_t n, const float4 *src, const uint32_t *pid, double *out, cudaStream_t s);
cudaError_t launch_profile(const SimParams &P, const Ptrs &D, int bin_axis, int vel_axis, int nbins,
                           int nblocks, cudaStream_t s);
cudaError_t launch_pair_rng(uint64_t seed, uint64_t step, int64_t m, const uint32_t *ti, const uint32_t *tj,
                            uint32_t *out_hash, float *out_xi, cudaStream_t s);
int scan_blocks_for(int ncell);
// the bounded device wait on a transaction that never arrives (failure-detection probe)
cudaError_t launch_wait_probe(const Ptrs &D, uint32_t polls, cudaStream_t s);
cudaError_t time_alu_peak(int kind, int reps, double *lane_ops_per_s, double *ms_per_launch);
// one-time kernel attributes (dynamic shared memory of the brick kernels)
cudaError_t init_kernel_attributes();
// largest brick_cap the builder's shared-memory limit allows
int max_brick_cap();
int observe_blocks_for(int n);

}  // namespace dpd
