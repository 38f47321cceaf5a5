/*
 * dpd_oracle.c -- plain FP64 CPU oracle for the DPD short-range pair
 * interaction of Tang & Karniadakis, "Accelerating Dissipative Particle
 * Dynamics Simulations on GPUs" (arXiv:1311.0402).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load this library.  The
 * product path (the CUDA library under paper_1311_0402_gb300/) shares no
 * code, header, table or constant with this file and never calls it.
 *
 * What is computed, and where the paper defines it:
 *   - equations of motion, Sec. 2 Eq. 1 (unit mass);
 *   - pairwise-additive force, Sec. 2 Eq. 2, with the conservative,
 *     dissipative and random parts of Eqs. 3-5, the cutoff of Eq. 6 and the
 *     weight functions / fluctuation-dissipation relation of Eqs. 7-9;
 *   - the TEA block hash and the per-particle signature of Algorithm 4
 *     (Sec. 3.5), with the pair hash of 4 rounds on the two signatures;
 *   - the basic Box-Muller transform of Sec. 3.5, with the sign bit / 31-bit
 *     phase split the paper describes for its cosine;
 *   - velocity-Verlet time stepping, Sec. 3.1 / Algorithm 1 (phases 1 and 2),
 *     written in the lambda form whose lambda = 1/2 case is exactly that
 *     kick-drift-kick scheme;
 *   - harmonic bonds F = K (r - r0), Sec. 4.5.
 *
 * The neighbour list, cell list and particle reordering of Secs. 3.2-3.3
 * are exact accelerations of the plain definition "all pairs with
 * |r_ij| < r_c under the periodic minimum image", so the force routine
 * below evaluates that definition directly (a brute-force O(N^2) loop, or a
 * simple linked-cell loop that visits every pair exactly once and is pinned
 * against the brute-force loop in the tests).
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - TEA constants: delta = 0x9E3779B9, k0 = low 32 bits of the seed,
 *     k1 = high 32 bits, k2 = 0x243F6A88, k3 = 0x85A308D3.
 *   - The signature's second word is the step number (u32), not velocity
 *     mantissa bits, so that the hash is a function of (seed, step, tag).
 *   - The pair hash is TEA-4 on (min(sig_i, sig_j), max(sig_i, sig_j)), so
 *     xi_ij = xi_ji.
 *   - xi = sign * sqrt(-2 ln u1) * cos(pi u2) with u1 = (A + 1) 2^-32 and
 *     u2 = (B & 0x7FFFFFFF) 2^-31, sign = -1 iff the top bit of B is set.
 *   - r_ij = r_i - r_j, e_ij = r_ij / |r_ij|; a pair at r = 0 contributes 0.
 *   - m = 1; sigma = sqrt(2 gamma kT).
 *   - Where floating point decides whether a pair interacts, the decision
 *     can be taken with the FP32 predicate the GPU kernels use (see
 *     oc_fp32_d2), so both sides admit the same pairs; w is then clamped to
 *     be >= 0 for a pair the FP32 test admits at an FP64 distance a rounding
 *     error above r_c.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math, no
 * contraction: the FP32 predicate must round every operation on its own).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_OK 0
#define OC_ERR_ARG 1
#define OC_ERR_OOM 2
#define OC_ERR_CAP 3

/* ------------------------------------------------------------------------ */
/* Tiny Encryption Algorithm, Algorithm 4 (Sec. 3.5).                        */
/* ------------------------------------------------------------------------ */

/* One call applies `rounds` TEA rounds to (v[0], v[1]) under the key k[4].
 * Each round adds delta to the running sum, then updates v0 from v1 and v1
 * from the new v0 with the three-term exclusive-or of Algorithm 4.  All
 * arithmetic is unsigned 32-bit with wrap-around and logical shifts. */
void oc_tea(int rounds, const uint32_t k[4], uint32_t v[2])
{
    const uint32_t delta = 0x9E3779B9u;
    uint32_t v0 = v[0], v1 = v[1], sum = 0u;
    for (int r = 0; r < rounds; ++r) {
        sum += delta;
        uint32_t t0 = (uint32_t)((v1 << 4) + k[0]);
        uint32_t t1 = (uint32_t)(v1 + sum);
        uint32_t t2 = (uint32_t)((v1 >> 5) + k[1]);
        v0 += t0 ^ t1 ^ t2;
        uint32_t s0 = (uint32_t)((v0 << 4) + k[2]);
        uint32_t s1 = (uint32_t)(v0 + sum);
        uint32_t s2 = (uint32_t)((v0 >> 5) + k[3]);
        v1 += s0 ^ s1 ^ s2;
    }
    v[0] = v0;
    v[1] = v1;
}

/* The key the method uses for a global seed (reading of the unprinted
 * constants of Algorithm 4). */
void oc_key(uint64_t seed, uint32_t k[4])
{
    k[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    k[1] = (uint32_t)(seed >> 32);
    k[2] = 0x243F6A88u;
    k[3] = 0x85A308D3u;
}

/* Bit reversal of a 32-bit word, bit by bit (Algorithm 4, BitReverse). */
uint32_t oc_bitrev32(uint32_t x)
{
    uint32_t y = 0u;
    for (int b = 0; b < 32; ++b) {
        y = (y << 1) | (x & 1u);
        x >>= 1;
    }
    return y;
}

/* Per-particle binary signature, Algorithm 4 "Preprocess": v0 = the bit-
 * reversed identity tag, v1 = the step number, 16 TEA rounds, then
 * v0 XOR v1. */
uint32_t oc_signature(uint64_t seed, uint32_t tag, uint64_t step)
{
    uint32_t k[4], v[2];
    oc_key(seed, k);
    v[0] = oc_bitrev32(tag);
    v[1] = (uint32_t)step;
    oc_tea(16, k, v);
    return v[0] ^ v[1];
}

/* Pair hash (Sec. 3.5): 4 TEA rounds on the ordered pair of signatures.
 * out[0] = A', out[1] = B'. */
void oc_pair_hash(uint64_t seed, uint64_t step, uint32_t tag_i, uint32_t tag_j,
                  uint32_t out[2])
{
    uint32_t k[4];
    oc_key(seed, k);
    uint32_t si = oc_signature(seed, tag_i, step);
    uint32_t sj = oc_signature(seed, tag_j, step);
    out[0] = si < sj ? si : sj;
    out[1] = si < sj ? sj : si;
    oc_tea(4, k, out);
}

/* Basic Box-Muller (Sec. 3.5) from two 32-bit words: the radial part uses
 * u1 = (a + 1) 2^-32 in (0, 1], the phase uses the low 31 bits of b as
 * u2 in [0, 1) and the top bit of b as the sign of the cosine, so that
 * sign * cos(pi u2) is distributed as cos(2 pi U). */
double oc_gauss(uint32_t a, uint32_t b)
{
    const double two_m32 = 1.0 / 4294967296.0;
    const double two_m31 = 1.0 / 2147483648.0;
    const double pi = 3.14159265358979323846;
    double u1 = ((double)a + 1.0) * two_m32;
    double u2 = (double)(b & 0x7FFFFFFFu) * two_m31;
    double sgn = (b >> 31) ? -1.0 : 1.0;
    return sgn * sqrt(-2.0 * log(u1)) * cos(pi * u2);
}

/* The Gaussian xi_ij for a pair at a step. */
double oc_xi(uint64_t seed, uint64_t step, uint32_t tag_i, uint32_t tag_j)
{
    uint32_t h[2];
    oc_pair_hash(seed, step, tag_i, tag_j, h);
    return oc_gauss(h[0], h[1]);
}

/* xi for many pairs at one step: out[k] = xi(seed, step, ti[k], tj[k]). */
void oc_xi_batch(uint64_t seed, uint64_t step, int64_t m, const uint32_t *ti, const uint32_t *tj,
                 double *out)
{
    for (int64_t k = 0; k < m; ++k) out[k] = oc_xi(seed, step, ti[k], tj[k]);
}

/* The pair-hash words for many pairs at one step (Sec. 3.5):
 * out[2k], out[2k + 1] = oc_pair_hash(seed, step, ti[k], tj[k]). */
void oc_pair_hash_batch(uint64_t seed, uint64_t step, int64_t m, const uint32_t *ti, const uint32_t *tj,
                        uint32_t *out)
{
    for (int64_t k = 0; k < m; ++k) oc_pair_hash(seed, step, ti[k], tj[k], out + 2 * k);
}

/* ------------------------------------------------------------------------ */
/* FP32 pair predicate (Sec. 3.4: the neighbour builder works in single      */
/* precision).  Every operation is rounded on its own, in this order:        */
/*   d = x_j - x_i;  if d > L/2: d -= L  else if d < -L/2: d += L;           */
/*   d2 = (dx*dx + dy*dy) + dz*dz.                                           */
/* ------------------------------------------------------------------------ */
float oc_fp32_d2(const float xi[3], const float xj[3], const float box[3])
{
    float d[3];
    for (int a = 0; a < 3; ++a) {
        float L = box[a];
        float h = 0.5f * L;
        float t = xj[a] - xi[a];
        if (t > h)
            t = t - L;
        else if (t < -h)
            t = t + L;
        d[a] = t;
    }
    float xx = d[0] * d[0];
    float yy = d[1] * d[1];
    float zz = d[2] * d[2];
    float s = xx + yy;
    return s + zz;
}

/* All pairs (i < j) with d2 < r^2 in the FP32 predicate, by brute force
 * (the plain definition of the neighbour set).  x is n x 3 floats.
 * Writes up to cap pairs as (i, j) into out; returns the total count. */
int64_t oc_pairs_fp32_brute(int64_t n, const float *x, const float box[3], float r,
                            uint32_t *out, int64_t cap)
{
    float r2 = r * r;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            if (oc_fp32_d2(x + 3 * i, x + 3 * j, box) < r2) {
                if (out && cnt < cap) {
                    out[2 * cnt] = (uint32_t)i;
                    out[2 * cnt + 1] = (uint32_t)j;
                }
                ++cnt;
            }
        }
    return cnt;
}

/* All j != i with d2 < r^2 for one particle i (for sampled checks at large
 * n).  Writes up to cap indices in increasing order; returns the count. */
int64_t oc_neighbors_of(int64_t n, const float *x, const float box[3], float r, int64_t i,
                        uint32_t *out, int64_t cap)
{
    float r2 = r * r;
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        if (oc_fp32_d2(x + 3 * i, x + 3 * j, box) < r2) {
            if (out && cnt < cap) out[cnt] = (uint32_t)j;
            ++cnt;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Forces, Eqs. 2-9, bonds (Sec. 4.5), body force (Sec. 4.2).               */
/* ------------------------------------------------------------------------ */

typedef struct {
    double box[3];
    int32_t n_species;
    int32_t cut_fp32;       /* 1: pair admitted iff the FP32 predicate holds */
    const double *a;        /* n_species x n_species, symmetric */
    double gamma, kT, rc, s, dt, lambda;
    uint64_t seed;
    int32_t body_mode;      /* 0 none, 1 uniform, 2 +g for y < Ly/2 and -g above */
    int32_t brute;          /* 1: O(N^2) pair loop, 0: linked cells */
    double body[3];
    int64_t nbonds;
    const uint32_t *bonds;  /* nbonds x 2 particle indices (array positions) */
    double k_bond, r0_bond;
} oc_params;

/* Minimum-image difference a - b along one axis of length L. */
static double min_image(double d, double L)
{
    double h = 0.5 * L;
    if (d > h)
        d -= L;
    else if (d < -h)
        d += L;
    return d;
}

/* w_R = w^s (Eq. 8), for w in [0, 1]. */
static double weight_R(double w, double s)
{
    if (w <= 0.0) return 0.0;
    return pow(w, s);
}

/* Force of one pair on particle i (F_ij of Eqs. 3-5); f_j gets -F_ij.
 * Adds the conservative virial r_ij . F^C_ij to *vir. */
static void pair_force(const oc_params *p, double sigma, double inv_sqrt_dt,
                       int64_t i, int64_t j, const double *x, const double *v,
                       const int32_t *sp, const uint32_t *sig, double *f, double *vir)
{
    double rij[3];
    for (int a = 0; a < 3; ++a) rij[a] = min_image(x[3 * i + a] - x[3 * j + a], p->box[a]);
    double r2 = rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2];
    if (p->cut_fp32) {
        float xi[3], xj[3], bx[3];
        for (int a = 0; a < 3; ++a) {
            xi[a] = (float)x[3 * i + a];
            xj[a] = (float)x[3 * j + a];
            bx[a] = (float)p->box[a];
        }
        float rcf = (float)p->rc;
        if (!(oc_fp32_d2(xi, xj, bx) < rcf * rcf)) return;
    } else {
        if (!(r2 < p->rc * p->rc)) return;
    }
    double r = sqrt(r2);
    if (r == 0.0) return;
    double e[3] = {rij[0] / r, rij[1] / r, rij[2] / r};
    double w = 1.0 - r / p->rc;
    if (w < 0.0) w = 0.0;
    double wR = weight_R(w, p->s);
    double wD = wR * wR;
    double vij[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
    double ev = e[0] * vij[0] + e[1] * vij[1] + e[2] * vij[2];
    int ti = sp ? sp[i] : 0, tj = sp ? sp[j] : 0;
    double aij = p->a[ti * p->n_species + tj];
    /* pair hash on the two per-step signatures (Sec. 3.5), then Box-Muller */
    uint32_t k[4], h[2];
    oc_key(p->seed, k);
    h[0] = sig[i] < sig[j] ? sig[i] : sig[j];
    h[1] = sig[i] < sig[j] ? sig[j] : sig[i];
    oc_tea(4, k, h);
    double xi = oc_gauss(h[0], h[1]);
    double FC = aij * w;                       /* Eq. 3, w_C = w */
    double FD = -p->gamma * wD * ev;           /* Eq. 4 */
    double FR = sigma * wR * xi * inv_sqrt_dt; /* Eq. 5 */
    double F = FC + FD + FR;
    for (int a = 0; a < 3; ++a) {
        f[3 * i + a] += F * e[a];
        f[3 * j + a] -= F * e[a];
    }
    *vir += FC * r; /* r_ij . (FC e_ij) */
}

/* Harmonic bond (Sec. 4.5): magnitude K (r - r0), pulling the ends
 * together when stretched.  Adds r_ij . F_ij to *vir. */
static void bond_force(const oc_params *p, int64_t i, int64_t j, const double *x, double *f,
                       double *vir)
{
    double rij[3];
    for (int a = 0; a < 3; ++a) rij[a] = min_image(x[3 * i + a] - x[3 * j + a], p->box[a]);
    double r = sqrt(rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2]);
    if (r == 0.0) return;
    double F = -p->k_bond * (r - p->r0_bond);
    for (int a = 0; a < 3; ++a) {
        f[3 * i + a] += F * rij[a] / r;
        f[3 * j + a] -= F * rij[a] / r;
    }
    *vir += F * r;
}

static int cell_of(double x, double L, int nc)
{
    int c = (int)floor(x / L * nc);
    c %= nc;
    if (c < 0) c += nc;
    return c;
}

/* Total force on every particle at one step: f = sum_j F_ij (Eq. 2) + bonds
 * + body force.  x, v, f are n x 3 doubles in the caller's order; sp and tag
 * may be NULL (species 0, tag = index).  *virial receives the conservative
 * + bond virial sum_{i<j} r_ij . F_ij. */
int oc_forces(const oc_params *p, int64_t n, const double *x, const double *v, const int32_t *sp,
              const uint32_t *tag, uint64_t step, double *f, double *virial)
{
    if (!p || n < 0 || !x || !v || !f || p->rc <= 0 || p->dt <= 0) return OC_ERR_ARG;
    double sigma = sqrt(2.0 * p->gamma * p->kT); /* Eq. 9 */
    double inv_sqrt_dt = 1.0 / sqrt(p->dt);
    double vir = 0.0;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    /* Algorithm 4 preprocessing: one signature per particle for this step. */
    uint32_t *sig = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!sig) return OC_ERR_OOM;
    for (int64_t i = 0; i < n; ++i)
        sig[i] = oc_signature(p->seed, tag ? tag[i] : (uint32_t)i, step);

    if (p->brute) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 1; j < n; ++j)
                pair_force(p, sigma, inv_sqrt_dt, i, j, x, v, sp, sig, f, &vir);
    } else {
        /* Linked cells of side >= r_c (1 + 1e-4): the margin covers the
         * rounding of the FP32 predicate, which can admit a pair whose FP64
         * distance exceeds r_c by a few parts in 1e6.  Every pair i < j in
         * the same or an adjacent cell is visited once. */
        int nc[3];
        for (int a = 0; a < 3; ++a) {
            nc[a] = (int)floor(p->box[a] / (p->rc * (1.0 + 1e-4)));
            if (nc[a] < 1) nc[a] = 1;
        }
        int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
        int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        int *cid = (int *)malloc(sizeof(int) * 3 * (size_t)(n > 0 ? n : 1));
        if (!head || !next || !cid) {
            free(head); free(next); free(cid); free(sig);
            return OC_ERR_OOM;
        }
        for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
        for (int64_t i = n - 1; i >= 0; --i) {
            int c3[3];
            for (int a = 0; a < 3; ++a) c3[a] = cell_of(x[3 * i + a], p->box[a], nc[a]);
            memcpy(cid + 3 * i, c3, sizeof(c3));
            int64_t c = ((int64_t)c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
            next[i] = head[c];
            head[c] = i;
        }
        /* Distinct neighbour offsets per axis: {-1,0,1}, or fewer when the
         * axis has fewer than three cells (so no cell is visited twice). */
        int off[3][3], noff[3];
        for (int a = 0; a < 3; ++a) {
            if (nc[a] >= 3) { off[a][0] = -1; off[a][1] = 0; off[a][2] = 1; noff[a] = 3; }
            else if (nc[a] == 2) { off[a][0] = 0; off[a][1] = 1; noff[a] = 2; }
            else { off[a][0] = 0; noff[a] = 1; }
        }
        for (int64_t i = 0; i < n; ++i) {
            const int *c3 = cid + 3 * i;
            for (int oz = 0; oz < noff[2]; ++oz)
                for (int oy = 0; oy < noff[1]; ++oy)
                    for (int ox = 0; ox < noff[0]; ++ox) {
                        int cx = (c3[0] + off[0][ox] + nc[0]) % nc[0];
                        int cy = (c3[1] + off[1][oy] + nc[1]) % nc[1];
                        int cz = (c3[2] + off[2][oz] + nc[2]) % nc[2];
                        int64_t c = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
                        for (int64_t j = head[c]; j >= 0; j = next[j])
                            if (j > i)
                                pair_force(p, sigma, inv_sqrt_dt, i, j, x, v, sp, sig, f, &vir);
                    }
        }
        free(head); free(next); free(cid);
    }
    free(sig);

    for (int64_t b = 0; b < p->nbonds; ++b) {
        int64_t i = p->bonds[2 * b], j = p->bonds[2 * b + 1];
        if (i >= n || j >= n) return OC_ERR_ARG;
        bond_force(p, i, j, x, f, &vir);
    }

    if (p->body_mode == 1) {
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) f[3 * i + a] += p->body[a];
    } else if (p->body_mode == 2) {
        double half = 0.5 * p->box[1];
        for (int64_t i = 0; i < n; ++i) {
            double sgn = x[3 * i + 1] < half ? 1.0 : -1.0;
            for (int a = 0; a < 3; ++a) f[3 * i + a] += sgn * p->body[a];
        }
    }
    if (virial) *virial = vir;
    return OC_OK;
}

/* ------------------------------------------------------------------------ */
/* Time stepping (Sec. 3.1, Algorithm 1) and observables.                   */
/* ------------------------------------------------------------------------ */

static double wrap(double x, double L)
{
    x -= L * floor(x / L);
    if (x >= L) x -= L;
    if (x < 0.0) x = 0.0;
    return x;
}

/* Per-step observables: out[0] = sum v^2 (= 2 KE, m = 1), out[1] = the
 * virial of oc_forces, out[2..4] = total momentum. */
static void observe(int64_t n, const double *v, double vir, double *out)
{
    double v2 = 0, px = 0, py = 0, pz = 0;
    for (int64_t i = 0; i < n; ++i) {
        v2 += v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        px += v[3 * i];
        py += v[3 * i + 1];
        pz += v[3 * i + 2];
    }
    out[0] = v2;
    out[1] = vir;
    out[2] = px;
    out[3] = py;
    out[4] = pz;
}

/* Advance nsteps steps of the lambda form of velocity Verlet.  With f the
 * force at (x_k, step k):
 *     x_{k+1} = x_k + dt v_k + dt^2/2 f_k          (phase 1: kick + drift)
 *     v~      = v_k + lambda dt f_k
 *     f_{k+1} = F(x_{k+1}, v~, step k+1)           (force, RNG keyed on k+1)
 *     v_{k+1} = v_k + dt/2 (f_k + f_{k+1})         (phase 2: kick)
 * With lambda = 1/2 this is exactly the paper's kick-drift-kick scheme.
 * f must hold F(x_k, v_k, k) on entry (call oc_forces first) and holds
 * f_{k+1} on exit.  Positions are wrapped into [0, L).
 *
 * obs (nullable) receives nsteps rows of 5 (see observe) taken after each
 * step.  prof_sum / prof_cnt (nullable) accumulate v_x and counts in
 * prof_nbins bins along y for steps with index >= prof_from (step count
 * since this call's start, 1-based). */
int oc_run(const oc_params *p, int64_t n, double *x, double *v, double *f, const int32_t *sp,
           const uint32_t *tag, uint64_t *step, int64_t nsteps, double *obs, int32_t prof_nbins,
           int64_t prof_from, double *prof_sum, double *prof_cnt)
{
    if (!p || !x || !v || !f || !step || nsteps < 0) return OC_ERR_ARG;
    double dt = p->dt;
    double *vt = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *fn = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!vt || !fn) { free(vt); free(fn); return OC_ERR_OOM; }
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) {
            int a = (int)(i % 3);
            x[i] = wrap(x[i] + dt * v[i] + 0.5 * dt * dt * f[i], p->box[a]);
            vt[i] = v[i] + p->lambda * dt * f[i];
        }
        double vir = 0.0;
        int rc = oc_forces(p, n, x, vt, sp, tag, *step + 1, fn, &vir);
        if (rc) { free(vt); free(fn); return rc; }
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] = v[i] + 0.5 * dt * (f[i] + fn[i]);
            f[i] = fn[i];
        }
        *step += 1;
        if (obs) observe(n, v, vir, obs + 5 * s);
        if (prof_sum && prof_cnt && prof_nbins > 0 && s + 1 >= prof_from) {
            for (int64_t i = 0; i < n; ++i) {
                int b = (int)floor(x[3 * i + 1] / p->box[1] * prof_nbins);
                if (b < 0) b = 0;
                if (b >= prof_nbins) b = prof_nbins - 1;
                prof_sum[b] += v[3 * i];
                prof_cnt[b] += 1.0;
            }
        }
    }
    free(vt);
    free(fn);
    return OC_OK;
}
