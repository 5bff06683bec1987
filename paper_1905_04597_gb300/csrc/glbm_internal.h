// Internal declarations shared by the CUDA translation units of libglbm.
// Not part of the public C ABI (include/glbm.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/glbm.h"

// Record the thread's error message (glbm_last_error) and return `st`.
glbm_status glbm_set_error(glbm_status st, const char *fmt, ...);

#define GLBM_MAXN 8                       // highest level N = k + 1 compiled
#define GLBM_MAXQ1 (2 * GLBM_MAXN + 1)    // velocities per axis at GLBM_MAXN

// Equilibrium of one axis at level N in lattice units (velocities -N..N,
// temperature N/3), as a polynomial in the velocity u:
//   E_n(u) = sum_j C[n][j] u^j,  n = -N..N, j = 0..2N,
// the coefficient of z^n in (P- / z + P0 + P+ z)^N with
//   P+- = 1/6 +- u/(2N) + u^2/(2N^2),  P0 = 2/3 - u^2/N^2     (Sec. 2, Eqs. maineq03-05).
// Stored split into even and odd powers so that E_n and E_-n = E_n(-u) share
// one evaluation: with v = u^2,
//   E_{+-n}(u) = W_n + Ae_n(v) +- u Bo_n(v),
//   Ae_n(v) = sum_{i=1..N} Ce[n][i] v^i,  Bo_n(v) = sum_{i=0..N-1} Co[n][i] v^i,
// and W_n = C[n][0] the rest weight.
struct AxisTable {
    int N;
    int pad_;
    double W[GLBM_MAXQ1];                    // index n + N
    double WN[GLBM_MAXQ1];                   // n W_n
    double Ce[GLBM_MAXN + 1][GLBM_MAXN + 1];  // [n][i] = C[n][2i], n = 0..N
    double Co[GLBM_MAXN + 1][GLBM_MAXN];      // [n][i] = C[n][2i+1]
    float Wf[GLBM_MAXQ1];
    float WNf[GLBM_MAXQ1];
    float Cef[GLBM_MAXN + 1][GLBM_MAXN + 1];
    float Cof[GLBM_MAXN + 1][GLBM_MAXN];
    float Co1lo[GLBM_MAXN + 1];  // C[n][1] - Cof[n][0]: low part of the linear coefficient
};

// Host: build the table of level N by N exact polynomial convolutions
// (the N-fold summation of D1Q3, Sec. 2). Also returns the full C[n][j]
// array (row-major, (2N+1) x (2N+1)) when `full` is non-null.
// The largest FP64 coefficient of each power j is then adjusted so that the
// identities of the exact polynomials, sum_n C[n][j] = [j == 0] (mass) and
// sum_n n C[n][j] = [j == 1] (momentum), hold to half an ulp of that entry.
// With plainly rounded coefficients the residual (up to several ulps) acts as
// a mass and momentum source of the same sign at every step of a steady flow.
void glbm_build_axis_table(int N, AxisTable *t, double *full);

// Per-instance constants read by the step kernels (one per lattice instance).
struct InstParams {
    double omega;      // 1 / (tau + 1/2)                         (Eq. maineq01)
    double g_theta;    // g / theta_x: force F_i = W_i xi_x g/theta_x   (Sec. 5.4)
    double inv_den;    // 1 / sum_{n>0} n W^y_n: wall emission normaliser
    double g_theta_om; // g / (theta_x omega): force folded into the equilibrium
    double ew_lo[GLBM_MAXQ1];  // E^x_n(u_wall_lo)
    double ew_hi[GLBM_MAXQ1];  // E^x_n(u_wall_hi)
    float omega_f, g_theta_f, inv_den_f, g_theta_om_f;
    float dw_lo_f[GLBM_MAXQ1];  // E^x_n(u_wall_lo) - W_n
    float dw_hi_f[GLBM_MAXQ1];  // E^x_n(u_wall_hi) - W_n
    // geometry of the instance (heterogeneous batches keep their own)
    int N;            // level along y (along both axes unless NX differs)
    int Lx, Ly;       // nodes
    int pitch;        // row pitch in elements (multiple of 32)
    int bc;           // GLBM_BC_*
    int NX;           // level along x
    long long off;    // element offset of this instance in the population buffers
    long long plane;  // elements per velocity plane (Ly * pitch)
};

// Arguments of one uniform (same geometry for every instance) 2D step.
struct Step2DArgs {
    AxisTable tab;        // level along y (and x for isotropic lattices)
    AxisTable tabx;       // level along x of anisotropic products (else unused)
    const void *fin;      // populations read (post-collision of the last step)
    void *fout;           // populations written
    const InstParams *ip; // n_inst entries
    unsigned *status;     // bit 0: non-positive density / positivity domain left
    unsigned *step_ctr;   // launches so far: seeds the FP32 dithered rounding
    unsigned *done_ctr;   // CTAs finished in the current launch
    int Lx, Ly, pitch, bc;
    long long plane;      // elements per velocity plane
    long long inst_stride;// elements per instance
};

// Tile shape of the fused 2D step: G warps share a node's velocity rows, R node
// rows per CTA, V x-adjacent nodes per thread (the candidates per level are
// listed in glbm_tiles.h).
struct TileShape {
    int G, R, V;
};
// Candidate shapes of level N (1..GLBM_MAXN) in precision prec (0 FP64, 1 FP32
// deviations): fills out[0..count) and returns count (0 for an invalid level).
int glbm_tile_shapes(int N, int prec, TileShape *out);

// Arguments of one step of a heterogeneous batch: one launch per level over
// that level's slice of a work list of (instance, x0, y0, N) tiles.
struct BatchArgs {
    AxisTable tab[GLBM_MAXN];  // tab[N - 1]
    const void *fin;           // pool read
    void *fout;                // pool written
    const InstParams *ip;      // per instance (offset, geometry, constants)
    const int4 *items;         // work list, sorted by level
    int n_items;
    int group[GLBM_MAXN + 2];  // items of level N: [group[N], group[N + 1]) (group[0] unused)
    int shape[GLBM_MAXN + 1];  // FP32 tile shape index of each level
    unsigned *status, *step_ctr, *done_ctr;
};
int glbm_batched_launches(const BatchArgs &a);  // launches per step (levels present)
cudaError_t glbm_launch_batched_f32(const BatchArgs &a, cudaStream_t s);
cudaError_t glbm_launch_batched_level(int N, const BatchArgs &a, bool advance, cudaStream_t s);
// One level's launch of a batch step; `advance` moves the launch counter on.
template <int N>
cudaError_t glbm_batched_level(const BatchArgs &a, bool advance, cudaStream_t s);

// Launchers of the uniform step with tile shape index `shape` (return the
// cudaError_t of the launch; cudaErrorInvalidValue for an unknown level/shape).
cudaError_t glbm_launch_step2d_f32(int N, int shape, const Step2DArgs &a, int n_inst,
                                   cudaStream_t s);
cudaError_t glbm_launch_step2d_f64(int N, int shape, const Step2DArgs &a, int n_inst,
                                   cudaStream_t s);
template <int N, typename T>
cudaError_t glbm_step2d_level(int shape, const Step2DArgs &a, int n_inst, cudaStream_t s);
// Anisotropic products with D1Q3 along x (level 1) and level N along y: the
// step with tile shape `shape` of the list glbm_tile_shapes_x1 gives.
cudaError_t glbm_launch_step2d_x1(int N, int prec, int shape, const Step2DArgs &a, int n_inst,
                                  cudaStream_t s);
int glbm_tile_shapes_x1(int N, int prec, TileShape *out);

// Auxiliary kernels (glbm_aux.cu).
struct AuxArgs {
    AxisTable tab;        // level N along y (the only axis in 1D)
    AxisTable tabx;       // level NX along x (2D; equal to tab for isotropic lattices)
    const InstParams *ip;
    int dims, prec;       // prec: 0 = FP64, 1 = FP32 deviations
    int Lx, Ly, pitch, bc, N, NX;
    long long plane, inst_stride;
};
cudaError_t glbm_launch_set_equilibrium(const AuxArgs &a, void *f, int inst, const double *rho,
                                        const double *ux, const double *uy, cudaStream_t s);
cudaError_t glbm_launch_set_populations(const AuxArgs &a, void *f, int inst, const double *src,
                                        cudaStream_t s);
cudaError_t glbm_launch_get_populations(const AuxArgs &a, const void *f, int inst, double *dst,
                                        cudaStream_t s);
cudaError_t glbm_launch_moments(const AuxArgs &a, const void *f, int inst, double *out,
                                cudaStream_t s);
cudaError_t glbm_launch_field_sums(const double *fields, int nfields, long long n, double *partials,
                                   int nblocks, double *out, cudaStream_t s);
int glbm_field_sum_blocks(long long n);
cudaError_t glbm_launch_step1d(const AuxArgs &a, const void *fin, void *fout, int inst,
                               unsigned *status, cudaStream_t s);
cudaError_t glbm_launch_run1d_resident(const AuxArgs &a, void *f, int inst, long long steps,
                                       unsigned *status, cudaStream_t s, int *ok);

// Adjoint step of one instance (glbm_adjoint.cu).
struct AdjArgs {
    AxisTable tab;
    const InstParams *ip;  // this instance
    const void *X;         // forward state X_t of the instance (FP64, or FP32 deviations)
    const double *mu_in;   // mu_{t+1} = dJ/dF_{t+1}, pitched like the populations
    double *mu_out;        // mu_t
    const double *G;       // [2][Lx] wall sums of mu_in (lower, upper)
    double *Gw;            // the same array, written by the wall kernel
    double *gpart;         // [blocks][2] partials of dJ/dtau, dJ/dg, summed over steps
    int Lx, Ly, pitch, bc, N, prec;
    long long plane;
};
long long glbm_adj_blocks(int Lx, int Ly);
cudaError_t glbm_launch_adj_seed(const AdjArgs &a, cudaStream_t s);
cudaError_t glbm_launch_adj_step(const AdjArgs &a, cudaStream_t s);
cudaError_t glbm_launch_adj_sum(const double *gpart, long long nblocks, double *out, cudaStream_t s);
