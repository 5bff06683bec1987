// Internal declarations shared by the CUDA translation units of libglbm.
// Not part of the public C ABI (include/glbm.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/glbm.h"

// Record the thread's error message (glbm_last_error) and return `st`.
glbm_status glbm_set_error(glbm_status st, const char *fmt, ...);

#define GLBM_MAXN 13                      // highest level N = k + 1 of any lattice
#define GLBM_MAXN_2N1 8                   // highest level of the 2N+1 hierarchy and of
                                          // the 2N+2 axes of D2Q(2N+2)^2 lattices
#define GLBM_MAXQ1 (2 * GLBM_MAXN + 1)    // velocities per axis at GLBM_MAXN
#define GLBM_MAXQA (2 * GLBM_MAXN + 2)    // the same on the 2N+2 hierarchy
#include <type_traits>

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
//
// On the 2N+2 hierarchy (Sec. 4, zero velocity removed; zv = 1) the axis has
// the 2N+2 velocities (m + 1/2) c, written as the odd integers v = +-(2m+1),
// m = 0..N, on a lattice of spacing c/2, whose equilibria are the means of the
// 2N+1 equilibria at the neighbouring velocities m c and (m+1) c
// (Eqs. maineq01_noball - maineq04_noball). They are again polynomials of
// degree 2N in u with E_{-v}(u) = E_v(-u), so the same split holds with the
// magnitude index m in place of n (and no velocity without a mirror):
//   E_{+-(2m+1)}(u) = W_m + Ae_m(v) +- u Bo_m(v).
// Velocity index i of the axis: v = i - N (2N+1 velocities) or
// v = 2i - (2N+1) (2N+2 velocities); W and WN are indexed by i.
// M is the capacity (highest level the arrays hold): the step kernels of
// levels up to 8 take AxisTable, whose small size keeps eight of them (the
// batch kernels' parameters) within the kernel-parameter limit; the levels up
// to 13 of the D1Q3 x D1Q(2N+2) channels and the auxiliary kernels take
// AxisTableHi.
template <int M>
struct AxisTableT {
    int N;
    int zv;                          // 1: the 2N+2 hierarchy
    double W[2 * M + 2];             // by velocity index i
    double WN[2 * M + 2];            // v_i W_i
    double Ce[M + 1][M + 1];         // [n][i] = C[n][2i], n = 0..N
    double Co[M + 1][M];             // [n][i] = C[n][2i+1]
    float Wf[2 * M + 2];
    float WNf[2 * M + 2];
    float Cef[M + 1][M + 1];
    float Cof[M + 1][M];
    float Co1lo[M + 1];  // C[n][1] - Cof[n][0]: low part of the linear coefficient
};
using AxisTable = AxisTableT<GLBM_MAXN_2N1>;
using AxisTableHi = AxisTableT<GLBM_MAXN>;

// Velocities of one axis at compile time: level N, Z = 1 on the 2N+2 hierarchy.
// m is the magnitude index of a +- pair (the zero velocity of the 2N+1
// hierarchy is m = 0 with ipos(0) == ineg(0)).
template <int N, int Z>
struct AxisVel {
    static constexpr int Q = 2 * N + 1 + Z;        // velocities
    static constexpr int VMAX = Z ? 2 * N + 1 : N;  // largest |v|
    static constexpr int M0 = Z ? 0 : 1;           // first m with a +- pair
    static constexpr int NPAIR = Z ? (N + 1) * (N + 1) : N * (N + 1) / 2;  // sum of |v| over v > 0
    __host__ __device__ static constexpr int vel(int i) { return Z ? 2 * i - (2 * N + 1) : i - N; }
    __host__ __device__ static constexpr int vmag(int m) { return Z ? 2 * m + 1 : m; }
    __host__ __device__ static constexpr int ipos(int m) { return Z ? N + 1 + m : N + m; }
    __host__ __device__ static constexpr int ineg(int m) { return N - m; }
    // lattice temperature of the axis: N/3, or (4N+3)/3 in the half-spacing
    // units of the 2N+2 hierarchy (Eq. temp_2N2)
    static constexpr double THETA = Z ? (4.0 * N + 3.0) / 3.0 : N / 3.0;
    // v_i^2 / theta - 1: the coefficient of u_x in Guo's force term
    __host__ __device__ static constexpr double ck(int i) { return (double)vel(i) * vel(i) / THETA - 1.0; }
};

// The same at run time from a table.
template <class Tab>
__host__ __device__ inline int ax_q(const Tab &t)
{
    return 2 * t.N + 1 + t.zv;
}
template <class Tab>
__host__ __device__ inline int ax_vel(const Tab &t, int i)
{
    return t.zv ? 2 * i - (2 * t.N + 1) : i - t.N;
}

// Host: build the table of level N by N exact polynomial convolutions
// (the N-fold summation of D1Q3, Sec. 2). Also returns the full C[n][j]
// array (row-major, (2N+1) x (2N+1)) when `full` is non-null.
// The largest FP64 coefficient of each power j is then adjusted so that the
// identities of the exact polynomials, sum_n C[n][j] = [j == 0] (mass) and
// sum_n n C[n][j] = [j == 1] (momentum), hold to half an ulp of that entry.
// With plainly rounded coefficients the residual (up to several ulps) acts as
// a mass and momentum source of the same sign at every step of a steady flow.
void glbm_build_axis_table(int N, AxisTableHi *t, double *full);
// Host: the table of level N on the 2N+2 hierarchy (zv = 1), from the exact
// 2N+1 coefficients: C'_v[j] = (C_m[j] + C_{m+1}[j]) / 2^{j+1} for v = 2m+1
// (u in units of c/2), with the same half-ulp adjustment of the mass and
// momentum identities.
void glbm_build_axis_table_zv(int N, AxisTableHi *t);
// Host: E_i(u) - W_i of velocity index i from a table (FP64 Horner).
double glbm_eq_dev_host(const AxisTableHi &t, double u, int i);
// Host: the same table in the small layout (level N <= 8).
AxisTable glbm_narrow_table(const AxisTableHi &t);

// Words of a context's device status array: ST_FLAGS bit 0 is set by any node
// that leaves the positivity domain; ST_CLOCK counts the steps launched (it
// seeds the FP32 dither and follows the step clock); ST_DONE counts the CTAs
// finished in the current launch; ST_STEPS counts the steps completed since the
// host last cleared it; ST_HALT is set at the end of a step whose flags are
// set, after which the launches of later steps do nothing. Every CTA reads
// ST_CLOCK and ST_HALT when it starts and adds to ST_DONE when it ends: the
// counter has a 128-byte line of its own, so that those reads do not queue
// behind its atomics at L2. ST_BASE is the step clock at the start of a
// dataflow chunk (below); ST_FLAGS bit 1 records a dataflow wait that ran out
// of time.
enum {
    ST_FLAGS = 0, ST_CLOCK = 32, ST_HALT = 33, ST_BASE = 34, ST_DONE = 64, ST_STEPS = 65,
    ST_WORDS = 96
};
enum { ST_UNSTABLE = 1u, ST_TIMEOUT = 2u };  // bits of ST_FLAGS

// Dataflow stepping of uniform 2D contexts: the launches of a chunk of steps
// overlap. Every CTA lets the next step's grid launch as soon as it starts
// (griddepcontrol.launch_dependents), and instead of waiting for the whole
// previous grid it waits only for the row bands its pulls read and its stores
// overwrite: a CTA covering rows [y0, y0 + R) of step k waits until every
// tile of the bands holding rows [y0 - V, y0 + R - 1 + V] (V the largest y
// speed) has finished step k - 1. Finished tiles are counted per (instance,
// band) in `bands`, reset at the start of each chunk, so step k of the chunk
// waits for k times the tiles of a band. A chunk's first step and a launch
// that follows anything else wait for the whole previous work as usual.
constexpr int GLBM_DF_CHUNK = 64;  // steps per dataflow chunk (the graph chunk)
// Zero the n counting words of a chunk and set ST_BASE from ST_CLOCK.
cudaError_t glbm_launch_df_start(unsigned *status, unsigned *words, long long n, cudaStream_t s);

// Per-instance constants read by the step kernels (one per lattice instance).
struct InstParams {
    double omega;      // 1 / (tau + 1/2)                         (Eq. maineq01)
    double g_theta;    // g / theta_x: force F_i = W_i xi_x g/theta_x   (Sec. 5.4)
    double inv_den;    // 1 / sum_{n>0} n W^y_n: wall emission normaliser
    double g_theta_om; // g / (theta_x omega): force folded into the equilibrium
                       // ((1 - omega/2) g / (theta_x omega) in Guo's form)
    double ew_lo[GLBM_MAXQA];  // E^x_i(u_wall_lo) by x velocity index
    double ew_hi[GLBM_MAXQA];  // E^x_i(u_wall_hi)
    float omega_f, g_theta_f, inv_den_f, g_theta_om_f;
    float dw_lo_f[GLBM_MAXQA];  // E^x_i(u_wall_lo) - W_i
    float dw_hi_f[GLBM_MAXQA];  // E^x_i(u_wall_hi) - W_i
    // geometry of the instance (heterogeneous batches keep their own)
    int N;            // level along y (along both axes unless NX differs)
    int Lx, Ly;       // nodes
    int pitch;        // row pitch in elements (multiple of 64)
    int bc;           // GLBM_BC_*
    int NX;           // level along x
    long long off;    // element offset of this instance in the population buffers
    long long plane;  // elements per velocity plane (Ly * pitch)
    double g_half;    // g / 2: Guo's half-force velocity shift (0 otherwise)
    float g_half_f;
    double dew_lo[GLBM_MAXQA];  // dE^x_i/du at u_wall_lo (2N+1 x axis; the adjoint)
    double dew_hi[GLBM_MAXQA];  // dE^x_i/du at u_wall_hi
};

// Arguments of one uniform (same geometry for every instance) 2D step; TY is
// the table type of the y axis (AxisTableHi above level 8).
template <class TY>
struct Step2DArgsT {
    TY tab;               // level along y (and x for isotropic lattices)
    AxisTable tabx;       // level along x of anisotropic products (else unused)
    const void *fin;      // populations read (post-collision of the last step)
    void *fout;           // populations written
    const InstParams *ip; // n_inst entries
    unsigned *status;     // bit 0: non-positive density / positivity domain left
    unsigned *step_ctr;   // launches so far: seeds the FP32 dithered rounding
    unsigned *done_ctr;   // CTAs finished in the current launch
    void *rw;             // wall densities, 2 x pitch per instance (k_wall_rho), or null:
                          // then every tile near a wall sums them itself
    unsigned *bands;      // dataflow: finished tiles per (instance, row band), or null
    unsigned *node_done;  // dataflow: CTAs finished per step of the chunk
    int node;             // dataflow: this step's index in its chunk
    int Lx, Ly, pitch, bc;
    long long plane;      // elements per velocity plane
    long long inst_stride;// elements per instance
};
using Step2DArgs = Step2DArgsT<AxisTable>;
using Step2DArgsHi = Step2DArgsT<AxisTableHi>;
template <int N>
using Step2DArgsOf = std::conditional_t<(N > GLBM_MAXN_2N1), Step2DArgsHi, Step2DArgs>;

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
    AxisTable tab[GLBM_MAXN_2N1];  // tab[N - 1] (batches take the 2N+1 levels 1..8)
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
// Lattices on the 2N+2 hierarchy: kind GLBM_ZVK_X1 is D1Q3 along x times the
// level-N 2N+2 axis along y; GLBM_ZVK_XY has the level-N 2N+2 axis on both.
enum { GLBM_ZVK_X1 = 0, GLBM_ZVK_XY = 1 };
// Lattice kinds of the 2D step with Guo's force (glbm_step2d_guo.cuh): the
// level-N lattice on both axes, D1Q3 x level N, D1Q3 x the level-N 2N+2 axis.
enum { GLBM_GUOK_ISO = 0, GLBM_GUOK_X1 = 1, GLBM_GUOK_ZV = 2 };
template <int N, typename T, int KIND>
cudaError_t glbm_step2d_guo_level(const Step2DArgs &a, int n_inst, cudaStream_t s);
// Step with Guo's force of level N (1..8), kind GLBM_GUOK_*, precision prec,
// in its one tile shape (glbm_tile_shape_guo).
cudaError_t glbm_launch_step2d_guo(int N, int kind, int prec, const Step2DArgs &a, int n_inst,
                                   cudaStream_t s);
int glbm_tile_shape_guo(int N, int kind, int prec, TileShape *out);
cudaError_t glbm_launch_step2d_zv(int N, int kind, int prec, int shape, const Step2DArgs &a,
                                  int n_inst, cudaStream_t s);
// Levels 9..13 (kind GLBM_ZVK_X1 only).
cudaError_t glbm_launch_step2d_zv_hi(int N, int prec, int shape, const Step2DArgsHi &a,
                                     int n_inst, cudaStream_t s);
int glbm_tile_shapes_zv(int N, int kind, int prec, TileShape *out);
template <int N, typename T>
cudaError_t glbm_step2d_zv_level(int kind, int shape, const Step2DArgsOf<N> &a, int n_inst,
                                 cudaStream_t s);

// 3D tensor products (glbm_step3d.cu): levels 1..3, isotropic, periodic in x
// and z, walls or periodicity in y.
struct Step3DArgs {
    AxisTable tab;         // level N (all three axes)
    const void *fin;
    void *fout;
    const InstParams *ip;
    unsigned *status, *step_ctr, *done_ctr;
    int Lx, Ly, Lz, pitch, bc;
    long long plane;       // elements per velocity plane (Lz * Ly * pitch)
    long long inst_stride; // elements per instance
};
#define GLBM_MAXN_3D 3
cudaError_t glbm_launch_step3d(int N, int prec, int shape, const Step3DArgs &a, int n_inst,
                               cudaStream_t s);
int glbm_tile_shapes_3d(int N, int prec, TileShape *out);

// Auxiliary kernels (glbm_aux.cu).
struct AuxArgs {
    AxisTableHi tab;      // level N along y (the only axis in 1D)
    AxisTableHi tabx;     // level NX along x (2D; equal to tab for isotropic lattices)
    const InstParams *ip;
    int dims, prec;       // prec: 0 = FP64, 1 = FP32 deviations
    int Lx, Ly, pitch, bc, N, NX;
    long long plane, inst_stride;
    int Lz;               // nodes along z (3D; 1 otherwise)
};
cudaError_t glbm_launch_set_equilibrium(const AuxArgs &a, void *f, int inst, const double *rho,
                                        const double *ux, const double *uy, cudaStream_t s);
cudaError_t glbm_launch_set_populations(const AuxArgs &a, void *f, int inst, const double *src,
                                        cudaStream_t s);
cudaError_t glbm_launch_get_populations(const AuxArgs &a, const void *f, int inst, double *dst,
                                        cudaStream_t s);
cudaError_t glbm_launch_moments(const AuxArgs &a, const void *f, int inst, double *out,
                                cudaStream_t s);
// 3D: initial equilibrium with u_z, and the nine moment fields.
cudaError_t glbm_launch_set_equilibrium3d(const AuxArgs &a, void *f, int inst, const double *rho,
                                          const double *ux, const double *uy, const double *uz,
                                          cudaStream_t s);
cudaError_t glbm_launch_moments3d(const AuxArgs &a, const void *f, int inst, double *out,
                                  cudaStream_t s);
// Channel diagnostics (Sec. 5.3, 5.4) of one instance from its moment fields
// (glbm_launch_moments / glbm_launch_moments3d output): prof[0..Ly) the row
// means of u_x, prof[Ly..2Ly) of rho u_x, stats[GLBM_CH_*] the scalars.
struct ChannelParams {
    double theta_y, tau, g;  // lattice temperature of the y axis, relaxation time, force
    double u_lo, u_hi;       // wall speeds (x direction)
    int walls;               // diffuse walls along y (else the wall entries are NaN)
};
cudaError_t glbm_launch_channel_diagnostics(const double *mom, int Lx, int Ly, int Lz,
                                            const ChannelParams &p, double *prof, double *stats,
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
    double *gpart;         // [blocks][GLBM_ADJ_NG] partials of dJ/dtau, dJ/dg, dJ/du_lo,
                           // dJ/du_hi, summed over steps
    int Lx, Ly, pitch, bc, N, prec;
    long long plane;
};
enum { GLBM_ADJ_NG = 4 };  // gradient components of the adjoint
long long glbm_adj_blocks(int Lx, int Ly);
cudaError_t glbm_launch_adj_seed(const AdjArgs &a, cudaStream_t s);
// the wall speeds' term of F_T = S(X_T) (a.X = X_T, mu_T the seed), into gpart
cudaError_t glbm_launch_adj_final_walls(const AdjArgs &a, cudaStream_t s);
cudaError_t glbm_launch_adj_step(const AdjArgs &a, cudaStream_t s);
cudaError_t glbm_launch_adj_sum(const double *gpart, long long nblocks, double *out, cudaStream_t s);
