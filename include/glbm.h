/*
 * glbm.h -- C ABI of libglbm, the GB300 (sm_103a) hot path of the Gaussian
 * lattice Boltzmann method (O. Ilyin, arXiv:1905.04597).
 *
 * The method (Sec. 2, Eq. maineq01): populations f_n, one per integer
 * velocity n = -N..N of level N (k = N-1 summations of D1Q3), follow
 *   f_n(t+1, x+n) - f_n(t, x) = omega (f^eq_{n;N} - f_n)(t, x),
 *   omega = 1 / (tau + 1/2),
 * with the summed ("Gaussian") equilibrium of Eqs. maineq02-05; 2D lattices
 * are tensor products of two 1D levels (Sec. 4). Everything here is in
 * lattice units: node spacing 1, time step 1, lattice temperature N/3.
 *
 * Time convention. A context holds, per instance, the post-collision
 * populations X_t. glbm_step advances X_{t+1} = C(S(X_t)) (S = streaming
 * with the boundary rule, C = BGK collision plus body force). The
 * macroscopic fields "at time t" are the moments of S(X_t).
 *
 * Population layout exchanged through this ABI: FP64, logical order
 * f[q][y][x] with x fastest, q = (ny+N)*(2N+1) + (nx+N) in 2D and q = n+N in
 * 1D. Internally the library stores FP64 or FP32 deviations from the rest
 * weights in pitched planes; conversion happens on the device.
 *
 * Errors. Every call returns a glbm_status; on failure nothing changes except
 * where a call says otherwise, and glbm_last_error() gives a message (per
 * thread). Device pointers and streams are CUDA runtime objects of the
 * current device. All calls are asynchronous on the context's stream unless
 * stated otherwise.
 */
#ifndef GLBM_H
#define GLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glbm_ctx glbm_ctx; /* opaque, owned by the library */

typedef enum {
    GLBM_OK = 0,
    GLBM_E_INVAL = -1,       /* bad argument or configuration */
    GLBM_E_NOMEM = -2,       /* device or host allocation failed */
    GLBM_E_CUDA = -3,        /* a CUDA runtime call failed */
    GLBM_E_UNSTABLE = -4,    /* a node left the positivity domain (Sec. 3) or rho <= 0 */
    GLBM_E_TIMEOUT = -5,     /* a bounded device wait ran out */
    GLBM_E_IO = -6,          /* checkpoint file error */
    GLBM_E_UNSUPPORTED = -7  /* valid request not compiled into this build */
} glbm_status;

typedef enum {
    GLBM_BC_WALLS = 0,       /* 2D: periodic in x, diffuse walls at y = -1/2 and y = ny-1/2 */
    GLBM_BC_BOUNCEBACK = 1,  /* 1D: halfway bounce-back at x = -1/2 and x = nx-1/2 */
    GLBM_BC_PERIODIC = 2     /* periodic along every axis */
} glbm_bc;

typedef enum {
    GLBM_FP64 = 0,           /* populations stored and updated in FP64 */
    GLBM_FP32_DEV = 1        /* FP32 deviations f - W from the rest weights, compensated sums */
} glbm_prec;

typedef enum {
    GLBM_ZV_X = 1,           /* x axis on the 2N+2 hierarchy (zero velocity removed, Sec. 4) */
    GLBM_ZV_Y = 2            /* y axis on the 2N+2 hierarchy */
} glbm_zv;

typedef enum {
    GLBM_FORCE_LINEAR = 0,   /* F_i = W_i xi_x g / theta_x, the linearised force of Sec. 5.4 */
    GLBM_FORCE_GUO = 1       /* Guo, Zheng and Shi (2002); not used by the paper */
} glbm_force;

/*
 * One lattice instance.
 *   dims      1, 2 or 3.
 *   nx, ny    nodes (ny ignored when dims == 1). With walls ny >= k+1; with
 *             bounce-back nx >= k+1.
 *   k         summations of D1Q3 per axis (level N = k+1, 2N+1 velocities per
 *             axis, Sec. 2); 0 <= k <= 7, and up to 12 for the channel models
 *             D1Q3 x D1Q(2k+4) of the 2N+2 hierarchy (zv_axes GLBM_ZV_Y with
 *             x_level 1; the paper's G-D1Q22 x D1Q3 .. G-D1Q28 x D1Q3).
 *   x_level   level along x of a 2D lattice: 0 (or k+1) takes the level of k
 *             on both axes; 1 makes the anisotropic product D1Q3 (x) times
 *             the level-(k+1) lattice (y), the tensor product of Sec. 4 with
 *             3 (2k+3) velocities that the paper uses for channel flows. The
 *             x axis then has its own lattice units (theta_x = 1/3): the force
 *             and the wall speeds are x quantities. Velocity q of the layout is
 *             (ny + N) (2 N_x + 1) + (nx + N_x). Not for 1D lattices,
 *             heterogeneous batches or the adjoint.
 *   tau       relaxation time (> 0), used when kn <= 0.
 *   kn        Knudsen number of Eq. (kn), Sec. 5.2: when > 0 it sets
 *             tau = kn * H / sqrt(2 theta), theta = N/3, H = ny (2D) or nx (1D);
 *             theta = (4N+3)/3 when y is on the 2N+2 hierarchy.
 *   bc, prec  glbm_bc, glbm_prec.
 *   u_wall_lo, u_wall_hi  x-velocities of the walls (GLBM_BC_WALLS).
 *   g         body force along x (2D), added after relaxation as
 *             F_i = W_i xi_x g / theta_x (the linearised force of Sec. 5.4),
 *             or in Guo's form (see force). Either way g is a force density:
 *             every node gains exactly g of x momentum per step.
 *   zv_axes   axes of a 2D lattice on the 2N+2 hierarchy of Sec. 4 (the zero
 *             velocity removed, Eqs. maineq01_noball - maineq04_noball), a
 *             mask of glbm_zv; 0 keeps the 2N+1 hierarchy. Such an axis has
 *             the 2N+2 velocities (m + 1/2) c, m = -N-1..N, each with the mean
 *             of the two neighbouring 2N+1 equilibria. It is written on a
 *             lattice of half the spacing, so its velocities are the odd
 *             integers v = 2i - (2N+1) of index i = 0..2N+1 and its lattice
 *             temperature is (4N+3)/3 (Eq. temp_2N2); speeds along it (wall
 *             speeds, u) are in those units. Compiled: GLBM_ZV_Y with
 *             x_level 1 (D1Q3 x D1Q(2N+2), the channel models G-D1Q6 x D1Q3,
 *             G-D1Q8 x D1Q3 of Sec. 5) and GLBM_ZV_X | GLBM_ZV_Y on an
 *             isotropic lattice (D2Q(2N+2)^2); other masks return
 *             GLBM_E_UNSUPPORTED. Walls then need ny >= 2N+1. Velocity q of
 *             the layout is iy Q_x + ix with the velocity indices of the axes.
 *             Not for heterogeneous batches or the adjoint.
 *   nz        nodes along z of a 3D lattice (dims 3): the product of the
 *             level-(k+1) axis on x, y and z (Sec. 4), D3Q(2k+3)^3, k <= 2,
 *             periodic in x and z, bc along y as in 2D; layout [q][z][y][x]
 *             with q = (n_z + N) (2N+1)^2 + (n_y + N) (2N+1) + (n_x + N);
 *             ny * nz <= 65535. Ignored below 3D. Not for heterogeneous
 *             batches or the adjoint.
 *   force     glbm_force. GLBM_FORCE_GUO takes the force of Guo, Zheng and
 *             Shi (Phys. Rev. E 65, 046308, 2002) instead of the paper's: the
 *             equilibrium and the reported velocity use u = (j + g/2) / rho,
 *             j = sum xi f, and F_i = (1 - omega/2) W_i [(xi_i - u).G +
 *             (xi_i.U)(xi_i.G)] with G = (g / theta_x, 0) and U_a = u_a /
 *             theta_a (Guo's second-order term, each axis's temperature in
 *             place of c_s^2). 2D lattices with k <= 7, isotropic, D1Q3 x
 *             level k+1 (x_level 1) or D1Q3 x the 2N+2 axis (zv_axes
 *             GLBM_ZV_Y); one tile shape per level (glbm_tune has nothing to
 *             choose); not for heterogeneous batches or the adjoint
 *             (GLBM_E_UNSUPPORTED). Every instance of a context takes the
 *             same form.
 */
typedef struct {
    int dims;
    int nx, ny;
    int k;
    int x_level;
    double tau;
    double kn;
    int bc;
    int prec;
    double u_wall_lo, u_wall_hi;
    double g;
    int zv_axes;
    int nz;
    int force;
} glbm_config;

/*
 * Create a context of n instances. When every instance shares dims, nx, ny,
 * k, bc and prec the batch is stepped by one launch with the instance as the
 * grid's third dimension; otherwise GLBM_E_UNSUPPORTED (heterogeneous
 * batches go through glbm_batch_create). `stream` is a cudaStream_t (NULL =
 * legacy default stream) on which all work of the context is ordered. Every
 * instance starts at rest (rho = 1, u = 0, X = W). The library allocates
 * its device memory here with cudaMalloc (or the allocator installed by
 * glbm_set_allocator) and frees it in glbm_destroy.
 */
glbm_status glbm_create(const glbm_config *cfgs, int n, void *stream, glbm_ctx **out);

/* Heterogeneous batch: instances may differ in k, ny, nx, tau, walls and
 * force (2D, GLBM_BC_WALLS or GLBM_BC_PERIODIC, one precision). Stepped by a
 * persistent kernel over a work list of (instance, tile). */
glbm_status glbm_batch_create(const glbm_config *cfgs, int n, void *stream, glbm_ctx **out);

void glbm_destroy(glbm_ctx *ctx);

/* Install device allocation callbacks used by later glbm_create calls
 * (NULL, NULL restores cudaMalloc/cudaFree). alloc(bytes, stream, user)
 * returns a device pointer or NULL; release(ptr, stream, user). */
typedef void *(*glbm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*glbm_free_fn)(void *ptr, void *stream, void *user);
glbm_status glbm_set_allocator(glbm_alloc_fn alloc, glbm_free_fn release, void *user);

/* Set instance `inst` to the local equilibrium X = rho E^x(u_x) E^y(u_y)
 * (Eq. maineq02 with the product form of Sec. 4) of the given fields, each
 * ny*nx FP64 values (uy ignored in 1D), on the device when on_device != 0,
 * else in host memory (copied in this call). Resets the step counter. */
glbm_status glbm_set_equilibrium(glbm_ctx *ctx, int inst, const double *rho, const double *ux,
                                 const double *uy, int on_device);
/* The same for a 3D context with the z velocity uz (NULL: u_z = 0); every
 * field nz*ny*nx values [z][y][x]. GLBM_E_INVAL for other contexts. */
glbm_status glbm_set_equilibrium_3d(glbm_ctx *ctx, int inst, const double *rho, const double *ux,
                                    const double *uy, const double *uz, int on_device);

/* Set / read the populations X of instance `inst` in the FP64 logical layout
 * described above (Q*ny*nx values). */
glbm_status glbm_set_populations(glbm_ctx *ctx, int inst, const double *f, int on_device);
glbm_status glbm_get_populations(glbm_ctx *ctx, int inst, double *f, int on_device);

/* Halo columns of an x-slab decomposition (one lattice split along the
 * periodic x axis over several contexts; the paper has no counterpart). Copy
 * the x-columns [x0, x0 + ncols) of every velocity plane and (z, y) row of
 * instance `inst`, exactly as stored (FP32 deviations or FP64, glbm_elem_size
 * bytes per element, no conversion), from the current state X_t to a packed
 * buffer laid out [q][z][y][ncols] (pack), or from such a buffer into the
 * state (unpack). `on_device` selects device or host memory for the buffer;
 * host copies synchronise. GLBM_E_INVAL for columns outside 0..nx. */
glbm_status glbm_pack_columns(glbm_ctx *ctx, int inst, int x0, int ncols, void *dst,
                              int on_device);
glbm_status glbm_unpack_columns(glbm_ctx *ctx, int inst, int x0, int ncols, const void *src,
                                int on_device);
/* Bytes per stored population element (4 in FP32 deviations, 8 in FP64); 0
 * for a null context. */
size_t glbm_elem_size(const glbm_ctx *ctx);

/* Advance every instance by n >= 0 steps (Eq. maineq01 with the boundary
 * rule). The steps are enqueued on the context's stream (repeated chunks of
 * 64 are replayed from a CUDA graph); the call then waits for them and
 * returns.
 * Failure: a step in which any node leaves the positivity domain of Sec. 3
 * (|u| > sqrt(2/3) N per axis, twice that on a 2N+2 axis, or rho <= 0)
 * completes, and the device then skips every later step of the call: the
 * state is X_{t0+k} after the k completed steps, glbm_time() returns t0 + k,
 * and the call returns GLBM_E_UNSTABLE with "k of n steps completed" in
 * glbm_last_error(). Further glbm_step calls complete no step (k = 0) until a
 * new state is set (glbm_set_equilibrium, glbm_set_populations, glbm_load).
 * 1D contexts step their instances one after another, each stopping at its
 * own failing step; there glbm_time() advances by the fewest steps any
 * instance completed. In dataflow mode (glbm_set_dataflow; calls of 2 or more
 * steps) the chunks' launches overlap; the contract is the same: the call
 * writes only the other two of three state buffers (the third is allocated on
 * the first such call), so its starting state survives, and when a node fails
 * the call replays itself launch after launch from it. GLBM_E_TIMEOUT reports
 * a dataflow wait that ran out, with the state that of the call's start.
 * GLBM_E_CUDA: a launch failed (the state is then undefined). */
glbm_status glbm_step(glbm_ctx *ctx, int64_t n);

/* Wait for the context's stream; GLBM_E_UNSTABLE if any step flagged a node. */
glbm_status glbm_sync(glbm_ctx *ctx);

/* Macroscopic fields of instance `inst` at the current time (moments of
 * S(X), FP64, lattice units), fields packed in this order for the bits set
 * in `mask`, each ny*nx values [y][x]:
 *   bit 0 rho, bit 1 u_x, bit 2 u_y, bit 3 T = sum |xi-u|^2 f / (D rho),
 *   bit 4 q_x, bit 5 q_y (q = (1/2) sum (xi-u) |xi-u|^2 f),
 *   bit 6 sigma_xy = sum (xi_x-u_x)(xi_y-u_y) f.
 * In 1D only bits 0, 1, 3, 4 apply. 3D lattices (fields nz*ny*nx values
 * [z][y][x]) add bit 7 u_z and bit 8 q_z, with T = sum |xi-u|^2 f / (3 rho).
 * `out_len` is the capacity in doubles.
 * Synchronises the stream when out is host memory. */
#define GLBM_M_RHO 0x01u
#define GLBM_M_UX 0x02u
#define GLBM_M_UY 0x04u
#define GLBM_M_T 0x08u
#define GLBM_M_QX 0x10u
#define GLBM_M_QY 0x20u
#define GLBM_M_SXY 0x40u
#define GLBM_M_ALL 0x7Fu
#define GLBM_M_UZ 0x80u
#define GLBM_M_QZ 0x100u
#define GLBM_M_ALL3 0x1FFu
glbm_status glbm_moments(glbm_ctx *ctx, int inst, unsigned mask, double *out, size_t out_len,
                         int out_on_device);

/* Global FP64 sums at the current time: total mass, x- and y-momentum of
 * instance `inst` (fixed-order block reduction, deterministic): sum rho,
 * sum rho u_x, sum rho u_y over the moments of S(X), so with Guo's force the
 * x-momentum is that of the shifted velocity, sum (j_x + g/2). Synchronises. */
glbm_status glbm_conservation(glbm_ctx *ctx, int inst, double *mass, double *mom_x,
                              double *mom_y);

/*
 * Channel diagnostics of instance `inst` (2D, or 3D averaged over z) at the
 * current time, from the moments of S(X) (FP64, lattice units, every sum in a
 * fixed order on the device, so repeated calls agree bit for bit):
 *   profile[y] = <u_x>(y) = (1/(nx nz)) sum_{x,z} u_x        (ny values)
 *   stats[GLBM_CH_FLOW_RATE]  J = sum_y (1/(nx nz)) sum_{x,z} rho u_x, the
 *       flow rate (momentum per unit width), as in glbm_adjoint_flowrate;
 *   stats[GLBM_CH_VOLUMETRIC] Q = (1/Kn) sum_y <u_x>(y) / (4 U0 H), the
 *       volumetric flow of Sec. 5.4 with H = ny, U0 = g H^2 / (8 nu),
 *       nu = theta_y tau, Kn = sqrt(2/theta_y) nu / H (Eq. kn); NaN if g = 0;
 *   stats[GLBM_CH_U_LO], stats[GLBM_CH_U_HI] the gas velocity at the wall
 *       planes y = -1/2 and y = ny - 1/2: <u_x> extrapolated linearly from
 *       the two nearest rows, (3 <u_x>(0) - <u_x>(1)) / 2 and its mirror;
 *   stats[GLBM_CH_SLIP_LO] = (u(-1/2) - u_wall_lo) / (u_wall_hi - u_wall_lo),
 *   stats[GLBM_CH_SLIP_HI] = (u_wall_hi - u(ny-1/2)) / (u_wall_hi - u_wall_lo):
 *       the Couette slip of Sec. 5.3, u(0)/(2 U_w) in the frame of each wall
 *       (NaN when the walls have equal speeds).
 * The four wall entries are NaN without walls. `profile` (ny doubles) and
 * `stats` (GLBM_CH_COUNT doubles) may each be NULL; both are host or both
 * device memory (on_device). Synchronises when they are host memory.
 * GLBM_E_UNSUPPORTED for 1D contexts.
 */
#define GLBM_CH_FLOW_RATE 0
#define GLBM_CH_VOLUMETRIC 1
#define GLBM_CH_U_LO 2
#define GLBM_CH_U_HI 3
#define GLBM_CH_SLIP_LO 4
#define GLBM_CH_SLIP_HI 5
#define GLBM_CH_COUNT 6
glbm_status glbm_channel_diagnostics(glbm_ctx *ctx, int inst, double *profile, double *stats,
                                     int on_device);

/*
 * Conservation sums without allocation. The paper has no counterpart: this is
 * a runtime convenience. It computes the same deterministic sums as
 * glbm_conservation (total mass, x- and y-momentum: sum rho, sum rho u_x,
 * sum rho u_y), but it owns no context and allocates nothing. The block
 * partials go to a static 24 KiB array in the library's device memory.
 *
 * It is for callers that may not call cudaMalloc: real-time loops that
 * cannot take the allocator's device-wide synchronisation, applications whose
 * memory pool owns all device memory, and code that runs inside such a pool's
 * own callbacks, where a nested allocation would deadlock or recurse.
 *
 *   fields  device pointer to the moment fields as glbm_moments writes them
 *           with mask GLBM_M_RHO | GLBM_M_UX | GLBM_M_UY: rho, u_x, u_y (2D,
 *           dims = 2) or rho, u_x (1D, dims = 1), each `nodes` doubles.
 *   nodes   1 .. GLBM_NOALLOC_MAX_NODES; larger counts return GLBM_E_INVAL.
 *   sums    device pointer to 3 doubles: mass, x-momentum, y-momentum
 *           (0 in 1D).
 *   stream  cudaStream_t; the call is asynchronous on it.
 *
 * The first call on a device looks up the scratch's device address, and it
 * should come before any stream capture. The address is kept for the life of
 * the device's primary context: after cudaDeviceReset (or anything else that
 * destroys that context) the library must be reloaded before this call is
 * used again. Every call shares the one scratch
 * array, which keeps the last call's contents. Nothing in it needs clearing,
 * because each call overwrites every partial it reads. Calls that overlap on
 * the GPU (different streams, or the same graph launched concurrently) race
 * on the scratch and must be serialised by the caller.
 */
#define GLBM_NOALLOC_MAX_NODES (4096LL * 1024LL)
glbm_status glbm_conservation_noalloc(const double *fields, int dims, int64_t nodes, double *sums,
                                      void *stream);

/*
 * Dataflow stepping (an engineering choice; the paper has no counterpart).
 * With it (the default), glbm_step runs uniform 2D contexts of levels k <= 7
 * whose wall densities come from the step tiles (glbm_get_wall_launch 0, or
 * no walls) in chunks of 64 steps whose launches overlap: a tile of step t+1
 * starts as soon as the rows of step t it reads and overwrites are done,
 * instead of after the whole of step t. The results are identical to
 * launching the steps one after another (same arithmetic, same dither), and so
 * is the failure contract: a glbm_step call of n >= 2 steps leaves the buffer
 * of its starting state unwritten (its first step reads it into a second
 * buffer, and the later steps alternate between that one and a third, one
 * state's memory allocated on first use; the three rotate from call to call,
 * no state is copied) and, if a node leaves the positivity domain, takes that
 * state back and replays the call one step after another, which stops after
 * the failing step. A wait that takes longer than 0.5 s (none should) returns
 * GLBM_E_TIMEOUT with the state of the call's start.
 * on = 0 launches the steps one after another. on = 2 is a test of the timeout
 * path: every wait of a chunk's later steps asks for more tiles than a band
 * has, so the first call of glbm_step waits 0.5 s and returns GLBM_E_TIMEOUT
 * with the state unchanged. If the counters or the third state buffer cannot
 * be allocated, the context steps launch after launch from then on.
 * glbm_get_dataflow returns 1 when the context's steps take this path.
 */
glbm_status glbm_set_dataflow(glbm_ctx *ctx, int on);
int glbm_get_dataflow(const glbm_ctx *ctx);

/*
 * Measured FP64 FMA throughput of the current device (a measurement aid for
 * the FP64 roofline; the paper has no counterpart): a probe kernel in which
 * every thread runs 8 independent FMA chains, 8 CTAs of 256 threads per SM,
 * timed with CUDA events on `stream` (a cudaStream_t; NULL = legacy default),
 * best of two runs after a warm-up. *fma_per_s receives FP64 FMA thread
 * instructions per second. Allocates 2 KB for the duration of the call;
 * synchronises the stream.
 */
glbm_status glbm_measure_fp64_rate(void *stream, double *fma_per_s);

/*
 * Gradient of the flow rate by the discrete adjoint. From the current state
 * X_t0 the context advances `steps` steps (the state afterwards is X_t0+steps,
 * as after glbm_step) keeping a checkpoint every `ckpt_every` steps. It then
 * sweeps backwards: it recomputes each segment from its checkpoint and
 * applies the hand-written adjoint stream-collide step (reverse streaming,
 * transposed diffuse-wall rule, rank-3 transposed BGK Jacobian). Per instance
 * it returns
 *   J        = (1/nx) sum over nodes of the x-momentum of S(X_T) (the
 *              volumetric flow rate per unit width, Sec. 5.4),
 *   dJ_dtau  = dJ/dtau  (omega = 1/(tau + 1/2)),
 *   dJ_dg    = dJ/dg    (body force along x),
 *   dJ_du_lo, dJ_du_hi = dJ/du_wall_lo, dJ/du_wall_hi (the wall speeds of
 *              Sec. 5.3; a wall speed enters only through E^x(u_w) of the
 *              populations the wall re-emits; 0 without walls).
 * Each output is an array of n_inst doubles in host memory; dJ_du_lo and
 * dJ_du_hi may be NULL. 2D uniform contexts of isotropic 2N+1 lattices with
 * the linearised force only (else GLBM_E_UNSUPPORTED). The adjoint state and
 * the gradient sums are FP64. The call allocates steps/ckpt_every +
 * ckpt_every state copies for the duration of the call. Synchronises.
 */
glbm_status glbm_adjoint_flowrate(glbm_ctx *ctx, int64_t steps, int64_t ckpt_every, double *J,
                                  double *dJ_dtau, double *dJ_dg, double *dJ_du_lo,
                                  double *dJ_du_hi);

/*
 * Tile shapes of the fused 2D step (an engineering choice; the paper has no
 * counterpart). A CTA of the stream-collide kernel covers 32 V columns x R
 * node rows: each thread updates V x-adjacent nodes (V = 2: FP32 pairs with
 * packed two-lane arithmetic), and each node's 2k+3 velocity rows are dealt
 * to G warps. Every level k (0..GLBM_LEVELS-1) and precision has up to
 * GLBM_MAX_TILES candidate shapes; entry 0 is the default of a new context.
 *
 * glbm_tile_count returns the number of candidates of level k in precision
 * prec (0 for an invalid pair); glbm_tile_shape returns candidate idx. Both
 * describe isotropic lattices of the 2N+1 hierarchy (levels k <= 7);
 * anisotropic contexts (x_level 1) and the 2N+2 lattices (zv_axes) have their
 * own lists, which glbm_autotune, glbm_set_tiles and glbm_get_tile_shape use.
 * glbm_get_tiles writes the index in use for every level (array of
 * GLBM_LEVELS ints, entry k for level k); glbm_set_tiles sets them (-1 keeps
 * a level's index; GLBM_E_INVAL and no change if an index is out of range).
 *
 * glbm_autotune times every candidate of every level the context steps: reps
 * launches each (1..1000) from the current state into the spare buffer, with
 * CUDA events on the context's stream, and keeps the fastest; with walls it
 * then times both ways of summing the wall densities (glbm_set_wall_launch)
 * with the chosen shapes and keeps the faster. A uniform 2D context of level
 * k <= 7 then steps 128 steps from its state (put back afterwards) with that
 * choice, and with every tile shape in dataflow chunks (glbm_set_dataflow,
 * wall densities from the tiles), and keeps the fastest of all, dataflow on
 * or off. The state, the step clock and the dither sequence are unchanged;
 * the first call allocates the third state buffer of dataflow calls (the
 * timed steps run through it and leave the state's buffer unwritten). If us is non-NULL it
 * receives the microseconds per launch, us[k * GLBM_MAX_TILES + idx], -1 for
 * pairs not timed (GLBM_LEVELS * GLBM_MAX_TILES doubles, host memory). R and
 * V change only which CTA and thread update a node; G also groups the
 * partial moments before their compensated sum, so shapes of different G may
 * differ in the last bits of FP32 results. 2D contexts only. Synchronises.
 */
#define GLBM_LEVELS 13
#define GLBM_MAX_TILES 8
int glbm_tile_count(int k, glbm_prec prec);
glbm_status glbm_tile_shape(int k, glbm_prec prec, int idx, int *G, int *R, int *V);
glbm_status glbm_get_tiles(const glbm_ctx *ctx, int *tiles);
/* The (G, R, V) shape the context uses for level k (for an anisotropic
 * context, from its own candidate list). */
glbm_status glbm_get_tile_shape(const glbm_ctx *ctx, int k, int *G, int *R, int *V);
glbm_status glbm_set_tiles(glbm_ctx *ctx, const int *tiles);
glbm_status glbm_autotune(glbm_ctx *ctx, int reps, double *us);

/* Wall densities (GLBM_BC_WALLS). Every step turns the mass that streams
 * into each diffuse wall into the wall's density rho_w(x), which sets the
 * populations the wall re-emits (diffuse reflection, Sec. 5.3). Either every
 * tile within reach of a wall sums that mass for its own columns before its
 * update (mode 0), or one launch before the stream-collide kernel sums it once
 * per column and wall into a small device buffer (mode 1, one more launch per
 * step). The sums are the same, in the same order: both modes give identical
 * results. A new context takes mode 1 where the tiles near the walls would
 * repeat the sums for more than a tenth of a step's own loads (high levels,
 * narrow channels), else mode 0. glbm_set_wall_launch sets the mode (0 or 1;
 * -1 restores that default; GLBM_E_INVAL otherwise, GLBM_E_UNSUPPORTED for a
 * context without walls, a batch of mixed levels or a 3D context;
 * synchronises). glbm_get_wall_launch returns the mode, -1 where none applies.
 */
glbm_status glbm_set_wall_launch(glbm_ctx *ctx, int mode);
int glbm_get_wall_launch(const glbm_ctx *ctx);

/* Checkpoint of every instance's state (header, raw device image, CRC-32).
 * glbm_load requires a context created with the same configuration. */
glbm_status glbm_save(glbm_ctx *ctx, const char *path);
glbm_status glbm_load(glbm_ctx *ctx, const char *path);

/* Number of steps taken since creation or the last state reset. */
int64_t glbm_time(const glbm_ctx *ctx);

/* Number of kernels the library has launched (graph nodes counted once per
 * replay). */
int64_t glbm_kernel_launches(const glbm_ctx *ctx);

/* Relaxation time actually used by instance `inst` (after the Kn mapping). */
double glbm_tau(const glbm_ctx *ctx, int inst);

/* Coefficients C[n][j] of the equilibrium polynomial E_n(u) = sum_j C[n][j] u^j
 * of level N = k+1 (lattice units), row-major (2N+1) x (2N+1), n = -N..N. */
glbm_status glbm_eq_table(int k, double *out, size_t out_len);

const char *glbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GLBM_H */
