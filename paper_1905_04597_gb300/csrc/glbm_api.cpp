// C ABI of libglbm (include/glbm.h): contexts, device buffers, the step loop
// with CUDA-graph replay, moments, conservation sums and checkpoints.
//
// A context holds n lattice instances in one pool of device memory (two
// copies: ping-pong). Every instance has its own geometry record (level,
// nodes, pitch, offset into the pool). A uniform context (every instance
// alike) is stepped by one launch of the tile kernel with the instance as the
// grid's third dimension; a heterogeneous one by a persistent kernel over a
// work list of (instance, tile) items.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/glbm.h"
#include "glbm_internal.h"

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

glbm_status glbm_set_error(glbm_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}
#define fail glbm_set_error

#define CUDA_TRY(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(GLBM_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

static glbm_alloc_fn g_alloc = nullptr;
static glbm_free_fn g_free = nullptr;
static void *g_alloc_user = nullptr;

extern "C" glbm_status glbm_set_allocator(glbm_alloc_fn alloc, glbm_free_fn release, void *user)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(GLBM_E_INVAL, "allocator and release must both be set or both be NULL");
    g_alloc = alloc;
    g_free = release;
    g_alloc_user = user;
    return GLBM_OK;
}

extern "C" const char *glbm_last_error(void) { return g_err; }

struct DevAlloc {
    glbm_alloc_fn alloc;
    glbm_free_fn release;
    void *user;
};

static void *dev_alloc(const DevAlloc &A, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 256;
    if (A.alloc) return A.alloc(bytes, (void *)s, A.user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dev_free(const DevAlloc &A, void *p, cudaStream_t s)
{
    if (!p) return;
    if (A.release)
        A.release(p, (void *)s, A.user);
    else
        cudaFree(p);
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct Geo {
    int N, NX, Lx, Ly, pitch, Q;  // N: level along y (and x), NX: level along x
    int zv;           // axes on the 2N+2 hierarchy (GLBM_ZV_X | GLBM_ZV_Y)
    int Lz;           // nodes along z (3D; 1 otherwise)
    long long plane;  // elements per velocity plane
    long long off;    // element offset of the instance in the pool
    long long nodes() const { return (long long)Lx * Ly * Lz; }
};

// A captured chunk of kGraphChunk steps: step 0 reads p0 and writes pa, then the
// steps alternate pa -> pb, pb -> pa (a chunk from buffer b into b' is
// (b, b', b)); df marks the dataflow form.
struct ChunkGraph {
    const void *p0, *pa, *pb;
    bool df;
    cudaGraphExec_t exec;
};

struct glbm_ctx {
    int n_inst = 0;
    int dims = 2, prec = 0;
    bool hetero = false;
    size_t elem = 8;
    std::vector<Geo> geo;
    std::vector<glbm_config> cfg;
    std::vector<AxisTableHi> tabs;     // index N (1..GLBM_MAXN)
    std::vector<AxisTableHi> tabs_zv;  // the same levels on the 2N+2 hierarchy
    std::vector<InstParams> h_ip;
    std::vector<double> tau;
    DevAlloc A{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    long long pool_elems = 0;    // elements per buffer
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;                 // buffer holding X_t
    InstParams *d_ip = nullptr;
    unsigned *d_status = nullptr;  // ST_WORDS status words (ST_FLAGS .. ST_HALT, glbm_internal.h)
    unsigned *h_status = nullptr;  // pinned copy of them, read after every glbm_step
    double *d_mom = nullptr;       // 7 (2D) or 9 (3D) fields of one instance
    double *d_part = nullptr;      // block partials of the conservation sums
    double *d_sums = nullptr;      // 3 sums
    double *d_diag = nullptr;      // channel diagnostics: row means and scalars
    size_t diag_len = 0;
    double *d_stage = nullptr;     // staging of host inputs
    size_t stage_len = 0;
    void *d_rw = nullptr;          // wall densities of the current step (k_wall_rho)
    bool wall_launch = false;      // whether k_wall_rho computes them (else each wall tile)
    int4 *d_items = nullptr;       // heterogeneous work list, sorted by level
    int n_items = 0;
    int group[GLBM_MAXN + 2] = {0};  // first item of each level
    int tile[GLBM_MAXN + 1] = {0};   // tile shape index per level (glbm_tiles.h)
    std::vector<ChunkGraph> graphs;  // captured chunks, by their buffers and form
    int dataflow = 1;              // 1: dataflow chunks where the context allows them
    unsigned *d_df = nullptr;      // per-step CTA counts of a chunk, then the band counts
    long long df_words = 0;
    void *spare = nullptr;         // third state buffer of dataflow calls (allocated on first use)
    bool halted = false;           // a glbm_step stopped at a failing step (until a new state)
    int64_t t = 0;
    int64_t launches = 0;
    unsigned clock_word = 0;  // host copy uploaded by set_clock (lives as long as the context)
};

static const int kGraphChunk = 64;  // steps per captured graph (even: a chunk from b ends in b)

static size_t bytes_state(const glbm_ctx *c) { return (size_t)c->pool_elems * c->elem; }

// Tables of the y axis (level N) and the x axis (level NX) of a geometry.
static const AxisTableHi &tab_y(const glbm_ctx *c, const Geo &g)
{
    return (g.zv & GLBM_ZV_Y) ? c->tabs_zv[g.N] : c->tabs[g.N];
}
static const AxisTableHi &tab_x(const glbm_ctx *c, const Geo &g)
{
    return (g.zv & GLBM_ZV_X) ? c->tabs_zv[g.NX] : c->tabs[g.NX];
}

// Lattice temperature of one axis: N/3, or (4N+3)/3 on the 2N+2 hierarchy
// (Eq. temp_2N2 in units of half the lattice spacing).
static double axis_theta(int N, bool zv) { return zv ? (4.0 * N + 3.0) / 3.0 : N / 3.0; }

static void fill_inst(const glbm_ctx *c, const glbm_config &cfg, const Geo &g, InstParams &ip,
                      double tau)
{
    memset(&ip, 0, sizeof(ip));
    const int N = g.N, NX = g.NX;
    const AxisTableHi &tab = tab_y(c, g);
    const double theta_x = axis_theta(NX, (g.zv & GLBM_ZV_X) != 0);
    ip.omega = 1.0 / (tau + 0.5);
    ip.g_theta = c->dims >= 2 ? cfg.g / theta_x : 0.0;
    double den = 0.0;  // the wall's normaliser runs over the y velocities
    for (int i = 0; i < ax_q(tab); ++i)
        if (ax_vel(tab, i) > 0) den += ax_vel(tab, i) * tab.W[i];
    ip.inv_den = 1.0 / den;
    if (g.zv & GLBM_ZV_X) {
        // E^x_i(u_w) of a 2N+2 x axis by Horner on its table
        const AxisTableHi &tx = tab_x(c, g);
        for (int i = 0; i < ax_q(tx); ++i) {
            const double dlo = glbm_eq_dev_host(tx, cfg.u_wall_lo, i);
            const double dhi = glbm_eq_dev_host(tx, cfg.u_wall_hi, i);
            ip.ew_lo[i] = tx.W[i] + dlo;
            ip.ew_hi[i] = tx.W[i] + dhi;
            ip.dw_lo_f[i] = (float)dlo;
            ip.dw_hi_f[i] = (float)dhi;
        }
    }
    // E^x_n(u_w) of a 2N+1 x axis from its coefficient table (FP64 Horner)
    double full[GLBM_MAXQ1 * GLBM_MAXQ1];
    AxisTableHi tmp;
    glbm_build_axis_table(NX, &tmp, full);
    const int Q1 = (g.zv & GLBM_ZV_X) ? 0 : 2 * NX + 1;
    for (int n = 0; n < Q1; ++n) {
        double elo = 0.0, ehi = 0.0;
        for (int j = Q1 - 1; j >= 0; --j) {
            elo = elo * cfg.u_wall_lo + full[n * Q1 + j];
            ehi = ehi * cfg.u_wall_hi + full[n * Q1 + j];
        }
        ip.ew_lo[n] = elo;
        ip.ew_hi[n] = ehi;
        // deviation computed without the constant term
        double dlo = 0.0, dhi = 0.0;
        for (int j = Q1 - 1; j >= 1; --j) {
            dlo = dlo * cfg.u_wall_lo + full[n * Q1 + j];
            dhi = dhi * cfg.u_wall_hi + full[n * Q1 + j];
        }
        ip.dw_lo_f[n] = (float)(dlo * cfg.u_wall_lo);
        ip.dw_hi_f[n] = (float)(dhi * cfg.u_wall_hi);
        // dE^x_n/du at the wall speeds (the adjoint's wall-speed term)
        double slo = 0.0, shi = 0.0;
        for (int j = Q1 - 1; j >= 1; --j) {
            slo = slo * cfg.u_wall_lo + j * full[n * Q1 + j];
            shi = shi * cfg.u_wall_hi + j * full[n * Q1 + j];
        }
        ip.dew_lo[n] = slo;
        ip.dew_hi[n] = shi;
    }
    ip.g_theta_om = ip.g_theta / ip.omega;
    if (cfg.force == GLBM_FORCE_GUO) {
        // Guo's form: F_i carries (1 - omega/2) g, the relaxation towards the
        // half-force-shifted u the other omega g/2
        ip.g_theta_om *= 1.0 - 0.5 * ip.omega;
        ip.g_half = 0.5 * cfg.g;
    }
    ip.g_half_f = (float)ip.g_half;
    ip.omega_f = (float)ip.omega;
    ip.g_theta_f = (float)ip.g_theta;
    ip.g_theta_om_f = (float)ip.g_theta_om;
    ip.inv_den_f = (float)ip.inv_den;
    ip.N = N;
    ip.NX = NX;
    ip.Lx = g.Lx;
    ip.Ly = g.Ly;
    ip.pitch = g.pitch;
    ip.bc = cfg.bc;
    ip.off = g.off;
    ip.plane = g.plane;
}

static glbm_status validate(const glbm_config &c)
{
    if (c.dims < 1 || c.dims > 3) return fail(GLBM_E_INVAL, "dims must be 1, 2 or 3 (got %d)", c.dims);
    if (c.force != GLBM_FORCE_LINEAR && c.force != GLBM_FORCE_GUO)
        return fail(GLBM_E_INVAL, "force must be GLBM_FORCE_LINEAR or GLBM_FORCE_GUO (got %d)", c.force);
    if (c.force == GLBM_FORCE_GUO) {
        if (c.dims != 2) return fail(GLBM_E_UNSUPPORTED, "Guo's force is compiled for 2D lattices");
        if (c.k > GLBM_MAXN_2N1 - 1)
            return fail(GLBM_E_UNSUPPORTED, "Guo's force is compiled for k <= %d", GLBM_MAXN_2N1 - 1);
        if (c.zv_axes == (GLBM_ZV_X | GLBM_ZV_Y))
            return fail(GLBM_E_UNSUPPORTED,
                        "Guo's force is compiled for the 2N+2 hierarchy along y only");
    }
    if (c.dims == 3) {
        if (c.k < 0 || c.k > GLBM_MAXN_3D - 1)
            return fail(GLBM_E_UNSUPPORTED, "3D lattices take k in 0..%d (got %d)", GLBM_MAXN_3D - 1, c.k);
        if (c.x_level != 0 || c.zv_axes != 0)
            return fail(GLBM_E_UNSUPPORTED, "3D lattices take the level of k on every axis");
        if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(GLBM_E_INVAL, "nx, ny, nz must be >= 1");
        if ((long long)c.ny * c.nz > 65535)
            return fail(GLBM_E_UNSUPPORTED, "3D lattices take ny * nz <= 65535");
        if (c.bc != GLBM_BC_WALLS && c.bc != GLBM_BC_PERIODIC)
            return fail(GLBM_E_INVAL, "3D lattices take GLBM_BC_WALLS or GLBM_BC_PERIODIC");
        if (c.bc == GLBM_BC_WALLS && c.ny < c.k + 1) return fail(GLBM_E_INVAL, "walls need ny >= k+1");
        if (c.prec != GLBM_FP64 && c.prec != GLBM_FP32_DEV) return fail(GLBM_E_INVAL, "bad precision %d", c.prec);
        if (!(c.kn > 0.0) && !(c.tau > 0.0)) return fail(GLBM_E_INVAL, "tau must be > 0 (or kn > 0)");
        const double umax = sqrt(2.0 / 3.0) * (c.k + 1);
        if (!(fabs(c.u_wall_lo) < umax) || !(fabs(c.u_wall_hi) < umax) || !isfinite(c.g))
            return fail(GLBM_E_INVAL, "wall speed outside the positivity domain or bad force");
        return GLBM_OK;
    }
    if (c.k < 0 || c.k > GLBM_MAXN - 1)
        return fail(GLBM_E_UNSUPPORTED, "k must be in 0..%d (got %d)", GLBM_MAXN - 1, c.k);
    const int N = c.k + 1;
    // levels above 8: only the channel models D1Q3 x D1Q(2N+2) (Sec. 5.4 uses N = 10..13)
    if (N > GLBM_MAXN_2N1 && !(c.dims == 2 && c.zv_axes == GLBM_ZV_Y && c.x_level == 1))
        return fail(GLBM_E_UNSUPPORTED,
                    "k > %d is compiled for D1Q3 x D1Q(2k+4) (x_level 1, zv_axes GLBM_ZV_Y) only",
                    GLBM_MAXN_2N1 - 1);
    if (c.x_level < 0 || c.x_level > GLBM_MAXN)
        return fail(GLBM_E_INVAL, "x_level must be in 0..%d (got %d)", GLBM_MAXN, c.x_level);
    if (c.x_level != 0 && c.x_level != 1 && c.x_level != N)
        return fail(GLBM_E_UNSUPPORTED,
                    "anisotropic lattices take D1Q3 along x (x_level 1) or the level of k");
    if (c.x_level != 0 && c.dims != 2) return fail(GLBM_E_INVAL, "x_level applies to 2D lattices");
    const int NX = c.x_level > 0 ? c.x_level : N;
    const int zv = c.zv_axes;
    if (zv < 0 || zv > (GLBM_ZV_X | GLBM_ZV_Y))
        return fail(GLBM_E_INVAL, "zv_axes must be a mask of GLBM_ZV_X and GLBM_ZV_Y (got %d)", zv);
    if (zv != 0 && c.dims != 2) return fail(GLBM_E_INVAL, "the 2N+2 hierarchy applies to 2D lattices");
    if (zv != 0 && !(zv == GLBM_ZV_Y && NX == 1) &&
        !(zv == (GLBM_ZV_X | GLBM_ZV_Y) && NX == N))
        return fail(GLBM_E_UNSUPPORTED,
                    "the 2N+2 hierarchy is compiled along y with D1Q3 along x (x_level 1) "
                    "or along both axes of an isotropic lattice");
    if (c.nx < 1 || (c.dims == 2 && c.ny < 1)) return fail(GLBM_E_INVAL, "nx, ny must be >= 1");
    if (c.prec != GLBM_FP64 && c.prec != GLBM_FP32_DEV) return fail(GLBM_E_INVAL, "bad precision %d", c.prec);
    if (c.dims == 1) {
        if (c.bc != GLBM_BC_BOUNCEBACK && c.bc != GLBM_BC_PERIODIC)
            return fail(GLBM_E_INVAL, "1D lattices take GLBM_BC_BOUNCEBACK or GLBM_BC_PERIODIC");
        if (c.bc == GLBM_BC_BOUNCEBACK && c.nx < N)
            return fail(GLBM_E_INVAL, "bounce-back needs nx >= k+1");
    } else {
        if (c.bc != GLBM_BC_WALLS && c.bc != GLBM_BC_PERIODIC)
            return fail(GLBM_E_INVAL, "2D lattices take GLBM_BC_WALLS or GLBM_BC_PERIODIC");
        const int vmax = (zv & GLBM_ZV_Y) ? 2 * N + 1 : N;  // fastest y velocity
        if (c.bc == GLBM_BC_WALLS && c.ny < vmax)
            return fail(GLBM_E_INVAL, "walls need ny >= %d (the fastest y velocity)", vmax);
    }
    if (!(c.kn > 0.0) && !(c.tau > 0.0)) return fail(GLBM_E_INVAL, "tau must be > 0 (or kn > 0)");
    // the wall speeds are x velocities (half-spacing units on a 2N+2 x axis)
    const double umax = sqrt(2.0 / 3.0) * NX * ((zv & GLBM_ZV_X) ? 2.0 : 1.0);
    if (!(fabs(c.u_wall_lo) < umax) || !(fabs(c.u_wall_hi) < umax) || !isfinite(c.g))
        return fail(GLBM_E_INVAL, "wall speed outside the positivity domain or bad force");
    return GLBM_OK;
}

static double tau_of(const glbm_config &c)
{
    if (c.kn > 0.0) {
        const int N = c.k + 1;
        const double theta = axis_theta(N, c.dims == 2 && (c.zv_axes & GLBM_ZV_Y));
        const double H = c.dims >= 2 ? c.ny : c.nx;
        return c.kn * H / sqrt(2.0 * theta);  // Eq. (kn), nu = theta tau
    }
    return c.tau;
}

static Geo make_geo(const glbm_config &c)
{
    Geo g;
    g.N = c.k + 1;
    g.NX = c.dims == 2 && c.x_level > 0 ? c.x_level : g.N;
    g.Lx = c.nx;
    g.Ly = c.dims >= 2 ? c.ny : 1;
    g.Lz = c.dims == 3 ? c.nz : 1;
    // rows padded to 64 elements and, in 2D and 3D, one spare row after the
    // Lz Ly rows of each velocity plane: the step tiles store every thread's
    // result unconditionally, the columns past Lx of a ragged tile into the
    // padding and the rows past Ly into the spare row; no pull, reducer or
    // copy reads either
    g.pitch = ((g.Lx + 63) / 64) * 64;
    g.zv = c.dims == 2 ? c.zv_axes : 0;
    const int Q1 = 2 * g.N + 1 + ((g.zv & GLBM_ZV_Y) ? 1 : 0);
    g.Q = c.dims == 2 ? Q1 * (2 * g.NX + 1 + ((g.zv & GLBM_ZV_X) ? 1 : 0)) : Q1;
    if (c.dims == 3) g.Q = Q1 * Q1 * Q1;
    g.plane = ((long long)g.Lz * g.Ly + (c.dims >= 2 ? 1 : 0)) * g.pitch;
    g.off = 0;
    return g;
}

static void drop_graphs(glbm_ctx *c)
{
    for (ChunkGraph &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

static void destroy_resources(glbm_ctx *c)
{
    drop_graphs(c);
    cudaStreamSynchronize(c->stream);
    dev_free(c->A, c->d_df, c->stream);
    dev_free(c->A, c->spare, c->stream);
    dev_free(c->A, c->buf[0], c->stream);
    dev_free(c->A, c->buf[1], c->stream);
    dev_free(c->A, c->d_ip, c->stream);
    dev_free(c->A, c->d_status, c->stream);
    dev_free(c->A, c->d_mom, c->stream);
    dev_free(c->A, c->d_diag, c->stream);
    dev_free(c->A, c->d_part, c->stream);
    dev_free(c->A, c->d_sums, c->stream);
    dev_free(c->A, c->d_stage, c->stream);
    dev_free(c->A, c->d_items, c->stream);
    dev_free(c->A, c->d_rw, c->stream);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->cap) cudaStreamDestroy(c->cap);
}

// Arguments of the auxiliary kernels for one instance: the pool pointer is
// advanced to the instance and the kernels are called with instance 0.
static AuxArgs aux_args(const glbm_ctx *c, int inst)
{
    const Geo &g = c->geo[inst];
    AuxArgs a;
    memset(&a, 0, sizeof(a));
    a.tab = tab_y(c, g);
    a.tabx = tab_x(c, g);
    a.ip = c->d_ip + inst;
    a.dims = c->dims;
    a.prec = c->prec;
    a.Lx = g.Lx;
    a.Ly = g.Ly;
    a.pitch = g.pitch;
    a.bc = c->cfg[inst].bc;
    a.N = g.N;
    a.NX = g.NX;
    a.plane = g.plane;
    a.inst_stride = 0;
    a.Lz = g.Lz;
    return a;
}

static void *inst_ptr(const glbm_ctx *c, int b, int inst)
{
    return (char *)c->buf[b] + (size_t)c->geo[inst].off * c->elem;
}

// The launch counter that seeds the dithered FP32 stores follows the step
// clock, so a run resumed from a checkpoint repeats the same dither sequence.
static cudaError_t set_clock(glbm_ctx *c, int64_t t)
{
    c->t = t;
    c->clock_word = (unsigned)t;
    return cudaMemcpyAsync(c->d_status + ST_CLOCK, &c->clock_word, sizeof(unsigned), cudaMemcpyHostToDevice,
                           c->stream);
}

// A new state (set_equilibrium, set_populations, load): clear the positivity
// flags and the halt word, so that stepping resumes.
static cudaError_t clear_unstable(glbm_ctx *c)
{
    c->halted = false;
    cudaError_t e = cudaMemsetAsync(c->d_status + ST_FLAGS, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status + ST_HALT, 0, sizeof(unsigned), c->stream);
    return e;
}

static glbm_status ensure_stage(glbm_ctx *c, size_t n)
{
    if (c->stage_len >= n) return GLBM_OK;
    dev_free(c->A, c->d_stage, c->stream);
    c->d_stage = (double *)dev_alloc(c->A, n * sizeof(double), c->stream);
    c->stage_len = c->d_stage ? n : 0;
    if (!c->d_stage) return fail(GLBM_E_NOMEM, "staging allocation of %zu doubles failed", n);
    return GLBM_OK;
}

// Allocation and initial state shared by both kinds of context.
// Whether the wall densities of a step get a launch of their own (k_wall_rho,
// once per column and wall) instead of the prologue of every tile within reach
// of a wall: when those tiles, at one node row each, would repeat the wall sums
// for more than a tenth of the step's own loads. Uniform 2D lattices with walls.
static bool wall_rho_pays(int N, int NX, int zv, int Ly)
{
    const bool zy = (zv & GLBM_ZV_Y) != 0, zx = (zv & GLBM_ZV_X) != 0;
    // largest y speed and number of (velocity, row) pairs of one wall: the 2N+1
    // speeds 1..N, or the 2N+2 odd speeds 1, 3, .., 2N+1
    const long long vmax = zy ? 2 * N + 1 : N;
    const long long npair = zy ? (long long)(N + 1) * (N + 1) : (long long)N * (N + 1) / 2;
    const long long qx = zx ? 2 * NX + 2 : 2 * NX + 1, qy = zy ? 2 * N + 2 : 2 * N + 1;
    const long long repeated = 2 * std::min<long long>(vmax, Ly) * npair * qx;
    return 10 * repeated > (long long)Ly * qx * qy;
}

static bool wall_rho_possible(const glbm_ctx *c)
{
    return c->dims == 2 && !c->hetero && c->cfg[0].bc == GLBM_BC_WALLS;
}
static bool wall_rho_launch(const glbm_ctx *c)
{
    const Geo &g = c->geo[0];
    return wall_rho_possible(c) && wall_rho_pays(g.N, g.NX, g.zv, g.Ly);
}
static glbm_status alloc_wall_rho(glbm_ctx *c)
{
    if (c->d_rw) return GLBM_OK;
    c->d_rw = dev_alloc(c->A, (size_t)c->n_inst * 2 * c->geo[0].pitch * c->elem, c->stream);
    return c->d_rw ? GLBM_OK : fail(GLBM_E_NOMEM, "device allocation of the wall densities failed");
}

static glbm_status finish_create(glbm_ctx *c, const glbm_config *cfgs, int n, void *stream)
{
    c->n_inst = n;
    c->dims = cfgs[0].dims;
    c->prec = cfgs[0].prec;
    c->elem = c->prec == GLBM_FP64 ? 8 : 4;
    c->A = DevAlloc{g_alloc, g_free, g_alloc_user};
    c->stream = (cudaStream_t)stream;
    c->cfg.assign(cfgs, cfgs + n);
    c->tabs.resize(GLBM_MAXN + 1);
    c->tabs_zv.resize(GLBM_MAXN + 1);
    for (int N = 1; N <= GLBM_MAXN; ++N) {
        glbm_build_axis_table(N, &c->tabs[N], nullptr);
        glbm_build_axis_table_zv(N, &c->tabs_zv[N]);
    }
    // pool layout: instances back to back, each starting on a 256-byte boundary
    c->geo.resize(n);
    long long off = 0;
    long long max_nodes = 1;
    const long long align = 256 / (long long)c->elem;
    for (int i = 0; i < n; ++i) {
        Geo g = make_geo(cfgs[i]);
        if ((long long)g.Q * g.plane >= (1LL << 31))
            return fail(GLBM_E_UNSUPPORTED, "instance %d holds %lld populations; at most 2^31 - 1", i,
                        (long long)g.Q * g.plane);
        g.off = off;
        off += ((g.Q * g.plane + align - 1) / align) * align;
        max_nodes = std::max(max_nodes, g.nodes());
        c->geo[i] = g;
    }
    c->pool_elems = off;
    c->h_ip.resize(n);
    c->tau.resize(n);
    for (int i = 0; i < n; ++i) {
        c->tau[i] = tau_of(cfgs[i]);
        fill_inst(c, cfgs[i], c->geo[i], c->h_ip[i], c->tau[i]);
    }

    cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(GLBM_E_CUDA, "stream creation failed: %s", cudaGetErrorString(e));
    if (cudaHostAlloc((void **)&c->h_status, ST_WORDS * sizeof(unsigned), cudaHostAllocDefault) !=
        cudaSuccess)
        return fail(GLBM_E_NOMEM, "pinned status allocation failed");
    memset(c->h_status, 0, ST_WORDS * sizeof(unsigned));
    const int blocks = glbm_field_sum_blocks(max_nodes);
    c->buf[0] = dev_alloc(c->A, bytes_state(c), c->stream);
    c->buf[1] = dev_alloc(c->A, bytes_state(c), c->stream);
    c->d_ip = (InstParams *)dev_alloc(c->A, sizeof(InstParams) * n, c->stream);
    c->d_status = (unsigned *)dev_alloc(c->A, ST_WORDS * sizeof(unsigned), c->stream);
    c->d_mom = (double *)dev_alloc(c->A, (c->dims == 3 ? 9 : 7) * (size_t)max_nodes * sizeof(double),
                                   c->stream);
    c->d_part = (double *)dev_alloc(c->A, 3 * (size_t)blocks * sizeof(double), c->stream);
    c->d_sums = (double *)dev_alloc(c->A, 3 * sizeof(double), c->stream);
    if (wall_rho_launch(c)) {
        glbm_status ws = alloc_wall_rho(c);
        if (ws != GLBM_OK) return ws;
        c->wall_launch = true;
    }
    if (!c->buf[0] || !c->buf[1] || !c->d_ip || !c->d_status || !c->d_mom || !c->d_part || !c->d_sums)
        return fail(GLBM_E_NOMEM, "device allocation of %.1f MB failed", 2.0 * bytes_state(c) / 1e6);
    CUDA_TRY(cudaMemcpyAsync(c->d_ip, c->h_ip.data(), sizeof(InstParams) * n, cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_status, 0, ST_WORDS * sizeof(unsigned), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->buf[0], 0, bytes_state(c), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->buf[1], 0, bytes_state(c), c->stream));
    // rest state X = W everywhere
    glbm_status st = ensure_stage(c, 4 * (size_t)max_nodes);
    if (st != GLBM_OK) return st;
    std::vector<double> one(max_nodes, 1.0), zero(max_nodes, 0.0);
    CUDA_TRY(cudaMemcpy(c->d_stage, one.data(), max_nodes * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_stage + max_nodes, zero.data(), max_nodes * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_stage + 2 * max_nodes, zero.data(), max_nodes * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_stage + 3 * max_nodes, zero.data(), max_nodes * 8, cudaMemcpyHostToDevice));
    for (int i = 0; i < n; ++i) {
        if (c->dims == 3)
            CUDA_TRY(glbm_launch_set_equilibrium3d(aux_args(c, i), inst_ptr(c, 0, i), 0, c->d_stage,
                                                   c->d_stage + max_nodes, c->d_stage + 2 * max_nodes,
                                                   c->d_stage + 3 * max_nodes, c->stream));
        else
            CUDA_TRY(glbm_launch_set_equilibrium(aux_args(c, i), inst_ptr(c, 0, i), 0, c->d_stage,
                                                 c->d_stage + max_nodes, c->d_stage + 2 * max_nodes,
                                                 c->stream));
        c->launches += 1;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

extern "C" glbm_status glbm_create(const glbm_config *cfgs, int n, void *stream, glbm_ctx **out)
{
    if (!cfgs || n < 1 || !out) return fail(GLBM_E_INVAL, "null argument or n < 1");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        glbm_status st = validate(cfgs[i]);
        if (st != GLBM_OK) return st;
        const glbm_config &a = cfgs[0], &b = cfgs[i];
        if (a.dims != b.dims || a.nx != b.nx || (a.dims >= 2 && a.ny != b.ny) ||
            (a.dims == 3 && a.nz != b.nz) || a.k != b.k ||
            a.bc != b.bc || a.prec != b.prec || make_geo(a).NX != make_geo(b).NX ||
            make_geo(a).zv != make_geo(b).zv)
            return fail(GLBM_E_UNSUPPORTED,
                        "instances differ in geometry; use glbm_batch_create for mixed batches");
        if (a.force != b.force) return fail(GLBM_E_UNSUPPORTED, "instances differ in the force form");
    }
    if (cfgs[0].dims == 3 && (long long)n * cfgs[0].nz > 65535)
        return fail(GLBM_E_UNSUPPORTED, "3D contexts take instances * nz <= 65535");
    glbm_ctx *c = new (std::nothrow) glbm_ctx();
    if (!c) return fail(GLBM_E_NOMEM, "host allocation failed");
    glbm_status st = finish_create(c, cfgs, n, stream);
    if (st != GLBM_OK) {
        destroy_resources(c);
        delete c;
        return st;
    }
    *out = c;
    return GLBM_OK;
}

// Whether the context steps an anisotropic product (D1Q3 along x).
static bool is_x1(const glbm_ctx *c) { return c->dims == 2 && c->geo[0].NX != c->geo[0].N; }
// Whether it steps a lattice with an axis on the 2N+2 hierarchy, and which kind.
static bool is_zv(const glbm_ctx *c) { return c->dims == 2 && c->geo[0].zv != 0; }
static int zv_kind(const glbm_ctx *c)
{
    return c->geo[0].zv == GLBM_ZV_Y ? GLBM_ZVK_X1 : GLBM_ZVK_XY;
}

// Whether the context steps with Guo's force, and its lattice kind.
static bool is_guo(const glbm_ctx *c) { return !c->hetero && c->cfg[0].force == GLBM_FORCE_GUO; }
static int guo_kind(const glbm_ctx *c)
{
    return is_zv(c) ? GLBM_GUOK_ZV : is_x1(c) ? GLBM_GUOK_X1 : GLBM_GUOK_ISO;
}

// Candidate tile shapes of level N for this context's lattices.
static int ctx_tile_shapes(const glbm_ctx *c, int N, TileShape *out)
{
    if (is_guo(c)) return glbm_tile_shape_guo(N, guo_kind(c), c->prec, out);
    if (c->dims == 3) return glbm_tile_shapes_3d(N, c->prec, out);
    if (is_zv(c)) return glbm_tile_shapes_zv(N, zv_kind(c), c->prec, out);
    return is_x1(c) ? glbm_tile_shapes_x1(N, c->prec, out) : glbm_tile_shapes(N, c->prec, out);
}

static TileShape tile_of(const glbm_ctx *c, int N)
{
    TileShape sh[GLBM_MAX_TILES];
    const int n = ctx_tile_shapes(c, N, sh);
    return n > 0 ? sh[c->tile[N] < n ? c->tile[N] : 0] : TileShape{1, 1, 1};
}

// Work list of a heterogeneous batch: every (instance, tile) with the rows of
// its level's tile shape, grouped by level (instance order within a level).
static glbm_status build_items(glbm_ctx *c)
{
    std::vector<int4> items;
    for (int i = 0; i < c->n_inst; ++i) {
        const Geo &g = c->geo[i];
        const TileShape t = tile_of(c, g.N);
        for (int y0 = 0; y0 < g.Ly; y0 += t.R)
            for (int x0 = 0; x0 < g.Lx; x0 += 32 * t.V) items.push_back(make_int4(i, x0, y0, g.N));
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const int4 &a, const int4 &b) { return a.w < b.w; });
    for (int N = 0; N <= GLBM_MAXN + 1; ++N) {  // first item of level >= N
        int k = 0;
        while (k < (int)items.size() && items[k].w < N) ++k;
        c->group[N] = k;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));  // no launch still reads the old list
    dev_free(c->A, c->d_items, c->stream);
    c->n_items = (int)items.size();
    c->d_items = (int4 *)dev_alloc(c->A, sizeof(int4) * items.size(), c->stream);
    if (!c->d_items) return fail(GLBM_E_NOMEM, "work list allocation failed");
    CUDA_TRY(cudaMemcpyAsync(c->d_items, items.data(), sizeof(int4) * items.size(),
                             cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

extern "C" glbm_status glbm_batch_create(const glbm_config *cfgs, int n, void *stream, glbm_ctx **out)
{
    if (!cfgs || n < 1 || !out) return fail(GLBM_E_INVAL, "null argument or n < 1");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        glbm_status st = validate(cfgs[i]);
        if (st != GLBM_OK) return st;
        if (cfgs[i].dims != 2) return fail(GLBM_E_UNSUPPORTED, "heterogeneous batches are 2D");
        if (make_geo(cfgs[i]).NX != cfgs[i].k + 1 || cfgs[i].zv_axes != 0)
            return fail(GLBM_E_UNSUPPORTED,
                        "heterogeneous batches take isotropic lattices of the 2N+1 hierarchy");
        if (cfgs[i].prec != GLBM_FP32_DEV)
            return fail(GLBM_E_UNSUPPORTED,
                        "heterogeneous batches store FP32 deviations (FP64 instances go through "
                        "glbm_create)");
        if (cfgs[i].force != GLBM_FORCE_LINEAR)
            return fail(GLBM_E_UNSUPPORTED, "heterogeneous batches take the linearised force");
    }
    glbm_ctx *c = new (std::nothrow) glbm_ctx();
    if (!c) return fail(GLBM_E_NOMEM, "host allocation failed");
    c->hetero = true;
    glbm_status st = finish_create(c, cfgs, n, stream);
    if (st == GLBM_OK) st = build_items(c);
    if (st != GLBM_OK) {
        destroy_resources(c);
        delete c;
        return st;
    }
    *out = c;
    return GLBM_OK;
}

extern "C" void glbm_destroy(glbm_ctx *c)
{
    if (!c) return;
    destroy_resources(c);
    delete c;
}

extern "C" int64_t glbm_time(const glbm_ctx *c) { return c ? c->t : -1; }
extern "C" int64_t glbm_kernel_launches(const glbm_ctx *c) { return c ? c->launches : -1; }
extern "C" double glbm_tau(const glbm_ctx *c, int inst)
{
    if (!c || inst < 0 || inst >= c->n_inst) return -1.0;
    return c->tau[inst];
}

extern "C" glbm_status glbm_eq_table(int k, double *out, size_t out_len)
{
    if (k < 0 || k > GLBM_MAXN - 1 || !out) return fail(GLBM_E_INVAL, "bad k or null output");
    const int N = k + 1, Q1 = 2 * N + 1;
    if (out_len < (size_t)Q1 * Q1) return fail(GLBM_E_INVAL, "output needs %d doubles", Q1 * Q1);
    AxisTableHi t;
    glbm_build_axis_table(N, &t, out);
    return GLBM_OK;
}

// ---------------------------------------------------------------------------
// state import / export
// ---------------------------------------------------------------------------
static glbm_status check_inst(const glbm_ctx *c, int inst)
{
    if (!c) return fail(GLBM_E_INVAL, "null context");
    if (inst < 0 || inst >= c->n_inst) return fail(GLBM_E_INVAL, "instance %d out of range", inst);
    return GLBM_OK;
}

// Equilibrium of fields rho, ux, uy (2D, 3D) and uz (3D; NULL = 0).
static glbm_status set_equilibrium_impl(glbm_ctx *c, int inst, const double *rho, const double *ux,
                                        const double *uy, const double *uz, int on_device)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    if (!rho || !ux || (c->dims >= 2 && !uy)) return fail(GLBM_E_INVAL, "null field");
    const size_t nodes = (size_t)c->geo[inst].nodes();
    const double *dr = rho, *du = ux, *dv = uy, *dw = uz;
    if (!on_device || (c->dims == 3 && !uz)) {
        st = ensure_stage(c, 4 * nodes);
        if (st != GLBM_OK) return st;
    }
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(c->d_stage, rho, nodes * 8, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->d_stage + nodes, ux, nodes * 8, cudaMemcpyHostToDevice, c->stream));
        if (c->dims >= 2)
            CUDA_TRY(cudaMemcpyAsync(c->d_stage + 2 * nodes, uy, nodes * 8, cudaMemcpyHostToDevice, c->stream));
        if (c->dims == 3 && uz)
            CUDA_TRY(cudaMemcpyAsync(c->d_stage + 3 * nodes, uz, nodes * 8, cudaMemcpyHostToDevice, c->stream));
        dr = c->d_stage;
        du = c->d_stage + nodes;
        dv = c->dims >= 2 ? c->d_stage + 2 * nodes : c->d_stage;
        if (uz) dw = c->d_stage + 3 * nodes;
    }
    if (!dv) dv = du;
    if (c->dims == 3) {
        if (!dw) {  // u_z = 0
            CUDA_TRY(cudaMemsetAsync(c->d_stage + 3 * nodes, 0, nodes * 8, c->stream));
            dw = c->d_stage + 3 * nodes;
        }
        CUDA_TRY(glbm_launch_set_equilibrium3d(aux_args(c, inst), inst_ptr(c, c->cur, inst), 0, dr, du,
                                               dv, dw, c->stream));
    } else {
        CUDA_TRY(glbm_launch_set_equilibrium(aux_args(c, inst), inst_ptr(c, c->cur, inst), 0, dr, du,
                                             dv, c->stream));
    }
    c->launches += 1;
    CUDA_TRY(set_clock(c, 0));
    CUDA_TRY(clear_unstable(c));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));  // host buffers reusable on return
    return GLBM_OK;
}

extern "C" glbm_status glbm_set_equilibrium(glbm_ctx *c, int inst, const double *rho,
                                            const double *ux, const double *uy, int on_device)
{
    return set_equilibrium_impl(c, inst, rho, ux, uy, nullptr, on_device);
}

extern "C" glbm_status glbm_set_equilibrium_3d(glbm_ctx *c, int inst, const double *rho,
                                               const double *ux, const double *uy, const double *uz,
                                               int on_device)
{
    if (c && c->dims != 3) return fail(GLBM_E_INVAL, "glbm_set_equilibrium_3d takes 3D contexts");
    return set_equilibrium_impl(c, inst, rho, ux, uy, uz, on_device);
}

extern "C" glbm_status glbm_set_populations(glbm_ctx *c, int inst, const double *f, int on_device)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    if (!f) return fail(GLBM_E_INVAL, "null populations");
    const size_t n = (size_t)c->geo[inst].Q * c->geo[inst].nodes();
    const double *src = f;
    if (!on_device) {
        st = ensure_stage(c, n);
        if (st != GLBM_OK) return st;
        CUDA_TRY(cudaMemcpyAsync(c->d_stage, f, n * 8, cudaMemcpyHostToDevice, c->stream));
        src = c->d_stage;
    }
    CUDA_TRY(glbm_launch_set_populations(aux_args(c, inst), inst_ptr(c, c->cur, inst), 0, src,
                                         c->stream));
    c->launches += 1;
    CUDA_TRY(set_clock(c, 0));
    CUDA_TRY(clear_unstable(c));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

extern "C" glbm_status glbm_get_populations(glbm_ctx *c, int inst, double *f, int on_device)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    if (!f) return fail(GLBM_E_INVAL, "null output");
    const size_t n = (size_t)c->geo[inst].Q * c->geo[inst].nodes();
    double *dst = f;
    if (!on_device) {
        st = ensure_stage(c, n);
        if (st != GLBM_OK) return st;
        dst = c->d_stage;
    }
    CUDA_TRY(glbm_launch_get_populations(aux_args(c, inst), inst_ptr(c, c->cur, inst), 0, dst,
                                         c->stream));
    c->launches += 1;
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(f, dst, n * 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return GLBM_OK;
}

// Copy x-columns [x0, x0 + ncols) of every (velocity, z, y) row of instance
// inst as stored, between the current buffer and a packed [q][z][y][ncols]
// buffer (one strided 2D copy).
static glbm_status copy_columns(glbm_ctx *c, int inst, int x0, int ncols, void *buf, int on_device,
                                bool pack)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    const Geo &g = c->geo[inst];
    if (!buf) return fail(GLBM_E_INVAL, "null buffer");
    if (ncols < 1 || x0 < 0 || x0 + ncols > g.Lx)
        return fail(GLBM_E_INVAL, "columns [%d, %d) outside 0..%d", x0, x0 + ncols, g.Lx);
    const size_t e = c->elem;
    char *base = (char *)inst_ptr(c, c->cur, inst) + (size_t)x0 * e;
    // the (z, y) rows of each velocity plane, planes g.plane elements apart
    // (2D planes hold a spare row after the Ly rows of data)
    const size_t rows = (size_t)g.Ly * g.Lz, width = (size_t)ncols * e, spitch = (size_t)g.pitch * e;
    const size_t plane_rows = (size_t)(g.plane / g.pitch);
    cudaMemcpy3DParms p = {};
    cudaPitchedPtr state = make_cudaPitchedPtr(base, spitch, width, plane_rows);
    cudaPitchedPtr packed = make_cudaPitchedPtr(buf, width, width, rows);
    p.srcPtr = pack ? state : packed;
    p.dstPtr = pack ? packed : state;
    p.extent = make_cudaExtent(width, rows, (size_t)g.Q);
    p.kind = on_device ? cudaMemcpyDeviceToDevice
                       : (pack ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    CUDA_TRY(cudaMemcpy3DAsync(&p, c->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

extern "C" glbm_status glbm_pack_columns(glbm_ctx *c, int inst, int x0, int ncols, void *dst,
                                         int on_device)
{
    return copy_columns(c, inst, x0, ncols, dst, on_device, true);
}

extern "C" glbm_status glbm_unpack_columns(glbm_ctx *c, int inst, int x0, int ncols,
                                           const void *src, int on_device)
{
    return copy_columns(c, inst, x0, ncols, const_cast<void *>(src), on_device, false);
}

extern "C" size_t glbm_elem_size(const glbm_ctx *c) { return c ? c->elem : 0; }

// ---------------------------------------------------------------------------
// stepping
// ---------------------------------------------------------------------------
// Arguments of the uniform step from fin into fout; TY is AxisTable for levels
// up to 8 and AxisTableHi above.
template <class TY>
static Step2DArgsT<TY> step_args_t(const glbm_ctx *c, const void *fin, void *fout)
{
    const Geo &g = c->geo[0];
    Step2DArgsT<TY> a;
    memset(&a, 0, sizeof(a));
    if constexpr (std::is_same<TY, AxisTableHi>::value)
        a.tab = tab_y(c, g);
    else
        a.tab = glbm_narrow_table(tab_y(c, g));
    a.tabx = glbm_narrow_table(tab_x(c, g));
    a.fin = fin;
    a.fout = fout;
    a.ip = c->d_ip;
    a.status = c->d_status;
    a.step_ctr = c->d_status + ST_CLOCK;
    a.done_ctr = c->d_status + ST_DONE;
    a.rw = c->wall_launch ? c->d_rw : nullptr;
    a.Lx = g.Lx;
    a.Ly = g.Ly;
    a.pitch = g.pitch;
    a.bc = c->cfg[0].bc;
    a.plane = g.plane;
    a.inst_stride = c->n_inst > 1 ? c->geo[1].off : 0;
    return a;
}
static Step2DArgs step_args(const glbm_ctx *c, int from)
{
    return step_args_t<AxisTable>(c, c->buf[from], c->buf[1 - from]);
}

static Step3DArgs step3d_args(const glbm_ctx *c, const void *fin, void *fout)
{
    const Geo &g = c->geo[0];
    Step3DArgs a;
    memset(&a, 0, sizeof(a));
    a.tab = glbm_narrow_table(c->tabs[g.N]);
    a.fin = fin;
    a.fout = fout;
    a.ip = c->d_ip;
    a.status = c->d_status;
    a.step_ctr = c->d_status + ST_CLOCK;
    a.done_ctr = c->d_status + ST_DONE;
    a.Lx = g.Lx;
    a.Ly = g.Ly;
    a.Lz = g.Lz;
    a.pitch = g.pitch;
    a.bc = c->cfg[0].bc;
    a.plane = g.plane;
    a.inst_stride = c->n_inst > 1 ? c->geo[1].off : 0;
    return a;
}

static BatchArgs batch_args(const glbm_ctx *c, const void *fin, void *fout)
{
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    for (int N = 1; N <= GLBM_MAXN_2N1; ++N) b.tab[N - 1] = glbm_narrow_table(c->tabs[N]);
    b.fin = fin;
    b.fout = fout;
    b.ip = c->d_ip;
    b.items = c->d_items;
    b.n_items = c->n_items;
    for (int N = 0; N <= GLBM_MAXN + 1; ++N) b.group[N] = c->group[N];
    for (int N = 0; N <= GLBM_MAXN; ++N) b.shape[N] = c->tile[N];
    b.status = c->d_status;
    b.step_ctr = c->d_status + ST_CLOCK;
    b.done_ctr = c->d_status + ST_DONE;
    return b;
}
static BatchArgs batch_args(const glbm_ctx *c, int from)
{
    return batch_args(c, c->buf[from], c->buf[1 - from]);
}

// Kernel launches of one 2D step.
static int launches_per_step(const glbm_ctx *c)
{
    return c->hetero ? glbm_batched_launches(batch_args(c, 0)) : (c->wall_launch ? 2 : 1);
}

// Dataflow chunks (glbm_internal.h): uniform 2D contexts of levels up to 8
// whose wall densities come from the tiles themselves (a separate wall launch
// would be a second grid per step to order).
static bool df_eligible(const glbm_ctx *c)
{
    return c->dataflow && !c->hetero && c->dims == 2 && c->geo[0].N <= GLBM_MAXN_2N1 &&
           !c->wall_launch;
}

// One 2D (or 3D) step of every instance from state buffer fin into fout, on
// stream s; node >= 0 makes it step `node` of a dataflow chunk.
static cudaError_t launch_step(const glbm_ctx *c, const void *fin, void *fout, cudaStream_t s,
                               int node = -1)
{
    if (c->hetero) return glbm_launch_batched_f32(batch_args(c, fin, fout), s);
    const int N = c->geo[0].N;
    if (c->dims == 3)
        return glbm_launch_step3d(N, c->prec, c->tile[N], step3d_args(c, fin, fout), c->n_inst, s);
    if (N > GLBM_MAXN_2N1)
        return glbm_launch_step2d_zv_hi(N, c->prec, c->tile[N],
                                        step_args_t<AxisTableHi>(c, fin, fout), c->n_inst, s);
    Step2DArgs a = step_args_t<AxisTable>(c, fin, fout);
    if (node >= 0) {
        a.node_done = c->d_df;
        a.bands = c->d_df + GLBM_DF_CHUNK;
        a.node = node;
        if (c->dataflow == 2) {
            // the timeout test: steps far beyond the chunk's, whose waits no
            // count can satisfy (the per-step counts stay indexed by `node`)
            const int far = 1 << 20;
            a.node += far;
            a.node_done -= far;
        }
    }
    if (is_guo(c)) return glbm_launch_step2d_guo(N, guo_kind(c), c->prec, a, c->n_inst, s);
    if (is_zv(c)) return glbm_launch_step2d_zv(N, zv_kind(c), c->prec, c->tile[N], a, c->n_inst, s);
    if (is_x1(c)) return glbm_launch_step2d_x1(N, c->prec, c->tile[N], a, c->n_inst, s);
    return c->prec == GLBM_FP64 ? glbm_launch_step2d_f64(N, c->tile[N], a, c->n_inst, s)
                                : glbm_launch_step2d_f32(N, c->tile[N], a, c->n_inst, s);
}

// One step from buffer `from` into the other.
static cudaError_t launch_one_2d(const glbm_ctx *c, int from, cudaStream_t s)
{
    return launch_step(c, c->buf[from], c->buf[1 - from], s);
}

// The counting words of dataflow chunks: GLBM_DF_CHUNK per-step CTA counts,
// then one band count per (instance, row) (bands of R rows use the first
// ceil(Ly / R) of an instance's Ly words).
static glbm_status df_words_ready(glbm_ctx *c)
{
    const long long n = GLBM_DF_CHUNK + (long long)c->n_inst * c->geo[0].Ly;
    if (c->d_df && c->df_words >= n) return GLBM_OK;
    dev_free(c->A, c->d_df, c->stream);
    c->d_df = (unsigned *)dev_alloc(c->A, n * sizeof(unsigned), c->stream);
    if (!c->d_df) return fail(GLBM_E_NOMEM, "dataflow counters");
    c->df_words = n;
    return GLBM_OK;
}

// Enqueue `count` steps on stream s: step 0 from p0 into pa, then pa -> pb,
// pb -> pa, ... (ChunkGraph); df: as a dataflow chunk (its counting words reset
// first, the steps numbered 0..count-1).
static cudaError_t launch_chunk(glbm_ctx *c, const void *p0, void *pa, void *pb, int count,
                                cudaStream_t s, bool df)
{
    cudaError_t e = df ? glbm_launch_df_start(c->d_status, c->d_df, c->df_words, s) : cudaSuccess;
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const void *fin = i == 0 ? p0 : ((i & 1) ? pa : pb);
        void *fout = (i & 1) ? pb : pa;
        e = launch_step(c, fin, fout, s, df ? i : -1);
    }
    return e;
}

// The graph of a full chunk (p0, pa, pb) in the given form, captured on first
// use (three state buffers give at most 12 per form).
static glbm_status chunk_graph(glbm_ctx *c, const void *p0, void *pa, void *pb, bool df,
                               cudaGraphExec_t *out)
{
    for (const ChunkGraph &g : c->graphs)
        if (g.p0 == p0 && g.pa == pa && g.pb == pb && g.df == df) {
            *out = g.exec;
            return GLBM_OK;
        }
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_chunk(c, p0, pa, pb, kGraphChunk, c->cap, df);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(GLBM_E_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(GLBM_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    c->graphs.push_back(ChunkGraph{p0, pa, pb, df, exec});
    *out = exec;
    return GLBM_OK;
}

// Enqueue n steps as chunks whose first step reads p0 and writes pa, the steps
// then alternating between pa and pb; full chunks replay graphs. Returns the
// buffer that holds the state after the n steps (pa for odd n, else pb).
static glbm_status enqueue_steps(glbm_ctx *c, int64_t n, const void *p0, void *pa, void *pb,
                                 bool df, void **last)
{
    *last = const_cast<void *>(p0);
    for (int64_t left = n; left > 0;) {
        const int m = (int)std::min<int64_t>(left, kGraphChunk);
        if (m == kGraphChunk) {
            cudaGraphExec_t g = nullptr;
            glbm_status st = chunk_graph(c, p0, pa, pb, df, &g);
            if (st != GLBM_OK) return st;
            CUDA_TRY(cudaGraphLaunch(g, c->stream));
        } else {
            CUDA_TRY(launch_chunk(c, p0, pa, pb, m, c->stream, df));
        }
        c->launches += (int64_t)m * launches_per_step(c) + (df ? 1 : 0);  // + k_df_start
        void *now = (m & 1) ? pa : pb, *other = (m & 1) ? pb : pa;
        p0 = now;  // the next chunk continues the alternation
        pa = other;
        pb = now;
        *last = now;
        left -= m;
    }
    return GLBM_OK;
}

// The status words after the work enqueued so far (waits for it).
static glbm_status read_status(glbm_ctx *c)
{
    CUDA_TRY(cudaMemcpyAsync(c->h_status, c->d_status, ST_WORDS * sizeof(unsigned),
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

// Steps of one 1D instance (all in one resident launch where the lattice fits
// one CTA's shared memory, else one launch per step); returns the steps
// completed, which stop after a step that left the positivity domain.
static glbm_status step_1d_instance(glbm_ctx *c, int i, int64_t n, int64_t *completed)
{
    const AuxArgs a = aux_args(c, i);
    CUDA_TRY(cudaMemsetAsync(c->d_status + ST_STEPS, 0, sizeof(unsigned), c->stream));
    int ok = 0;
    CUDA_TRY(glbm_launch_run1d_resident(a, inst_ptr(c, c->cur, i), 0, n, c->d_status, c->stream,
                                        &ok));
    int b = c->cur;
    if (ok) {
        c->launches += 1;
    } else {
        // too large for one CTA: one launch per step through both buffers
        for (int64_t s = 0; s < n; ++s) {
            CUDA_TRY(glbm_launch_step1d(a, inst_ptr(c, b, i), inst_ptr(c, 1 - b, i), 0, c->d_status,
                                        c->stream));
            b = 1 - b;
        }
        c->launches += n;
    }
    glbm_status st = read_status(c);
    if (st != GLBM_OK) return st;
    *completed = c->h_status[ST_STEPS];
    if (!ok && (*completed & 1)) {  // the last completed step wrote the other buffer
        const size_t bytes = (size_t)c->geo[i].Q * c->geo[i].plane * c->elem;
        CUDA_TRY(cudaMemcpyAsync(inst_ptr(c, c->cur, i), inst_ptr(c, 1 - c->cur, i), bytes,
                                 cudaMemcpyDeviceToDevice, c->stream));
    }
    return GLBM_OK;
}

// Enqueue n (< 2^31) 2D or 3D steps of every instance; returns the steps
// completed (each step's last launch counts itself, and once a step has left
// the positivity domain the launches of later steps do nothing).
static glbm_status step_nd(glbm_ctx *c, int64_t n, int64_t *completed)
{
    const int cur0 = c->cur;
    CUDA_TRY(cudaMemsetAsync(c->d_status + ST_STEPS, 0, sizeof(unsigned), c->stream));
    void *last = nullptr;
    glbm_status st = enqueue_steps(c, n, c->buf[cur0], c->buf[1 - cur0], c->buf[cur0], false, &last);
    if (st != GLBM_OK) return st;
    st = read_status(c);
    if (st != GLBM_OK) return st;
    *completed = c->h_status[ST_STEPS];
    c->cur = (int)((cur0 + *completed) & 1);  // X_{t + completed} is in this buffer
    return GLBM_OK;
}

// The third state buffer of dataflow calls (zeroed like the other two).
static glbm_status spare_ready(glbm_ctx *c)
{
    if (c->spare) return GLBM_OK;
    const size_t bytes = bytes_state(c);
    c->spare = dev_alloc(c->A, bytes, c->stream);
    if (!c->spare) return fail(GLBM_E_NOMEM, "third state buffer of %.1f MB", bytes / 1e6);
    CUDA_TRY(cudaMemsetAsync(c->spare, 0, bytes, c->stream));
    return GLBM_OK;
}

// Which buffers hold the state, the other step operand and the spare.
struct Binding {
    void *buf0, *buf1, *spare;
    int cur;
};
static Binding binding(const glbm_ctx *c) { return Binding{c->buf[0], c->buf[1], c->spare, c->cur}; }
static void rebind(glbm_ctx *c, const Binding &b)
{
    c->buf[0] = b.buf0;
    c->buf[1] = b.buf1;
    c->spare = b.spare;
    c->cur = b.cur;
}

// Enqueue n (1 <= n < 2^31) steps in dataflow chunks without writing the
// buffer S that holds X_t: the first step reads S into the second buffer X and
// the steps then alternate between X and the spare Y. On return buf[cur] holds
// the last state written, S is the spare, and the steps completed are returned:
// n, unless a node left the positivity domain or a wait ran out of time, when
// the caller binds S again (binding(), rebind()) and nothing is lost.
static glbm_status step_df(glbm_ctx *c, int64_t n, int64_t *completed)
{
    void *S = c->buf[c->cur], *X = c->buf[1 - c->cur], *Y = c->spare;
    CUDA_TRY(cudaMemsetAsync(c->d_status + ST_STEPS, 0, sizeof(unsigned), c->stream));
    void *last = nullptr;
    glbm_status st = enqueue_steps(c, n, S, X, Y, true, &last);
    if (st != GLBM_OK) return st;
    st = read_status(c);
    if (st != GLBM_OK) return st;
    *completed = c->h_status[ST_STEPS];
    c->buf[0] = last;
    c->buf[1] = last == X ? Y : X;
    c->cur = 0;
    c->spare = S;
    return GLBM_OK;
}

extern "C" glbm_status glbm_step(glbm_ctx *c, int64_t n)
{
    if (!c) return fail(GLBM_E_INVAL, "null context");
    if (n < 0) return fail(GLBM_E_INVAL, "negative step count");
    const int64_t t0 = c->t;
    int64_t done = 0;  // steps of every instance completed by this call
    bool bad = false;
    if (c->dims == 1) {
        // instances one after another; each stops at its own failing step
        done = n;
        for (int i = 0; i < c->n_inst; ++i) {
            int64_t k = 0;
            glbm_status st = step_1d_instance(c, i, n, &k);
            if (st != GLBM_OK) return st;
            if (k < n || (c->h_status[ST_FLAGS] & 1u)) bad = true;
            done = std::min(done, k);
        }
    } else {
        bool strict = true;
        if (n >= 2 && n <= ((int64_t)1 << 30) && df_eligible(c) && !c->halted) {
            // dataflow chunks: the steps of a chunk overlap, so a failing step
            // is not where the run stops. The buffer of X_{t0} is not written
            // (step_df); if a node leaves the positivity domain (or a wait runs
            // out of time) it is bound again and the call replayed one step
            // after another, which stops exactly after the failing step (same
            // arithmetic, same dither: the results are identical)
            glbm_status st = df_words_ready(c);
            if (st == GLBM_OK) st = spare_ready(c);
            if (st == GLBM_E_NOMEM) {
                // no memory for the counters or the third state buffer: this
                // context steps launch after launch from now on (same results)
                c->dataflow = 0;
                return glbm_step(c, n);
            }
            if (st != GLBM_OK) return st;
            const Binding start = binding(c);
            int64_t k = 0;
            st = step_df(c, n, &k);
            if (st != GLBM_OK) return st;
            const unsigned flags = c->h_status[ST_FLAGS] & (ST_UNSTABLE | ST_TIMEOUT);
            strict = flags != 0u;
            if (strict) {
                rebind(c, start);
                CUDA_TRY(set_clock(c, t0));
                CUDA_TRY(clear_unstable(c));
                if (flags & ST_TIMEOUT) {
                    CUDA_TRY(cudaStreamSynchronize(c->stream));
                    return fail(GLBM_E_TIMEOUT,
                                "a dataflow step waited more than 0.5 s for its rows; the state is "
                                "that of time %lld again (no step applied)", (long long)t0);
                }
            } else {
                done = k;
            }
        }
        for (int64_t left = strict ? n : 0; left > 0 && !bad;) {
            const int64_t m = std::min<int64_t>(left, (int64_t)1 << 30);
            int64_t k = 0;
            glbm_status st = step_nd(c, m, &k);
            if (st != GLBM_OK) return st;
            done += k;
            left -= m;
            bad = (c->h_status[ST_FLAGS] & 1u) != 0u;
        }
        if (n == 0) {
            glbm_status st = read_status(c);
            if (st != GLBM_OK) return st;
            bad = (c->h_status[ST_FLAGS] & 1u) != 0u;
        }
    }
    c->t = t0 + done;
    if (bad) c->halted = true;
    if (bad)
        return fail(GLBM_E_UNSTABLE,
                    "a node left the positivity domain (|u| > sqrt(2/3) N per axis, or rho <= 0); "
                    "%lld of %lld steps completed, the state is that of time %lld",
                    (long long)done, (long long)n, (long long)c->t);
    return GLBM_OK;
}

extern "C" glbm_status glbm_sync(glbm_ctx *c)
{
    if (!c) return fail(GLBM_E_INVAL, "null context");
    glbm_status st = read_status(c);
    if (st != GLBM_OK) return st;
    if (c->h_status[ST_FLAGS] & 1u) return fail(GLBM_E_UNSTABLE, "a node left the positivity domain");
    return GLBM_OK;
}

// ---------------------------------------------------------------------------
// moments and conservation
// ---------------------------------------------------------------------------
static glbm_status compute_moments(glbm_ctx *c, int inst)
{
    if (c->dims == 3)
        CUDA_TRY(glbm_launch_moments3d(aux_args(c, inst), inst_ptr(c, c->cur, inst), 0, c->d_mom, c->stream));
    else
        CUDA_TRY(glbm_launch_moments(aux_args(c, inst), inst_ptr(c, c->cur, inst), 0, c->d_mom, c->stream));
    c->launches += 1;
    return GLBM_OK;
}

extern "C" glbm_status glbm_channel_diagnostics(glbm_ctx *c, int inst, double *profile,
                                                double *stats, int on_device)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    if (c->dims < 2) return fail(GLBM_E_UNSUPPORTED, "channel diagnostics need a 2D or 3D lattice");
    const Geo &g = c->geo[inst];
    const size_t need = 2 * (size_t)g.Ly + GLBM_CH_COUNT;
    if (c->diag_len < need) {
        dev_free(c->A, c->d_diag, c->stream);
        c->d_diag = (double *)dev_alloc(c->A, need * sizeof(double), c->stream);
        c->diag_len = c->d_diag ? need : 0;
        if (!c->d_diag) return fail(GLBM_E_NOMEM, "diagnostics buffer of %zu doubles", need);
    }
    st = compute_moments(c, inst);
    if (st != GLBM_OK) return st;
    const glbm_config &cf = c->cfg[inst];
    ChannelParams p;
    p.theta_y = axis_theta(g.N, c->dims == 2 && (g.zv & GLBM_ZV_Y));
    p.tau = c->tau[inst];
    p.g = cf.g;
    p.u_lo = cf.u_wall_lo;
    p.u_hi = cf.u_wall_hi;
    p.walls = cf.bc == GLBM_BC_WALLS;
    double *d_prof = c->d_diag, *d_stats = c->d_diag + 2 * (size_t)g.Ly;
    CUDA_TRY(glbm_launch_channel_diagnostics(c->d_mom, g.Lx, g.Ly, g.Lz, p, d_prof, d_stats,
                                             c->stream));
    c->launches += 2;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (profile)
        CUDA_TRY(cudaMemcpyAsync(profile, d_prof, (size_t)g.Ly * sizeof(double), kind, c->stream));
    if (stats)
        CUDA_TRY(cudaMemcpyAsync(stats, d_stats, GLBM_CH_COUNT * sizeof(double), kind, c->stream));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

extern "C" glbm_status glbm_moments(glbm_ctx *c, int inst, unsigned mask, double *out,
                                    size_t out_len, int out_on_device)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    if (!out) return fail(GLBM_E_INVAL, "null output");
    // field slot of each mask bit in the reducer's output
    const int slot2d[9] = {0, 1, 2, 3, 4, 5, 6, -1, -1};
    const int slot1d[9] = {0, 1, -1, 2, 3, -1, -1, -1, -1};
    const int slot3d[9] = {0, 1, 2, 3, 4, 5, 6, 7, 8};
    const int *slot = c->dims == 3 ? slot3d : (c->dims == 2 ? slot2d : slot1d);
    const size_t nodes = (size_t)c->geo[inst].nodes();
    size_t need = 0;
    if (mask >> 9) return fail(GLBM_E_INVAL, "unknown field bits in mask 0x%x", mask);
    for (int b = 0; b < 9; ++b) {
        if (!(mask & (1u << b))) continue;
        if (slot[b] < 0) return fail(GLBM_E_INVAL, "field bit %d has no %dD meaning", b, c->dims);
        need += nodes;
    }
    if (need == 0) return fail(GLBM_E_INVAL, "empty field mask");
    if (out_len < need) return fail(GLBM_E_INVAL, "output holds %zu doubles, needs %zu", out_len, need);
    st = compute_moments(c, inst);
    if (st != GLBM_OK) return st;
    size_t o = 0;
    for (int b = 0; b < 9; ++b) {
        if (!(mask & (1u << b))) continue;
        CUDA_TRY(cudaMemcpyAsync(out + o, c->d_mom + (size_t)slot[b] * nodes, nodes * 8,
                                 out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
        o += nodes;
    }
    if (!out_on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

extern "C" glbm_status glbm_conservation(glbm_ctx *c, int inst, double *mass, double *mom_x,
                                         double *mom_y)
{
    glbm_status st = check_inst(c, inst);
    if (st != GLBM_OK) return st;
    st = compute_moments(c, inst);
    if (st != GLBM_OK) return st;
    const long long nodes = c->geo[inst].nodes();
    CUDA_TRY(glbm_launch_field_sums(c->d_mom, c->dims >= 2 ? 3 : 2, nodes, c->d_part,
                                    glbm_field_sum_blocks(nodes), c->d_sums, c->stream));
    c->launches += 2;
    double h[3];
    CUDA_TRY(cudaMemcpyAsync(h, c->d_sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (mass) *mass = h[0];
    if (mom_x) *mom_x = h[1];
    if (mom_y) *mom_y = c->dims >= 2 ? h[2] : 0.0;
    return GLBM_OK;
}

// ---------------------------------------------------------------------------
// checkpoints: header, raw pool image of every instance, CRC-32
// ---------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int32_t version, dims, prec, n_inst, hetero, pad;
    int64_t t;
    uint64_t bytes;
    uint64_t config_crc;  // CRC-32 of every instance's geometry, level and boundary
};

static uint32_t crc32_update(uint32_t crc, const unsigned char *p, size_t n)
{
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int b = 0; b < 8; ++b) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

static void fill_header(const glbm_ctx *c, CkptHeader &h)
{
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "GLBMCKP2", 8);
    h.version = 2;
    h.dims = c->dims;
    h.prec = c->prec;
    h.n_inst = c->n_inst;
    h.hetero = c->hetero ? 1 : 0;
    h.t = c->t;
    h.bytes = bytes_state(c);
    uint32_t crc = 0;
    for (const glbm_config &g : c->cfg) {
        const int geo[6] = {g.dims, g.nx, g.ny, g.k, g.bc, g.prec};
        crc = crc32_update(crc, (const unsigned char *)geo, sizeof(geo));
        const int nx_level = make_geo(g).NX;  // anisotropic lattices add their x level
        if (nx_level != g.k + 1) crc = crc32_update(crc, (const unsigned char *)&nx_level, sizeof(int));
        const int zv = make_geo(g).zv;  // and 2N+2 lattices their axes
        if (zv != 0) crc = crc32_update(crc, (const unsigned char *)&zv, sizeof(int));
        if (g.dims == 3) crc = crc32_update(crc, (const unsigned char *)&g.nz, sizeof(int));
    }
    h.config_crc = crc;
}

extern "C" glbm_status glbm_save(glbm_ctx *c, const char *path)
{
    if (!c || !path) return fail(GLBM_E_INVAL, "null argument");
    std::vector<unsigned char> img(bytes_state(c));
    CUDA_TRY(cudaMemcpyAsync(img.data(), c->buf[c->cur], img.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CkptHeader h;
    fill_header(c, h);
    uint32_t crc = crc32_update(0, (const unsigned char *)&h, sizeof(h));
    crc = crc32_update(crc, img.data(), img.size());
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(GLBM_E_IO, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1 && fwrite(img.data(), 1, img.size(), fp) == img.size() &&
              fwrite(&crc, sizeof(crc), 1, fp) == 1;
    ok = (fclose(fp) == 0) && ok;
    return ok ? GLBM_OK : fail(GLBM_E_IO, "write to %s failed", path);
}

extern "C" glbm_status glbm_load(glbm_ctx *c, const char *path)
{
    if (!c || !path) return fail(GLBM_E_INVAL, "null argument");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(GLBM_E_IO, "cannot open %s", path);
    CkptHeader h, want;
    fill_header(c, want);
    std::vector<unsigned char> img;
    uint32_t crc_file = 0;
    bool ok = fread(&h, sizeof(h), 1, fp) == 1;
    if (ok) {
        want.t = h.t;
        if (memcmp(&h, &want, sizeof(h)) != 0) {
            fclose(fp);
            return fail(GLBM_E_INVAL, "checkpoint %s does not match this context's configuration", path);
        }
        img.resize(h.bytes);
        ok = fread(img.data(), 1, img.size(), fp) == img.size() &&
             fread(&crc_file, sizeof(crc_file), 1, fp) == 1;
    }
    fclose(fp);
    if (!ok) return fail(GLBM_E_IO, "checkpoint %s is truncated", path);
    uint32_t crc = crc32_update(0, (const unsigned char *)&h, sizeof(h));
    crc = crc32_update(crc, img.data(), img.size());
    if (crc != crc_file) return fail(GLBM_E_IO, "checkpoint %s fails its CRC-32 check", path);
    CUDA_TRY(cudaMemcpyAsync(c->buf[c->cur], img.data(), img.size(), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(set_clock(c, h.t));
    CUDA_TRY(clear_unstable(c));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

// ---------------------------------------------------------------------------
// adjoint gradient of the flow rate
// ---------------------------------------------------------------------------
// One uniform 2D step from an arbitrary pool image `fin` into `fout`.
static cudaError_t launch_2d_between(const glbm_ctx *c, const void *fin, void *fout, cudaStream_t s)
{
    const int N = c->geo[0].N;
    if (N > GLBM_MAXN_2N1) return cudaErrorInvalidValue;  // the adjoint takes levels <= 8
    Step2DArgs a = step_args(c, 0);
    a.fin = fin;
    a.fout = fout;
    if (is_guo(c)) return glbm_launch_step2d_guo(N, guo_kind(c), c->prec, a, c->n_inst, s);
    if (is_zv(c)) return glbm_launch_step2d_zv(N, zv_kind(c), c->prec, c->tile[N], a, c->n_inst, s);
    if (is_x1(c)) return glbm_launch_step2d_x1(N, c->prec, c->tile[N], a, c->n_inst, s);
    return c->prec == GLBM_FP64 ? glbm_launch_step2d_f64(N, c->tile[N], a, c->n_inst, s)
                                : glbm_launch_step2d_f32(N, c->tile[N], a, c->n_inst, s);
}

struct Scratch {
    const DevAlloc &A;
    cudaStream_t s;
    std::vector<void *> ptrs;
    Scratch(const DevAlloc &a, cudaStream_t st) : A(a), s(st) {}
    void *get(size_t bytes)
    {
        void *p = dev_alloc(A, bytes, s);
        if (p) ptrs.push_back(p);
        return p;
    }
    ~Scratch()
    {
        cudaStreamSynchronize(s);
        for (void *p : ptrs) dev_free(A, p, s);
    }
};

extern "C" glbm_status glbm_adjoint_flowrate(glbm_ctx *c, int64_t steps, int64_t ckpt_every,
                                             double *J, double *dJ_dtau, double *dJ_dg,
                                             double *dJ_du_lo, double *dJ_du_hi)
{
    if (!c || !J || !dJ_dtau || !dJ_dg) return fail(GLBM_E_INVAL, "null argument");
    if (c->dims != 2 || c->hetero)
        return fail(GLBM_E_UNSUPPORTED, "the adjoint takes 2D uniform contexts");
    if (is_x1(c) || is_zv(c))
        return fail(GLBM_E_UNSUPPORTED, "the adjoint takes isotropic lattices of the 2N+1 hierarchy");
    if (is_guo(c)) return fail(GLBM_E_UNSUPPORTED, "the adjoint takes the linearised force");
    if (steps < 1 || ckpt_every < 1) return fail(GLBM_E_INVAL, "steps and ckpt_every must be >= 1");
    const int64_t K = ckpt_every < steps ? ckpt_every : steps;
    const int64_t nseg = (steps + K - 1) / K;
    const size_t pool = bytes_state(c);
    const Geo &g = c->geo[0];
    const size_t mu_bytes = (size_t)g.Q * g.plane * sizeof(double);
    const long long nblk = glbm_adj_blocks(g.Lx, g.Ly);
    Scratch S(c->A, c->stream);
    char *ck = (char *)S.get(pool * nseg);
    char *seg = (char *)S.get(pool * K);
    double *mu0 = (double *)S.get(mu_bytes), *mu1 = (double *)S.get(mu_bytes);
    double *G = (double *)S.get(2 * (size_t)g.Lx * sizeof(double));
    double *gpart = (double *)S.get(GLBM_ADJ_NG * (size_t)nblk * sizeof(double));
    double *gsum = (double *)S.get(GLBM_ADJ_NG * sizeof(double));
    if (!ck || !seg || !mu0 || !mu1 || !G || !gpart || !gsum)
        return fail(GLBM_E_NOMEM, "adjoint scratch of %.1f MB failed",
                    (pool * (nseg + K) + 2.0 * mu_bytes) / 1e6);
    const int64_t t_start = c->t;

    // forward with checkpoints
    for (int64_t s = 0; s < nseg; ++s) {
        CUDA_TRY(cudaMemcpyAsync(ck + pool * s, c->buf[c->cur], pool, cudaMemcpyDeviceToDevice, c->stream));
        const int64_t len = std::min<int64_t>(K, steps - s * K);
        glbm_status st = glbm_step(c, len);
        if (st != GLBM_OK) return st;
    }
    for (int i = 0; i < c->n_inst; ++i) {
        double mass, jx, jy;
        glbm_status st = glbm_conservation(c, i, &mass, &jx, &jy);
        if (st != GLBM_OK) return st;
        J[i] = jx / c->geo[i].Lx;
    }
    const int64_t t_end = c->t;

    // backward, one instance at a time
    for (int i = 0; i < c->n_inst; ++i) {
        AdjArgs a;
        memset(&a, 0, sizeof(a));
        a.tab = glbm_narrow_table(c->tabs[g.N]);
        a.ip = c->d_ip + i;
        a.G = G;
        a.Gw = G;
        a.gpart = gpart;
        a.Lx = g.Lx;
        a.Ly = g.Ly;
        a.pitch = g.pitch;
        a.bc = c->cfg[i].bc;
        a.N = g.N;
        a.prec = c->prec;
        a.plane = g.plane;
        double *mu_cur = mu0, *mu_nxt = mu1;
        a.mu_out = mu_cur;
        CUDA_TRY(glbm_launch_adj_seed(a, c->stream));
        CUDA_TRY(cudaMemsetAsync(gpart, 0, GLBM_ADJ_NG * (size_t)nblk * sizeof(double), c->stream));
        // the wall speeds' term of F_T, from X_T (the state after the forward run)
        a.X = (const char *)c->buf[c->cur] + (size_t)c->geo[i].off * c->elem;
        CUDA_TRY(glbm_launch_adj_final_walls(a, c->stream));
        for (int64_t s = nseg - 1; s >= 0; --s) {
            const int64_t t0 = s * K, len = std::min<int64_t>(K, steps - t0);
            // recompute X_t0 .. X_t0+len-1 with the dither counter of the forward pass
            CUDA_TRY(cudaMemcpyAsync(seg, ck + pool * s, pool, cudaMemcpyDeviceToDevice, c->stream));
            CUDA_TRY(set_clock(c, t_start + t0));
            for (int64_t r = 0; r + 1 < len; ++r) {
                CUDA_TRY(launch_2d_between(c, seg + pool * r, seg + pool * (r + 1), c->stream));
                c->launches += launches_per_step(c);
            }
            for (int64_t r = len - 1; r >= 0; --r) {
                a.X = seg + pool * r + (size_t)c->geo[i].off * c->elem;
                a.mu_in = mu_cur;
                a.mu_out = mu_nxt;
                CUDA_TRY(glbm_launch_adj_step(a, c->stream));
                c->launches += 2;
                std::swap(mu_cur, mu_nxt);
            }
        }
        CUDA_TRY(glbm_launch_adj_sum(gpart, nblk, gsum, c->stream));
        double h[GLBM_ADJ_NG];
        CUDA_TRY(cudaMemcpyAsync(h, gsum, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        dJ_dtau[i] = h[0];
        dJ_dg[i] = h[1];
        if (dJ_du_lo) dJ_du_lo[i] = h[2];
        if (dJ_du_hi) dJ_du_hi[i] = h[3];
    }
    CUDA_TRY(set_clock(c, t_end));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}

// ---------------------------------------------------------------------------
// tile shapes and the autotuner

extern "C" int glbm_tile_count(int k, glbm_prec prec)
{
    TileShape sh[GLBM_MAX_TILES];
    if (k < 0 || k >= GLBM_LEVELS || (prec != GLBM_FP64 && prec != GLBM_FP32_DEV)) return 0;
    return glbm_tile_shapes(k + 1, prec, sh);
}

extern "C" glbm_status glbm_tile_shape(int k, glbm_prec prec, int idx, int *G, int *R, int *V)
{
    TileShape sh[GLBM_MAX_TILES];
    const int n = glbm_tile_count(k, prec);
    if (!G || !R || !V) return fail(GLBM_E_INVAL, "null argument");
    if (idx < 0 || idx >= n) return fail(GLBM_E_INVAL, "no tile shape %d for k=%d", idx, k);
    glbm_tile_shapes(k + 1, prec, sh);
    *G = sh[idx].G;
    *R = sh[idx].R;
    *V = sh[idx].V;
    return GLBM_OK;
}

extern "C" glbm_status glbm_get_tiles(const glbm_ctx *c, int *tiles)
{
    if (!c || !tiles) return fail(GLBM_E_INVAL, "null argument");
    for (int k = 0; k < GLBM_LEVELS; ++k) tiles[k] = c->tile[k + 1];
    return GLBM_OK;
}

extern "C" glbm_status glbm_get_tile_shape(const glbm_ctx *c, int k, int *G, int *R, int *V)
{
    if (!c || !G || !R || !V) return fail(GLBM_E_INVAL, "null argument");
    if (k < 0 || k >= GLBM_LEVELS) return fail(GLBM_E_INVAL, "no level k=%d", k);
    const TileShape t = tile_of(c, k + 1);
    *G = t.G;
    *R = t.R;
    *V = t.V;
    return GLBM_OK;
}

// Graphs and (in batches) the work list follow the tile shapes.
static glbm_status tiles_changed(glbm_ctx *c)
{
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    return c->hetero ? build_items(c) : GLBM_OK;
}

extern "C" glbm_status glbm_set_dataflow(glbm_ctx *c, int on)
{
    if (!c) return fail(GLBM_E_INVAL, "null context");
    if (on < 0 || on > 2) return fail(GLBM_E_INVAL, "dataflow mode %d (0, 1 or 2)", on);
    const bool changed = on != c->dataflow;
    c->dataflow = on;
    return changed ? tiles_changed(c) : GLBM_OK;  // the chunk graphs carry the mode
}

extern "C" int glbm_get_dataflow(const glbm_ctx *c)
{
    return c && df_eligible(c) ? 1 : 0;
}

extern "C" glbm_status glbm_set_wall_launch(glbm_ctx *c, int mode)
{
    if (!c) return fail(GLBM_E_INVAL, "null context");
    if (mode < -1 || mode > 1) return fail(GLBM_E_INVAL, "wall launch mode %d (-1, 0 or 1)", mode);
    if (!wall_rho_possible(c))
        return fail(GLBM_E_UNSUPPORTED, "wall densities apply to uniform 2D contexts with walls");
    const bool on = mode < 0 ? wall_rho_launch(c) : mode == 1;
    if (on) {
        glbm_status st = alloc_wall_rho(c);
        if (st != GLBM_OK) return st;
    }
    c->wall_launch = on;
    return tiles_changed(c);  // the captured step graphs name the old launches
}

extern "C" int glbm_get_wall_launch(const glbm_ctx *c)
{
    if (!c || !wall_rho_possible(c)) return -1;
    return c->wall_launch ? 1 : 0;
}

extern "C" glbm_status glbm_set_tiles(glbm_ctx *c, const int *tiles)
{
    if (!c || !tiles) return fail(GLBM_E_INVAL, "null argument");
    TileShape sh[GLBM_MAX_TILES];
    // a level without candidates in this context keeps index 0 (accepted as given)
    for (int k = 0; k < GLBM_LEVELS; ++k) {
        const int n = ctx_tile_shapes(c, k + 1, sh);
        if (tiles[k] < -1 || tiles[k] >= (n > 0 ? n : 1))
            return fail(GLBM_E_INVAL, "tile index %d out of range for k=%d", tiles[k], k);
    }
    for (int k = 0; k < GLBM_LEVELS; ++k)
        if (tiles[k] >= 0) c->tile[k + 1] = tiles[k];
    return tiles_changed(c);
}

// Whether the context steps instances of level N.
static bool level_present(const glbm_ctx *c, int N)
{
    if (c->hetero) return c->group[N + 1] > c->group[N];
    return c->geo[0].N == N;
}

// One launch of level N's instances from the current buffer into the spare one.
static cudaError_t launch_level_once(const glbm_ctx *c, int N)
{
    if (c->hetero) return glbm_launch_batched_level(N, batch_args(c, c->cur), false, c->stream);
    return launch_one_2d(c, c->cur, c->stream);
}

// Time `steps` steps of the context from its current state, launch after
// launch or in dataflow chunks, through the three state buffers so that the
// current state's buffer is not written; the binding, the clock and the status
// are put back after each of the two runs (the first captures the graphs).
static glbm_status time_steps(glbm_ctx *c, int64_t steps, bool df, cudaEvent_t e0, cudaEvent_t e1,
                              float *ms)
{
    const Binding start = binding(c);
    const int64_t t0 = c->t;
    for (int rep = 0; rep < 2; ++rep) {
        CUDA_TRY(cudaEventRecord(e0, c->stream));
        void *last = nullptr;
        glbm_status st = enqueue_steps(c, steps, c->buf[c->cur], c->buf[1 - c->cur], c->spare, df,
                                       &last);
        if (st != GLBM_OK) return st;
        CUDA_TRY(cudaEventRecord(e1, c->stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        rebind(c, start);
        CUDA_TRY(set_clock(c, t0));
        CUDA_TRY(clear_unstable(c));
    }
    return GLBM_OK;
}

// The last stage of glbm_autotune for contexts whose steps can take dataflow
// chunks: 128 steps with the choice made so far (launch after launch), then
// 128 steps in dataflow chunks with every tile shape of the level (wall
// densities from the tiles); the fastest of all is kept, dataflow on or off.
static glbm_status autotune_dataflow(glbm_ctx *c, cudaEvent_t e0, cudaEvent_t e1)
{
    const int N = c->geo[0].N;
    glbm_status st = df_words_ready(c);
    if (st == GLBM_OK) st = spare_ready(c);
    if (st == GLBM_E_NOMEM) {  // no room for dataflow chunks: keep stepping launch after launch
        c->dataflow = 0;
        return tiles_changed(c);
    }
    if (st != GLBM_OK) return st;
    const int64_t steps = 2 * kGraphChunk;
    const int tile0 = c->tile[N];
    const bool wall0 = c->wall_launch;
    float best = 0.f;
    st = tiles_changed(c);
    if (st == GLBM_OK) st = time_steps(c, steps, false, e0, e1, &best);
    int best_tile = tile0;
    bool best_wall = wall0, best_df = false;
    TileShape sh[GLBM_MAX_TILES];
    const int n = ctx_tile_shapes(c, N, sh);
    for (int idx = 0; idx < n && st == GLBM_OK; ++idx) {
        c->tile[N] = idx;
        c->wall_launch = false;
        st = tiles_changed(c);
        float ms = 0.f;
        if (st == GLBM_OK) st = time_steps(c, steps, true, e0, e1, &ms);
        if (st == GLBM_OK && ms < best) {
            best = ms;
            best_tile = idx;
            best_wall = false;
            best_df = true;
        }
    }
    c->tile[N] = best_tile;
    c->wall_launch = best_wall;
    c->dataflow = best_df ? 1 : 0;
    return st;
}

extern "C" glbm_status glbm_autotune(glbm_ctx *c, int reps, double *us)
{
    if (!c) return fail(GLBM_E_INVAL, "null context");
    if (c->dims < 2) return fail(GLBM_E_UNSUPPORTED, "tile shapes apply to 2D and 3D lattices");
    if (reps < 1 || reps > 1000) return fail(GLBM_E_INVAL, "reps must be in 1..1000");
    if (us)
        for (int i = 0; i < GLBM_LEVELS * GLBM_MAX_TILES; ++i) us[i] = -1.0;
    // the trial launches must neither be skipped by an earlier failure nor leave
    // flags of their own: keep the status words and put them back afterwards
    unsigned saved[ST_WORDS];
    {
        glbm_status rs = read_status(c);
        if (rs != GLBM_OK) return rs;
        memcpy(saved, c->h_status, sizeof(saved));
        CUDA_TRY(clear_unstable(c));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    glbm_status st = ce == cudaSuccess ? GLBM_OK : fail(GLBM_E_CUDA, "event: %s", cudaGetErrorString(ce));
    for (int N = 1; N <= GLBM_MAXN && st == GLBM_OK; ++N) {
        if (!level_present(c, N)) continue;
        TileShape sh[GLBM_MAX_TILES];
        const int n = ctx_tile_shapes(c, N, sh);
        int best = c->tile[N];
        float best_ms = 0.f;
        for (int idx = 0; idx < n && st == GLBM_OK; ++idx) {
            c->tile[N] = idx;
            if (c->hetero && (st = build_items(c)) != GLBM_OK) break;
            cudaError_t e = launch_level_once(c, N);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_level_once(c, N);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = fail(GLBM_E_CUDA, "autotune launch: %s", cudaGetErrorString(e));
                break;
            }
            if (us) us[(N - 1) * GLBM_MAX_TILES + idx] = 1e3 * ms / reps;
            if (idx == 0 || ms < best_ms) {
                best_ms = ms;
                best = idx;
            }
        }
        c->tile[N] = best;
    }
    // then the way the wall densities are summed, with the chosen shapes: the
    // faster of the two modes (identical results)
    if (st == GLBM_OK && wall_rho_possible(c)) st = alloc_wall_rho(c);
    if (st == GLBM_OK && wall_rho_possible(c)) {
        const int N = c->geo[0].N;
        float ms_mode[2] = {0.f, 0.f};
        for (int m = 0; m < 2 && st == GLBM_OK; ++m) {
            c->wall_launch = m == 1;
            cudaError_t e = launch_level_once(c, N);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_level_once(c, N);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_mode[m], e0, e1);
            if (e != cudaSuccess) st = fail(GLBM_E_CUDA, "autotune launch: %s", cudaGetErrorString(e));
        }
        c->wall_launch = ms_mode[1] < ms_mode[0];
    }
    // and last, for contexts that can step in dataflow chunks, whole chunks of
    // steps both ways (a launch timed alone cannot show the overlap)
    if (st == GLBM_OK && !c->hetero && c->dims == 2 && c->geo[0].N <= GLBM_MAXN_2N1) {
        c->dataflow = 1;
        st = autotune_dataflow(c, e0, e1);
    }
    if (e1) cudaEventDestroy(e1);
    cudaEventDestroy(e0);
    if (st != GLBM_OK) return st;
    st = tiles_changed(c);
    if (st != GLBM_OK) return st;
    // the trial launches advanced the dither counter and may have set flags:
    // restore the status words, then the clock
    CUDA_TRY(cudaMemcpyAsync(c->d_status, saved, sizeof(saved), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(set_clock(c, c->t));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return GLBM_OK;
}
