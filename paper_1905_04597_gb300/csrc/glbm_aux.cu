// Auxiliary kernels of libglbm: initial equilibrium, import/export of
// populations in the FP64 logical layout, the moment reducer (moments of the
// streamed state, Sec. 2 for rho and u; temperature, heat flux and shear
// stress as central moments), deterministic global sums, and the 1D step
// (Sec. 5.1 shock tube, halfway bounce-back) both per launch and resident in
// one CTA for many steps.
#include <algorithm>
#include <mutex>

#include "glbm_device.cuh"

namespace {

// E_i(u) - W_i of velocity index i at runtime level t.N (FP64 Horner on the
// coefficient table; on the 2N+2 hierarchy the velocity is +-(2m+1)).
__device__ double eq_dev_rt(const AxisTableHi &t, double u, int i)
{
    const int N = t.N;
    const int n = ax_vel(t, i);
    const int an = n < 0 ? -n : n;
    const int m = t.zv ? (an - 1) / 2 : an;
    const double v = u * u;
    double ae = t.Ce[m][N];
    for (int k = N - 1; k >= 1; --k) ae = fma(ae, v, t.Ce[m][k]);
    ae *= v;
    double bo = 0.0;
    if (an > 0) {
        bo = t.Co[m][N - 1];
        for (int k = N - 2; k >= 0; --k) bo = fma(bo, v, t.Co[m][k]);
    }
    return n >= 0 ? fma(u, bo, ae) : fma(-u, bo, ae);
}

// E_i(u) - W_i of every velocity index of a runtime level, the mirror pairs
// (i, Q - 1 - i), whose velocities are opposite, from one evaluation of the
// even and odd parts each: the same operations as eq_dev_rt per index.
__device__ void eq_dev_all_rt(const AxisTableHi &t, double u, double *out)
{
    const int N = t.N, Q = ax_q(t);
    const double v = u * u;
    for (int p = 0; p < Q / 2; ++p) {
        const int an = ax_vel(t, Q - 1 - p);  // > 0
        const int m = t.zv ? (an - 1) / 2 : an;
        double ae = t.Ce[m][N];
        for (int k = N - 1; k >= 1; --k) ae = fma(ae, v, t.Ce[m][k]);
        ae *= v;
        double bo = t.Co[m][N - 1];
        for (int k = N - 2; k >= 0; --k) bo = fma(bo, v, t.Co[m][k]);
        out[Q - 1 - p] = fma(u, bo, ae);
        out[p] = fma(-u, bo, ae);
    }
    if (Q & 1) out[Q / 2] = eq_dev_rt(t, u, Q / 2);
}

__device__ __forceinline__ double load_full(const AuxArgs &a, const void *f, long long idx, int q)
{
    (void)q;
    if (a.prec == GLBM_FP64) return static_cast<const double *>(f)[idx];
    return (double)static_cast<const float *>(f)[idx];
}

// rest weight of flat velocity q (q = iy Qx + ix in 2D, (iz Q1 + iy) Q1 + ix in 3D)
__device__ __forceinline__ double rest_weight(const AuxArgs &a, int q)
{
    if (a.dims == 1) return a.tab.W[q];
    if (a.dims == 3) {
        const int Q1 = ax_q(a.tab);
        return a.tab.W[q / (Q1 * Q1)] * a.tab.W[(q / Q1) % Q1] * a.tab.W[q % Q1];
    }
    const int Qx = ax_q(a.tabx);
    return a.tab.W[q / Qx] * a.tabx.W[q % Qx];
}

__global__ void k_set_equilibrium(const __grid_constant__ AuxArgs a, void *f, int inst,
                                  const double *__restrict__ rho, const double *__restrict__ ux,
                                  const double *__restrict__ uy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.Lx) return;
    // 1D: the only axis is x, with table tab and level N
    const AxisTableHi &tx = a.dims == 2 ? a.tabx : a.tab;
    const int Q1x = ax_q(tx);
    const long long node = (long long)y * a.Lx + x;
    const double r = rho[node], u = ux[node], v = a.dims == 2 ? uy[node] : 0.0;
    const long long base = (long long)inst * a.inst_stride + (long long)y * a.pitch + x;
    const int Qy = a.dims == 2 ? ax_q(a.tab) : 1;
    const bool f64 = a.prec == GLBM_FP64;
    double exs[GLBM_MAXQA];  // per node: E^x (FP64 storage) or E^x - W^x (FP32 deviations)
    double dys[GLBM_MAXQA];  // E^y - W^y
    eq_dev_all_rt(tx, u, exs);
    if (f64)
        for (int ix = 0; ix < Q1x; ++ix) exs[ix] += tx.W[ix];
    if (a.dims == 2) eq_dev_all_rt(a.tab, v, dys);
    for (int iy = 0; iy < Qy; ++iy) {
        const double wy = a.dims == 2 ? a.tab.W[iy] : 1.0;
        const double dy = a.dims == 2 ? dys[iy] : 0.0;
        // per row: A = rho E^y and B = rho E^y - W^y = (rho - 1) W^y + rho d^y
        // (no cancellation); then rho E^x E^y = E^x A and, in deviations,
        // rho E^x E^y - W^x W^y = W^x B + d^x A: one or two FP64 operations
        // per population
        const double A = r * (wy + dy);
        const double B = fma(r - 1.0, wy, r * dy);
        const long long row = base + (long long)(iy * Q1x) * a.plane;
        if (f64) {
            double *out = static_cast<double *>(f) + row;
            for (int ix = 0; ix < Q1x; ++ix) out[(long long)ix * a.plane] = exs[ix] * A;
        } else {
            float *out = static_cast<float *>(f) + row;
            for (int ix = 0; ix < Q1x; ++ix)
                out[(long long)ix * a.plane] = (float)fma(exs[ix], A, tx.W[ix] * B);
        }
    }
}

__global__ void k_set_populations(const __grid_constant__ AuxArgs a, void *f, int inst,
                                  const double *__restrict__ src)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int q = blockIdx.z;
    if (x >= a.Lx) return;
    const long long rows = (long long)a.Ly * a.Lz;  // (z, y) rows of a velocity plane
    const double v = src[((long long)q * rows + y) * a.Lx + x];
    const long long idx =
        (long long)inst * a.inst_stride + (long long)q * a.plane + (long long)y * a.pitch + x;
    if (a.prec == GLBM_FP64)
        static_cast<double *>(f)[idx] = v;
    else
        static_cast<float *>(f)[idx] = (float)(v - rest_weight(a, q));
}

__global__ void k_get_populations(const __grid_constant__ AuxArgs a, const void *f, int inst,
                                  double *__restrict__ dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int q = blockIdx.z;
    if (x >= a.Lx) return;
    const long long idx =
        (long long)inst * a.inst_stride + (long long)q * a.plane + (long long)y * a.pitch + x;
    double v = load_full(a, f, idx, q);
    if (a.prec != GLBM_FP64) v += rest_weight(a, q);
    dst[((long long)q * a.Ly * a.Lz + y) * a.Lx + x] = v;
}

// Population of velocity (ix, iy) arriving at node (x, y) by streaming X
// (full FP64 value), including the boundary rule. rw_lo / rw_hi are the wall
// densities of column x.
__device__ double pulled(const AuxArgs &a, const InstParams &ip, const void *f, long long ibase,
                         int x, int y, int ix, int iy, double rw_lo, double rw_hi)
{
    const int N = a.N;
    if (a.dims == 1) {
        const int n = ix - N;
        int xs = x - n;
        int q = ix;
        if (a.bc == GLBM_BC_PERIODIC) {
            xs = wrap_index(xs, a.Lx);
        } else if (xs < 0) {
            xs = -1 - xs;
            q = 2 * N - ix;
        } else if (xs >= a.Lx) {
            xs = 2 * a.Lx - 1 - xs;
            q = 2 * N - ix;
        }
        double v = load_full(a, f, ibase + (long long)q * a.plane + xs, q);
        if (a.prec != GLBM_FP64) v += a.tab.W[q];
        return v;
    }
    const int nx = ax_vel(a.tabx, ix), ny = ax_vel(a.tab, iy);
    const int xs = wrap_index(x - nx, a.Lx);
    int ys = y - ny;
    if (a.bc == GLBM_BC_WALLS) {
        if (ys < 0) return rw_lo * ip.ew_lo[ix] * a.tab.W[iy];
        if (ys >= a.Ly) return rw_hi * ip.ew_hi[ix] * a.tab.W[iy];
    } else {
        ys = wrap_index(ys, a.Ly);
    }
    const int q = iy * ax_q(a.tabx) + ix;
    double v = load_full(a, f, ibase + (long long)q * a.plane + (long long)ys * a.pitch + xs, q);
    if (a.prec != GLBM_FP64) v += a.tab.W[iy] * a.tabx.W[ix];
    return v;
}

// Wall density of column x: absorbed mass / sum_{v>0} v W_v (FP64).
__device__ double wall_density(const AuxArgs &a, const InstParams &ip, const void *f,
                               long long ibase, int x, bool lower)
{
    const int N = a.N, Q1x = ax_q(a.tabx), zv = a.tab.zv;
    double D = 0.0;
    // velocity magnitudes |v| = m (2N+1) or 2m+1 (2N+2) in increasing order
    for (int m = zv ? 0 : 1; m <= N; ++m) {
        const int aa = zv ? 2 * m + 1 : m;
        for (int k = 0; k < aa; ++k) {
            const int iy = lower ? N - m : (zv ? N + 1 + m : N + m);
            const int row = lower ? k : a.Ly - 1 - k;
            for (int ix = 0; ix < Q1x; ++ix) {
                const int xs = wrap_index(x - ax_vel(a.tabx, ix), a.Lx);
                const int q = iy * Q1x + ix;
                double v = load_full(a, f, ibase + (long long)q * a.plane + (long long)row * a.pitch + xs, q);
                if (a.prec != GLBM_FP64) v += a.tab.W[iy] * a.tabx.W[ix];
                D += v;
            }
        }
    }
    return D * ip.inv_den;
}

// out[7][Ly][Lx] (2D) or out[4][Lx] (1D): moments of S(X) at every node.
__global__ void k_moments(const __grid_constant__ AuxArgs a, const void *f, int inst,
                          double *__restrict__ out)
{
    const AxisTableHi &tx = a.dims == 2 ? a.tabx : a.tab;
    const int Q1x = ax_q(tx);
    const bool f64 = a.prec == GLBM_FP64;
    // per block, from the x axis: (c, c^2, c^3) of every mirror pair's positive
    // velocity and, for FP32 deviations, m_p = sum_ix W^x xi_x^p (the rest
    // weights' part of a row's R_p is W^y m_p, added once per row)
    __shared__ double cpow[GLBM_MAXQA / 2][3];
    __shared__ double wmom[4];
    if ((int)threadIdx.x < Q1x / 2) {
        const double c = ax_vel(tx, Q1x - 1 - threadIdx.x), c2 = c * c;
        cpow[threadIdx.x][0] = c;
        cpow[threadIdx.x][1] = c2;
        cpow[threadIdx.x][2] = c2 * c;
    }
    if (threadIdx.x == 32) {
        double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
        if (!f64 && a.dims == 2) {
            for (int ix = 0; ix < Q1x; ++ix) {
                const double w = tx.W[ix], c = ax_vel(tx, ix);
                m0 += w;
                m1 = fma(c, w, m1);
                m2 = fma(c * c, w, m2);
                m3 = fma(c * c * c, w, m3);
            }
        }
        wmom[0] = m0;
        wmom[1] = m1;
        wmom[2] = m2;
        wmom[3] = m3;
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.Lx) return;
    const InstParams &ip = a.ip[inst];
    const int Qy = a.dims == 2 ? ax_q(a.tab) : 1;
    const int vmax = a.tab.zv ? 2 * a.N + 1 : a.N;  // fastest y velocity
    const long long ibase = (long long)inst * a.inst_stride;
    double rw_lo = 0.0, rw_hi = 0.0;
    if (a.dims == 2 && a.bc == GLBM_BC_WALLS) {
        if (y < vmax) rw_lo = wall_density(a, ip, f, ibase, x, true);
        if (y >= a.Ly - vmax) rw_hi = wall_density(a, ip, f, ibase, x, false);
    }
    // one pass of raw moments, row by row: R_p = sum_ix xi_x^p v for p = 0..3,
    // then the central moments about u from them (expanded in FP64)
    double M0 = 0.0, jx = 0.0, jy = 0.0, Pxx = 0.0, Pyy = 0.0, Pxy = 0.0, Mx = 0.0, My = 0.0;
    const int cmax = ax_vel(tx, Q1x - 1);  // the largest x speed
    const bool one_wrap = a.Lx > cmax;
    const double m0 = wmom[0], m1 = wmom[1], m2 = wmom[2], m3 = wmom[3];
    for (int iy = 0; iy < Qy; ++iy) {
        double R0 = 0.0, R1 = 0.0, R2 = 0.0, R3 = 0.0;
        const int ny = a.dims == 2 ? ax_vel(a.tab, iy) : 0;
        int ys = y - ny;
        if (a.dims == 1 || (a.bc == GLBM_BC_WALLS && (ys < 0 || ys >= a.Ly))) {
            // 1D (bounce-back ends) and rows emitted by a wall: value by value
            for (int ix = 0; ix < Q1x; ++ix) {
                const double v = pulled(a, ip, f, ibase, x, y, ix, iy, rw_lo, rw_hi);
                const double c = ax_vel(tx, ix);
                R0 += v;
                R1 = fma(c, v, R1);
                R2 = fma(c * c, v, R2);
                R3 = fma(c * c * c, v, R3);
            }
        } else {
            // a pulled row: the velocity columns in mirror pairs (+c, -c), so
            // that the odd powers take the pair's difference and the even ones
            // its sum; stored values (FP32: deviations) are summed and the rest
            // weights' part is added once
            if (a.bc != GLBM_BC_WALLS) ys = wrap_index(ys, a.Ly);
            const long long row = ibase + (long long)(iy * Q1x) * a.plane + (long long)ys * a.pitch;
#pragma unroll 4
            for (int p = 0; p < Q1x / 2; ++p) {
                const int ipos = Q1x - 1 - p;
                const int cv = ax_vel(tx, ipos);  // > 0; column p moves at -cv
                const long long ap = row + (long long)ipos * a.plane + wrap_shift(x - cv, a.Lx, one_wrap);
                const long long am = row + (long long)p * a.plane + wrap_shift(x + cv, a.Lx, one_wrap);
                const double vp = load_full(a, f, ap, 0), vm = load_full(a, f, am, 0);
                const double sp = vp + vm, dm = vp - vm;
                R0 += sp;
                R1 = fma(cpow[p][0], dm, R1);
                R2 = fma(cpow[p][1], sp, R2);
                R3 = fma(cpow[p][2], dm, R3);
            }
            if (Q1x & 1) R0 += load_full(a, f, row + (long long)(Q1x / 2) * a.plane + x, 0);
            if (!f64) {
                const double wy = a.tab.W[iy];
                R0 = fma(wy, m0, R0);
                R1 = fma(wy, m1, R1);
                R2 = fma(wy, m2, R2);
                R3 = fma(wy, m3, R3);
            }
        }
        const double cy = a.dims == 2 ? ax_vel(a.tab, iy) : 0.0;
        M0 += R0;
        jx += R1;
        jy = fma(cy, R0, jy);
        Pxx += R2;
        Pyy = fma(cy * cy, R0, Pyy);
        Pxy = fma(cy, R1, Pxy);
        Mx += fma(cy * cy, R1, R3);             // sum xi_x |xi|^2 v
        My += cy * fma(cy * cy, R0, R2);        // sum xi_y |xi|^2 v
    }
    const double rho = M0;
    // u_x = (j_x + g/2) / rho with Guo's force (g_half = 0 otherwise)
    const double ux = (jx + ip.g_half) / rho, uy = jy / rho;
    // central second moments: P_ab - u_a j_b - j_a u_b + rho u_a u_b
    const double cxx = Pxx - 2.0 * ux * jx + rho * ux * ux;
    const double cyy = Pyy - 2.0 * uy * jy + rho * uy * uy;
    const double sxy = Pxy - ux * jy - jx * uy + rho * ux * uy;
    // sum c_a |c|^2 v, c = xi - u: M3_a - u_a tr P - 2 u.P_a + 2 u_a u.j + |u|^2 j_a - u_a |u|^2 rho
    const double trP = Pxx + Pyy, uj = ux * jx + uy * jy, u2 = ux * ux + uy * uy;
    const double qx = Mx - ux * trP - 2.0 * (ux * Pxx + uy * Pxy) + 2.0 * ux * uj + u2 * jx -
                      ux * u2 * rho;
    const double qy = My - uy * trP - 2.0 * (ux * Pxy + uy * Pyy) + 2.0 * uy * uj + u2 * jy -
                      uy * u2 * rho;
    const double e2 = cxx + cyy;
    const long long plane = (long long)a.Lx * a.Ly;
    const long long node = (long long)y * a.Lx + x;
    if (a.dims == 2) {
        out[0 * plane + node] = rho;
        out[1 * plane + node] = ux;
        out[2 * plane + node] = uy;
        out[3 * plane + node] = e2 / (2.0 * rho);
        out[4 * plane + node] = 0.5 * qx;
        out[5 * plane + node] = 0.5 * qy;
        out[6 * plane + node] = sxy;
    } else {
        out[0 * plane + node] = rho;
        out[1 * plane + node] = ux;
        out[2 * plane + node] = e2 / rho;
        out[3 * plane + node] = 0.5 * qx;
    }
}

// Deterministic sums of rho, rho u_x, rho u_y over n nodes: every block sums a
// fixed contiguous range in a fixed tree order; a second launch adds the
// block partials in index order.
constexpr int SUM_THREADS = 256;

__global__ void k_field_partials(const double *__restrict__ fields, int nfields, long long n,
                                 double *__restrict__ partials)
{
    __shared__ double sh[3][SUM_THREADS];
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * per;
    const long long hi = min(n, lo + per);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += SUM_THREADS) {
        const double r = fields[i];
        s0 += r;
        s1 += r * fields[n + i];
        if (nfields > 2) s2 += r * fields[2 * n + i];
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int stride = SUM_THREADS / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
            for (int m = 0; m < 3; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x < 3) partials[blockIdx.x * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_field_final(const double *__restrict__ partials, int nblocks, double *out)
{
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * 3 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Channel diagnostics (Sec. 5.3, 5.4) from the moment fields of one instance
// (rho at field 0, u_x at field 1, each [z][y][x]): the row means over x (and
// z) of u_x and rho u_x, then the flow rate, the volumetric flow and the slip
// ratios. FP64, every sum in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int ROW_THREADS = 256;

// Fixed tree over ROW_THREADS shared values (two arrays at once).
__device__ __forceinline__ void tree2(double *a, double *b)
{
    __syncthreads();
    for (int stride = ROW_THREADS / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) {
            a[threadIdx.x] += a[threadIdx.x + stride];
            b[threadIdx.x] += b[threadIdx.x + stride];
        }
        __syncthreads();
    }
}

// Block y: prof[y] = mean over (z, x) of u_x, prof[Ly + y] = mean of rho u_x.
__global__ void k_row_means(const double *__restrict__ mom, int Lx, int Ly, int Lz,
                            double *__restrict__ prof)
{
    __shared__ double su[ROW_THREADS], sj[ROW_THREADS];
    const int y = blockIdx.x;
    const long long plane = (long long)Lx * Ly * Lz;
    double a = 0.0, b = 0.0;
    for (int z = 0; z < Lz; ++z)
        for (int x = threadIdx.x; x < Lx; x += ROW_THREADS) {
            const long long node = ((long long)z * Ly + y) * Lx + x;
            const double u = mom[plane + node];
            a += u;
            b += mom[node] * u;
        }
    su[threadIdx.x] = a;
    sj[threadIdx.x] = b;
    tree2(su, sj);
    if (threadIdx.x == 0) {
        const double n = (double)Lx * (double)Lz;
        prof[y] = su[0] / n;
        prof[Ly + y] = sj[0] / n;
    }
}

// One block: stats[GLBM_CH_*] from the row means (see glbm_channel_diagnostics).
__global__ void k_channel_stats(const double *__restrict__ prof, int Ly, ChannelParams p,
                                double *__restrict__ stats)
{
    __shared__ double su[ROW_THREADS], sj[ROW_THREADS];
    double a = 0.0, b = 0.0;
    for (int y = threadIdx.x; y < Ly; y += ROW_THREADS) {
        a += prof[y];
        b += prof[Ly + y];
    }
    su[threadIdx.x] = a;
    sj[threadIdx.x] = b;
    tree2(su, sj);
    if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7FF8000000000000LL);
        const double H = (double)Ly;
        // volumetric flow Q = (1/Kn) int_0^H u dy / (4 U0 H), U0 = g H^2 / (8 nu)
        const double nu = p.theta_y * p.tau;
        const double U0 = p.g * H * H / (8.0 * nu);
        const double kn = p.tau * sqrt(2.0 * p.theta_y) / H;  // Eq. (kn) with nu = theta tau
        stats[GLBM_CH_FLOW_RATE] = sj[0];
        stats[GLBM_CH_VOLUMETRIC] = p.g != 0.0 ? su[0] / (kn * 4.0 * U0 * H) : nan;
        // the row means extrapolated linearly to the wall planes y = -1/2, Ly - 1/2
        const double ulo = Ly > 1 ? 1.5 * prof[0] - 0.5 * prof[1] : prof[0];
        const double uhi = Ly > 1 ? 1.5 * prof[Ly - 1] - 0.5 * prof[Ly - 2] : prof[Ly - 1];
        const double du = p.u_hi - p.u_lo;
        stats[GLBM_CH_U_LO] = p.walls ? ulo : nan;
        stats[GLBM_CH_U_HI] = p.walls ? uhi : nan;
        stats[GLBM_CH_SLIP_LO] = p.walls && du != 0.0 ? (ulo - p.u_lo) / du : nan;
        stats[GLBM_CH_SLIP_HI] = p.walls && du != 0.0 ? (p.u_hi - uhi) / du : nan;
    }
}

// ---------------------------------------------------------------------------
// 1D step (Sec. 5.1): pull with halfway bounce-back or periodic ends, moments,
// equilibrium, relaxation. One thread per node.
// ---------------------------------------------------------------------------
template <int N, typename T>
__device__ __forceinline__ void node1d(const AuxArgs &a, const InstParams &ip, const T *fin,
                                       T *fout, int x, int L, long long plane, unsigned *status)
{
    constexpr int Q1 = 2 * N + 1;
    constexpr bool DEV = sizeof(T) == 4;
    using Acc = TabAcc<T>;
    T f[Q1];
#pragma unroll
    for (int ix = 0; ix < Q1; ++ix) {
        const int n = ix - N;
        int xs = x - n, q = ix;
        if (a.bc == GLBM_BC_PERIODIC) {
            xs = wrap_index(xs, L);
        } else if (xs < 0) {
            xs = -1 - xs;
            q = 2 * N - ix;
        } else if (xs >= L) {
            xs = 2 * L - 1 - xs;
            q = 2 * N - ix;
        }
        f[ix] = fin[(long long)q * plane + xs];
    }
    T s = T(0), c = T(0), sj = T(0), cj = T(0);
#pragma unroll
    for (int ix = 0; ix < Q1; ++ix) acc2(s, c, f[ix]);
#pragma unroll
    for (int n = 1; n <= N; ++n) acc2(sj, cj, T(n) * (f[N + n] - f[N - n]));
    const T m0 = s + c;
    const T rho = DEV ? T(1) + m0 : m0;
    const T drho = DEV ? m0 : m0 - T(1);
    const T j = sj + cj;
    T u = j / rho;
    // FP32: u = j / (1 + delta rho) from the unrounded density, by one
    // correction with the residual (j - u) - u delta rho (j - u is exact)
    if (DEV) u += fma(-u, drho, j - u) / rho;
    const T umax = (T)(0.816496580927726 * N);
    if (!(rho > T(0)) || !(fabs(u) <= umax)) flag_unstable(status);
    T d[Q1];
    eq_dev_all<N, T>(a.tab, u, d);
    const T om = DEV ? (T)ip.omega_f : (T)ip.omega;
#pragma unroll
    for (int ix = 0; ix < Q1; ++ix) {
        const T w = Acc::W(a.tab, ix);
        // FP32: delta f^eq = d + drho (W + d), the momentum-carrying d unscaled
        // by a rounded rho; FP64: f^eq = rho (W + d)
        const T eq = DEV ? fma(drho, w + d[ix], d[ix]) : rho * (w + d[ix]);
        fout[(long long)ix * plane + x] = fma(om, eq - f[ix], f[ix]);  // f + omega (f^eq - f)
    }
}

template <int N, typename T>
__global__ void k_step1d(const __grid_constant__ AuxArgs a, const T *__restrict__ fin,
                         T *__restrict__ fout, int inst, unsigned *status)
{
    if (step_halted(status)) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < a.Lx) node1d<N, T>(a, a.ip[inst], fin, fout, x, a.Lx, a.plane, status);
    finish_step(status);
}

// Many steps of one small 1D lattice inside one CTA: both population copies
// live in shared memory and a block barrier separates the steps, so the whole
// run is one launch (the shock tube is launch-latency bound, not HBM bound).
template <int N, typename T>
__global__ void k_run1d_resident(const __grid_constant__ AuxArgs a, T *__restrict__ f,
                                 int inst, long long steps, unsigned *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned bad;
    constexpr int Q1 = 2 * N + 1;
    if (step_halted(status)) return;  // an earlier step left the positivity domain
    const int L = a.Lx;
    T *A = reinterpret_cast<T *>(smem_raw);
    T *B = A + (long long)Q1 * L;
    for (int i = threadIdx.x; i < Q1 * L; i += blockDim.x) {
        const int q = i / L, x = i % L;
        A[i] = f[(long long)q * a.plane + x];
    }
    if (threadIdx.x == 0) bad = 0u;
    __syncthreads();
    long long done = 0;
    while (done < steps) {
        for (int x = threadIdx.x; x < L; x += blockDim.x)
            node1d<N, T>(a, a.ip[inst], A, B, x, L, L, status);
        __syncthreads();  // the step's flags (global atomics of this block) are visible
        T *tmp = A;
        A = B;
        B = tmp;
        ++done;
        // stop after a step that left the positivity domain: one read,
        // broadcast, so that every thread leaves the loop at the same step
        if (threadIdx.x == 0) bad = __ldcg(status + ST_FLAGS) & 1u;
        __syncthreads();
        if (bad) break;
    }
    for (int i = threadIdx.x; i < Q1 * L; i += blockDim.x) {
        const int q = i / L, x = i % L;
        f[(long long)q * a.plane + x] = A[i];
    }
    if (threadIdx.x == 0) {
        atomicAdd(status + ST_STEPS, (unsigned)done);
        if (bad) atomicExch(status + ST_HALT, 1u);
    }
}

template <typename T>
cudaError_t launch_step1d_t(const AuxArgs &a, const void *fin, void *fout, int inst,
                            unsigned *status, cudaStream_t s)
{
    const T *in = static_cast<const T *>(fin) + (long long)inst * a.inst_stride;
    T *out = static_cast<T *>(fout) + (long long)inst * a.inst_stride;
    const int threads = 128;
    const int blocks = (a.Lx + threads - 1) / threads;
    switch (a.N) {
#define GLBM_CASE(NN) \
    case NN: k_step1d<NN, T><<<blocks, threads, 0, s>>>(a, in, out, inst, status); break;
        GLBM_CASE(1) GLBM_CASE(2) GLBM_CASE(3) GLBM_CASE(4)
        GLBM_CASE(5) GLBM_CASE(6) GLBM_CASE(7) GLBM_CASE(8)
#undef GLBM_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int N, typename T>
cudaError_t launch_resident_n(const AuxArgs &a, T *f, int inst, long long steps,
                              unsigned *status, cudaStream_t s, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_run1d_resident<N, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = a.Lx >= 1024 ? 1024 : ((a.Lx + 31) / 32) * 32;
    k_run1d_resident<N, T><<<1, threads, smem, s>>>(a, f, inst, steps, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resident_t(const AuxArgs &a, void *fv, int inst, long long steps,
                              unsigned *status, cudaStream_t s, int *ok)
{
    const size_t smem = (size_t)2 * (2 * a.N + 1) * a.Lx * sizeof(T);
    *ok = 0;
    if (smem > 200 * 1024) return cudaSuccess;  // caller falls back to per-step launches
    *ok = 1;
    T *f = static_cast<T *>(fv) + (long long)inst * a.inst_stride;
    switch (a.N) {
#define GLBM_CASE(NN) \
    case NN: return launch_resident_n<NN, T>(a, f, inst, steps, status, s, smem);
        GLBM_CASE(1) GLBM_CASE(2) GLBM_CASE(3) GLBM_CASE(4)
        GLBM_CASE(5) GLBM_CASE(6) GLBM_CASE(7) GLBM_CASE(8)
#undef GLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// 3D tensor products: level N on every axis, layout f[q][z][y][x] with
// q = (iz Q1 + iy) Q1 + ix, periodic in x and z, walls or periodicity in y.
// ---------------------------------------------------------------------------
__global__ void k_set_equilibrium3d(const __grid_constant__ AuxArgs a, void *f, int inst,
                                    const double *__restrict__ rho, const double *__restrict__ ux,
                                    const double *__restrict__ uy, const double *__restrict__ uz)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int zy = blockIdx.y;  // z * Ly + y
    if (x >= a.Lx) return;
    const int Q1 = ax_q(a.tab);
    const long long node = (long long)zy * a.Lx + x;
    const double r = rho[node];
    const long long base = (long long)inst * a.inst_stride + (long long)zy * a.pitch + x;
    const bool f64 = a.prec == GLBM_FP64;
    // per node: E^x (FP64 storage) or E^x - W^x (FP32 deviations), and E^y - W^y
    double exs[GLBM_MAXQA], dys[GLBM_MAXQA], dzs[GLBM_MAXQA];
    eq_dev_all_rt(a.tab, ux[node], exs);
    eq_dev_all_rt(a.tab, uy[node], dys);
    eq_dev_all_rt(a.tab, uz[node], dzs);
    if (f64)
        for (int i = 0; i < Q1; ++i) exs[i] += a.tab.W[i];
    for (int iz = 0; iz < Q1; ++iz) {
        const double wz = a.tab.W[iz], dz = dzs[iz];
        for (int iy = 0; iy < Q1; ++iy) {
            const double wy = a.tab.W[iy], dy = dys[iy];
            // per row: A = rho E^y E^z and B = rho E^y E^z - W^y W^z =
            // (rho - 1) W^y W^z + rho (d^y E^z + W^y d^z) (no cancellation);
            // then rho E^x E^y E^z = E^x A, and in deviations W^x B + d^x A
            const double A = r * ((wy + dy) * (wz + dz));
            const double B = fma(r - 1.0, wy * wz, r * fma(dy, wz + dz, wy * dz));
            const long long row = base + (long long)((iz * Q1 + iy) * Q1) * a.plane;
            if (f64) {
                double *out = static_cast<double *>(f) + row;
                for (int ix = 0; ix < Q1; ++ix) out[(long long)ix * a.plane] = exs[ix] * A;
            } else {
                float *out = static_cast<float *>(f) + row;
                for (int ix = 0; ix < Q1; ++ix)
                    out[(long long)ix * a.plane] = (float)fma(exs[ix], A, a.tab.W[ix] * B);
            }
        }
    }
}

// Population of velocity (ix, iy, iz) arriving at node (x, y, z) by streaming
// X (full FP64 value), with the wall emission rho_w E^x(u_w) W^y W^z.
__device__ double pulled3d(const AuxArgs &a, const InstParams &ip, const void *f, long long ibase,
                           int x, int y, int z, int ix, int iy, int iz, double rw_lo, double rw_hi)
{
    const int N = a.N, Q1 = 2 * N + 1;
    const int xs = wrap_index(x - (ix - N), a.Lx), zs = wrap_index(z - (iz - N), a.Lz);
    int ys = y - (iy - N);
    const double wyz = a.tab.W[iy] * a.tab.W[iz];
    if (a.bc == GLBM_BC_WALLS) {
        if (ys < 0) return rw_lo * ip.ew_lo[ix] * wyz;
        if (ys >= a.Ly) return rw_hi * ip.ew_hi[ix] * wyz;
    } else {
        ys = wrap_index(ys, a.Ly);
    }
    const int q = (iz * Q1 + iy) * Q1 + ix;
    double v = load_full(a, f, ibase + (long long)q * a.plane +
                                   ((long long)zs * a.Ly + ys) * a.pitch + xs, q);
    if (a.prec != GLBM_FP64) v += a.tab.W[ix] * wyz;
    return v;
}

// Wall density of column (x, z): absorbed mass / sum_{n>0} n W_n.
__device__ double wall_density3d(const AuxArgs &a, const InstParams &ip, const void *f,
                                 long long ibase, int x, int z, bool lower)
{
    const int N = a.N, Q1 = 2 * N + 1;
    double D = 0.0;
    for (int aa = 1; aa <= N; ++aa)
        for (int k = 0; k < aa; ++k)
            for (int iz = 0; iz < Q1; ++iz) {
                const int iy = lower ? N - aa : N + aa;
                const int row = lower ? k : a.Ly - 1 - k;
                const int zs = wrap_index(z - (iz - N), a.Lz);
                for (int ix = 0; ix < Q1; ++ix) {
                    const int xs = wrap_index(x - (ix - N), a.Lx);
                    const int q = (iz * Q1 + iy) * Q1 + ix;
                    double v = load_full(a, f, ibase + (long long)q * a.plane +
                                                   ((long long)zs * a.Ly + row) * a.pitch + xs, q);
                    if (a.prec != GLBM_FP64) v += a.tab.W[ix] * a.tab.W[iy] * a.tab.W[iz];
                    D += v;
                }
            }
    return D * ip.inv_den;
}

// out[9][Lz][Ly][Lx]: rho, u_x, u_y, T = sum |xi-u|^2 f / (3 rho), q_x, q_y,
// sigma_xy, u_z, q_z of S(X).
__global__ void k_moments3d(const __grid_constant__ AuxArgs a, const void *f, int inst,
                            double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int zy = blockIdx.y;
    if (x >= a.Lx) return;
    const int y = zy % a.Ly, z = zy / a.Ly;
    const InstParams &ip = a.ip[inst];
    const int N = a.N, Q1 = 2 * N + 1;
    const long long ibase = (long long)inst * a.inst_stride;
    double rw_lo = 0.0, rw_hi = 0.0;
    if (a.bc == GLBM_BC_WALLS) {
        if (y < N) rw_lo = wall_density3d(a, ip, f, ibase, x, z, true);
        if (y >= a.Ly - N) rw_hi = wall_density3d(a, ip, f, ibase, x, z, false);
    }
    // one pass of raw moments, row by row (R_p = sum_ix xi_x^p v), then the
    // central moments about u from them (expanded in FP64)
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    double Pxx = 0.0, Pyy = 0.0, Pzz = 0.0, Pxy = 0.0, Pxz = 0.0, Pyz = 0.0;
    double Mx = 0.0, My = 0.0, Mz = 0.0;  // sum xi_a |xi|^2 v
    const bool f64 = a.prec == GLBM_FP64;
    const bool one_wrap = a.Lx > N;
    // FP32 deviations: the rest weights' part of a row's R_p is W^y W^z sum_ix
    // W^x xi_x^p, added once per row
    double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
    if (!f64) {
        for (int ix = 0; ix < Q1; ++ix) {
            const double w = a.tab.W[ix], c = ix - N;
            m0 += w;
            m1 = fma(c, w, m1);
            m2 = fma(c * c, w, m2);
            m3 = fma(c * c * c, w, m3);
        }
    }
    for (int iz = 0; iz < Q1; ++iz)
        for (int iy = 0; iy < Q1; ++iy) {
            double R0 = 0.0, R1 = 0.0, R2 = 0.0, R3 = 0.0;
            int ys = y - (iy - N);
            if (a.bc == GLBM_BC_WALLS && (ys < 0 || ys >= a.Ly)) {
                // a row emitted by a wall: value by value
                for (int ix = 0; ix < Q1; ++ix) {
                    const double v = pulled3d(a, ip, f, ibase, x, y, z, ix, iy, iz, rw_lo, rw_hi);
                    const double c = ix - N;
                    R0 += v;
                    R1 = fma(c, v, R1);
                    R2 = fma(c * c, v, R2);
                    R3 = fma(c * c * c, v, R3);
                }
            } else {
                // a pulled row: mirror pairs (+c, -c), odd powers on the pair's
                // difference, even ones on its sum; FP32 stores deviations, whose
                // rest weights' part is added once per row
                if (a.bc != GLBM_BC_WALLS) ys = wrap_index(ys, a.Ly);
                const int zs = wrap_index(z - (iz - N), a.Lz);
                const long long row = ibase + (long long)((iz * Q1 + iy) * Q1) * a.plane +
                                      ((long long)zs * a.Ly + ys) * a.pitch;
#pragma unroll 3
                for (int n = 1; n <= N; ++n) {
                    const double vp = load_full(a, f, row + (long long)(N + n) * a.plane +
                                                          wrap_shift(x - n, a.Lx, one_wrap), 0);
                    const double vm = load_full(a, f, row + (long long)(N - n) * a.plane +
                                                          wrap_shift(x + n, a.Lx, one_wrap), 0);
                    const double sp = vp + vm, dm = vp - vm;
                    const double c = n, c2 = c * c;
                    R0 += sp;
                    R1 = fma(c, dm, R1);
                    R2 = fma(c2, sp, R2);
                    R3 = fma(c2 * c, dm, R3);
                }
                R0 += load_full(a, f, row + (long long)N * a.plane + x, 0);
                if (!f64) {
                    const double wyz = a.tab.W[iy] * a.tab.W[iz];
                    R0 = fma(wyz, m0, R0);
                    R1 = fma(wyz, m1, R1);
                    R2 = fma(wyz, m2, R2);
                    R3 = fma(wyz, m3, R3);
                }
            }
            const double cy = iy - N, cz = iz - N, s2 = cy * cy + cz * cz;
            rho += R0;
            jx += R1;
            jy = fma(cy, R0, jy);
            jz = fma(cz, R0, jz);
            Pxx += R2;
            Pyy = fma(cy * cy, R0, Pyy);
            Pzz = fma(cz * cz, R0, Pzz);
            Pxy = fma(cy, R1, Pxy);
            Pxz = fma(cz, R1, Pxz);
            Pyz = fma(cy * cz, R0, Pyz);
            Mx += fma(s2, R1, R3);
            My += cy * fma(s2, R0, R2);
            Mz += cz * fma(s2, R0, R2);
        }
    const double ux = jx / rho, uy = jy / rho, uz = jz / rho;
    const double trP = Pxx + Pyy + Pzz, uj = ux * jx + uy * jy + uz * jz;
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double e2 = trP - 2.0 * uj + rho * u2;
    const double sxy = Pxy - ux * jy - jx * uy + rho * ux * uy;
    const double uPx = ux * Pxx + uy * Pxy + uz * Pxz, uPy = ux * Pxy + uy * Pyy + uz * Pyz,
                 uPz = ux * Pxz + uy * Pyz + uz * Pzz;
    const double qx = Mx - ux * trP - 2.0 * uPx + 2.0 * ux * uj + u2 * jx - ux * u2 * rho;
    const double qy = My - uy * trP - 2.0 * uPy + 2.0 * uy * uj + u2 * jy - uy * u2 * rho;
    const double qz = Mz - uz * trP - 2.0 * uPz + 2.0 * uz * uj + u2 * jz - uz * u2 * rho;
    const long long nodes = (long long)a.Lx * a.Ly * a.Lz;
    const long long node = (long long)zy * a.Lx + x;
    const double m[9] = {rho, ux, uy, e2 / (3.0 * rho), 0.5 * qx, 0.5 * qy, sxy, uz, 0.5 * qz};
    for (int k = 0; k < 9; ++k) out[k * nodes + node] = m[k];
}

}  // namespace

cudaError_t glbm_launch_set_equilibrium3d(const AuxArgs &a, void *f, int inst, const double *rho,
                                          const double *ux, const double *uy, const double *uz,
                                          cudaStream_t s)
{
    dim3 grid((a.Lx + 127) / 128, a.Ly * a.Lz);
    k_set_equilibrium3d<<<grid, 128, 0, s>>>(a, f, inst, rho, ux, uy, uz);
    return cudaGetLastError();
}

cudaError_t glbm_launch_moments3d(const AuxArgs &a, const void *f, int inst, double *out,
                                  cudaStream_t s)
{
    dim3 grid((a.Lx + 63) / 64, a.Ly * a.Lz);
    k_moments3d<<<grid, 64, 0, s>>>(a, f, inst, out);
    return cudaGetLastError();
}

cudaError_t glbm_launch_set_equilibrium(const AuxArgs &a, void *f, int inst, const double *rho,
                                        const double *ux, const double *uy, cudaStream_t s)
{
    dim3 grid((a.Lx + 127) / 128, a.Ly);
    k_set_equilibrium<<<grid, 128, 0, s>>>(a, f, inst, rho, ux, uy);
    return cudaGetLastError();
}

cudaError_t glbm_launch_set_populations(const AuxArgs &a, void *f, int inst, const double *src,
                                        cudaStream_t s)
{
    dim3 grid((a.Lx + 127) / 128, a.Ly * a.Lz,
              a.dims == 3 ? ax_q(a.tab) * ax_q(a.tab) * ax_q(a.tab)
                          : (a.dims == 2 ? ax_q(a.tab) * ax_q(a.tabx) : ax_q(a.tab)));
    k_set_populations<<<grid, 128, 0, s>>>(a, f, inst, src);
    return cudaGetLastError();
}

cudaError_t glbm_launch_get_populations(const AuxArgs &a, const void *f, int inst, double *dst,
                                        cudaStream_t s)
{
    dim3 grid((a.Lx + 127) / 128, a.Ly * a.Lz,
              a.dims == 3 ? ax_q(a.tab) * ax_q(a.tab) * ax_q(a.tab)
                          : (a.dims == 2 ? ax_q(a.tab) * ax_q(a.tabx) : ax_q(a.tab)));
    k_get_populations<<<grid, 128, 0, s>>>(a, f, inst, dst);
    return cudaGetLastError();
}

cudaError_t glbm_launch_moments(const AuxArgs &a, const void *f, int inst, double *out,
                                cudaStream_t s)
{
    dim3 grid((a.Lx + 63) / 64, a.Ly);
    k_moments<<<grid, 64, 0, s>>>(a, f, inst, out);
    return cudaGetLastError();
}

int glbm_field_sum_blocks(long long n)
{
    long long b = (n + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

cudaError_t glbm_launch_field_sums(const double *fields, int nfields, long long n, double *partials,
                                   int nblocks, double *out, cudaStream_t s)
{
    k_field_partials<<<nblocks, SUM_THREADS, 0, s>>>(fields, nfields, n, partials);
    k_field_final<<<1, 32, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t glbm_launch_step1d(const AuxArgs &a, const void *fin, void *fout, int inst,
                               unsigned *status, cudaStream_t s)
{
    if (a.prec == GLBM_FP64) return launch_step1d_t<double>(a, fin, fout, inst, status, s);
    return launch_step1d_t<float>(a, fin, fout, inst, status, s);
}

cudaError_t glbm_launch_run1d_resident(const AuxArgs &a, void *f, int inst, long long steps,
                                       unsigned *status, cudaStream_t s, int *ok)
{
    if (a.prec == GLBM_FP64) return launch_resident_t<double>(a, f, inst, steps, status, s, ok);
    return launch_resident_t<float>(a, f, inst, steps, status, s, ok);
}

// ---------------------------------------------------------------------------
// Conservation sums without allocation (glbm_conservation_noalloc).
//
// The block partials of the deterministic sum live in this file-scope device
// array instead of context memory, for callers that may not allocate device
// memory. Every GPU that loads the library holds it (24 KiB) until the process
// exits, and every call shares it.
// ---------------------------------------------------------------------------
#define GLBM_NOALLOC_MAX_BLOCKS 1024
static __device__ __align__(256) double g_noalloc_partials[3 * GLBM_NOALLOC_MAX_BLOCKS];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64];  // device address of g_noalloc_partials, per device

extern "C" glbm_status glbm_conservation_noalloc(const double *fields, int dims, int64_t nodes,
                                                 double *sums, void *stream)
{
    if (!fields || !sums) return glbm_set_error(GLBM_E_INVAL, "null fields or sums");
    if (dims != 1 && dims != 2) return glbm_set_error(GLBM_E_INVAL, "dims must be 1 or 2");
    if (nodes < 1 || nodes > GLBM_NOALLOC_MAX_NODES)
        return glbm_set_error(GLBM_E_INVAL,
                              "glbm_conservation_noalloc takes 1 to %lld nodes (got %lld): its "
                              "static scratch holds %d block partials of 4096 nodes",
                              (long long)GLBM_NOALLOC_MAX_NODES, (long long)nodes,
                              GLBM_NOALLOC_MAX_BLOCKS);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return glbm_set_error(GLBM_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return glbm_set_error(GLBM_E_UNSUPPORTED, "device index %d >= 64", dev);
    void *scratch = nullptr;
    {
        // set-up once per device, with that device current: in host code the
        // array's name is only a stand-in, its device address comes from here
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_partials);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                return glbm_set_error(GLBM_E_CUDA, "cudaGetSymbolAddress of the scratch: %s",
                                      cudaGetErrorString(e));
            }
        }
        scratch = g_noalloc_ptr[dev];
    }
    // every block writes all three of its partials before the final pass reads
    // them, so nothing has to be cleared between calls
    const int nblocks = glbm_field_sum_blocks(nodes);
    e = glbm_launch_field_sums(fields, dims == 2 ? 3 : 2, nodes, static_cast<double *>(scratch),
                               nblocks, sums, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return glbm_set_error(GLBM_E_CUDA, "launch: %s", cudaGetErrorString(e));
    return GLBM_OK;
}

cudaError_t glbm_launch_channel_diagnostics(const double *mom, int Lx, int Ly, int Lz,
                                            const ChannelParams &p, double *prof, double *stats,
                                            cudaStream_t s)
{
    k_row_means<<<Ly, ROW_THREADS, 0, s>>>(mom, Lx, Ly, Lz, prof);
    k_channel_stats<<<1, ROW_THREADS, 0, s>>>(prof, Ly, p, stats);
    return cudaGetLastError();
}

// FP64 FMA throughput probe (glbm_measure_fp64_rate): a measurement aid for the
// FP64 roofline, not part of the method. Every thread runs 8 independent FMA
// chains (enough independent work per warp to keep the FP64 pipe busy), and
// the sum goes to a sink only when it takes a value it never takes, so the
// chains are not removed.
namespace {
constexpr int PROBE_CHAINS = 8;

__global__ void k_fp64_rate(double *sink, int iters, double a, double b)
{
    double x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    if (s == -1.0) sink[threadIdx.x] = s;
}
}  // namespace

extern "C" glbm_status glbm_measure_fp64_rate(void *stream, double *fma_per_s)
{
    if (!fma_per_s) return glbm_set_error(GLBM_E_INVAL, "null argument");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, 256 * sizeof(double));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8, iters = 4096;
    double best = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        k_fp64_rate<<<blocks, threads, 0, s>>>(sink, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        const double rate = (double)blocks * threads * iters * PROBE_CHAINS / (ms * 1e-3);
        if (e == cudaSuccess && rep > 0 && rate > best) best = rate;  // the first run warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return glbm_set_error(GLBM_E_CUDA, "FP64 probe: %s", cudaGetErrorString(e));
    *fma_per_s = best;
    return GLBM_OK;
}

// Start of a dataflow chunk (glbm_internal.h): the band counts and the
// per-step CTA counts go back to zero, and ST_BASE takes the step clock that
// the chunk's first step starts from.
namespace {
__global__ void k_df_start(unsigned *status, unsigned *words, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        words[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) status[ST_BASE] = status[ST_CLOCK];
}
}  // namespace

cudaError_t glbm_launch_df_start(unsigned *status, unsigned *words, long long n, cudaStream_t s)
{
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    k_df_start<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(status, words, n);
    return cudaGetLastError();
}
