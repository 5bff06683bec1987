// Discrete adjoint of the 2D stream-collide step, for the gradient of the flow
// rate J = (1/Lx) sum_nodes sum_i xi_x,i F_i(T) (F = S(X): the streamed
// populations, Sec. 5.4 volumetric flow) with respect to the relaxation time
// tau, the body force g and the two wall speeds (Sec. 5.3).
//
// Forward: X_{t+1} = C(F_t), F_t = S(X_t). With mu_t = dJ/dF_t:
//   mu_T = xi_x / Lx,
//   lambda_{t+1} = S^T mu_{t+1}         (reverse streaming, wall terms below),
//   mu_t = (dC/dF)^T lambda_{t+1}        (rank-3 collision Jacobian, Eq. maineq01),
//   dJ/dtau += lambda_{t+1} . dC/dtau = -omega^2 lambda . (f^eq - f),
//   dJ/dg   += lambda_{t+1} . dC/dg   = lambda . W xi_x / theta.
// The collision Jacobian of f* = f + omega (f^eq(rho, u) - f) + F is
//   df*_i/df_j = (1 - omega) delta_ij
//              + omega [E_i + sum_a dE_i/du_a (xi_j,a - u_a)],
// so its transpose maps lambda to
//   mu_j = (1 - omega) lambda_j + omega [a0 + ax (xi_x,j - u_x) + ay (xi_y,j - u_y)],
//   a0 = sum_i lambda_i E_i,  a_a = sum_i lambda_i dE_i/du_a.
// Wall transpose: a population absorbed into a wall changes the wall density
// rho_w of the column it would reach by 1/den, and rho_w scales every emitted
// ghost rho_w E^x_i(u_w) W^y_i; so lambda of an absorbed population is
//   G(x_d) / den,  G(x) = sum_{emitted (i, y) of that wall} mu_i(x, y) E^x_i(u_w) W^y_i.
// A wall speed enters F_t only through E^x(u_w) of its emitted ghosts (rho_w
// balances the absorbed mass), so
//   dJ/du_w = sum_t sum_{emitted (x, y, i) of that wall} mu_t,i(x, y) rho_w,t(x)
//             dE^x_i/du(u_w) W^y_i,
// with rho_w,t from X_t: the step of time t adds its term at the wall rows,
// k_adj_final_walls the term of F_T.
#include "glbm_device.cuh"

namespace {

// E_n and dE_n/du (n = -N..N) at velocity u, FP64, from the even/odd table.
template <int N>
__device__ __forceinline__ void eq_and_slope(const AxisTable &t, double u, double (&E)[2 * N + 1],
                                             double (&dE)[2 * N + 1])
{
    const double v = u * u;
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        // Ae(v) = sum_{i=1..N} Ce[n][i] v^i and its derivative in v
        double a = t.Ce[n][N], da = 0.0;
#pragma unroll
        for (int i = N - 1; i >= 1; --i) {
            da = fma(da, v, a);
            a = fma(a, v, t.Ce[n][i]);
        }
        // a now is sum_{i>=1} Ce v^(i-1); Ae = a v, Ae' = a + v da
        const double Ae = a * v, dAe = fma(v, da, a);
        double b = 0.0, db = 0.0;
        if (n > 0) {
            b = t.Co[n][N - 1];
#pragma unroll
            for (int i = N - 2; i >= 0; --i) {
                db = fma(db, v, b);
                b = fma(b, v, t.Co[n][i]);
            }
        }
        // E_{+-n} = W + Ae(v) +- u Bo(v);  dE/du = 2u Ae'(v) +- (Bo + 2v Bo'(v))
        const double odd = u * b, dodd = fma(2.0 * v, db, b);
        E[N + n] = t.W[N + n] + Ae + odd;
        dE[N + n] = 2.0 * u * dAe + dodd;
        if (n > 0) {
            E[N - n] = t.W[N - n] + Ae - odd;
            dE[N - n] = 2.0 * u * dAe - dodd;
        }
    }
}

template <typename TF>
__device__ __forceinline__ double fwd_value(const AdjArgs &a, long long idx, int iy, int ix)
{
    double v = (double)static_cast<const TF *>(a.X)[idx];
    if (sizeof(TF) == 4) v += a.tab.W[iy] * a.tab.W[ix];  // FP32 stores deviations
    return v;
}

// Wall density of column x from the forward state (FP64 sum of the absorbed mass).
template <int N, typename TF>
__device__ double fwd_wall_density(const AdjArgs &a, int x, bool lower)
{
    constexpr int Q1 = 2 * N + 1;
    double D = 0.0;
    for (int aa = 1; aa <= N; ++aa) {
        for (int k = 0; k < aa; ++k) {
            const int iy = lower ? N - aa : N + aa;
            const int row = lower ? k : a.Ly - 1 - k;
            for (int ix = 0; ix < Q1; ++ix) {
                const int xs = wrap_index(x - (ix - N), a.Lx);
                D += fwd_value<TF>(a, (long long)(iy * Q1 + ix) * a.plane + (long long)row * a.pitch + xs,
                                   iy, ix);
            }
        }
    }
    return D * a.ip->inv_den;
}

// Forward pulled population F_t,i at (x, y) (ghosts from the wall densities).
template <int N, typename TF>
__device__ __forceinline__ double fwd_pull(const AdjArgs &a, int x, int y, int ix, int iy,
                                           double rw_lo, double rw_hi)
{
    constexpr int Q1 = 2 * N + 1;
    const int xs = wrap_index(x - (ix - N), a.Lx);
    int ys = y - (iy - N);
    if (a.bc == GLBM_BC_WALLS) {
        if (ys < 0) return rw_lo * a.ip->ew_lo[ix] * a.tab.W[iy];
        if (ys >= a.Ly) return rw_hi * a.ip->ew_hi[ix] * a.tab.W[iy];
    } else {
        ys = wrap_index(ys, a.Ly);
    }
    return fwd_value<TF>(a, (long long)(iy * Q1 + ix) * a.plane + (long long)ys * a.pitch + xs, iy, ix);
}

// lambda_{t+1,i} at (x, y) = (S^T mu_{t+1})_i: reverse pull from the node the
// population streams to, or the wall term when it streams into a wall.
template <int N>
__device__ __forceinline__ double adj_pull(const AdjArgs &a, int x, int y, int ix, int iy)
{
    constexpr int Q1 = 2 * N + 1;
    const int xd = wrap_index(x + (ix - N), a.Lx);
    int yd = y + (iy - N);
    if (a.bc == GLBM_BC_WALLS) {
        if (yd < 0) return a.G[xd] * a.ip->inv_den;
        if (yd >= a.Ly) return a.G[a.Lx + xd] * a.ip->inv_den;
    } else {
        yd = wrap_index(yd, a.Ly);
    }
    return a.mu_in[(long long)(iy * Q1 + ix) * a.plane + (long long)yd * a.pitch + xd];
}

// G(x) of both walls from mu_{t+1}: one thread per column.
template <int N>
__global__ void k_adj_wall(const __grid_constant__ AdjArgs a)
{
    constexpr int Q1 = 2 * N + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.Lx) return;
    double glo = 0.0, ghi = 0.0;
    for (int ny = 1; ny <= N; ++ny) {
        const double wy = a.tab.W[N + ny];
        for (int k = 0; k < ny; ++k) {
            for (int ix = 0; ix < Q1; ++ix) {
                // emitted by the lower wall: velocity +ny into rows 0..ny-1
                glo += a.mu_in[(long long)((N + ny) * Q1 + ix) * a.plane + (long long)k * a.pitch + x] *
                       a.ip->ew_lo[ix] * wy;
                // emitted by the upper wall: velocity -ny into rows Ly-ny..Ly-1
                ghi += a.mu_in[(long long)((N - ny) * Q1 + ix) * a.plane +
                               (long long)(a.Ly - 1 - k) * a.pitch + x] *
                       a.ip->ew_hi[ix] * wy;
            }
        }
    }
    a.Gw[x] = glo;
    a.Gw[a.Lx + x] = ghi;
}

constexpr int ADJ_THREADS = 64;

template <int N, typename TF>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_step(const __grid_constant__ AdjArgs a)
{
    constexpr int Q1 = 2 * N + 1;
    __shared__ double red[GLBM_ADJ_NG][ADJ_THREADS];
    const int x = blockIdx.x * ADJ_THREADS + threadIdx.x;
    const int y = blockIdx.y;
    const bool active = x < a.Lx;
    const int xc = active ? x : a.Lx - 1;
    const InstParams &ip = *a.ip;
    const double om = ip.omega;
    const double theta = N / 3.0;

    double rw_lo = 0.0, rw_hi = 0.0;
    if (a.bc == GLBM_BC_WALLS) {
        if (y < N) rw_lo = fwd_wall_density<N, TF>(a, xc, true);
        if (y >= a.Ly - N) rw_hi = fwd_wall_density<N, TF>(a, xc, false);
    }
    // forward moments of F_t at this node
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int iy = 0; iy < Q1; ++iy)
        for (int ix = 0; ix < Q1; ++ix) {
            const double f = fwd_pull<N, TF>(a, xc, y, ix, iy, rw_lo, rw_hi);
            rho += f;
            jx += (ix - N) * f;
            jy += (iy - N) * f;
        }
    const double ux = jx / rho, uy = jy / rho;
    double Ex[Q1], dEx[Q1], Ey[Q1], dEy[Q1];
    eq_and_slope<N>(a.tab, ux, Ex, dEx);
    eq_and_slope<N>(a.tab, uy, Ey, dEy);

    // contractions of lambda_{t+1} with the equilibrium and its slopes
    double a0 = 0.0, ax = 0.0, ay = 0.0, gt = 0.0, gg = 0.0;
    for (int iy = 0; iy < Q1; ++iy)
        for (int ix = 0; ix < Q1; ++ix) {
            const double lam = adj_pull<N>(a, xc, y, ix, iy);
            const double f = fwd_pull<N, TF>(a, xc, y, ix, iy, rw_lo, rw_hi);
            const double E = Ex[ix] * Ey[iy];
            a0 = fma(lam, E, a0);
            ax = fma(lam, dEx[ix] * Ey[iy], ax);
            ay = fma(lam, Ex[ix] * dEy[iy], ay);
            gt = fma(lam, rho * E - f, gt);
            gg = fma(lam, a.tab.W[ix] * a.tab.W[iy] * (ix - N), gg);
        }
    // mu_t = (dC/dF)^T lambda at this node (the density cancels: d f^eq_i / d f_j =
    // E_i + sum_a dE_i/du_a (xi_j,a - u_a))
    // and the wall speeds' term of F_t: mu_t of every ghost this node pulls
    // from a wall, times rho_w dE^x/du(u_w) W^y
    double glo = 0.0, ghi = 0.0;
    if (active) {
        for (int iy = 0; iy < Q1; ++iy)
            for (int ix = 0; ix < Q1; ++ix) {
                const double lam = adj_pull<N>(a, xc, y, ix, iy);
                const double m = (1.0 - om) * lam +
                                 om * (a0 + ax * ((ix - N) - ux) + ay * ((iy - N) - uy));
                a.mu_out[(long long)(iy * Q1 + ix) * a.plane + (long long)y * a.pitch + x] = m;
                if (a.bc == GLBM_BC_WALLS) {
                    const int ys = y - (iy - N);
                    if (ys < 0) glo = fma(m * rw_lo * ip.dew_lo[ix], a.tab.W[iy], glo);
                    if (ys >= a.Ly) ghi = fma(m * rw_hi * ip.dew_hi[ix], a.tab.W[iy], ghi);
                }
            }
    }
    // gradient partials of this block, summed in a fixed order
    red[0][threadIdx.x] = active ? -om * om * gt : 0.0;
    red[1][threadIdx.x] = active ? gg / theta : 0.0;
    red[2][threadIdx.x] = glo;
    red[3][threadIdx.x] = ghi;
    __syncthreads();
    for (int s = ADJ_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < GLBM_ADJ_NG; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
        for (int k = 0; k < GLBM_ADJ_NG; ++k) a.gpart[GLBM_ADJ_NG * b + k] += red[k][0];
    }
}

// The wall speeds' term of F_T = S(X_T): mu_T = xi_x / Lx (the seed) at every
// ghost a wall emits, times rho_w(X_T) dE^x/du(u_w) W^y, one thread per column,
// added to the partials of the blocks of row 0 (the grid of k_adj_step's first
// row), in a fixed order.
template <int N, typename TF>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_final_walls(const __grid_constant__ AdjArgs a)
{
    constexpr int Q1 = 2 * N + 1;
    __shared__ double red[2][ADJ_THREADS];
    const int x = blockIdx.x * ADJ_THREADS + threadIdx.x;
    const InstParams &ip = *a.ip;
    double glo = 0.0, ghi = 0.0;
    if (x < a.Lx) {
        const double rlo = fwd_wall_density<N, TF>(a, x, true);
        const double rhi = fwd_wall_density<N, TF>(a, x, false);
        for (int ny = 1; ny <= N; ++ny) {
            const double wy = a.tab.W[N + ny];
            for (int k = 0; k < ny; ++k)  // rows 0..ny-1 (lower), Ly-ny..Ly-1 (upper)
                for (int ix = 0; ix < Q1; ++ix) {
                    const double mu = (double)(ix - N) / a.Lx;
                    glo = fma(mu * rlo * ip.dew_lo[ix], wy, glo);
                    ghi = fma(mu * rhi * ip.dew_hi[ix], wy, ghi);
                }
        }
    }
    red[0][threadIdx.x] = glo;
    red[1][threadIdx.x] = ghi;
    __syncthreads();
    for (int s = ADJ_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.gpart[GLBM_ADJ_NG * blockIdx.x + 2] += red[0][0];
        a.gpart[GLBM_ADJ_NG * blockIdx.x + 3] += red[1][0];
    }
}

// mu_T = xi_x / Lx at every node, zero in the padding.
template <int N>
__global__ void k_adj_seed(const __grid_constant__ AdjArgs a)
{
    constexpr int Q1 = 2 * N + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int q = blockIdx.z;
    if (x >= a.pitch) return;
    const double v = x < a.Lx ? (double)(q % Q1 - N) / a.Lx : 0.0;
    a.mu_out[(long long)q * a.plane + (long long)y * a.pitch + x] = v;
}

__global__ void k_adj_sum(const double *gpart, long long nblocks, double *out)
{
    if (threadIdx.x < GLBM_ADJ_NG) {
        double s = 0.0;
        for (long long b = 0; b < nblocks; ++b) s += gpart[GLBM_ADJ_NG * b + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <int N>
cudaError_t adj_step_n(const AdjArgs &a, cudaStream_t s)
{
    k_adj_wall<N><<<(a.Lx + 63) / 64, 64, 0, s>>>(a);
    dim3 grid((a.Lx + ADJ_THREADS - 1) / ADJ_THREADS, a.Ly);
    if (a.prec == GLBM_FP64)
        k_adj_step<N, double><<<grid, ADJ_THREADS, 0, s>>>(a);
    else
        k_adj_step<N, float><<<grid, ADJ_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t adj_final_walls_n(const AdjArgs &a, cudaStream_t s)
{
    if (a.bc != GLBM_BC_WALLS) return cudaSuccess;
    const int blocks = (a.Lx + ADJ_THREADS - 1) / ADJ_THREADS;
    if (a.prec == GLBM_FP64)
        k_adj_final_walls<N, double><<<blocks, ADJ_THREADS, 0, s>>>(a);
    else
        k_adj_final_walls<N, float><<<blocks, ADJ_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t adj_seed_n(const AdjArgs &a, cudaStream_t s)
{
    dim3 grid((a.pitch + 127) / 128, a.Ly, (2 * N + 1) * (2 * N + 1));
    k_adj_seed<N><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

long long glbm_adj_blocks(int Lx, int Ly)
{
    return (long long)((Lx + ADJ_THREADS - 1) / ADJ_THREADS) * Ly;
}

cudaError_t glbm_launch_adj_seed(const AdjArgs &a, cudaStream_t s)
{
    switch (a.N) {
#define GLBM_CASE(NN) \
    case NN: return adj_seed_n<NN>(a, s);
        GLBM_CASE(1) GLBM_CASE(2) GLBM_CASE(3) GLBM_CASE(4)
        GLBM_CASE(5) GLBM_CASE(6) GLBM_CASE(7) GLBM_CASE(8)
#undef GLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_adj_final_walls(const AdjArgs &a, cudaStream_t s)
{
    switch (a.N) {
#define GLBM_CASE(NN) \
    case NN: return adj_final_walls_n<NN>(a, s);
        GLBM_CASE(1) GLBM_CASE(2) GLBM_CASE(3) GLBM_CASE(4)
        GLBM_CASE(5) GLBM_CASE(6) GLBM_CASE(7) GLBM_CASE(8)
#undef GLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_adj_step(const AdjArgs &a, cudaStream_t s)
{
    switch (a.N) {
#define GLBM_CASE(NN) \
    case NN: return adj_step_n<NN>(a, s);
        GLBM_CASE(1) GLBM_CASE(2) GLBM_CASE(3) GLBM_CASE(4)
        GLBM_CASE(5) GLBM_CASE(6) GLBM_CASE(7) GLBM_CASE(8)
#undef GLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_adj_sum(const double *gpart, long long nblocks, double *out, cudaStream_t s)
{
    k_adj_sum<<<1, 32, 0, s>>>(gpart, nblocks, out);
    return cudaGetLastError();
}
