// Fused pull-stream + BGK collide for the 3D tensor-product lattices (Sec. 4:
// the product of 1D levels on three axes, D3Q(2N+1)^3), with the diffuse
// walls at y = -1/2 and y = Ly - 1/2 (periodic in x and z), the linearised
// body force along x (Sec. 5.4) and the FP32-deviation or FP64 storage of the
// 2D step.
//
// One CTA covers 32 columns x R rows of one z-slice of one instance. A node's
// (2N+1)^3 populations form (2N+1)^2 velocity rows (n_z, n_y) of 2N+1
// columns (n_x); the rows are dealt to G warps, so a thread keeps
// ceil((2N+1)^2 / G) (2N+1) values in registers. Phases as in the 2D tile:
//   phase 0 (CTAs touching a wall): the mass streaming into each wall per
//           (x, z) column, turned into the wall density rho_w(x, z);
//   phase 1: pull (periodic in x and z; sources inside a wall take the
//           wall's emission rho_w E^x(u_w) W^y W^z), partial moments;
//   phase 2: moments, E - W per axis, relaxation plus force, store.
// The equilibrium deviation is built row by row:
//   delta f^eq = d^x rho e^y e^z + W^x (rho e^y e^z - W^y W^z),
//   rho e^y e^z - W^y W^z = d^y rho e^z + W^y (drho W^z + rho d^z),
// with e = W + d per axis.
#pragma once
#include "glbm_step2d.cuh"

template <int N, typename T, int G, int R>
struct Step3D {
    static constexpr int Q1 = 2 * N + 1;
    static constexpr int NROW = Q1 * Q1;               // velocity rows (n_z, n_y)
    static constexpr int RPG = (NROW + G - 1) / G;     // rows per warp group
    static constexpr int NW = G * R;
    static constexpr int NV = 4;                       // wall-flux accumulators
    static constexpr bool DEV = sizeof(T) == 4;
    using A = TabAcc<T>;
    // With G == 2N+1 warp groups, group g holds the rows (n_z = k - N, n_y = g - N):
    // n_z is a compile-time index of the unrolled loop and n_y is fixed per thread.
    static constexpr bool ZROW = G == Q1;
    __device__ static int row_z(int row, int k) { return ZROW ? k : row / Q1; }
    __device__ static int row_y(int row, int g) { return ZROW ? g : row % Q1; }

    struct Smem {
        T part[R][G][8][32];  // (s, c) of delta rho, j_x, j_y, j_z per row and group
        T rw[2][32];          // wall density (FP64) or its deviation (FP32): lo, hi
        T dsum[NV][2][32];
    };

    __device__ static void run(const AxisTable &tab, const InstParams &ip, int Lx, int Ly, int Lz,
                               int pitch, int plane, int bc, const T *__restrict__ fin,
                               T *__restrict__ fout, int x0, int y0, int z, Smem &sm,
                               unsigned *status, unsigned seed, bool live = true)
    {
        const int lane = threadIdx.x & 31;
        const int w = threadIdx.x >> 5;
        const int g = w % G;
        const int r = w / G;
        const bool walls = bc == GLBM_BC_WALLS;
        const int x = x0 + lane, y = y0 + r;
        // live: no earlier step halted the run (else nothing is stored)
        const bool active = (x < Lx) && (y < Ly) && live;
        const int xc = x < Lx ? x : Lx - 1;
        const int yc = y < Ly ? y : Ly - 1;
        const int slab = Ly * pitch;  // elements per z-slice of a velocity plane

        int cofs[Q1];
#pragma unroll
        for (int ix = 0; ix < Q1; ++ix) cofs[ix] = ix * plane + wrap_shift(xc - (ix - N), Lx, Lx > N);

        // ---- phase 0: wall densities of this tile's (x, z) columns ----------
        const bool need_lo = walls && (y0 < N);
        const bool need_hi = walls && (y0 + R > Ly - N);
        if (need_lo || need_hi) {
            // (n_y, row) pairs with row < |n_y| in order of |n_y|, each over
            // every n_z, through NV fixed accumulators (order independent of
            // the tile shape)
#pragma unroll 1
            for (int v = w; v < NV; v += NW) {
                T slo = T(0), shi = T(0);
#pragma unroll 1
                for (int p = v; p < N * (N + 1) / 2 * Q1; p += NV) {
                    const int iz = p % Q1;
                    int aa = 1, k = p / Q1;
                    while (k >= aa) {
                        k -= aa;
                        ++aa;
                    }
                    const int zs = wrap_shift(z - (iz - N), Lz, Lz > N);
                    if (need_lo) {  // n_y = -aa leaving row k through y = -1/2
                        const T *pl = fin + ((iz * Q1 + N - aa) * Q1 * plane + zs * slab + k * pitch);
#pragma unroll
                        for (int ix = 0; ix < Q1; ++ix) slo += __ldg(pl + cofs[ix]);
                    }
                    if (need_hi) {  // n_y = +aa leaving row Ly-1-k through y = Ly-1/2
                        const T *ph =
                            fin + ((iz * Q1 + N + aa) * Q1 * plane + zs * slab + (Ly - 1 - k) * pitch);
#pragma unroll
                        for (int ix = 0; ix < Q1; ++ix) shi += __ldg(ph + cofs[ix]);
                    }
                }
                sm.dsum[v][0][lane] = slo;
                sm.dsum[v][1][lane] = shi;
            }
            __syncthreads();
            if (w == 0) {
                T s0 = T(0), s1 = T(0);
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    s0 += sm.dsum[j][0][lane];
                    s1 += sm.dsum[j][1][lane];
                }
                const T inv_den = DEV ? (T)ip.inv_den_f : (T)ip.inv_den;
                sm.rw[0][lane] = s0 * inv_den;
                sm.rw[1][lane] = s1 * inv_den;
            }
            __syncthreads();
        }

        // ---- phase 1: pull and partial moments -----------------------------
        T f[RPG][Q1];
        T s_r = T(0), c_r = T(0), s_x = T(0), c_x = T(0), s_y = T(0), c_y = T(0), s_z = T(0),
          c_z = T(0);
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int row = g + k * G;
            if (row < NROW) {
                const int iz = row_z(row, k), iy = row_y(row, g);
                int ys = yc - (iy - N);
                ys = walls ? min(max(ys, 0), Ly - 1) : wrap_shift(ys, Ly, Ly > N);
                const int zs = wrap_shift(z - (iz - N), Lz, Lz > N);
                const T *rowp = fin + (row * Q1 * plane + zs * slab + ys * pitch);
#pragma unroll
                for (int ix = 0; ix < Q1; ++ix) f[k][ix] = __ldg(rowp + cofs[ix]);
            }
        }
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int row = g + k * G;
            if (row < NROW) {
                const int iz = row_z(row, k), iy = row_y(row, g);
                const int ny = iy - N, nz = iz - N;
                const int ys = yc - ny;
                if (walls && (ys < 0 || ys >= Ly)) {  // uniform across the warp
                    const bool lo = ys < 0;
                    const T wyz = mul_rn(A::W(tab, iy), A::W(tab, iz));
                    const T rw = sm.rw[lo ? 0 : 1][lane];
#pragma unroll
                    for (int ix = 0; ix < Q1; ++ix) {
                        if (DEV) {
                            const T dw = lo ? (T)ip.dw_lo_f[ix] : (T)ip.dw_hi_f[ix];
                            // no rounded 1 + drho_w scales the emitted momentum
                            f[k][ix] = mul_rn(wyz, fma(rw, A::W(tab, ix), fma(rw, dw, dw)));
                        } else {
                            const T ew = lo ? (T)ip.ew_lo[ix] : (T)ip.ew_hi[ix];
                            f[k][ix] = mul_rn(rw * ew, wyz);
                        }
                    }
                }
                T rs = T(0);
#pragma unroll
                for (int ix = 0; ix < Q1; ++ix) rs += f[k][ix];
                T jx = T(0);
#pragma unroll
                for (int n = 1; n <= N; ++n) jx = fma(T(n), f[k][N + n] - f[k][N - n], jx);
                acc2(s_r, c_r, rs);
                acc2(s_x, c_x, jx);
                if (ny != 0) acc2(s_y, c_y, mul_rn(T(ny), rs));
                if (nz != 0) acc2(s_z, c_z, mul_rn(T(nz), rs));
            }
        }
        {
            T *pp = &sm.part[r][g][0][lane];
            pp[0 * 32] = s_r;
            pp[1 * 32] = c_r;
            pp[2 * 32] = s_x;
            pp[3 * 32] = c_x;
            pp[4 * 32] = s_y;
            pp[5 * 32] = c_y;
            pp[6 * 32] = s_z;
            pp[7 * 32] = c_z;
        }
        __syncthreads();

        // ---- phase 2: moments, equilibrium, relaxation, store --------------
        T S_r = T(0), C_r = T(0), S_x = T(0), C_x = T(0), S_y = T(0), C_y = T(0), S_z = T(0),
          C_z = T(0);
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
            const T *pp = &sm.part[r][gi][0][lane];
            acc2(S_r, C_r, pp[0 * 32]);
            acc2(S_x, C_x, pp[2 * 32]);
            acc2(S_y, C_y, pp[4 * 32]);
            acc2(S_z, C_z, pp[6 * 32]);
            if (DEV) {
                C_r += pp[1 * 32];
                C_x += pp[3 * 32];
                C_y += pp[5 * 32];
                C_z += pp[7 * 32];
            }
        }
        const T m0 = S_r + C_r;
        const T rho = DEV ? T(1) + m0 : m0;
        const T drho = DEV ? m0 : m0 - T(1);
        const T inv_rho = T(1) / rho;
        const T jx = S_x + C_x, jy = S_y + C_y, jz = S_z + C_z;
        T ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
        const unsigned hnode = DEV ? hash32((unsigned)((z * Ly + y) * Lx + x) ^ seed) : 0u;
        if constexpr (DEV) {
            // u = j / (1 + delta rho), rounded stochastically (as in the 2D tile):
            // j times the rounded reciprocal alone carries a fixed relative bias
            // of up to 2^-24 where rho lies just below 1
            const T dux = dither_ulp(ux, dither_unit(dither_word_ux(hnode)));
            const T duy = dither_ulp(uy, dither_unit(dither_word_uy(hnode)));
            const T duz = dither_ulp(uz, dither_unit(dither_word_uz(hnode)));
            ux = fma(fma(-ux, drho, (S_x - ux) + C_x) + dux, inv_rho, ux);
            uy = fma(fma(-uy, drho, (S_y - uy) + C_y) + duy, inv_rho, uy);
            uz = fma(fma(-uz, drho, (S_z - uz) + C_z) + duz, inv_rho, uz);
        }
        if (active) {
            const T umax = (T)(0.816496580927726 * N);  // sqrt(2/3) N (Sec. 3)
            if (!(rho > T(0)) || !(fabs(ux) <= umax) || !(fabs(uy) <= umax) || !(fabs(uz) <= umax))
                flag_unstable(status);
        }
        T dx[Q1], dy[Q1], dz[Q1];
        if constexpr (DEV) {
            // polynomial values rounded stochastically, one draw per node and axis
            eq_dev_all_sr<N>(tab, ux, dither_unit2(dither_word_ex(hnode)), dx);
            eq_dev_all_sr<N>(tab, uy, dither_unit2(dither_word_ey(hnode)), dy);
            eq_dev_all_sr<N>(tab, uz, dither_unit2(dither_word_ez(hnode)), dz);
        } else {
            eq_dev_all<N, T>(tab, ux, dx);
            eq_dev_all<N, T>(tab, uy, dy);
            eq_dev_all<N, T>(tab, uz, dz);
#pragma unroll
            for (int ix = 0; ix < Q1; ++ix) dx[ix] += A::W(tab, ix);  // E^x, once per node
        }

        // ZROW: this thread's n_y deviation, selected once
        T dy_g = dy[0];
        if constexpr (ZROW) {
#pragma unroll
            for (int i = 1; i < Q1; ++i)
                if (g == i) dy_g = dy[i];
        }
        const T om = DEV ? (T)ip.omega_f : (T)ip.omega;
        const T gto = DEV ? (T)ip.g_theta_om_f : (T)ip.g_theta_om;  // g / (theta omega)
        if (!live) return;  // an earlier step halted the run: store nothing
        // rows past Ly store into the plane's spare row after its Lz Ly rows,
        // columns past Lx into the row padding (pitch is a multiple of 64): no
        // store needs a per-node condition, and nothing reads those places
        T *const obase = fout + ((y < Ly ? z * slab + y * pitch : Lz * slab) + x);
        const float iom = DEV ? 1.0f / ip.omega_f : 0.0f;  // the dither enters f^eq over omega
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int row = g + k * G;
            if (row < NROW) {
                const int iz = row_z(row, k), iy = row_y(row, g);
                const T wy = A::W(tab, iy), wz = A::W(tab, iz);
                // runtime row: the per-axis deviations by a select chain
                T dyv, dzv;
                if constexpr (ZROW) {
                    dzv = dz[k];
                    dyv = dy_g;
                } else {
                    dyv = dy[0];
                    dzv = dz[0];
#pragma unroll
                    for (int i = 1; i < Q1; ++i) {
                        if (iy == i) dyv = dy[i];
                        if (iz == i) dzv = dz[i];
                    }
                }
                const T rez = rho * (wz + dzv);       // rho e^z
                const T rez_y = rez * (wy + dyv);     // rho e^y e^z
                const T wyz = mul_rn(wy, wz);
                const T gr = mul_rn(gto, wyz);        // W^y W^z g / (theta omega)
                // FP32: B = rho e^y e^z - W^y W^z = d^y W^z + (W^y + d^y) Bz with
                // Bz = rho e^z - W^z = drho W^z + d^z + drho d^z: no momentum
                // carrier (d^y, d^z) is scaled by a rounded rho or e^y
                const T Bz = DEV ? fma(drho, wz, fma(drho, dzv, dzv)) : T(0);
                const T B = DEV ? fma(dyv, wz, fma(dyv, Bz, mul_rn(wy, Bz))) : T(0);
                T *const op = obase + row * Q1 * plane;
                const unsigned hrow = hnode + (unsigned)row * 0x85EBCA6Bu;
                // the row's dither draws, divided by omega
                const float ua = DEV ? mul_rn(dither_unit(hrow), iom) : 0.0f;
                const float ub = DEV ? mul_rn(dither_unit(dither_word_b(hrow)), iom) : 0.0f;
                if constexpr (DEV) {
                    // velocity columns in pairs (ix, ix + 1) on the two-lane FP32
                    // instructions, each lane doing exactly the scalar loop's
                    // operations in its order (bit-identical results); the last
                    // of the odd 2N+1 columns takes the scalar loop
                    const f32x2 B2 = pk2(B, B), gr2 = pk2(gr, gr), om2 = pk2(om, om),
                                nwy2 = pk2(-wy, -wy), wz2 = pk2(wz, wz);
#pragma unroll
                    for (int ix = 0; ix + 1 < Q1; ix += 2) {
                        const f32x2 f0 = pk2(f[k][ix], f[k][ix + 1]);
                        const f32x2 Bn = fma2(pk2(T(ix - N), T(ix + 1 - N)), gr2, B2);
                        const f32x2 dxv = pk2(dx[ix], dx[ix + 1]);
                        const float p0 = __int_as_float(__float_as_int(lo2(f0)) & 0x7F800000);
                        const float p1 = __int_as_float(__float_as_int(hi2(f0)) & 0x7F800000);
                        const f32x2 dith = mul2(pk2(dither_pick(ix, ua, ub, -ua, -ub),
                                                    dither_pick(ix + 1, ua, ub, -ua, -ub)),
                                                pk2(p0, p1));
                        const f32x2 t1 =
                            fma2(dxv, B2, fma2(pk2(A::W(tab, ix), A::W(tab, ix + 1)), Bn, dith));
                        const f32x2 rr = fma2(mul2(dxv, nwy2), wz2, f0);
                        const f32x2 v2 = fma2(om2, sub2(t1, rr), f0);
                        op[ix * plane] = lo2(v2);
                        op[(ix + 1) * plane] = hi2(v2);
                    }
                }
#pragma unroll
                for (int ix = (DEV ? Q1 - 1 : 0); ix < Q1; ++ix) {
                    const int nx = ix - N;
                    const T f0 = f[k][ix];
                    T v;
                    if (DEV) {
                        const T Bn = nx != 0 ? fma(T(nx), gr, B) : B;
                        // delta f^eq = d^x W^y W^z + E^x B + F/omega: the
                        // momentum-carrying d^x is rounded with W^y, then meets W^z
                        // in a fused rounding (no rounded rho or W^y W^z factor,
                        // whose fixed error would scale the momentum at every
                        // step); as in 2D, r = f0 - d^x W^y W^z, t1 holds the rest
                        // plus the dither (half an ulp of f0, over omega), and the
                        // store f0 + omega (t1 - r) is one rounding
                        const float u = dither_pick(ix, ua, ub, -ua, -ub);
                        const T dith = (T)dither_ulp((float)f0, u);
                        const T t1 = fma(dx[ix], B, fma(A::W(tab, ix), Bn, dith));
                        const T r = fma(-mul_rn(dx[ix], wy), wz, f0);  // f0 - d^x W^y W^z
                        v = fma(om, t1 - r, f0);
                    } else {
                        // dx holds E^x itself in FP64 mode; f^eq - f0 in one
                        // fused rounding, the force term, f0 + omega (...)
                        T d = fma(dx[ix], rez_y, -f0);
                        if (nx != 0) d = fma(A::WN(tab, ix), gr, d);
                        v = fma(om, d, f0);
                    }
                    op[ix * plane] = v;
                }
            }
        }
    }
};

template <int N, typename T, int G, int R>
__global__ void __launch_bounds__(32 * G * R) k_step3d(const __grid_constant__ Step3DArgs a)
{
    using S = Step3D<N, T, G, R>;
    __shared__ typename S::Smem sm;
    wait_prior_grid();
    const bool live = !step_halted(a.status);  // needed only at the stores
    const int inst = blockIdx.z / a.Lz;
    const int z = blockIdx.z - inst * a.Lz;
    const T *fin = static_cast<const T *>(a.fin) + (long long)inst * a.inst_stride;
    T *fout = static_cast<T *>(a.fout) + (long long)inst * a.inst_stride;
    const unsigned seed = S::DEV ? hash32(__ldcg(a.step_ctr) * 0x632BE5ABu + inst) : 0u;
    S::run(a.tab, a.ip[inst], a.Lx, a.Ly, a.Lz, a.pitch, (int)a.plane, a.bc, fin, fout,
           blockIdx.x * 32, blockIdx.y * R, z, sm, a.status, seed, live);
    if (live) finish_step(a.status);
}
