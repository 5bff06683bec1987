// Fused pull-stream + BGK collide for the 2D tensor-product Gaussian lattices
// (Sec. 2, Eq. maineq01, product equilibrium of Sec. 4), with the diffuse
// walls' density computed in a CTA prologue and the linearised body force
// (Sec. 5.4).
//
// One CTA covers a tile of 32 columns x R rows of one instance. Each node's
// (2N+1)^2 populations are split by velocity row (ny) over G warps, so a
// thread holds at most ceil((2N+1)/G) * (2N+1) values in registers:
//   phase 0 (CTAs touching a wall): per column, the mass streaming into each
//           wall is summed from the previous post-collision state and turned
//           into the wall density rho_w(x) (emission balances absorption);
//   phase 1: pull every population f_i(x - xi_i) (coalesced 32-wide loads per
//           velocity plane, periodic wrap in x; sources inside a wall take the
//           wall's re-emitted value rho_w(x) E^x_i(u_w) W^y_i), then partial
//           moments (density and momentum) per velocity row;
//   phase 2: partial moments exchanged through shared memory (fixed order),
//           u = j / rho, equilibrium polynomials by Horner, relaxation plus
//           force, and a coalesced store of each population at its own node.
// FP32 mode stores deviations delta f = f - W (rest density 1) and adds the
// moments with compensated row sums; FP64 mode stores f.
// ZY / ZX select the 2N+2 hierarchy (Sec. 4, zero velocity removed) along y /
// x: that axis has 2N+2 velocity indices i with the odd velocities
// v = 2i - (2N+1) on a lattice of half the spacing (AxisVel).
// GUO replaces the linearised force by the force of Guo, Zheng and Shi (Phys.
// Rev. E 65, 046308, 2002), which the paper does not use: u = (j + g/2) / rho
// in the equilibrium and F_i = (1 - omega/2) W_i [(xi_i - u).G + (xi_i.U)
// (xi_i.G)] with G = (g / theta_x, 0), U_a = u_a / theta_a.
#pragma once
#include "glbm_device.cuh"

template <int N, typename T, int G, int R, int NXL = N, int ZY = 0, int ZX = 0, bool GUO = false>
struct Step2D {
    using AY = AxisVel<N, ZY>;
    using AX = AxisVel<NXL, ZX>;
    static constexpr int Q1 = AY::Q;              // velocity rows (level N along y)
    static constexpr int QX = AX::Q;              // velocity columns (level NXL along x)
    static constexpr int RPG = (Q1 + G - 1) / G;  // velocity rows per warp group
    static constexpr int NW = G * R;              // warps per CTA
    static constexpr int NT = 32 * NW;
    static constexpr int NV = 4;                  // wall-flux accumulators
    static constexpr bool DX_SHARED = G > 1 && sizeof(T) == 4;  // E^x - W read from smem
    static constexpr bool DEV = sizeof(T) == 4;   // FP32 deviation storage
    using A = TabAcc<T>;

    struct Smem {
        T part[R][G][6][32];  // (s, c) pairs of delta rho, j_x, j_y per row and group
        T rw[2][32];          // wall density (FP64) or its deviation (FP32): lo, hi
        T dsum[NV][2][32];    // partial wall fluxes of the NV accumulators
        // E^x - W and E^y - W of the tile's nodes, shared by the warp groups
        T eqx[G > 1 ? R : 1][G > 1 ? QX : 1][32];
        T eqy[G > 1 ? R : 1][G > 1 ? Q1 : 1][32];
    };

    // Wall densities of the columns of cofs (phase 0): for each wall flagged,
    // the mass streaming into it, summed over the pairs (velocity, row) with
    // row < |ny| from the previous post-collision state fin, becomes rho_w(x)
    // (FP64) or rho_w(x) - 1 (FP32) in rw[0] (y = -1/2) or rw[1] (y = Ly - 1/2).
    // The pairs are enumerated in order of |ny| and summed by NV fixed
    // accumulators (pair number mod NV) that the nw warps share round robin, so
    // the order of the additions depends neither on the tile shape nor on the
    // launch. U pairs of an accumulator are loaded before they are added (more
    // loads in flight, same order of additions): the tiles' prologue keeps
    // U = 1 and its loops rolled (the code must not grow), k_wall_rho takes
    // more. Every thread of the CTA calls it.
    template <int U = 1>
    __device__ static void wall_densities(const InstParams &ip, const T *__restrict__ fin, int Ly,
                                          int pitch, int plane, const int (&cofs)[QX], bool need_lo,
                                          bool need_hi, int w, int nw, int lane,
                                          T (&dsum)[NV][2][32], T (&rw)[2][32])
    {
#pragma unroll 1
        for (int v = w; v < NV; v += nw) {
            T slo = T(0), shi = T(0);
#pragma unroll 1
            for (int p0 = v; p0 < AY::NPAIR; p0 += U * NV) {
                T vlo[U][QX], vhi[U][QX];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * NV;
                    if (p < AY::NPAIR) {
                        int m = AY::M0, k = p;
                        while (k >= AY::vmag(m)) {
                            k -= AY::vmag(m);
                            ++m;
                        }
                        if (need_lo) {  // velocity ny = -|v_m| leaving row k through y = -1/2
                            const T *pl = fin + (AY::ineg(m) * QX * plane + k * pitch);
#pragma unroll
                            for (int ix = 0; ix < QX; ++ix) vlo[u][ix] = ld_pop(pl + cofs[ix]);
                        }
                        if (need_hi) {  // velocity ny = +|v_m| leaving row Ly-1-k through y = Ly-1/2
                            const T *ph = fin + (AY::ipos(m) * QX * plane + (Ly - 1 - k) * pitch);
#pragma unroll
                            for (int ix = 0; ix < QX; ++ix) vhi[u][ix] = ld_pop(ph + cofs[ix]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (p0 + u * NV < AY::NPAIR) {
#pragma unroll
                        for (int ix = 0; ix < QX; ++ix) {
                            if (need_lo) slo += vlo[u][ix];
                            if (need_hi) shi += vhi[u][ix];
                        }
                    }
                }
            }
            dsum[v][0][lane] = slo;
            dsum[v][1][lane] = shi;
        }
        __syncthreads();
        if (w == 0) {
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                s0 += dsum[j][0][lane];
                s1 += dsum[j][1][lane];
            }
            const T inv_den = DEV ? (T)ip.inv_den_f : (T)ip.inv_den;
            // FP64: rho_w = D / den.  FP32: rho_w - 1 = (D - den) / den, and
            // D - den is the sum of the absorbed deviations.
            rw[0][lane] = s0 * inv_den;
            rw[1][lane] = s1 * inv_den;
        }
        __syncthreads();
    }

    // Loads of this warp group's velocity rows iy = g + k G of the pull, all
    // independent (rows beyond a wall clamp to the edge row; their values are
    // replaced by the wall's emission afterwards).
    __device__ static void pull_rows(const T *__restrict__ fin, int g, int yc, int Ly, int pitch,
                                     int plane, bool walls, const int (&cofs)[QX],
                                     T (&f)[RPG][QX])
    {
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int iy = g + k * G;
            if (iy < Q1) {
                const int ny = AY::vel(iy);
                int ys = yc - ny;
                ys = walls ? min(max(ys, 0), Ly - 1) : wrap_shift(ys, Ly, Ly > AY::VMAX);
                const T *rowp = fin + (iy * QX * plane + ys * pitch);
#pragma unroll
                for (int ix = 0; ix < QX; ++ix) f[k][ix] = ld_pop(rowp + cofs[ix]);
            }
        }
    }

    // One tile: columns x0..x0+31, rows y0..y0+R-1 of one instance whose
    // populations start at fin / fout; tab is the y axis's table, tabx the x
    // axis's (the same table for isotropic lattices). rwg, when set, holds the
    // instance's wall densities (rwg[x] at y = -1/2, rwg[pitch + x] at
    // y = Ly - 1/2) from k_wall_rho, and phase 0 is skipped. Every thread
    // calls it.
    template <class TY, class TX>
    __device__ static void run(const TY &tab, const TX &tabx, const InstParams &ip,
                               int Lx, int Ly,
                               int pitch, int plane, int bc, const T *__restrict__ fin,
                               T *__restrict__ fout, int x0, int y0, Smem &sm, unsigned *status,
                               unsigned seed, const T *__restrict__ rwg = nullptr,
                               bool live = true)
    {
        const int lane = threadIdx.x & 31;
        const int w = threadIdx.x >> 5;
        const int g = w % G;
        const int r = w / G;
        // plane < 2^31 / Q: instance offsets fit 31 bits (checked at creation)
        const bool walls = bc == GLBM_BC_WALLS;
        const int x = x0 + lane, y = y0 + r;
        // live: no earlier step halted the run (else nothing is stored)
        const bool active = (x < Lx) && (y < Ly) && live;
        const int xc = x < Lx ? x : Lx - 1;
        const int yc = y < Ly ? y : Ly - 1;

        // offset of velocity column ix's plane plus its periodic source column
        int cofs[QX];
#pragma unroll
        for (int ix = 0; ix < QX; ++ix)
            cofs[ix] = ix * plane + wrap_shift(xc - AX::vel(ix), Lx, Lx > AX::VMAX);

        // ---- phase 0: wall densities of this tile's columns ---------------
        // (read from rwg instead when a separate launch computed them)
        const bool need_lo = walls && (y0 < AY::VMAX);
        const bool need_hi = walls && (y0 + R > Ly - AY::VMAX);
        if ((need_lo || need_hi) && !rwg)
            wall_densities(ip, fin, Ly, pitch, plane, cofs, need_lo, need_hi, w, NW, lane, sm.dsum,
                           sm.rw);

        // ---- phase 1: pull and partial moments -----------------------------
        // This warp's velocity rows are iy = g + k G (k = 0..RPG-1): the row is a
        // run-time value while the register array f[k][ix] keeps compile-time
        // indices, so all G warp groups share one copy of the unrolled code.
        T f[RPG][QX];
        T s_r = T(0), c_r = T(0), s_x = T(0), c_x = T(0), s_y = T(0), c_y = T(0);
        // loads first, all independent
        pull_rows(fin, g, yc, Ly, pitch, plane, walls, cofs, f);
        // wall re-emission and row sums
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int iy = g + k * G;
            if (iy < Q1) {
                const int ny = AY::vel(iy);
                const int ys = yc - ny;
                if (walls && (ys < 0 || ys >= Ly)) {  // uniform across the warp
                    const bool lo = ys < 0;
                    const T wy = A::W(tab, iy);
                    const T rw = rwg ? __ldg(rwg + (lo ? xc : pitch + xc)) : sm.rw[lo ? 0 : 1][lane];
#pragma unroll
                    for (int ix = 0; ix < QX; ++ix) {
                        if (DEV) {
                            const T dw = lo ? (T)ip.dw_lo_f[ix] : (T)ip.dw_hi_f[ix];
                            // W^y (drho_w W^x + (E^x(u_w) - W^x) + drho_w (E^x(u_w) - W^x)):
                            // no rounded 1 + drho_w scales the emitted momentum
                            f[k][ix] = mul_rn(wy, fma(rw, A::W(tabx, ix), fma(rw, dw, dw)));
                        } else {
                            const T ew = lo ? (T)ip.ew_lo[ix] : (T)ip.ew_hi[ix];
                            f[k][ix] = mul_rn(rw * ew, wy);
                        }
                    }
                }
                T rs = T(0);
#pragma unroll
                for (int ix = 0; ix < QX; ++ix) rs += f[k][ix];
                T jx = T(0);
#pragma unroll
                for (int m = AX::M0; m <= NXL; ++m)
                    jx = fma(T(AX::vmag(m)), f[k][AX::ipos(m)] - f[k][AX::ineg(m)], jx);
                acc2(s_r, c_r, rs);
                acc2(s_x, c_x, jx);
                if (ny != 0) acc2(s_y, c_y, mul_rn(T(ny), rs));
            }
        }
        // ---- phase 2: moments, equilibrium, relaxation, store --------------
        T S_r = T(0), C_r = T(0), S_x = T(0), C_x = T(0), S_y = T(0), C_y = T(0);
        if constexpr (G == 1) {
            // one warp group holds a node's every row: its own sums are the
            // node's (adding them to zero as below changes nothing), so no
            // exchange and no barrier
            S_r = s_r;
            S_x = s_x;
            S_y = s_y;
            if (DEV) {
                C_r = c_r;
                C_x = c_x;
                C_y = c_y;
            }
        } else {
            sm.part[r][g][0][lane] = s_r;
            sm.part[r][g][1][lane] = c_r;
            sm.part[r][g][2][lane] = s_x;
            sm.part[r][g][3][lane] = c_x;
            sm.part[r][g][4][lane] = s_y;
            sm.part[r][g][5][lane] = c_y;
            __syncthreads();
#pragma unroll
            for (int gi = 0; gi < G; ++gi) {
                acc2(S_r, C_r, sm.part[r][gi][0][lane]);
                acc2(S_x, C_x, sm.part[r][gi][2][lane]);
                acc2(S_y, C_y, sm.part[r][gi][4][lane]);
                if (DEV) {
                    C_r += sm.part[r][gi][1][lane];
                    C_x += sm.part[r][gi][3][lane];
                    C_y += sm.part[r][gi][5][lane];
                }
            }
        }
        const T m0 = S_r + C_r;            // FP32: delta rho; FP64: rho
        const T rho = DEV ? T(1) + m0 : m0;
        const T drho = DEV ? m0 : m0 - T(1);
        const T inv_rho = T(1) / rho;
        T jx = S_x + C_x;
        const T jy = S_y + C_y;
        // Guo's form: the equilibrium takes u = (j + g/2) / rho
        const T gh = GUO ? (DEV ? (T)ip.g_half_f : (T)ip.g_half) : T(0);
        if constexpr (GUO) jx += gh;
        T ux = jx * inv_rho, uy = jy * inv_rho;
        // random word of this node and launch for the dithered FP32 roundings
        const unsigned hnode = DEV ? hash32((unsigned)(y * Lx + x) ^ seed) : 0u;
        if constexpr (DEV) {
            // u = j / (1 + delta rho) from the unrounded density, rounded
            // stochastically: one correction by the residual (j - u) - u delta rho
            // (S - u is exact) plus a dither of half an ulp of u, so that the
            // rounding error of u (and of the equilibrium's momentum rho u) is
            // zero-mean instead of repeating at every step of a steady flow. j
            // times the rounded reciprocal alone misses by up to 2^-24 of u, with
            // a fixed sign where rho lies just below 1.
            const T dux = dither_ulp(ux, dither_unit(dither_word_ux(hnode)));
            const T duy = dither_ulp(uy, dither_unit(dither_word_uy(hnode)));
            // (the residual takes the compensated sum S + C unrounded)
            T rx = (S_x - ux) + C_x;
            if constexpr (GUO) rx += gh;
            ux = fma(fma(-ux, drho, rx) + dux, inv_rho, ux);
            uy = fma(fma(-uy, drho, (S_y - uy) + C_y) + duy, inv_rho, uy);
        }
        if (active) {
            // sqrt(2/3) N per axis: positivity bound (Sec. 3), twice that in
            // the half-spacing units of a 2N+2 axis
            const T umax = (T)(0.816496580927726 * (ZY ? 2 * N : N));
            const T umaxx = (T)(0.816496580927726 * (ZX ? 2 * NXL : NXL));
            if (!(rho > T(0)) || !(fabs(ux) <= umaxx) || !(fabs(uy) <= umax)) flag_unstable(status);
        }

        T dx[QX];
        T dyall[G == 1 ? Q1 : 1];  // one warp group: E^y - W for every row at once
        // FP32: the polynomial values are rounded stochastically, one draw per
        // node and axis (eq_pm_sr)
        const float rex = DEV ? dither_unit2(dither_word_ex(hnode)) : 0.0f;
        const float rey_ = DEV ? dither_unit2(dither_word_ey(hnode)) : 0.0f;
        if constexpr (G == 1) {
            if constexpr (DEV) {
                eq_dev_all_sr<NXL, ZX>(tabx, ux, rex, dx);
                eq_dev_all_sr<N, ZY>(tab, uy, rey_, dyall);
            } else {
                eq_dev_all<NXL, T, ZX>(tabx, ux, dx);
                eq_dev_all<N, T, ZY>(tab, uy, dyall);
            }
        } else {
            // the G warp groups of a node row share the polynomial work: group g
            // evaluates E^x - W and E^y - W for |n| = g, g + G, ..., and the
            // values meet in shared memory
            const T vx = ux * ux, vy = uy * uy;
#pragma unroll
            for (int n = 0; n <= (N > NXL ? N : NXL); ++n) {
                if (n % G != g) continue;
                T ae, bo, b0, dp, dm;
                if (n <= NXL) {
                    const bool single = n == 0 && !ZX;  // the zero velocity
                    if constexpr (DEV) {
                        eq_pm_sr<NXL, ZX>(tabx, n, ux, vx, rex, dp, dm);
                    } else {
                        eq_parts<NXL, T, ZX>(tabx, n, vx, ae, bo, b0);
                        eq_pm(ux, ae, bo, b0, dp, dm);
                        if (single) dp = ae;
                    }
                    sm.eqx[r][AX::ipos(n)][lane] = dp;
                    if (!single) sm.eqx[r][AX::ineg(n)][lane] = dm;
                }
                if (n <= N) {
                    const bool single = n == 0 && !ZY;
                    if constexpr (DEV) {
                        eq_pm_sr<N, ZY>(tab, n, uy, vy, rey_, dp, dm);
                    } else {
                        eq_parts<N, T, ZY>(tab, n, vy, ae, bo, b0);
                        eq_pm(uy, ae, bo, b0, dp, dm);
                        if (single) dp = ae;
                    }
                    sm.eqy[r][AY::ipos(n)][lane] = dp;
                    if (!single) sm.eqy[r][AY::ineg(n)][lane] = dm;
                }
            }
            __syncthreads();
            if constexpr (!DX_SHARED) {
#pragma unroll
                for (int ix = 0; ix < QX; ++ix) dx[ix] = sm.eqx[r][ix][lane];
            }
        }
        T ex[QX];  // FP64 mode: E^x = W + d^x
#pragma unroll
        for (int ix = 0; ix < QX; ++ix) ex[ix] = DEV ? T(0) : A::W(tabx, ix) + dx[ix];
        const T om = DEV ? (T)ip.omega_f : (T)ip.omega;
        const T gto = DEV ? (T)ip.g_theta_om_f : (T)ip.g_theta_om;  // g / (theta omega)
        const T cyv = GUO ? uy * T(1.0 / AY::THETA) : T(0);        // Guo: U_y = u_y / theta_y
        if (!live) return;  // an earlier step halted the run: store nothing
        // rows past Ly store into the plane's spare row y = Ly, columns past
        // Lx into the row padding (pitch is a multiple of 64): no store needs a
        // per-node condition, and nothing ever reads those places
        T *const obase = fout + ((y < Ly ? y : Ly) * pitch + x);
        // the store's dither enters the equilibrium divided by omega (below)
        const float iom = DEV ? 1.0f / ip.omega_f : 0.0f;

        // f* = f + omega (f^eq + F/omega - f): the relaxation is written as a
        // correction to f (no rounded (1 - omega) factor biases mass or momentum)
        // and the force F_i = W^x_i xi_x W^y_i g/theta joins the equilibrium
        // through the per-row factor gr = W^y g / (theta omega).
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int iy = g + k * G;
            if (iy < Q1) {
                const T wy = A::W(tab, iy), nwy = -wy;
                T dy;
                if constexpr (G == 1)
                    dy = dyall[k];
                else
                    dy = sm.eqy[r][iy][lane];
                const T rey = rho * (wy + dy);  // rho e^y
                const T gr = mul_rn(gto, wy);
                // Guo's form: F_i / omega = W^x_i (v_x grA + ck_i grB) with
                // grA = gr (1 + v_y U_y), grB = gr u_x, ck_i = v_x^2 / theta_x - 1
                T grA = gr, grB = T(0);
                if constexpr (GUO) {
                    grA = fma(gr, T(AY::vel(iy)) * cyv, gr);
                    grB = gr * ux;
                }
                // FP32: delta f^eq = d^x W^y + E^x B with B = rho e^y - W^y =
                // drho W^y + d^y + drho d^y: the y momentum's carrier d^y is not
                // scaled by a rounded rho
                const T B = DEV ? fma(drho, wy, fma(drho, dy, dy)) : T(0);
                T *const op = obase + iy * QX * plane;
                // random word of this row: node word plus a multiple of the row;
                // the row's two dither draws, divided by omega
                const unsigned hrow = hnode + (unsigned)iy * 0x85EBCA6Bu;
                const float ua = DEV ? mul_rn(dither_unit(hrow), iom) : 0.0f;
                const float ub = DEV ? mul_rn(dither_unit(dither_word_b(hrow)), iom) : 0.0f;
                if constexpr (DEV) {
                    // velocity columns in pairs (ix, ix + 1) on the two-lane FP32
                    // instructions: each lane does exactly the scalar operations
                    // below, in the same order, so the results are those of the
                    // scalar loop bit for bit; the last column of an odd count
                    // takes the scalar loop
                    const f32x2 B2 = pk2(B, B), nwy2 = pk2(nwy, nwy), om2 = pk2(om, om),
                                gr2 = pk2(grA, grA), grB2 = pk2(grB, grB);
#pragma unroll
                    for (int ix = 0; ix + 1 < QX; ix += 2) {
                        const f32x2 f0 = pk2(f[k][ix], f[k][ix + 1]);
                        const f32x2 Bn =
                            GUO ? fma2(pk2(T(AX::vel(ix)), T(AX::vel(ix + 1))), gr2,
                                       fma2(pk2(T(AX::ck(ix)), T(AX::ck(ix + 1))), grB2, B2))
                                : fma2(pk2(T(AX::vel(ix)), T(AX::vel(ix + 1))), gr2, B2);
                        const f32x2 dxv = DX_SHARED ? pk2(sm.eqx[r][ix][lane], sm.eqx[r][ix + 1][lane])
                                                    : pk2(dx[ix], dx[ix + 1]);
                        const float p0 = __int_as_float(__float_as_int(lo2(f0)) & 0x7F800000);
                        const float p1 = __int_as_float(__float_as_int(hi2(f0)) & 0x7F800000);
                        const f32x2 dith = mul2(pk2(dither_pick(ix, ua, ub, -ua, -ub),
                                                    dither_pick(ix + 1, ua, ub, -ua, -ub)),
                                                pk2(p0, p1));
                        const f32x2 t1 = fma2(dxv, B2, fma2(pk2(A::W(tabx, ix), A::W(tabx, ix + 1)), Bn, dith));
                        const f32x2 rr = fma2(dxv, nwy2, f0);
                        const f32x2 v2 = fma2(om2, sub2(t1, rr), f0);
                        op[ix * plane] = lo2(v2);
                        op[(ix + 1) * plane] = hi2(v2);
                    }
                }
#pragma unroll
                for (int ix = (DEV ? QX - (QX & 1) : 0); ix < QX; ++ix) {
                    const int nx = AX::vel(ix);
                    const T f0 = f[k][ix];
                    T v;
                    if (DEV) {
                        const T Bn = GUO ? fma(T(nx), grA, fma(T(AX::ck(ix)), grB, B))
                                         : (nx != 0 ? fma(T(nx), gr, B) : B);
                        // split FP32 tiles read E^x - W where it is used (fewer registers)
                        const T dxv = DX_SHARED ? sm.eqx[r][ix][lane] : dx[ix];
                        // delta f^eq = d^x W^y + E^x B + F/omega: the momentum-
                        // carrying d^x meets only the float weight W^y (whose row
                        // sum is exactly 1); a rounded rho e^y there would scale
                        // the momentum by a fixed 1 + O(2^-24) at every step of a
                        // steady flow. f^eq is never rounded at the scale of f:
                        // r = f0 - d^x W^y cancels (one fused rounding, of a small
                        // value when the flow runs along x), t1 holds the rest of
                        // f^eq plus the dither (half an ulp of f0, over omega),
                        // and the store f0 + omega (t1 - r) is one rounding that
                        // sees the whole dither: zero-mean.
                        const float u = dither_pick(ix, ua, ub, -ua, -ub);
                        const T dith = (T)dither_ulp((float)f0, u);
                        const T t1 = fma(dxv, B, fma(A::W(tabx, ix), Bn, dith));
                        const T r = fma(dxv, nwy, f0);
                        v = fma(om, t1 - r, f0);
                    } else {
                        // f^eq - f0 in one fused rounding, then the force term,
                        // then f0 + omega (f^eq + F/omega - f0): three FP64
                        // instructions (two without a force term)
                        T d = fma(ex[ix], rey, -f0);
                        if constexpr (GUO)
                            d = fma(A::W(tabx, ix), fma(T(nx), grA, T(AX::ck(ix)) * grB), d);
                        else if (nx != 0)
                            d = fma(A::WN(tabx, ix), gr, d);
                        v = fma(om, d, f0);
                    }
                    op[ix * plane] = v;
                }
            }
        }
    }
};

template <int N, typename T, int G, int R, int NXL = N, int ZY = 0, int ZX = 0, bool GUO = false>
__global__ void __launch_bounds__(32 * G * R)
    k_step2d(const __grid_constant__ Step2DArgsOf<N> a)
{
    using S = Step2D<N, T, G, R, NXL, ZY, ZX, GUO>;
    __shared__ typename S::Smem sm;
    const int inst = blockIdx.z;
    const bool df = a.bands != nullptr;  // dataflow chunk (glbm_internal.h)
    if (df) {
        df_launch_next();
        if (a.node > 0) {
            constexpr int V = S::AY::VMAX;
            const int y0 = blockIdx.y * R;
            df_wait_rows(a.bands, a.status, inst, y0 - V, y0 + R - 1 + V, a.Ly, R,
                         a.bc != GLBM_BC_WALLS, (unsigned)a.node * gridDim.x);
        }
    } else {
        wait_prior_grid();
    }
    // read here, needed only at the stores: no CTA waits for it before its loads
    const bool live = !step_halted(a.status);
    const T *fin = static_cast<const T *>(a.fin) + (long long)inst * a.inst_stride;
    T *fout = static_cast<T *>(a.fout) + (long long)inst * a.inst_stride;
    // the step clock: the launch counter (read before any CTA of this launch
    // can advance it), or the chunk's base plus this step's index
    const unsigned clk = df ? __ldcg(a.status + ST_BASE) + (unsigned)a.node : __ldcg(a.step_ctr);
    const unsigned seed = S::DEV ? hash32(clk * 0x632BE5ABu + inst) : 0u;
    const T *rwg = a.rw ? static_cast<const T *>(a.rw) + (long long)inst * 2 * a.pitch : nullptr;
    if constexpr (NXL == N && ZX == ZY)
        S::run(a.tab, a.tab, a.ip[inst], a.Lx, a.Ly, a.pitch, (int)a.plane, a.bc, fin, fout,
               blockIdx.x * 32, blockIdx.y * R, sm, a.status, seed, rwg, live);
    else
        S::run(a.tab, a.tabx, a.ip[inst], a.Lx, a.Ly, a.pitch, (int)a.plane, a.bc, fin, fout,
               blockIdx.x * 32, blockIdx.y * R, sm, a.status, seed, rwg, live);
    if (df) {
        df_tile_done(a.bands, inst);
        if (live) finish_step_df(a.status, a.node_done + a.node);
    } else if (live) {
        finish_step(a.status);
    }
}

// Wall densities of one step computed once per column and wall, for lattices
// whose tiles within reach of a wall would otherwise each repeat the sums of
// phase 0 (the step launched next reads them through Step2DArgs::rw). Grid
// (ceil(Lx / 32), instances, 2 walls) of NV warps; writes rho_w (FP64) or
// rho_w - 1 (FP32) of column x and wall h (0: y = -1/2, 1: y = Ly - 1/2) at
// rw[(inst * 2 + h) * pitch + x]. The sums are those of phase 0, in the same
// order, so the step's result does not depend on which of the two ran.
template <int N, typename T, int NXL, int ZY, int ZX>
__global__ void __launch_bounds__(32 * Step2D<N, T, 1, 1, NXL, ZY, ZX>::NV)
    k_wall_rho(const __grid_constant__ Step2DArgsOf<N> a)
{
    using S = Step2D<N, T, 1, 1, NXL, ZY, ZX>;
    using AX = typename S::AX;
    __shared__ T dsum[S::NV][2][32];
    __shared__ T rw[2][32];
    wait_prior_grid();
    const bool live = !step_halted(a.status);  // needed only at the store
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inst = blockIdx.y, h = blockIdx.z;
    const int x = blockIdx.x * 32 + lane;
    const int xc = x < a.Lx ? x : a.Lx - 1;
    const T *fin = static_cast<const T *>(a.fin) + (long long)inst * a.inst_stride;
    int cofs[S::QX];
#pragma unroll
    for (int ix = 0; ix < S::QX; ++ix)
        cofs[ix] = ix * (int)a.plane + wrap_shift(xc - AX::vel(ix), a.Lx, a.Lx > AX::VMAX);
    // up to 192 bytes of loads (U pairs) in flight per thread
    constexpr int LMAX = 192 / (int)sizeof(T);
    constexpr int U = S::QX >= LMAX ? 1 : LMAX / S::QX;
    S::template wall_densities<U>(a.ip[inst], fin, a.Ly, a.pitch, (int)a.plane, cofs, h == 0, h == 1,
                                  w, S::NV, lane, dsum, rw);
    if (w == 0 && x < a.Lx && live)
        static_cast<T *>(a.rw)[((long long)inst * 2 + h) * a.pitch + x] = rw[h][lane];
}
