// FP32-deviation form of the fused pull-stream + BGK collide tile (Sec. 2,
// Eq. maineq01, product equilibrium of Sec. 4, diffuse walls, linearised
// force of Sec. 5.4) working on PAIRS of x-adjacent nodes with the packed
// two-lane FP32 instructions of sm_100 and later (add/sub/mul/fma .f32x2).
//
// A thread owns nodes (x, y) and (x + 1, y), x even, and keeps each
// population of the two nodes in one 64-bit register pair (low word: node x).
// Every lane of a packed instruction is rounded exactly like the scalar
// instruction of the one-node tile (glbm_step2d.cuh), and the operations are
// done in the same order, so a pair tile and a one-node tile of the same G
// give bit-identical results. What the pairing saves is instructions: one
// packed op updates two populations, a pull whose velocity has even n_x is one
// 8-byte load, and the store of both nodes is one 8-byte store.
//
// A CTA covers 64 columns x R rows with G warps per node row (32 G R
// threads); phases as in the one-node tile:
//   phase 0 (CTAs touching a wall): wall densities of the tile's columns;
//   phase 1: pull every population of both nodes (periodic wrap in x; sources
//            inside a wall take the wall's re-emitted value), partial moments
//            per velocity row with compensated sums;
//   phase 2: moments, equilibrium, relaxation plus force, dithered store.
// ZY = 1 / ZX = 1 put the y / x axis on the 2N+2 hierarchy (Sec. 4, zero
// velocity removed: odd velocities on a half-spacing lattice).
#pragma once
#include "glbm_step2d.cuh"

// Wall densities of a pair tile's 64 columns (row a2 of the fused step): the
// mass streaming into each wall, summed through NV fixed accumulators (pair
// p mod NV of the (|n_y|, row) pairs) in the order of the one-node tile,
// whatever the tile shape; the NW warps of the CTA share the accumulators.
// Leaves rho_w - 1 of both walls in rw[2][64]. Every thread calls it.
template <int N, int NX, int NV, int ZY = 0, int ZX = 0>
__device__ __forceinline__ void pair_wall_densities(const InstParams &ip, const float *__restrict__ fin,
                                                    int Ly, int pitch, int plane, const int *win,
                                                    bool need_lo, bool need_hi, int w, int NW,
                                                    int lane, float (*dsum)[2][64], float (*rw)[64])
{
    using AY = AxisVel<N, ZY>;
    using AX = AxisVel<NX, ZX>;
    constexpr int Q1 = AX::Q;  // velocity columns (N: level along y)
#pragma unroll 1
    for (int v = w; v < NV; v += NW) {
        float slo0 = 0.f, slo1 = 0.f, shi0 = 0.f, shi1 = 0.f;
#pragma unroll 1
        for (int p = v; p < AY::NPAIR; p += NV) {
            int m = AY::M0, k = p;
            while (k >= AY::vmag(m)) {
                k -= AY::vmag(m);
                ++m;
            }
            if (need_lo) {  // velocity ny = -|v_m| leaving row k through y = -1/2
                const float *pl = fin + (AY::ineg(m) * Q1 * plane + k * pitch);
#pragma unroll
                for (int ix = 0; ix < Q1; ++ix) {
                    slo0 += ld_pop(pl + (ix * plane + win[AX::VMAX - AX::vel(ix)]));
                    slo1 += ld_pop(pl + (ix * plane + win[AX::VMAX - AX::vel(ix) + 1]));
                }
            }
            if (need_hi) {  // velocity ny = +|v_m| leaving row Ly-1-k through y = Ly-1/2
                const float *ph = fin + (AY::ipos(m) * Q1 * plane + (Ly - 1 - k) * pitch);
#pragma unroll
                for (int ix = 0; ix < Q1; ++ix) {
                    shi0 += ld_pop(ph + (ix * plane + win[AX::VMAX - AX::vel(ix)]));
                    shi1 += ld_pop(ph + (ix * plane + win[AX::VMAX - AX::vel(ix) + 1]));
                }
            }
        }
        dsum[v][0][2 * lane] = slo0;
        dsum[v][0][2 * lane + 1] = slo1;
        dsum[v][1][2 * lane] = shi0;
        dsum[v][1][2 * lane + 1] = shi1;
    }
    __syncthreads();
    if (w == 0) {
        const float inv_den = ip.inv_den_f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = 2 * lane + h;
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                s0 += dsum[j][0][col];
                s1 += dsum[j][1][col];
            }
            // rho_w - 1 = (D - den) / den: D - den is the absorbed deviation
            rw[0][col] = s0 * inv_den;
            rw[1][col] = s1 * inv_den;
        }
    }
    __syncthreads();
}

// Pull of one velocity row iy (source row ys) for a node pair: f[ix] holds
// both nodes' populations of x velocity index ix; N is the x level (ZX: its
// 2N+2 hierarchy). The window win[j] is column x - VMAX + j.
template <int N, int ZX = 0>
__device__ __forceinline__ void pair_load_row(const float *__restrict__ fin, int iy, int ys,
                                              int pitch, int plane, int x, bool inner,
                                              const int *win, f32x2 (&f)[2 * N + 1 + ZX])
{
    using AX = AxisVel<N, ZX>;
    constexpr int Q1 = AX::Q;
    const float *rowp = fin + (iy * Q1 * plane + ys * pitch);
    if (inner) {
#pragma unroll
        for (int ix = 0; ix < Q1; ++ix) {
            const int nx = AX::vel(ix);
            const float *p = rowp + (ix * plane + (x - nx));
            if ((nx & 1) == 0)  // (x - nx) even: one aligned 8-byte load
                f[ix] = ld_pop(reinterpret_cast<const f32x2 *>(p));
            else
                f[ix] = pk2(ld_pop(p), ld_pop(p + 1));
        }
    } else {
#pragma unroll
        for (int ix = 0; ix < Q1; ++ix) {
            const float *p = rowp + ix * plane;
            const int j = AX::VMAX - AX::vel(ix);
            f[ix] = pk2(ld_pop(p + win[j]), ld_pop(p + win[j + 1]));
        }
    }
}

// The populations a wall re-emits into velocity row iy of a node pair
// (sources inside the wall): W^y (drho_w W^x + rho_w (E^x(u_w) - W^x)).
template <int N, int ZX, class TY, class TX>
__device__ __forceinline__ void pair_wall_row(const TY &tab, const TX &tabx,
                                              const InstParams &ip, int iy, bool lo, float rw0,
                                              float rw1, f32x2 (&f)[2 * N + 1 + ZX])
{
    using A = TabAcc<float>;
    const float wy = A::W(tab, iy);  // tab: y axis; tabx and N: x axis
#pragma unroll
    for (int ix = 0; ix < 2 * N + 1 + ZX; ++ix) {
        const float dw = lo ? ip.dw_lo_f[ix] : ip.dw_hi_f[ix];
        const float wx = A::W(tabx, ix);
        // no rounded 1 + drho_w scales the emitted momentum (as in the one-node tile)
        f[ix] = pk2(mul_rn(wy, fmaf(rw0, wx, fmaf(rw0, dw, dw))),
                    mul_rn(wy, fmaf(rw1, wx, fmaf(rw1, dw, dw))));
    }
}

// Relaxation plus force and the dithered FP32 store of velocity row iy of a
// node pair: f* = f + omega (f^eq + F/omega - f) with
// delta f^eq = d^x W^y + E^x B, B = drho W^y + d^y + drho d^y, the force through the
// row factor gr = W^y g / (theta omega), and a dither of half an ulp from the
// two draws of each node's row word (h0, h1 and the row), taken in turn with
// alternating signs along the row. E^x - W comes from the
// registers dxr, or from shared memory at dxs (stride 32 pairs) when DXS.
// N and tabx: the x axis.
template <int N, bool DXS, int ZX, class TX>
__device__ __forceinline__ void pair_collide_row(const TX &tabx, int iy, float wy, f32x2 dy,
                                                 f32x2 drho, f32x2 om, float iom, float gto,
                                                 const f32x2 (&f)[2 * N + 1 + ZX],
                                                 const f32x2 (&dxr)[2 * N + 1 + ZX], const f32x2 *dxs,
                                                 float *op, int plane, unsigned h0, unsigned h1)
{
    using A = TabAcc<float>;
    const f32x2 wy2 = pk2(wy, wy), nwy2 = pk2(-wy, -wy);
    const float grs = mul_rn(gto, wy);
    const f32x2 gr = pk2(grs, grs);
    const f32x2 B = fma2(drho, wy2, fma2(drho, dy, dy));  // rho e^y - W^y
    const unsigned hr0 = h0 + (unsigned)iy * 0x85EBCA6Bu;  // row words
    const unsigned hr1 = h1 + (unsigned)iy * 0x85EBCA6Bu;
    // the row's two dither draws of each node (divided by omega) and their negatives
    const float a0 = mul_rn(dither_unit(hr0), iom), a1 = mul_rn(dither_unit(hr1), iom);
    const float b0 = mul_rn(dither_unit(dither_word_b(hr0)), iom);
    const float b1 = mul_rn(dither_unit(dither_word_b(hr1)), iom);
    const f32x2 ua = pk2(a0, a1), ub = pk2(b0, b1), na = pk2(-a0, -a1), nb = pk2(-b0, -b1);
#pragma unroll
    for (int ix = 0; ix < 2 * N + 1 + ZX; ++ix) {
        const int nx = AxisVel<N, ZX>::vel(ix);
        const f32x2 f0 = f[ix];
        const f32x2 Bn = nx != 0 ? fma2(pk2((float)nx, (float)nx), gr, B) : B;
        const float wx = A::W(tabx, ix);
        const f32x2 dxv = DXS ? dxs[ix * 32] : dxr[ix];
        // the one-node tile's order: t1 = d^x B + W^x Bn + dither / omega,
        // r = f0 - d^x W^y, one rounding of the store f0 + omega (t1 - r)
        const float p0 = __int_as_float(__float_as_int(lo2(f0)) & 0x7F800000);
        const float p1 = __int_as_float(__float_as_int(hi2(f0)) & 0x7F800000);
        const f32x2 dith = mul2(dither_pick(ix, ua, ub, na, nb), pk2(p0, p1));
        const f32x2 t1 = fma2(dxv, B, fma2(pk2(wx, wx), Bn, dith));
        const f32x2 r = fma2(dxv, nwy2, f0);
        const f32x2 v = fma2(om, sub2(t1, r), f0);
        // every thread stores both nodes: columns past Lx land in the row
        // padding, rows past Ly in the plane's spare row (the caller's op)
        *reinterpret_cast<f32x2 *>(op + ix * plane) = v;
    }
}

template <int N, int G, int R, int NXL = N, int ZY = 0, int ZX = 0>
struct Step2DPair {
    using AY = AxisVel<N, ZY>;
    using AX = AxisVel<NXL, ZX>;
    static constexpr int Q1 = AY::Q;              // velocity rows (level N along y)
    static constexpr int QX = AX::Q;              // velocity columns (level NXL along x)
    static constexpr int RPG = (Q1 + G - 1) / G;  // velocity rows per warp group
    static constexpr int NW = G * R;              // warps per CTA
    static constexpr int TW = 64;                 // tile width (columns)
    static constexpr int NWIN = 2 * AX::VMAX + 2; // source columns of a node pair
    static constexpr int NV = Step2D<N, float, G, R>::NV;  // wall-flux accumulators
    using A = TabAcc<float>;

    struct Smem {
        float part[R][G][6][TW];  // (s, c) of delta rho, j_x, j_y per row, group, column
        float rw[2][TW];          // wall density deviations: lo, hi
        float dsum[NV][2][TW];    // partial wall fluxes of the NV accumulators
        // E^x - W and E^y - W of the tile's nodes, shared by the warp groups
        float eqx[G > 1 ? R : 1][G > 1 ? QX : 1][TW];
        float eqy[G > 1 ? R : 1][G > 1 ? Q1 : 1][TW];
    };

    // One tile: columns x0..x0+63 (x0 a multiple of 64), rows y0..y0+R-1 of one
    // instance whose populations start at fin / fout (8-byte aligned planes);
    // tab is the y axis's table, tabx the x axis's (the same when isotropic).
    // rwg, when set, holds the instance's wall densities from k_wall_rho
    // (rwg[x] at y = -1/2, rwg[pitch + x] at y = Ly - 1/2).
    template <class TY, class TX>
    __device__ static void run(const TY &tab, const TX &tabx, const InstParams &ip,
                               int Lx, int Ly,
                               int pitch, int plane, int bc, const float *__restrict__ fin,
                               float *__restrict__ fout, int x0, int y0, Smem &sm,
                               unsigned *status, unsigned seed,
                               const float *__restrict__ rwg = nullptr, bool live = true)
    {
        const int lane = threadIdx.x & 31;
        const int w = threadIdx.x >> 5;
        const int g = w % G;
        const int r = w / G;
        const bool walls = bc == GLBM_BC_WALLS;
        const int x = x0 + 2 * lane, y = y0 + r;
        const bool yin = y < Ly;
        // live: no earlier step halted the run (else nothing is stored)
        const bool act0 = yin && x < Lx && live, act1 = yin && x + 1 < Lx && live;
        const int xc = x < Lx ? x : Lx - 1;
        const int yc = yin ? y : Ly - 1;
        // the tile pulls from columns x0-VMAX .. x0+63+VMAX without wrapping
        const bool inner = x0 >= AX::VMAX && x0 + TW + AX::VMAX <= Lx;

        // source columns of the pair: node x pulls velocity n_x from column
        // win[VMAX - n_x], node x + 1 from win[VMAX - n_x + 1]
        int win[NWIN];
        const bool one_wrap = Lx > AX::VMAX + 1;
#pragma unroll
        for (int j = 0; j < NWIN; ++j) win[j] = wrap_shift(xc - AX::VMAX + j, Lx, one_wrap);

        // ---- phase 0: wall densities of this tile's columns ---------------
        const bool need_lo = walls && (y0 < AY::VMAX);
        const bool need_hi = walls && (y0 + R > Ly - AY::VMAX);
        if ((need_lo || need_hi) && !rwg)  // else computed by k_wall_rho
            pair_wall_densities<N, NXL, NV, ZY, ZX>(ip, fin, Ly, pitch, plane, win, need_lo, need_hi,
                                                    w, NW, lane, sm.dsum, sm.rw);

        // ---- phase 1: pull and partial moments -----------------------------
        // rows iy = g + k G of this warp group; f[k][ix] holds both nodes
        f32x2 f[RPG][QX];
        f32x2 s_r = 0ull, c_r = 0ull, s_x = 0ull, c_x = 0ull, s_y = 0ull, c_y = 0ull;
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int iy = g + k * G;
            if (iy < Q1) {
                const int ny = AY::vel(iy);
                int ys = yc - ny;
                ys = walls ? min(max(ys, 0), Ly - 1) : wrap_shift(ys, Ly, Ly > AY::VMAX);
                pair_load_row<NXL, ZX>(fin, iy, ys, pitch, plane, x, inner, win, f[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int iy = g + k * G;
            if (iy < Q1) {
                const int ny = AY::vel(iy);
                const int ys = yc - ny;
                if (walls && (ys < 0 || ys >= Ly)) {  // uniform across the warp
                    const bool lo = ys < 0;
                    float rw0, rw1;
                    if (rwg) {
                        const float *rl = rwg + (lo ? 0 : pitch);
                        rw0 = __ldg(rl + xc);
                        rw1 = __ldg(rl + (x + 1 < Lx ? x + 1 : xc));
                    } else {
                        rw0 = sm.rw[lo ? 0 : 1][2 * lane];
                        rw1 = sm.rw[lo ? 0 : 1][2 * lane + 1];
                    }
                    pair_wall_row<NXL, ZX>(tab, tabx, ip, iy, lo, rw0, rw1, f[k]);
                }
                f32x2 rs = 0ull;
#pragma unroll
                for (int ix = 0; ix < QX; ++ix) rs = add2(rs, f[k][ix]);
                f32x2 jx = 0ull;
#pragma unroll
                for (int m = AX::M0; m <= NXL; ++m)
                    jx = fma2(pk2((float)AX::vmag(m), (float)AX::vmag(m)),
                              sub2(f[k][AX::ipos(m)], f[k][AX::ineg(m)]), jx);
                acc2x2(s_r, c_r, rs);
                acc2x2(s_x, c_x, jx);
                if (ny != 0)  // products rounded per lane, as in the one-node tile
                    acc2x2(s_y, c_y, pk2(mul_rn((float)ny, lo2(rs)), mul_rn((float)ny, hi2(rs))));
            }
        }
        {
            f32x2 *pp = reinterpret_cast<f32x2 *>(&sm.part[r][g][0][2 * lane]);
            constexpr int st = TW / 2;  // f32x2 stride between the six rows
            pp[0 * st] = s_r;
            pp[1 * st] = c_r;
            pp[2 * st] = s_x;
            pp[3 * st] = c_x;
            pp[4 * st] = s_y;
            pp[5 * st] = c_y;
        }
        __syncthreads();

        // ---- phase 2: moments, equilibrium, relaxation, store --------------
        f32x2 S_r = 0ull, C_r = 0ull, S_x = 0ull, C_x = 0ull, S_y = 0ull, C_y = 0ull;
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
            const f32x2 *pp = reinterpret_cast<const f32x2 *>(&sm.part[r][gi][0][2 * lane]);
            constexpr int st = TW / 2;
            acc2x2(S_r, C_r, pp[0 * st]);
            acc2x2(S_x, C_x, pp[2 * st]);
            acc2x2(S_y, C_y, pp[4 * st]);
            C_r = add2(C_r, pp[1 * st]);
            C_x = add2(C_x, pp[3 * st]);
            C_y = add2(C_y, pp[5 * st]);
        }
        const f32x2 drho = add2(S_r, C_r);  // delta rho of both nodes
        const f32x2 rho = add2(pk2(1.f, 1.f), drho);
        const f32x2 inv_rho = pk2(1.f / lo2(rho), 1.f / hi2(rho));
        const f32x2 jx = add2(S_x, C_x), jy = add2(S_y, C_y);
        f32x2 ux = mul2(jx, inv_rho), uy = mul2(jy, inv_rho);
        // random words of the two nodes and this launch (dithered roundings)
        const unsigned h0 = hash32((unsigned)(y * Lx + x) ^ seed);
        const unsigned h1 = hash32((unsigned)(y * Lx + x + 1) ^ seed);
        {
            // u = j / (1 + delta rho), rounded stochastically (the one-node
            // tile's correction and dither, lane by lane)
            constexpr f32x2 SIGN2 = 0x8000000080000000ull;
            const f32x2 dux = pk2(dither_ulp(lo2(ux), dither_unit(dither_word_ux(h0))),
                                  dither_ulp(hi2(ux), dither_unit(dither_word_ux(h1))));
            const f32x2 duy = pk2(dither_ulp(lo2(uy), dither_unit(dither_word_uy(h0))),
                                  dither_ulp(hi2(uy), dither_unit(dither_word_uy(h1))));
            ux = fma2(add2(fma2(ux ^ SIGN2, drho, add2(sub2(S_x, ux), C_x)), dux), inv_rho, ux);
            uy = fma2(add2(fma2(uy ^ SIGN2, drho, add2(sub2(S_y, uy), C_y)), duy), inv_rho, uy);
        }
        {
            // sqrt(2/3) N per axis (Sec. 3), twice that on a 2N+2 axis
            const float umax = (float)(0.816496580927726 * (ZY ? 2 * N : N));
            const float umaxx = (float)(0.816496580927726 * (ZX ? 2 * NXL : NXL));
            const bool bad0 = act0 && (!(lo2(rho) > 0.f) || !(fabsf(lo2(ux)) <= umaxx) ||
                                       !(fabsf(lo2(uy)) <= umax));
            const bool bad1 = act1 && (!(hi2(rho) > 0.f) || !(fabsf(hi2(ux)) <= umaxx) ||
                                       !(fabsf(hi2(uy)) <= umax));
            if (bad0 || bad1) flag_unstable(status);
        }

        // E^x - W and E^y - W for both nodes
        f32x2 dx[QX];
        float dy0all[G == 1 ? Q1 : 1], dy1all[G == 1 ? Q1 : 1];
        // polynomial values rounded stochastically: one draw per node and axis
        const float rx0 = dither_unit2(dither_word_ex(h0)), rx1 = dither_unit2(dither_word_ex(h1));
        const float ry0 = dither_unit2(dither_word_ey(h0)), ry1 = dither_unit2(dither_word_ey(h1));
        if constexpr (G == 1) {
            float d0[QX], d1[QX];
            eq_dev_all_sr<NXL, ZX>(tabx, lo2(ux), rx0, d0);
            eq_dev_all_sr<NXL, ZX>(tabx, hi2(ux), rx1, d1);
#pragma unroll
            for (int ix = 0; ix < QX; ++ix) dx[ix] = pk2(d0[ix], d1[ix]);
            eq_dev_all_sr<N, ZY>(tab, lo2(uy), ry0, dy0all);
            eq_dev_all_sr<N, ZY>(tab, hi2(uy), ry1, dy1all);
        } else {
            // the G warp groups share the polynomial work: group g evaluates
            // |n| = g, g + G, ... for both nodes and both axes, and the values
            // meet in shared memory
            const float u[4] = {lo2(ux), hi2(ux), lo2(uy), hi2(uy)};
            const float rr[4] = {rx0, rx1, ry0, ry1};
#pragma unroll
            for (int n = 0; n <= (N > NXL ? N : NXL); ++n) {
                if (n % G != g) continue;
                float plus[4], minus[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c < 2 ? n > NXL : n > N) continue;  // x nodes: level NXL; y: N
                    if (c < 2)
                        eq_pm_sr<NXL, ZX>(tabx, n, u[c], u[c] * u[c], rr[c], plus[c], minus[c]);
                    else
                        eq_pm_sr<N, ZY>(tab, n, u[c], u[c] * u[c], rr[c], plus[c], minus[c]);
                }
                if (n <= NXL) {
                    *reinterpret_cast<f32x2 *>(&sm.eqx[r][AX::ipos(n)][2 * lane]) =
                        pk2(plus[0], plus[1]);
                    if (n != 0 || ZX)
                        *reinterpret_cast<f32x2 *>(&sm.eqx[r][AX::ineg(n)][2 * lane]) =
                            pk2(minus[0], minus[1]);
                }
                if (n <= N) {
                    *reinterpret_cast<f32x2 *>(&sm.eqy[r][AY::ipos(n)][2 * lane]) =
                        pk2(plus[2], plus[3]);
                    if (n != 0 || ZY)
                        *reinterpret_cast<f32x2 *>(&sm.eqy[r][AY::ineg(n)][2 * lane]) =
                            pk2(minus[2], minus[3]);
                }
            }
            __syncthreads();  // E^x - W is read from shared memory where it is used
        }
        const f32x2 om = pk2(ip.omega_f, ip.omega_f);
        const float iom = 1.0f / ip.omega_f;
        const float gto = ip.g_theta_om_f;  // g / (theta omega)
        if (!live) return;  // an earlier step halted the run: store nothing
        // rows past Ly store into the plane's spare row y = Ly, columns past
        // Lx into the row padding (pitch is a multiple of 64): no store needs a
        // per-node condition, and nothing ever reads those places
        float *const obase = fout + ((yin ? y : Ly) * pitch + x);

#pragma unroll
        for (int k = 0; k < RPG; ++k) {
            const int iy = g + k * G;
            if (iy < Q1) {
                const float wy = A::W(tab, iy);
                f32x2 dy;
                if constexpr (G == 1)
                    dy = pk2(dy0all[k], dy1all[k]);
                else
                    dy = *reinterpret_cast<const f32x2 *>(&sm.eqy[r][iy][2 * lane]);
                const f32x2 *dxs = reinterpret_cast<const f32x2 *>(&sm.eqx[G > 1 ? r : 0][0][2 * lane]);
                pair_collide_row<NXL, (G > 1), ZX>(tabx, iy, wy, dy, drho, om, iom, gto, f[k], dx, dxs,
                                               obase + iy * QX * plane, plane, h0, h1);
            }
        }
    }
};

