// Equilibrium-coefficient table of one axis (built once per level N, FP64).
//
// The equilibrium of level N is the distribution of a sum of N independent
// three-outcome variables (Sec. 2): its generating function in z is
// (P- / z + P0 + P+ z)^N, and with P+- and P0 quadratic in the velocity u
// (Eqs. maineq04-05 in lattice units, c = 1, c_s^2 = N/3)
//   P+- = 1/6 +- u/(2N) + u^2/(2N^2),   P0 = 2/3 - u^2/N^2,
// each population E_n(u) is a polynomial of degree 2N in u. The table holds
// its coefficients, obtained by N exact convolutions of the quadratic
// trinomial (the N-fold summation itself); the kernels evaluate E_n by Horner
// and never touch factorials.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "glbm_internal.h"

// Make the conservation identity of column j hold to within half an ulp of
// its largest entry:
//   even j: sum_n C[n][j] = [j == 0]          (mass; c[0] absorbs the residual)
//   odd j:  sum_n n C[n][j] = [j == 1]        (momentum; c[+-1] absorb it)
// with c[n] = C[n][j] for n = 0..N and C[-n][j] = (-1)^j c[n]. The residual of
// the correctly rounded entries is computed exactly: every entry is an integer
// multiple of the smallest entry's ulp, so the weighted sum is an exact
// 128-bit integer. All other entries keep full relative precision.
// On the 2N+2 hierarchy (zv) c[m] belongs to the velocities +-(2m+1): the
// weights are 2 (mass) and 2 (2m+1) (momentum), and c[0] absorbs both.
static void fix_identity(double *c, int N, int j, bool zv = false)
{
    int emin = 0;
    bool any = false;
    for (int n = 0; n <= N; ++n) {
        if (c[n] == 0.0) continue;
        const int e = ilogb(c[n]) - 52;  // ulp exponent of c[n]
        if (!any || e < emin) emin = e;
        any = true;
    }
    if (!any) return;
    const double delta = (j == 0 || j == 1) ? 1.0 : 0.0;
    // largest magnitude of any term in units of 2^emin must fit the accumulator
    double big = fabs(delta);
    for (int n = 0; n <= N; ++n) big = fmax(big, (zv ? 4.0 : 2.0) * (n + 1) * fabs(c[n]));
    if (ilogb(big) - emin > 120) return;  // span too wide for exact integers: keep as is
    __int128 S = 0;
    for (int n = 0; n <= N; ++n) {
        const __int128 I = (__int128)ldexp(c[n], -emin);  // exact integer
        const int mult = zv ? ((j % 2 == 0) ? 2 : 2 * (2 * n + 1))
                            : ((j % 2 == 0) ? (n == 0 ? 1 : 2) : 2 * n);
        S += (__int128)mult * I;
    }
    const __int128 T = (__int128)ldexp(delta, -emin);
    const double R = ldexp((double)(T - S), emin);  // residual (rounded once)
    if (zv)
        c[0] += 0.5 * R;
    else if (j % 2 == 0)
        c[0] += R;
    else
        c[1] += 0.5 * R;
}

// Exact N-fold convolution: cur[n + N][j] = coefficient of z^n u^j.
static void convolve(int N, double (&cur)[GLBM_MAXQ1][GLBM_MAXQ1])
{
    const int Q1 = 2 * N + 1;
    double nxt[GLBM_MAXQ1][GLBM_MAXQ1];
    memset(cur, 0, sizeof(cur));
    cur[N][0] = 1.0;
    // trinomial factors: index 0 -> z^-1 (P-), 1 -> z^0 (P0), 2 -> z^+1 (P+);
    // each a quadratic in u with coefficients [u^0, u^1, u^2]
    const double inv2N = 1.0 / (2.0 * N), inv2N2 = 1.0 / (2.0 * N * (double)N);
    const double fac[3][3] = {
        {1.0 / 6.0, -inv2N, inv2N2},
        {2.0 / 3.0, 0.0, -2.0 * inv2N2},
        {1.0 / 6.0, inv2N, inv2N2},
    };
    for (int step = 0; step < N; ++step) {
        memset(nxt, 0, sizeof(nxt));
        for (int n = 0; n < Q1; ++n) {
            for (int j = 0; j < Q1; ++j) {
                double a = cur[n][j];
                if (a == 0.0) continue;
                for (int dz = 0; dz < 3; ++dz) {
                    int nn = n + dz - 1;
                    for (int dj = 0; dj < 3; ++dj) {
                        if (nn < 0 || nn >= Q1 || j + dj >= Q1) continue;
                        nxt[nn][j + dj] += a * fac[dz][dj];
                    }
                }
            }
        }
        memcpy(cur, nxt, sizeof(cur));
    }
}

// Exact value of a float in units of 2^-80 (the weights lie in (2^-40, 1)).
static __int128 float_units(float f) { return (__int128)ldexp((double)f, 80); }

// FP32 rest weights whose exact sum is 1 as closely as the floats allow. The
// weight sum of one axis multiplies the other axis's momentum in the FP32
// deviation equilibrium (delta f^eq = d^x rho e^y + W^x (...)), so a sum of
// 1 + eps would scale the momentum by 1 + eps at every collision (nearest
// rounding gives eps up to 4e-8; D1Q3: 1/6 + 2/3 + 1/6 = 1 + 3e-8). Starting
// from the nearest floats, the weight whose one-ulp move (a velocity and its
// mirror move together) brings the exact sum closest to 1 is moved, until no
// move helps; no weight moves more than 8 ulps.
static void balance_weights_f32(AxisTableHi *t, int Q)
{
    const int nd = (Q + 1) / 2;  // distinct weights: index i < nd and its mirror Q-1-i
    float w[GLBM_MAXN + 1];
    int mult[GLBM_MAXN + 1], moved[GLBM_MAXN + 1];
    __int128 R = -((__int128)1 << 80);  // sum - 1
    for (int j = 0; j < nd; ++j) {
        w[j] = (float)t->W[j];
        mult[j] = (j == Q - 1 - j) ? 1 : 2;
        moved[j] = 0;
        R += mult[j] * float_units(w[j]);
    }
    for (int it = 0; it < 16 * nd; ++it) {
        int bj = -1, bd = 0;
        __int128 bR = R;
        for (int j = 0; j < nd; ++j) {
            for (int d = -1; d <= 1; d += 2) {
                if (moved[j] + d > 8 || moved[j] + d < -8) continue;
                const float g = nextafterf(w[j], d > 0 ? 2.0f : 0.0f);
                const __int128 R2 = R + mult[j] * (float_units(g) - float_units(w[j]));
                const __int128 a2 = R2 < 0 ? -R2 : R2, ab = bR < 0 ? -bR : bR;
                if (a2 < ab) {
                    bj = j;
                    bd = d;
                    bR = R2;
                }
            }
        }
        if (bj < 0) break;
        w[bj] = nextafterf(w[bj], bd > 0 ? 2.0f : 0.0f);
        moved[bj] += bd;
        R = bR;
    }
    for (int j = 0; j < nd; ++j) t->Wf[j] = t->Wf[Q - 1 - j] = w[j];
}

// FP32 copies and the hi + lo split of the linear coefficient.
static void fill_f32(AxisTableHi *t, int Q)
{
    const int N = t->N;
    for (int i = 0; i < Q; ++i) t->WNf[i] = (float)t->WN[i];
    balance_weights_f32(t, Q);
    for (int n = 0; n <= N; ++n) {
        for (int i = 0; i <= N; ++i) t->Cef[n][i] = (float)t->Ce[n][i];
        for (int i = 0; i < N; ++i) t->Cof[n][i] = (float)t->Co[n][i];
        // FP32 keeps the linear coefficient as hi + lo so that the momentum
        // identity is not broken by its rounding
        t->Co1lo[n] = (float)(t->Co[n][0] - (double)t->Cof[n][0]);
    }
}

void glbm_build_axis_table(int N, AxisTableHi *t, double *full)
{
    const int Q1 = 2 * N + 1;
    // cur[n + N][j]: coefficient of z^n u^j; sized for the largest level
    double cur[GLBM_MAXQ1][GLBM_MAXQ1];
    convolve(N, cur);

    // conservation identities of the FP64 coefficients to half an ulp
    for (int j = 0; j < Q1; ++j) {
        double c[GLBM_MAXN + 1];
        for (int n = 0; n <= N; ++n) c[n] = cur[n + N][j];
        fix_identity(c, N, j);
        for (int n = 0; n <= N; ++n) {
            cur[n + N][j] = c[n];
            cur[N - n][j] = (j % 2 == 0) ? c[n] : -c[n];
        }
    }

    memset(t, 0, sizeof(*t));
    t->N = N;
    for (int n = -N; n <= N; ++n) {
        t->W[n + N] = cur[n + N][0];
        t->WN[n + N] = n * cur[n + N][0];
    }
    for (int n = 0; n <= N; ++n) {
        for (int i = 0; i <= N; ++i) t->Ce[n][i] = cur[n + N][2 * i];
        for (int i = 0; i < N; ++i) t->Co[n][i] = cur[n + N][2 * i + 1];
    }
    fill_f32(t, Q1);
    if (full) {
        for (int n = 0; n < Q1; ++n)
            for (int j = 0; j < Q1; ++j) full[n * Q1 + j] = cur[n][j];
    }
}

void glbm_build_axis_table_zv(int N, AxisTableHi *t)
{
    double cur[GLBM_MAXQ1][GLBM_MAXQ1];
    convolve(N, cur);
    // c[m][j]: coefficient of u^j of E_{2m+1}(u) = (E_m(u/2) + E_{m+1}(u/2)) / 2,
    // u in units of c/2 (E_{N+1} = 0); halving and the powers of two are exact,
    // the sum of the two neighbours is rounded once
    double c[GLBM_MAXN + 1][GLBM_MAXQ1];
    for (int m = 0; m <= N; ++m)
        for (int j = 0; j <= 2 * N; ++j) {
            const double hi = m + 1 <= N ? cur[m + 1 + N][j] : 0.0;
            c[m][j] = ldexp(cur[m + N][j] + hi, -(j + 1));
        }
    for (int j = 0; j <= 2 * N; ++j) {
        double col[GLBM_MAXN + 1];
        for (int m = 0; m <= N; ++m) col[m] = c[m][j];
        fix_identity(col, N, j, true);
        for (int m = 0; m <= N; ++m) c[m][j] = col[m];
    }
    memset(t, 0, sizeof(*t));
    t->N = N;
    t->zv = 1;
    for (int m = 0; m <= N; ++m) {
        const int ip = N + 1 + m, in = N - m, v = 2 * m + 1;
        t->W[ip] = t->W[in] = c[m][0];
        t->WN[ip] = v * c[m][0];
        t->WN[in] = -v * c[m][0];
        for (int i = 0; i <= N; ++i) t->Ce[m][i] = c[m][2 * i];
        for (int i = 0; i < N; ++i) t->Co[m][i] = c[m][2 * i + 1];
    }
    fill_f32(t, 2 * N + 2);
}

double glbm_eq_dev_host(const AxisTableHi &t, double u, int i)
{
    const int N = t.N;
    const int v = ax_vel(t, i);
    const int m = t.zv ? (abs(v) - 1) / 2 : abs(v);
    const double w = u * u;
    double ae = t.Ce[m][N];
    for (int k = N - 1; k >= 1; --k) ae = fma(ae, w, t.Ce[m][k]);
    ae *= w;
    double bo = 0.0;
    if (v != 0) {
        bo = t.Co[m][N - 1];
        for (int k = N - 2; k >= 0; --k) bo = fma(bo, w, t.Co[m][k]);
    }
    return v >= 0 ? fma(u, bo, ae) : fma(-u, bo, ae);
}

AxisTable glbm_narrow_table(const AxisTableHi &t)
{
    AxisTable o;
    memset(&o, 0, sizeof(o));
    o.N = t.N;
    o.zv = t.zv;
    const int M = GLBM_MAXN_2N1;
    for (int i = 0; i < 2 * M + 2; ++i) {
        o.W[i] = t.W[i];
        o.WN[i] = t.WN[i];
        o.Wf[i] = t.Wf[i];
        o.WNf[i] = t.WNf[i];
    }
    for (int n = 0; n <= M; ++n) {
        for (int i = 0; i <= M; ++i) {
            o.Ce[n][i] = t.Ce[n][i];
            o.Cef[n][i] = t.Cef[n][i];
        }
        for (int i = 0; i < M; ++i) {
            o.Co[n][i] = t.Co[n][i];
            o.Cof[n][i] = t.Cof[n][i];
        }
        o.Co1lo[n] = t.Co1lo[n];
    }
    return o;
}
