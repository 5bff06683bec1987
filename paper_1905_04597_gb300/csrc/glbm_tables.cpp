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
static void fix_identity(double *c, int N, int j)
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
    for (int n = 0; n <= N; ++n) big = fmax(big, 2.0 * (n + 1) * fabs(c[n]));
    if (ilogb(big) - emin > 120) return;  // span too wide for exact integers: keep as is
    __int128 S = 0;
    for (int n = 0; n <= N; ++n) {
        const __int128 I = (__int128)ldexp(c[n], -emin);  // exact integer
        const int mult = (j % 2 == 0) ? (n == 0 ? 1 : 2) : 2 * n;
        S += (__int128)mult * I;
    }
    const __int128 T = (__int128)ldexp(delta, -emin);
    const double R = ldexp((double)(T - S), emin);  // residual (rounded once)
    if (j % 2 == 0)
        c[0] += R;
    else
        c[1] += 0.5 * R;
}

void glbm_build_axis_table(int N, AxisTable *t, double *full)
{
    const int Q1 = 2 * N + 1;
    // poly[n + N][j]: coefficient of z^n u^j; sized for the largest level
    double cur[GLBM_MAXQ1][GLBM_MAXQ1];
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
        t->Wf[n + N] = (float)cur[n + N][0];
        t->WN[n + N] = n * cur[n + N][0];
        t->WNf[n + N] = (float)(n * cur[n + N][0]);
    }
    for (int n = 0; n <= N; ++n) {
        for (int i = 0; i <= N; ++i) {
            t->Ce[n][i] = cur[n + N][2 * i];
            t->Cef[n][i] = (float)cur[n + N][2 * i];
        }
        for (int i = 0; i < N; ++i) {
            t->Co[n][i] = cur[n + N][2 * i + 1];
            t->Cof[n][i] = (float)cur[n + N][2 * i + 1];
        }
        // FP32 keeps the linear coefficient as hi + lo so that the momentum
        // identity sum_n n C[n][1] = 1 is not broken by its rounding
        t->Co1lo[n] = (float)(cur[n + N][1] - (double)t->Cof[n][0]);
    }
    if (full) {
        for (int n = 0; n < Q1; ++n)
            for (int j = 0; j < Q1; ++j) full[n * Q1 + j] = cur[n][j];
    }
}
