/*
 * glbm_oracle.c -- plain FP64 CPU oracle for the Gaussian lattice Boltzmann
 * method of O. Ilyin, "Gaussian Lattice Boltzmann method and its applications
 * to rarefied flows" (arXiv:1905.04597).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or helper with the CUDA path:
 *   - the equilibrium is evaluated at every node from the factorial sum of
 *     Sec. 2 (Eq. maineq03 with Eqs. maineq04-05), never from a polynomial
 *     coefficient table;
 *   - streaming is written in push form (each population is moved from its
 *     source node); the CUDA path pulls.
 *
 * Units. Lattice units per axis: node spacing c(N)*dt = 1 and dt = 1, so the
 * discrete velocities of level N are the integers n = -N..N and the lattice
 * temperature is theta = c_s^2 = N/3 (Eq. maineq05 with c = 1).
 *
 * Time stepping. The state X_t is the array of post-collision populations.
 * One step is X_{t+1} = C(S(X_t)) with S the streaming (including boundary
 * rules) and C the BGK collision of Eq. maineq01 with frequency
 * 1/(tau + 1/2). The macroscopic fields "at time t" are the moments of the
 * streamed populations S(X_t).
 *
 * Layout. Populations f[q][y][x], x fastest, q = (ny+NY)*(2NX+1) + (nx+NX)
 * for the 2D tensor-product lattice (Sec. 4) and q = n+N in 1D; on the 2N+2
 * lattices below, q = iy*Qx + ix with the velocity indices of each axis.
 *
 * The 2N+2 hierarchy (Sec. 4, "zero velocity is removed"): the velocities
 * (n + 1/2) c, n = 0..N, and (n - 1/2) c, n = -N..0, with the equilibrium of
 * each taken as the mean of the 2N+1 hierarchy's equilibria at the two
 * neighbouring velocities (Eqs. maineq01_noball - maineq04_noball). Written on
 * a lattice of spacing c/2, its velocities are the odd integers -(2N+1) ..
 * 2N+1, the 2N+1 equilibria are evaluated at u/c = u/2, and the lattice
 * temperature is (4N+3)/3 (Eq. temp_2N2 with c = 2). 2D lattices only, per
 * axis (orc_cfg.zv): the paper's channel models G-D1Q6 x D1Q3 and
 * G-D1Q8 x D1Q3 take it along the wall normal y only, G-D2Q784 along both.
 *
 * 3D lattices (Sec. 4: the product extends to any number of axes) take the
 * product of three 1D levels, q = (iz Qy + iy) Qx + ix and f[q][z][y][x],
 * periodic in x and z, walls (or periodicity) in y as in 2D; the wall
 * re-emits rho_w(x, z) E^x(u_w) E^y(0) E^z(0).
 *
 * Boundary readings (the paper cites its wall condition but states no
 * formula; Sec. 5.3-5.4):
 *   - walls sit halfway between nodes, at y = -1/2 and y = Ly - 1/2;
 *   - diffuse (kinetic) reflection: every population that streams into a wall
 *     is absorbed and its mass is attributed to the column x it would have
 *     reached; the wall re-emits, into every (node, velocity) whose source lies
 *     inside the wall, rho_w(x) * E^x_{nx}(u_w) * E^y_{ny}(0), with rho_w(x)
 *     chosen so that the emitted mass equals the absorbed mass of column x;
 *   - 1D ends use halfway bounce-back;
 *   - the body force is F_i = W_i * xi_{x,i} * g / theta_x added after the
 *     relaxation (the linearised force of Sec. 5.4 written for the lattice
 *     used along the flow);
 *   - or, when orc_cfg.guo is set, the force of Guo, Zheng and Shi (Phys.
 *     Rev. E 65, 046308, 2002), which the paper does not use: the
 *     equilibrium and the reported velocity take u = (j + g/2) / rho, and
 *     F_i = (1 - omega/2) W_i [(xi_i - u).G + (xi_i.U)(xi_i.G)] with
 *     G_a = g_a / theta_a and U_a = u_a / theta_a per axis (Guo's second-order
 *     Hermite form, c_s^2 replaced by each axis's temperature). g is a force
 *     density in both forms: each injects exactly g of x momentum per node and
 *     step (here omega g/2 through the relaxation towards the shifted u and
 *     (1 - omega/2) g through F).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_N 16

enum { ORC_BC_WALLS = 0, ORC_BC_BOUNCEBACK = 1, ORC_BC_PERIODIC = 2 };
enum { ORC_ZV_X = 1, ORC_ZV_Y = 2 };

/* Configuration of one lattice; mirrored by a ctypes.Structure in oracle.py. */
typedef struct {
    int dims;  /* 1 or 2 */
    int NX;    /* level N along x (velocities -NX..NX) */
    int NY;    /* level N along y (2D only) */
    int Lx;    /* nodes along x */
    int Ly;    /* nodes along y (1 in 1D) */
    int bc;    /* ORC_BC_* */
    double tau;   /* relaxation time; omega = 1/(tau + 1/2) */
    double uw_lo; /* x-velocity of the wall at y = -1/2 (lattice units) */
    double uw_hi; /* x-velocity of the wall at y = Ly - 1/2 */
    double g;     /* body force along x (lattice units), 2D only */
    int zv;       /* 2D axes that take the 2N+2 hierarchy without zero velocity:
                     bit 0 (ORC_ZV_X) x, bit 1 (ORC_ZV_Y) y; 0 = none */
    int NZ;       /* level N along z (3D only) */
    int Lz;       /* nodes along z (1 below 3D) */
    int guo;      /* 1: Guo's force and half-force velocity shift; 0: linearised */
} orc_cfg;

static double orc_factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i;
    return r;
}

/*
 * Sub-probabilities of one three-outcome variable at level N, Eqs. maineq04
 * and the line after it: P_{N,+-} = (c_s^2 +- c*u + u^2/N) / (2 c^2 N) and
 * P_{N,0} = 1 - P_{N,+} - P_{N,-}.
 */
static void orc_subprob(int N, double c, double cs2, double u,
                        double *Pp, double *Pm, double *P0)
{
    *Pp = (cs2 + c * u + u * u / N) / (2.0 * c * c * N);
    *Pm = (cs2 - c * u + u * u / N) / (2.0 * c * c * N);
    *P0 = 1.0 - *Pp - *Pm;
}

/*
 * Prob(sum_{j=1}^N X_j = n c), Eq. maineq03: for n >= 0,
 *   sum_{m=0}^{floor((N-n)/2)} N!/((n+m)! m! (N-n-2m)!) P+^{n+m} P-^m P0^{N-n-2m};
 * for n < 0 the same with |n| and P+ and P- exchanged (end of Sec. 2).
 */
static double orc_trinomial(int N, int n, double Pp, double Pm, double P0)
{
    if (n < 0) {
        double t = Pp;
        Pp = Pm;
        Pm = t;
        n = -n;
    }
    double s = 0.0;
    for (int m = 0; m <= (N - n) / 2; ++m) {
        double ways = orc_factorial(N) /
                      (orc_factorial(n + m) * orc_factorial(m) * orc_factorial(N - n - 2 * m));
        s += ways * pow(Pp, n + m) * pow(Pm, m) * pow(P0, N - n - 2 * m);
    }
    return s;
}

/*
 * Equilibrium probabilities of level N in physical units (Eqs. maineq02-05):
 * out[n+N] = Prob(sum = n c) for n = -N..N, lattice speed c and temperature
 * cs2 = c_s^2 given independently so the worked example of App. A (unit
 * temperature, c = sqrt(3/2)) can be evaluated. Returns 1 when a
 * sub-probability is negative (outside the positivity domain of Sec. 3),
 * else 0.
 */
int orc_prob(int N, double c, double cs2, double u, double *out)
{
    double Pp, Pm, P0;
    if (N < 1 || N > ORC_MAX_N) return -1;
    orc_subprob(N, c, cs2, u, &Pp, &Pm, &P0);
    for (int n = -N; n <= N; ++n) out[n + N] = orc_trinomial(N, n, Pp, Pm, P0);
    return (Pp < 0.0 || Pm < 0.0 || P0 < 0.0) ? 1 : 0;
}

/* Lattice-unit equilibrium f^eq_n / rho at level N: c = 1, c_s^2 = N/3. */
static void orc_eq_lattice(int N, double u, double *out)
{
    double Pp, Pm, P0;
    orc_subprob(N, 1.0, N / 3.0, u, &Pp, &Pm, &P0);
    for (int n = -N; n <= N; ++n) out[n + N] = orc_trinomial(N, n, Pp, Pm, P0);
}

/* Public wrapper of orc_eq_lattice (density 1). */
void orc_eq1d(int N, double u, double *out)
{
    orc_eq_lattice(N, u, out);
}

/* Rest weights W_n = f^eq_{n;N}(rho = 1, u = 0) (Sec. 5.4, App. A). */
void orc_weights(int N, double *out)
{
    orc_eq_lattice(N, 0.0, out);
}

/* One axis of a 2D lattice: level N, hierarchy (zv = 0: 2N+1 velocities
 * -N..N; zv = 1: 2N+2 velocities, the odd integers -(2N+1)..2N+1). */
typedef struct {
    int N, zv, Q;
    int v[2 * ORC_MAX_N + 2];
} orc_axis;

static void orc_axis_make(int N, int zv, orc_axis *a)
{
    a->N = N;
    a->zv = zv;
    a->Q = zv ? 2 * N + 2 : 2 * N + 1;
    for (int j = 0; j < a->Q; ++j) a->v[j] = zv ? 2 * j - (2 * N + 1) : j - N;
}

/*
 * f^eq_j / rho of the axis at velocity u (its lattice units). On the 2N+2
 * hierarchy the velocity v = 2n +- 1 (that is (n +- 1/2) c) takes the mean
 * of the 2N+1 equilibria at its neighbours n and n +- 1 (c units, u / c =
 * u / 2), an equilibrium beyond -N..N counting zero (Eqs. maineq01_noball -
 * maineq04_noball).
 */
static void orc_axis_eq(const orc_axis *a, double u, double *E)
{
    if (!a->zv) {
        orc_eq_lattice(a->N, u, E);
        return;
    }
    const int N = a->N;
    double En[2 * ORC_MAX_N + 1];
    orc_eq_lattice(N, 0.5 * u, En);
    for (int j = 0; j < a->Q; ++j) {
        const int lo = (a->v[j] - 1) / 2, hi = (a->v[j] + 1) / 2;
        const double elo = (lo >= -N && lo <= N) ? En[lo + N] : 0.0;
        const double ehi = (hi >= -N && hi <= N) ? En[hi + N] : 0.0;
        E[j] = 0.5 * (elo + ehi);
    }
}

/* Lattice temperature of the axis: N/3, or (4N+3)/3 on the 2N+2 hierarchy. */
static double orc_axis_theta(const orc_axis *a)
{
    return a->zv ? (4.0 * a->N + 3.0) / 3.0 : a->N / 3.0;
}

/* Positivity bound on |u| (Sec. 3: |u/c| <= sqrt(2/3) N). */
static double orc_axis_umax(const orc_axis *a)
{
    return (a->zv ? 2.0 : 1.0) * sqrt(2.0 / 3.0) * a->N;
}

/* Public: f^eq / rho of one axis (Q values), hierarchy zv. */
void orc_eq_axis(int N, int zv, double u, double *out)
{
    orc_axis a;
    orc_axis_make(N, zv, &a);
    orc_axis_eq(&a, u, out);
}

/* Public: Eq. (kn) with the lattice temperature of the hierarchy. */
double orc_tau_from_kn_axis(int N, int zv, double H, double kn)
{
    orc_axis a;
    orc_axis_make(N, zv, &a);
    return kn * H / sqrt(2.0 * orc_axis_theta(&a));
}

/*
 * Knudsen number to relaxation time, Eq. (kn): Kn = sqrt(2/theta) nu / H with
 * nu = theta * tau (Sec. 5.2), in lattice units theta = N/3.
 */
double orc_tau_from_kn(int N, double H, double kn)
{
    double theta = N / 3.0;
    return kn * H / sqrt(2.0 * theta);
}

#define ORC_ZVX(c) (((c)->zv & ORC_ZV_X) != 0)
#define ORC_ZVY(c) (((c)->zv & ORC_ZV_Y) != 0)

static int orc_check(const orc_cfg *c)
{
    if (c->zv < 0 || c->zv > 3 || (c->zv && c->dims != 2)) return -1;
    if (c->guo != 0 && (c->guo != 1 || c->dims == 1)) return -1;
    if (c->dims == 3) {
        if (c->NX < 1 || c->NX > ORC_MAX_N || c->NY < 1 || c->NY > ORC_MAX_N || c->NZ < 1 ||
            c->NZ > ORC_MAX_N)
            return -1;
        if (c->Lx < 1 || c->Ly < 1 || c->Lz < 1) return -1;
        if (c->bc == ORC_BC_WALLS && c->Ly < c->NY) return -1;
        if (c->bc != ORC_BC_WALLS && c->bc != ORC_BC_PERIODIC) return -1;
        return c->tau > 0.0 ? 0 : -1;
    }
    if (c->Lz != 1 && c->Lz != 0) return -1;
    if (c->dims == 1) {
        if (c->NX < 1 || c->NX > ORC_MAX_N || c->Lx < 1 || c->Ly != 1) return -1;
        if (c->bc == ORC_BC_BOUNCEBACK && c->Lx < c->NX) return -1;
        if (c->bc != ORC_BC_BOUNCEBACK && c->bc != ORC_BC_PERIODIC) return -1;
    } else if (c->dims == 2) {
        if (c->NX < 1 || c->NX > ORC_MAX_N || c->NY < 1 || c->NY > ORC_MAX_N) return -1;
        if (c->Lx < 1 || c->Ly < 1) return -1;
        if (c->bc == ORC_BC_WALLS && c->Ly < (ORC_ZVY(c) ? 2 * c->NY + 1 : c->NY)) return -1;
        if (c->bc != ORC_BC_WALLS && c->bc != ORC_BC_PERIODIC) return -1;
    } else {
        return -1;
    }
    return c->tau > 0.0 ? 0 : -1;
}

static int orc_nq(const orc_cfg *c)
{
    if (c->dims == 3) return (2 * c->NX + 1) * (2 * c->NY + 1) * (2 * c->NZ + 1);
    return c->dims == 1 ? 2 * c->NX + 1 : (2 * c->NX + 1 + ORC_ZVX(c)) * (2 * c->NY + 1 + ORC_ZVY(c));
}

/* ------------------------------------------------------------------------ */
/* Streaming (push form)                                                     */
/* ------------------------------------------------------------------------ */

/* Nodes of the lattice (all axes). */
static size_t orc_nodes(const orc_cfg *c)
{
    return (size_t)c->Lx * c->Ly * (c->dims == 3 ? c->Lz : 1);
}

static int orc_wrap(int i, int L)
{
    i %= L;
    return i < 0 ? i + L : i;
}

/*
 * 1D streaming: f_n(x + n) <- X_n(x). Periodic, or halfway bounce-back at
 * x = -1/2 and x = L - 1/2 (a population leaving through an end comes back
 * with the opposite velocity, having travelled the same distance).
 */
static void orc_stream1d(const orc_cfg *c, const double *X, double *F)
{
    int N = c->NX, L = c->Lx;
    for (int n = -N; n <= N; ++n) {
        for (int x = 0; x < L; ++x) {
            double v = X[(n + N) * L + x];
            int xd = x + n;
            if (c->bc == ORC_BC_PERIODIC) {
                F[(n + N) * L + orc_wrap(xd, L)] = v;
            } else if (xd < 0) {
                F[(-n + N) * L + (-1 - xd)] = v;
            } else if (xd >= L) {
                F[(-n + N) * L + (2 * L - 1 - xd)] = v;
            } else {
                F[(n + N) * L + xd] = v;
            }
        }
    }
}

/*
 * 2D streaming: f_i(x + xi_x, y + xi_y) <- X_i(x, y), periodic in x. With
 * walls, populations crossing y = -1/2 or y = Ly - 1/2 are absorbed into the
 * wall of that side, booked under the column they would have reached; then
 * each wall re-emits its absorbed mass of column x as
 * rho_w(x) E^x(u_w) W^y into the rows whose source lies inside the wall.
 */
static void orc_stream2d(const orc_cfg *c, const double *X, double *F)
{
    orc_axis ax, ay;
    orc_axis_make(c->NX, ORC_ZVX(c), &ax);
    orc_axis_make(c->NY, ORC_ZVY(c), &ay);
    int Lx = c->Lx, Ly = c->Ly;
    size_t plane = (size_t)Lx * Ly;
    double *Dlo = (double *)calloc((size_t)Lx, sizeof(double));
    double *Dhi = (double *)calloc((size_t)Lx, sizeof(double));

    for (int iy = 0; iy < ay.Q; ++iy) {
        for (int ix = 0; ix < ax.Q; ++ix) {
            int q = iy * ax.Q + ix, nx = ax.v[ix], ny = ay.v[iy];
            for (int y = 0; y < Ly; ++y) {
                for (int x = 0; x < Lx; ++x) {
                    double v = X[q * plane + (size_t)y * Lx + x];
                    int xd = orc_wrap(x + nx, Lx);
                    int yd = y + ny;
                    if (c->bc == ORC_BC_PERIODIC) {
                        F[q * plane + (size_t)orc_wrap(yd, Ly) * Lx + xd] = v;
                    } else if (yd < 0) {
                        Dlo[xd] += v;
                    } else if (yd >= Ly) {
                        Dhi[xd] += v;
                    } else {
                        F[q * plane + (size_t)yd * Lx + xd] = v;
                    }
                }
            }
        }
    }

    if (c->bc == ORC_BC_WALLS) {
        double Wy[2 * ORC_MAX_N + 2], Elo[2 * ORC_MAX_N + 2], Ehi[2 * ORC_MAX_N + 2];
        orc_axis_eq(&ay, 0.0, Wy);
        orc_axis_eq(&ax, c->uw_lo, Elo);
        orc_axis_eq(&ax, c->uw_hi, Ehi);
        /* emitted mass per unit rho_w: sum over velocities leaving the wall of
           |xi_y| * E^x * W^y, i.e. one population per row it fills */
        double den = 0.0, den_hi = 0.0;
        for (int iy = 0; iy < ay.Q; ++iy) {
            for (int ix = 0; ix < ax.Q; ++ix) {
                if (ay.v[iy] > 0) den += ay.v[iy] * Elo[ix] * Wy[iy];
                if (ay.v[iy] < 0) den_hi += -ay.v[iy] * Ehi[ix] * Wy[iy];
            }
        }
        for (int x = 0; x < Lx; ++x) {
            double rlo = Dlo[x] / den;
            double rhi = Dhi[x] / den_hi;
            for (int iy = 0; iy < ay.Q; ++iy) {
                int ny = ay.v[iy];
                for (int ix = 0; ix < ax.Q; ++ix) {
                    int q = iy * ax.Q + ix;
                    /* ny > 0 leaves the lower wall into rows 0..ny-1, ny < 0 the
                       upper wall into rows Ly-1 .. Ly+ny */
                    for (int k = 0; k < (ny > 0 ? ny : -ny); ++k) {
                        if (ny > 0)
                            F[q * plane + (size_t)k * Lx + x] = rlo * Elo[ix] * Wy[iy];
                        else
                            F[q * plane + (size_t)(Ly - 1 - k) * Lx + x] = rhi * Ehi[ix] * Wy[iy];
                    }
                }
            }
        }
    }
    free(Dlo);
    free(Dhi);
}

/*
 * 3D push streaming: periodic in x and z; in y as in 2D (periodic, or the
 * diffuse walls with the absorbed mass of each (x, z) column re-emitted with
 * the shape E^x(u_w) W^y W^z).
 */
static void orc_stream3d(const orc_cfg *c, const double *X, double *F)
{
    const int NX = c->NX, NY = c->NY, NZ = c->NZ, Lx = c->Lx, Ly = c->Ly, Lz = c->Lz;
    const int Qx = 2 * NX + 1, Qy = 2 * NY + 1, Qz = 2 * NZ + 1;
    const size_t plane = (size_t)Lx * Ly * Lz, col = (size_t)Lx * Lz;
    double *Dlo = (double *)calloc(col, sizeof(double));
    double *Dhi = (double *)calloc(col, sizeof(double));
    for (int iz = 0; iz < Qz; ++iz)
        for (int iy = 0; iy < Qy; ++iy)
            for (int ix = 0; ix < Qx; ++ix) {
                const int q = (iz * Qy + iy) * Qx + ix, nx = ix - NX, ny = iy - NY, nz = iz - NZ;
                for (int z = 0; z < Lz; ++z)
                    for (int y = 0; y < Ly; ++y)
                        for (int x = 0; x < Lx; ++x) {
                            const double v = X[q * plane + ((size_t)z * Ly + y) * Lx + x];
                            const int xd = orc_wrap(x + nx, Lx), zd = orc_wrap(z + nz, Lz);
                            const int yd = y + ny;
                            if (c->bc == ORC_BC_PERIODIC)
                                F[q * plane + ((size_t)zd * Ly + orc_wrap(yd, Ly)) * Lx + xd] = v;
                            else if (yd < 0)
                                Dlo[(size_t)zd * Lx + xd] += v;
                            else if (yd >= Ly)
                                Dhi[(size_t)zd * Lx + xd] += v;
                            else
                                F[q * plane + ((size_t)zd * Ly + yd) * Lx + xd] = v;
                        }
            }
    if (c->bc == ORC_BC_WALLS) {
        double Wy[2 * ORC_MAX_N + 1], Wz[2 * ORC_MAX_N + 1];
        double Elo[2 * ORC_MAX_N + 1], Ehi[2 * ORC_MAX_N + 1];
        orc_eq_lattice(NY, 0.0, Wy);
        orc_eq_lattice(NZ, 0.0, Wz);
        orc_eq_lattice(NX, c->uw_lo, Elo);
        orc_eq_lattice(NX, c->uw_hi, Ehi);
        /* emitted mass per unit rho_w: sum over velocities leaving the wall of
           |xi_y| E^x W^y W^z */
        double den = 0.0, den_hi = 0.0;
        for (int iz = 0; iz < Qz; ++iz)
            for (int iy = 0; iy < Qy; ++iy)
                for (int ix = 0; ix < Qx; ++ix) {
                    const int ny = iy - NY;
                    if (ny > 0) den += ny * Elo[ix] * Wy[iy] * Wz[iz];
                    if (ny < 0) den_hi += -ny * Ehi[ix] * Wy[iy] * Wz[iz];
                }
        for (int z = 0; z < Lz; ++z)
            for (int x = 0; x < Lx; ++x) {
                const double rlo = Dlo[(size_t)z * Lx + x] / den;
                const double rhi = Dhi[(size_t)z * Lx + x] / den_hi;
                for (int iz = 0; iz < Qz; ++iz)
                    for (int iy = 0; iy < Qy; ++iy) {
                        const int ny = iy - NY;
                        for (int ix = 0; ix < Qx; ++ix) {
                            const int q = (iz * Qy + iy) * Qx + ix;
                            for (int k = 0; k < (ny > 0 ? ny : -ny); ++k) {
                                if (ny > 0)
                                    F[q * plane + ((size_t)z * Ly + k) * Lx + x] =
                                        rlo * Elo[ix] * Wy[iy] * Wz[iz];
                                else
                                    F[q * plane + ((size_t)z * Ly + (Ly - 1 - k)) * Lx + x] =
                                        rhi * Ehi[ix] * Wy[iy] * Wz[iz];
                            }
                        }
                    }
            }
    }
    free(Dlo);
    free(Dhi);
}

int orc_stream(const orc_cfg *c, const double *X, double *F)
{
    if (orc_check(c)) return -1;
    if (c->dims == 1)
        orc_stream1d(c, X, F);
    else if (c->dims == 3)
        orc_stream3d(c, X, F);
    else
        orc_stream2d(c, X, F);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Collision (Eq. maineq01 right-hand side)                                  */
/* ------------------------------------------------------------------------ */

/*
 * Velocity that the equilibrium and the reported fields use: j / rho, or
 * (j_x + g/2) / rho along x in Guo's form.
 */
static double orc_ux(const orc_cfg *c, double jx, double rho)
{
    return (c->guo ? jx + 0.5 * c->g : jx) / rho;
}

/*
 * Body force on the population of velocity (vx, vy, vz) at a node of velocity
 * (ux, uy, uz), W the product of its rest weights, thx, thy, thz the axis
 * temperatures: linearised W vx g / theta_x (Sec. 5.4), or Guo's
 * (1 - omega/2) W [(xi - u).G + (xi.U)(xi.G)] with G = (g/theta_x, 0, 0) and
 * U_a = u_a / theta_a.
 */
static double orc_force(const orc_cfg *c, double omega, double W, double vx, double vy,
                        double vz, double ux, double uy, double uz, double thx, double thy,
                        double thz)
{
    const double Gx = c->g / thx;
    if (!c->guo) return W * vx * Gx;
    const double xiU = vx * ux / thx + vy * uy / thy + vz * uz / thz;
    return (1.0 - 0.5 * omega) * W * ((vx - ux) * Gx + xiU * vx * Gx);
}

/*
 * BGK relaxation at every node: f* = f + omega (f^eq - f) + F_i with
 * omega = 1/(tau + 1/2), f^eq = rho E^x(u_x) E^y(u_y) (product form, Sec. 4)
 * and rho, rho u the zeroth and first moments of f. Returns the number of
 * nodes whose equilibrium left the positivity domain (Sec. 3) or whose
 * density is not positive.
 */
int orc_collide(const orc_cfg *c, const double *F, double *X)
{
    if (orc_check(c)) return -1;
    double omega = 1.0 / (c->tau + 0.5);
    int bad = 0;
    if (c->dims == 1) {
        int N = c->NX, L = c->Lx;
        double E[2 * ORC_MAX_N + 1];
        for (int x = 0; x < L; ++x) {
            double rho = 0.0, j = 0.0;
            for (int n = -N; n <= N; ++n) {
                rho += F[(n + N) * L + x];
                j += n * F[(n + N) * L + x];
            }
            double u = j / rho;
            if (!(rho > 0.0) || fabs(u) > sqrt(2.0 / 3.0) * N) ++bad;
            orc_eq_lattice(N, u, E);
            for (int n = -N; n <= N; ++n) {
                double f = F[(n + N) * L + x];
                X[(n + N) * L + x] = f + omega * (rho * E[n + N] - f);
            }
        }
        return bad;
    }
    if (c->dims == 3) {
        const int NX = c->NX, NY = c->NY, NZ = c->NZ;
        const int Qx = 2 * NX + 1, Qy = 2 * NY + 1, Qz = 2 * NZ + 1;
        const size_t plane = orc_nodes(c);
        double Wx[2 * ORC_MAX_N + 1], Wy[2 * ORC_MAX_N + 1], Wz[2 * ORC_MAX_N + 1];
        double Ex[2 * ORC_MAX_N + 1], Ey[2 * ORC_MAX_N + 1], Ez[2 * ORC_MAX_N + 1];
        orc_eq_lattice(NX, 0.0, Wx);
        orc_eq_lattice(NY, 0.0, Wy);
        orc_eq_lattice(NZ, 0.0, Wz);
        const double theta_x = NX / 3.0;
        for (size_t node = 0; node < plane; ++node) {
            double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
            for (int iz = 0; iz < Qz; ++iz)
                for (int iy = 0; iy < Qy; ++iy)
                    for (int ix = 0; ix < Qx; ++ix) {
                        const double f = F[((iz * Qy + iy) * Qx + ix) * plane + node];
                        rho += f;
                        jx += (ix - NX) * f;
                        jy += (iy - NY) * f;
                        jz += (iz - NZ) * f;
                    }
            const double ux = orc_ux(c, jx, rho), uy = jy / rho, uz = jz / rho;
            const double b = sqrt(2.0 / 3.0);
            if (!(rho > 0.0) || fabs(ux) > b * NX || fabs(uy) > b * NY || fabs(uz) > b * NZ) ++bad;
            orc_eq_lattice(NX, ux, Ex);
            orc_eq_lattice(NY, uy, Ey);
            orc_eq_lattice(NZ, uz, Ez);
            for (int iz = 0; iz < Qz; ++iz)
                for (int iy = 0; iy < Qy; ++iy)
                    for (int ix = 0; ix < Qx; ++ix) {
                        const size_t idx = ((iz * Qy + iy) * Qx + ix) * plane + node;
                        const double f = F[idx];
                        const double feq = rho * Ex[ix] * Ey[iy] * Ez[iz];
                        const double force =
                            orc_force(c, omega, Wx[ix] * Wy[iy] * Wz[iz], ix - NX, iy - NY, iz - NZ,
                                      ux, uy, uz, theta_x, NY / 3.0, NZ / 3.0);
                        X[idx] = f + omega * (feq - f) + force;
                    }
        }
        return bad;
    }

    orc_axis ax, ay;
    orc_axis_make(c->NX, ORC_ZVX(c), &ax);
    orc_axis_make(c->NY, ORC_ZVY(c), &ay);
    int Lx = c->Lx, Ly = c->Ly;
    size_t plane = (size_t)Lx * Ly;
    double Wx[2 * ORC_MAX_N + 2], Wy[2 * ORC_MAX_N + 2];
    orc_axis_eq(&ax, 0.0, Wx);
    orc_axis_eq(&ay, 0.0, Wy);
    double theta_x = orc_axis_theta(&ax), theta_y = orc_axis_theta(&ay);
    /* every node collides on its own: rows may run on several threads (an
       -fopenmp build, used only to time the oracle on all cores) with results
       identical to the serial loop */
#pragma omp parallel for reduction(+ : bad)
    for (int y = 0; y < Ly; ++y) {
        double Ex[2 * ORC_MAX_N + 2], Ey[2 * ORC_MAX_N + 2];
        for (int x = 0; x < Lx; ++x) {
            size_t node = (size_t)y * Lx + x;
            double rho = 0.0, jx = 0.0, jy = 0.0;
            for (int iy = 0; iy < ay.Q; ++iy) {
                for (int ix = 0; ix < ax.Q; ++ix) {
                    double f = F[(iy * ax.Q + ix) * plane + node];
                    rho += f;
                    jx += ax.v[ix] * f;
                    jy += ay.v[iy] * f;
                }
            }
            double ux = orc_ux(c, jx, rho), uy = jy / rho;
            if (!(rho > 0.0) || fabs(ux) > orc_axis_umax(&ax) || fabs(uy) > orc_axis_umax(&ay))
                ++bad;
            orc_axis_eq(&ax, ux, Ex);
            orc_axis_eq(&ay, uy, Ey);
            for (int iy = 0; iy < ay.Q; ++iy) {
                for (int ix = 0; ix < ax.Q; ++ix) {
                    size_t idx = (iy * ax.Q + ix) * plane + node;
                    double f = F[idx];
                    double feq = rho * Ex[ix] * Ey[iy];
                    double force = orc_force(c, omega, Wx[ix] * Wy[iy], ax.v[ix], ay.v[iy], 0.0,
                                             ux, uy, 0.0, theta_x, theta_y, 1.0);
                    X[idx] = f + omega * (feq - f) + force;
                }
            }
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Macroscopic fields                                                        */
/* ------------------------------------------------------------------------ */

/*
 * Moments of populations F at every node (Sec. 2 for rho, rho u; the
 * temperature, heat flux and shear stress are the usual central moments,
 * taken about u; u_x = (j_x + g/2) / rho in Guo's form):
 * 2D out[7][Ly][Lx] = rho, u_x, u_y, T = sum |xi-u|^2 f / (2 rho),
 *   q_x, q_y = (1/2) sum (xi-u)_a |xi-u|^2 f, sigma_xy = sum (xi-u)_x (xi-u)_y f;
 * 1D out[4][L] = rho, u, T = sum (xi-u)^2 f / rho, q = (1/2) sum (xi-u)^3 f;
 * 3D out[9][Lz][Ly][Lx] = rho, u_x, u_y, T = sum |xi-u|^2 f / (3 rho), q_x,
 *   q_y, sigma_xy, u_z, q_z (the 2D fields first, then the z ones).
 */
int orc_macro(const orc_cfg *c, const double *F, double *out)
{
    if (orc_check(c)) return -1;
    if (c->dims == 3) {
        const int NX = c->NX, NY = c->NY, NZ = c->NZ;
        const int Qx = 2 * NX + 1, Qy = 2 * NY + 1, Qz = 2 * NZ + 1;
        const size_t plane = orc_nodes(c);
        for (size_t node = 0; node < plane; ++node) {
            double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
            for (int iz = 0; iz < Qz; ++iz)
                for (int iy = 0; iy < Qy; ++iy)
                    for (int ix = 0; ix < Qx; ++ix) {
                        const double f = F[((iz * Qy + iy) * Qx + ix) * plane + node];
                        rho += f;
                        jx += (ix - NX) * f;
                        jy += (iy - NY) * f;
                        jz += (iz - NZ) * f;
                    }
            const double ux = orc_ux(c, jx, rho), uy = jy / rho, uz = jz / rho;
            double e2 = 0.0, qx = 0.0, qy = 0.0, qz = 0.0, sxy = 0.0;
            for (int iz = 0; iz < Qz; ++iz)
                for (int iy = 0; iy < Qy; ++iy)
                    for (int ix = 0; ix < Qx; ++ix) {
                        const double f = F[((iz * Qy + iy) * Qx + ix) * plane + node];
                        const double dx = ix - NX - ux, dy = iy - NY - uy, dz = iz - NZ - uz;
                        const double d2 = dx * dx + dy * dy + dz * dz;
                        e2 += d2 * f;
                        qx += dx * d2 * f;
                        qy += dy * d2 * f;
                        qz += dz * d2 * f;
                        sxy += dx * dy * f;
                    }
            const double m[9] = {rho, ux, uy, e2 / (3.0 * rho), 0.5 * qx, 0.5 * qy, sxy, uz, 0.5 * qz};
            for (int k = 0; k < 9; ++k) out[k * plane + node] = m[k];
        }
        return 0;
    }
    if (c->dims == 1) {
        int N = c->NX, L = c->Lx;
        for (int x = 0; x < L; ++x) {
            double rho = 0.0, j = 0.0;
            for (int n = -N; n <= N; ++n) {
                rho += F[(n + N) * L + x];
                j += n * F[(n + N) * L + x];
            }
            double u = j / rho, e2 = 0.0, e3 = 0.0;
            for (int n = -N; n <= N; ++n) {
                double d = n - u, f = F[(n + N) * L + x];
                e2 += d * d * f;
                e3 += d * d * d * f;
            }
            out[0 * L + x] = rho;
            out[1 * L + x] = u;
            out[2 * L + x] = e2 / rho;
            out[3 * L + x] = 0.5 * e3;
        }
        return 0;
    }
    orc_axis ax, ay;
    orc_axis_make(c->NX, ORC_ZVX(c), &ax);
    orc_axis_make(c->NY, ORC_ZVY(c), &ay);
    size_t plane = (size_t)c->Lx * c->Ly;
    for (size_t node = 0; node < plane; ++node) {
        double rho = 0.0, jx = 0.0, jy = 0.0;
        for (int iy = 0; iy < ay.Q; ++iy) {
            for (int ix = 0; ix < ax.Q; ++ix) {
                double f = F[(iy * ax.Q + ix) * plane + node];
                rho += f;
                jx += ax.v[ix] * f;
                jy += ay.v[iy] * f;
            }
        }
        double ux = orc_ux(c, jx, rho), uy = jy / rho;
        double e2 = 0.0, qx = 0.0, qy = 0.0, sxy = 0.0;
        for (int iy = 0; iy < ay.Q; ++iy) {
            for (int ix = 0; ix < ax.Q; ++ix) {
                double f = F[(iy * ax.Q + ix) * plane + node];
                double dx = ax.v[ix] - ux, dy = ay.v[iy] - uy, d2 = dx * dx + dy * dy;
                e2 += d2 * f;
                qx += dx * d2 * f;
                qy += dy * d2 * f;
                sxy += dx * dy * f;
            }
        }
        out[0 * plane + node] = rho;
        out[1 * plane + node] = ux;
        out[2 * plane + node] = uy;
        out[3 * plane + node] = e2 / (2.0 * rho);
        out[4 * plane + node] = 0.5 * qx;
        out[5 * plane + node] = 0.5 * qy;
        out[6 * plane + node] = sxy;
    }
    return 0;
}

/*
 * Local equilibrium initial state X_0 = rho E^x(u_x) E^y(u_y) at every node
 * (rho, ux, uy given per node; uy ignored in 1D).
 */
int orc_equilibrium(const orc_cfg *c, const double *rho, const double *ux, const double *uy,
                    double *X)
{
    if (orc_check(c) || c->dims == 3) return -1;
    if (c->dims == 1) {
        int N = c->NX, L = c->Lx;
        double E[2 * ORC_MAX_N + 1];
        for (int x = 0; x < L; ++x) {
            orc_eq_lattice(N, ux[x], E);
            for (int n = -N; n <= N; ++n) X[(n + N) * L + x] = rho[x] * E[n + N];
        }
        return 0;
    }
    orc_axis ax, ay;
    orc_axis_make(c->NX, ORC_ZVX(c), &ax);
    orc_axis_make(c->NY, ORC_ZVY(c), &ay);
    size_t plane = (size_t)c->Lx * c->Ly;
    double Ex[2 * ORC_MAX_N + 2], Ey[2 * ORC_MAX_N + 2];
    for (size_t node = 0; node < plane; ++node) {
        orc_axis_eq(&ax, ux[node], Ex);
        orc_axis_eq(&ay, uy[node], Ey);
        for (int iy = 0; iy < ay.Q; ++iy)
            for (int ix = 0; ix < ax.Q; ++ix)
                X[(iy * ax.Q + ix) * plane + node] = rho[node] * Ex[ix] * Ey[iy];
    }
    return 0;
}

/*
 * 3D local equilibrium X_0 = rho E^x(u_x) E^y(u_y) E^z(u_z) at every node.
 */
int orc_equilibrium3d(const orc_cfg *c, const double *rho, const double *ux, const double *uy,
                      const double *uz, double *X)
{
    if (orc_check(c) || c->dims != 3) return -1;
    const int NX = c->NX, NY = c->NY, NZ = c->NZ;
    const int Qx = 2 * NX + 1, Qy = 2 * NY + 1, Qz = 2 * NZ + 1;
    const size_t plane = orc_nodes(c);
    double Ex[2 * ORC_MAX_N + 1], Ey[2 * ORC_MAX_N + 1], Ez[2 * ORC_MAX_N + 1];
    for (size_t node = 0; node < plane; ++node) {
        orc_eq_lattice(NX, ux[node], Ex);
        orc_eq_lattice(NY, uy[node], Ey);
        orc_eq_lattice(NZ, uz[node], Ez);
        for (int iz = 0; iz < Qz; ++iz)
            for (int iy = 0; iy < Qy; ++iy)
                for (int ix = 0; ix < Qx; ++ix)
                    X[((iz * Qy + iy) * Qx + ix) * plane + node] = rho[node] * Ex[ix] * Ey[iy] * Ez[iz];
    }
    return 0;
}

/*
 * Advance X in place by `steps` steps X <- C(S(X)). Returns the number of
 * collisions that left the positivity domain, or -1 on a bad configuration.
 */
long orc_run(const orc_cfg *c, double *X, long steps)
{
    if (orc_check(c)) return -1;
    size_t n = (size_t)orc_nq(c) * orc_nodes(c);
    double *F = (double *)malloc(n * sizeof(double));
    long bad = 0;
    for (long t = 0; t < steps; ++t) {
        orc_stream(c, X, F);
        bad += orc_collide(c, F, X);
    }
    free(F);
    return bad;
}

/* Moments at the current time: moments of S(X). */
int orc_observe(const orc_cfg *c, const double *X, double *out)
{
    if (orc_check(c)) return -1;
    size_t n = (size_t)orc_nq(c) * orc_nodes(c);
    double *F = (double *)malloc(n * sizeof(double));
    orc_stream(c, X, F);
    orc_macro(c, F, out);
    free(F);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode gradient of the flow rate (dual numbers)                     */
/* ------------------------------------------------------------------------ */

/*
 * Equilibrium and its derivative in u at level N (lattice units): E[n+N] as in
 * orc_eq_lattice and dE[n+N] = dE_n/du, by differentiating every term of the
 * factorial sum of Eq. maineq03 with P+- = (N/3 +- u + u^2/N)/(2N) and
 * P0 = 1 - P+ - P-:  dP+-/du = (+-1 + 2u/N)/(2N),  dP0/du = -2u/N^2.
 */
static void orc_eq_lattice_du(int N, double u, double *E, double *dE)
{
    const double Pp = (N / 3.0 + u + u * u / N) / (2.0 * N);
    const double Pm = (N / 3.0 - u + u * u / N) / (2.0 * N);
    const double P0 = 1.0 - Pp - Pm;
    const double dPp = (1.0 + 2.0 * u / N) / (2.0 * N);
    const double dPm = (-1.0 + 2.0 * u / N) / (2.0 * N);
    const double dP0 = -dPp - dPm;
    for (int n = -N; n <= N; ++n) {
        double pp = Pp, pm = Pm, dpp = dPp, dpm = dPm;
        int an = n;
        if (n < 0) { /* mirror: exchange P+ and P- */
            pp = Pm; pm = Pp; dpp = dPm; dpm = dPp; an = -n;
        }
        double s = 0.0, ds = 0.0;
        for (int m = 0; m <= (N - an) / 2; ++m) {
            const int a = an + m, b = m, c = N - an - 2 * m;
            const double ways = orc_factorial(N) /
                                (orc_factorial(a) * orc_factorial(b) * orc_factorial(c));
            const double t = pow(pp, a) * pow(pm, b) * pow(P0, c);
            s += ways * t;
            /* product rule over the three powers */
            double dt = 0.0;
            if (a > 0) dt += a * pow(pp, a - 1) * dpp * pow(pm, b) * pow(P0, c);
            if (b > 0) dt += b * pow(pp, a) * pow(pm, b - 1) * dpm * pow(P0, c);
            if (c > 0) dt += c * pow(pp, a) * pow(pm, b) * pow(P0, c - 1) * dP0;
            ds += ways * dt;
        }
        E[n + N] = s;
        dE[n + N] = ds;
    }
}

/* States of the dual numbers: the value and its derivatives by tau, g and the
   two wall speeds. */
#define ORC_NT 5

/*
 * Collision of a dual state: X = C(F) for the values and, for each parameter p
 * in (tau, g, u_wall_lo, u_wall_hi), dX/dp = dC/dF . dF/dp + dC/dp, with
 *   f* = f + omega (f^eq - f) + F_i,  omega = 1/(tau + 1/2),
 *   d omega / d tau = -omega^2,  dF_i/dg = W_i xi_x / theta_x,
 *   d f^eq_i = E_i d rho + rho (dE^x_i/du_x du_x E^y_i + E^x_i dE^y_i/du_y du_y),
 *   du = (dj - u d rho) / rho;
 * the collision has no explicit dependence on the wall speeds (they enter
 * through the streaming, orc_emission_du). F, X hold ORC_NT arrays of n
 * populations: [value | d/dtau | d/dg | d/du_wall_lo | d/du_wall_hi].
 */
static void orc_collide_dual(const orc_cfg *c, const double *F, double *X)
{
    const int NX = c->NX, NY = c->NY, Lx = c->Lx, Ly = c->Ly;
    const int Q1x = 2 * NX + 1;
    const size_t plane = (size_t)Lx * Ly;
    const size_t n = (size_t)orc_nq(c) * plane;
    const double omega = 1.0 / (c->tau + 0.5);
    const double domega = -omega * omega;
    const double theta_x = NX / 3.0;
    double Wx[2 * ORC_MAX_N + 1], Wy[2 * ORC_MAX_N + 1];
    double Ex[2 * ORC_MAX_N + 1], Ey[2 * ORC_MAX_N + 1], dEx[2 * ORC_MAX_N + 1], dEy[2 * ORC_MAX_N + 1];
    orc_eq_lattice(NX, 0.0, Wx);
    orc_eq_lattice(NY, 0.0, Wy);
    for (size_t node = 0; node < plane; ++node) {
        double rho[ORC_NT] = {0}, jx[ORC_NT] = {0}, jy[ORC_NT] = {0};
        for (int ny = -NY; ny <= NY; ++ny)
            for (int nx = -NX; nx <= NX; ++nx) {
                const size_t idx = ((ny + NY) * Q1x + (nx + NX)) * plane + node;
                for (int d = 0; d < ORC_NT; ++d) {
                    const double f = F[d * n + idx];
                    rho[d] += f;
                    jx[d] += nx * f;
                    jy[d] += ny * f;
                }
            }
        const double ux = jx[0] / rho[0], uy = jy[0] / rho[0];
        double dux[ORC_NT], duy[ORC_NT];
        for (int d = 1; d < ORC_NT; ++d) {
            dux[d] = (jx[d] - ux * rho[d]) / rho[0];
            duy[d] = (jy[d] - uy * rho[d]) / rho[0];
        }
        orc_eq_lattice_du(NX, ux, Ex, dEx);
        orc_eq_lattice_du(NY, uy, Ey, dEy);
        for (int ny = -NY; ny <= NY; ++ny)
            for (int nx = -NX; nx <= NX; ++nx) {
                const size_t idx = ((ny + NY) * Q1x + (nx + NX)) * plane + node;
                const double f = F[idx];
                const double feq = rho[0] * Ex[nx + NX] * Ey[ny + NY];
                const double wxg = Wx[nx + NX] * Wy[ny + NY] * nx / theta_x;
                X[idx] = f + omega * (feq - f) + wxg * c->g;
                for (int d = 1; d < ORC_NT; ++d) {
                    const double df = F[d * n + idx];
                    const double dfeq = rho[d] * Ex[nx + NX] * Ey[ny + NY] +
                                        rho[0] * (dEx[nx + NX] * dux[d] * Ey[ny + NY] +
                                                  Ex[nx + NX] * dEy[ny + NY] * duy[d]);
                    double v = df + omega * (dfeq - df);
                    if (d == 1) v += domega * (feq - f); /* d/dtau */
                    if (d == 2) v += wxg;                /* d/dg */
                    X[d * n + idx] = v;
                }
            }
    }
}

/*
 * Derivative by the speed of one wall (upper = 0: y = -1/2, 1: y = Ly - 1/2) of
 * streaming the value state X, added to dF: the wall re-emits
 * rho_w(x) E^x_i(u_w) W^y_i (reading R5), where rho_w balances the mass X
 * sends into the wall and so does not depend on u_w (the emitted mass per unit
 * rho_w, sum_{n>0} n W^y_n sum_i E^x_i(u_w), is the same at every u_w because
 * sum_i E^x_i = 1); the derivative is rho_w(x) dE^x_i/du(u_w) W^y_i at every
 * emitted (node, velocity) of that wall. Isotropic 2N+1 lattices.
 */
static void orc_emission_du(const orc_cfg *c, const double *X, int upper, double *dF)
{
    const int NX = c->NX, NY = c->NY, Q1x = 2 * NX + 1;
    const int Lx = c->Lx, Ly = c->Ly;
    const size_t plane = (size_t)Lx * Ly;
    const double uw = upper ? c->uw_hi : c->uw_lo;
    double Wy[2 * ORC_MAX_N + 1], E[2 * ORC_MAX_N + 1], dE[2 * ORC_MAX_N + 1];
    orc_eq_lattice(NY, 0.0, Wy);
    orc_eq_lattice_du(NX, uw, E, dE);
    double den = 0.0;
    for (int ny = 1; ny <= NY; ++ny)
        for (int ix = 0; ix < Q1x; ++ix) den += ny * E[ix] * Wy[ny + NY];
    double *D = (double *)calloc((size_t)Lx, sizeof(double));
    /* the mass that streams into the wall, booked under the column it reaches */
    for (int ny = -NY; ny <= NY; ++ny) {
        if ((upper && ny <= 0) || (!upper && ny >= 0)) continue;
        for (int nx = -NX; nx <= NX; ++nx) {
            const int q = (ny + NY) * Q1x + (nx + NX);
            for (int y = 0; y < Ly; ++y) {
                const int yd = y + ny;
                if ((upper && yd < Ly) || (!upper && yd >= 0)) continue;
                for (int x = 0; x < Lx; ++x)
                    D[orc_wrap(x + nx, Lx)] += X[q * plane + (size_t)y * Lx + x];
            }
        }
    }
    for (int x = 0; x < Lx; ++x) {
        const double rw = D[x] / den;
        for (int a = 1; a <= NY; ++a) {
            const int ny = upper ? -a : a;  /* velocities leaving the wall */
            for (int nx = -NX; nx <= NX; ++nx) {
                const int q = (ny + NY) * Q1x + (nx + NX);
                for (int k = 0; k < a; ++k) {
                    const int y = upper ? Ly - 1 - k : k;
                    dF[q * plane + (size_t)y * Lx + x] += rw * dE[nx + NX] * Wy[ny + NY];
                }
            }
        }
    }
    free(D);
}

/*
 * Flow rate J = (1/Lx) sum over nodes of the x-momentum of S(X_T) after `steps`
 * steps from X (2D), and its derivatives by tau, g, u_wall_lo and u_wall_hi by
 * forward-mode differentiation of every step (streaming is linear in the
 * populations, so the tangents stream like the values, plus the wall speeds'
 * own term of the emission). X holds the initial populations (independent of
 * the parameters); out = {J, dJ/dtau, dJ/dg, dJ/du_wall_lo, dJ/du_wall_hi}.
 * Returns -1 on a bad configuration.
 */
int orc_flowrate_grad(const orc_cfg *c, const double *X0, long steps, double *out)
{
    if (orc_check(c) || c->dims != 2 || c->zv || c->guo) return -1;  /* 2N+1, linearised force */
    const size_t plane = (size_t)c->Lx * c->Ly;
    const size_t n = (size_t)orc_nq(c) * plane;
    double *X = (double *)calloc(ORC_NT * n, sizeof(double));
    double *F = (double *)malloc(ORC_NT * n * sizeof(double));
    memcpy(X, X0, n * sizeof(double));
    for (long t = 0; t <= steps; ++t) {
        for (int d = 0; d < ORC_NT; ++d) orc_stream2d(c, X + d * n, F + d * n);
        if (c->bc == ORC_BC_WALLS) {
            orc_emission_du(c, X, 0, F + 3 * n);
            orc_emission_du(c, X, 1, F + 4 * n);
        }
        if (t < steps) orc_collide_dual(c, F, X);
    }
    const int NX = c->NX, NY = c->NY, Q1x = 2 * NX + 1;
    for (int d = 0; d < ORC_NT; ++d) {
        double s = 0.0;
        for (int ny = -NY; ny <= NY; ++ny)
            for (int nx = -NX; nx <= NX; ++nx)
                for (size_t node = 0; node < plane; ++node)
                    s += nx * F[d * n + ((ny + NY) * Q1x + (nx + NX)) * plane + node];
        out[d] = s / c->Lx;
    }
    free(X);
    free(F);
    return 0;
}
