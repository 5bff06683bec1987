"""Pins of the oracle's Guo forcing option (Guo, Zheng and Shi, Phys. Rev. E 65,
046308, 2002; an alternative to the linearised force of Sec. 5.4).

What fixes the form, independent of how the oracle writes it:
  - Guo's moment conditions on the force term F_i: sum F_i = 0,
    sum xi F_i = (1 - omega/2) g and sum xi xi F_i = (1 - omega/2)(g u + u g),
    with u the half-force-shifted velocity (j + g/2) / rho;
  - the collision increment then carries exactly g of x momentum and no mass
    (omega g/2 through the relaxation, (1 - omega/2) g through F);
  - from rest in a periodic box the reported velocity is (t + 1/2) g / rho at
    step t: the half-force shift;
  - D2Q9 (level 1 on both axes, c_s^2 = 1/3) reproduces Guo's published
    D2Q9 term;
  - a force-driven channel at small Knudsen number has the Navier-Stokes
    curvature u'' = -g / (rho nu), nu = theta tau.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import inputs

ZV_Y = 2


def _axis_vel(N, zv):
    return (2 * np.arange(2 * N + 2) - (2 * N + 1)) if zv else np.arange(-N, N + 1)


def _axis_theta(N, zv):
    return (4 * N + 3) / 3.0 if zv else N / 3.0


def _vel2(NX, NY, zvy=0):
    vx = _axis_vel(NX, 0).astype(float)
    vy = _axis_vel(NY, zvy).astype(float)
    return np.tile(vx, len(vy)), np.repeat(vy, len(vx))


def _mom(w, A):
    return np.tensordot(w, A, axes=1)


# (NX, NY, zv along y): isotropic levels, the anisotropic channel lattice
# D1Q3 x D1Q9 and the 2N+2 channel lattice D1Q3 x D1Q8
LATTICES = [(1, 1, 0), (3, 3, 0), (1, 4, 0), (1, 3, ZV_Y)]


def _force_terms(NX, NY, zvy, tau, g, seed):
    """F, the populations after Guo's collision, and the force term F_i
    isolated as X - F - omega (f^eq(rho, u_shifted) - F)."""
    Lx, Ly = 5, 4
    lat = orc.Lattice(2, NX, NY, Lx, Ly, orc.BC_PERIODIC, tau, g=g, zv=zvy, guo=1)
    F = inputs.random_populations(seed, lat.Q, Ly, Lx, lo=0.8, hi=1.2) / lat.Q
    X, _ = lat.collide(F)
    vx, vy = _vel2(NX, NY, zvy)
    rho = _mom(np.ones_like(vx), F)
    ux = (_mom(vx, F) + 0.5 * g) / rho
    uy = _mom(vy, F) / rho
    feq = lat.equilibrium(rho, ux, uy)
    om = 1.0 / (tau + 0.5)
    return F, X, X - F - om * (feq - F), (vx, vy, rho, ux, uy, om)


@pytest.mark.parametrize("NX,NY,zvy", LATTICES)
def test_guo_increment_carries_exactly_g(NX, NY, zvy):
    g = 2.3e-4
    F, X, _, (vx, vy, rho, ux, uy, om) = _force_terms(NX, NY, zvy, 0.37, g, 11)
    d = X - F
    np.testing.assert_allclose(_mom(np.ones_like(vx), d), 0.0, atol=1e-16)
    np.testing.assert_allclose(_mom(vx, d), g, rtol=1e-11)
    np.testing.assert_allclose(_mom(vy, d), 0.0, atol=1e-16)


@pytest.mark.parametrize("NX,NY,zvy", LATTICES)
def test_guo_moment_conditions(NX, NY, zvy):
    g, tau = 1.7e-4, 0.83
    _, _, Fi, (vx, vy, rho, ux, uy, om) = _force_terms(NX, NY, zvy, tau, g, 12)
    a = (1.0 - 0.5 * om) * g
    np.testing.assert_allclose(_mom(np.ones_like(vx), Fi), 0.0, atol=1e-15)
    np.testing.assert_allclose(_mom(vx, Fi), a, rtol=1e-10)
    np.testing.assert_allclose(_mom(vy, Fi), 0.0, atol=1e-15)
    # second moments (g u + u g) with g along x
    np.testing.assert_allclose(_mom(vx * vx, Fi), 2 * a * ux, rtol=1e-8, atol=1e-15)
    np.testing.assert_allclose(_mom(vx * vy, Fi), a * uy, rtol=1e-8, atol=1e-15)
    np.testing.assert_allclose(_mom(vy * vy, Fi), 0.0, atol=1e-15)


def test_guo_d2q9_is_the_published_term():
    """Level 1 on both axes is D2Q9 with c_s^2 = 1/3: Guo's term
    F_i = (1 - omega/2) w_i [(e_i - u)/c_s^2 + (e_i . u) e_i / c_s^4] . g."""
    g, tau = 3.1e-4, 0.61
    _, _, Fi, (vx, vy, rho, ux, uy, om) = _force_terms(1, 1, 0, tau, g, 13)
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    cs2 = 1.0 / 3.0
    for q in range(9):
        ex, ey = vx[q], vy[q]
        w = w1[int(ex)] * w1[int(ey)]
        eu = ex * ux + ey * uy
        want = (1 - 0.5 * om) * w * ((ex - ux) / cs2 + eu * ex / cs2 ** 2) * g
        np.testing.assert_allclose(Fi[q], want, rtol=1e-8, atol=1e-16)


@pytest.mark.parametrize("NX,NY,zvy", LATTICES)
def test_guo_half_force_shift_from_rest(NX, NY, zvy):
    """Uniform periodic box: j grows by g per step and the reported velocity
    is (t + 1/2) g / rho at step t."""
    g, rho0, tau = 4e-5, 1.3, 0.9
    lat = orc.Lattice(2, NX, NY, 3, 2, orc.BC_PERIODIC, tau, g=g, zv=zvy, guo=1)
    X = lat.equilibrium(np.full((2, 3), rho0), np.zeros((2, 3)), np.zeros((2, 3)))
    for t in range(4):
        m = lat.observe(X)
        np.testing.assert_allclose(m[0], rho0, rtol=1e-14)
        np.testing.assert_allclose(m[1], (t + 0.5) * g / rho0, rtol=1e-10)
        np.testing.assert_allclose(m[2], 0.0, atol=1e-15)
        X, bad = lat.run(X, 1)
        assert bad == 0


def test_guo_3d_increment_and_moments():
    g, tau, N = 1.9e-4, 0.7, 2
    Lx, Ly, Lz = 3, 3, 2
    lat = orc.Lattice(3, N, N, Lx, Ly, orc.BC_PERIODIC, tau, g=g, NZ=N, Lz=Lz, guo=1)
    F = inputs.random_populations(14, lat.Q, Lz * Ly, Lx, lo=0.8, hi=1.2).reshape(lat.shape) / lat.Q
    X, _ = lat.collide(F)
    v = np.arange(-N, N + 1).astype(float)
    Q1 = len(v)
    vx = np.tile(v, Q1 * Q1)
    vy = np.tile(np.repeat(v, Q1), Q1)
    vz = np.repeat(v, Q1 * Q1)
    rho = _mom(np.ones_like(vx), F)
    ux, uy, uz = (_mom(vx, F) + 0.5 * g) / rho, _mom(vy, F) / rho, _mom(vz, F) / rho
    om = 1.0 / (tau + 0.5)
    Fi = X - F - om * (lat.equilibrium(rho, ux, uy, uz) - F)
    a = (1 - 0.5 * om) * g
    np.testing.assert_allclose(_mom(vx, X - F), g, rtol=1e-11)
    np.testing.assert_allclose(_mom(np.ones_like(vx), Fi), 0.0, atol=1e-15)
    np.testing.assert_allclose(_mom(vx, Fi), a, rtol=1e-10)
    np.testing.assert_allclose(_mom(vx * vx, Fi), 2 * a * ux, rtol=1e-8, atol=1e-15)
    np.testing.assert_allclose(_mom(vx * vz, Fi), a * uz, rtol=1e-8, atol=1e-15)
    np.testing.assert_allclose(_mom(vy * vz, Fi), 0.0, atol=1e-15)


def test_guo_rejected_in_1d_and_by_the_adjoint():
    with pytest.raises(ValueError):
        orc.Lattice(1, 2, 0, 8, 1, orc.BC_PERIODIC, 0.8, guo=1).run(np.ones((5, 8)), 1)
    lat = orc.Lattice(2, 1, 1, 2, 4, orc.BC_WALLS, 0.8, g=1e-5, guo=1)
    X = lat.equilibrium(np.ones((4, 2)), np.zeros((4, 2)), np.zeros((4, 2)))
    with pytest.raises(ValueError):
        lat.flowrate_grad(X, 2)


def _steady(lat, X, chunk, tol=1e-13, limit=200):
    for _ in range(limit):
        Y, bad = lat.run(X, chunk)
        assert bad == 0
        if np.max(np.abs(Y - X)) < tol:
            return Y
        X = Y
    raise AssertionError("no steady state")


@pytest.mark.parametrize("N", [1, 2, 3])
def test_guo_poiseuille_curvature(N):
    """Force-driven channel between diffuse walls at rest, Kn = 0.01: the
    reported (shifted) velocity is symmetric with the Navier-Stokes curvature
    -g / nu, nu = theta tau: at every bulk node on D2Q9 (whose unidirectional
    steady state is an exact parabola), by a quadratic fit over the middle half
    on the larger lattices (whose short-wave modes ripple the second
    differences); the total reported momentum exceeds the raw momentum by g/2
    per node; and the profile is the linearised force's plus g/2 (both forms
    inject g per node and step, and the terms that differ feed only the
    xx stress, which a unidirectional flow never reads)."""
    Ly, g = 24, 1e-5
    theta = N / 3.0
    tau = orc.tau_from_kn(N, Ly, 0.01)
    nu = theta * tau
    prof = {}
    for guo in (0, 1):
        lat = orc.Lattice(2, N, N, 1, Ly, orc.BC_WALLS, tau, g=g, guo=guo)
        X = lat.equilibrium(np.ones((Ly, 1)), np.zeros((Ly, 1)), np.zeros((Ly, 1)))
        X = _steady(lat, X, chunk=2000)
        prof[guo] = (lat, X, lat.observe(X))
    lat, X, m = prof[1]
    u = m[1][:, 0]
    np.testing.assert_allclose(u, u[::-1], rtol=1e-11)
    mid = slice(Ly // 4, 3 * Ly // 4)
    if N == 1:
        d2 = u[2:] - 2 * u[1:-1] + u[:-2]
        np.testing.assert_allclose(d2[mid], -g / nu, rtol=1e-9)
    else:
        y = np.arange(Ly) + 0.5 - Ly / 2.0
        a = np.polyfit(y[mid], u[mid], 2)[0]
        assert 2 * a == pytest.approx(-g / nu, rel=1e-2)
    F = lat.stream(X)
    vx, _ = _vel2(N, N)
    j = _mom(vx, F)[:, 0]
    np.testing.assert_allclose(np.sum(m[0][:, 0] * u) - np.sum(j), 0.5 * g * Ly, rtol=1e-8)
    np.testing.assert_allclose(u - prof[0][2][1][:, 0], 0.5 * g, rtol=1e-8)
