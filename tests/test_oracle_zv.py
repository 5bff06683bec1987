"""Pins of the oracle on the 2N+2 hierarchy (Sec. 4: the zero velocity removed).

The velocities (n +- 1/2) c take the mean of the 2N+1 equilibria at their two
neighbours (Eqs. maineq01_noball - maineq04_noball). On the lattice of spacing
c/2 the oracle uses, the velocities are the odd integers -(2N+1)..2N+1 and the
lattice temperature is (4N+3)/3 (Eq. temp_2N2 with c = 2).

Checked against what the mathematics fixes, never against the oracle's own
formulas: brute-force enumeration (the mean of two neighbouring equilibria is
the law of N D1Q3 steps plus one fair half-step coin), the mass, momentum and
shifted second moment of Sec. 4, the third moment of App. B, positivity on
the domain of Sec. 3, conservation by the collision, the exact momentum of the
force with theta_x of the hierarchy, periodic streaming as numpy.roll, the
wall rule's mass balance, rest state and emission shape, and the Navier-Stokes
Poiseuille curvature with nu = theta_y tau, for the channel models
G-D1Q6 x D1Q3 and G-D1Q8 x D1Q3 of Sec. 5 (2N+2 along y only) and the fully
symmetric lattices (2N+2 along both axes).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import inputs

ZV_X, ZV_Y = orc.ZV_X, orc.ZV_Y


def _axis_v(N, zv):
    if zv:
        return np.arange(-(2 * N + 1), 2 * N + 2, 2).astype(float)
    return np.arange(-N, N + 1).astype(float)


def _vel(NX, NY, zv):
    vx, vy = _axis_v(NX, zv & ZV_X), _axis_v(NY, zv & ZV_Y)
    return np.tile(vx, len(vy)), np.repeat(vy, len(vx))


def _theta(N, zv):
    return (4 * N + 3) / 3.0 if zv else N / 3.0


def _lat(NX, NY, Lx, Ly, zv, bc=orc.BC_WALLS, tau=0.8, uw_lo=0.0, uw_hi=0.0, g=0.0):
    return orc.Lattice(2, NX, NY, Lx, Ly, bc, tau, uw_lo, uw_hi, g, zv=zv)


def _dice_and_coin(N, u):
    """Exact law of 2 S + B, S the sum of N D1Q3 steps at speed u / 2 (units of c),
    B = +-1 with probability 1/2 each: the velocity in units of c/2."""
    uc = u / 2
    Pp = (Fraction(N, 3) + uc + uc * uc / N) / (2 * N)
    Pm = (Fraction(N, 3) - uc + uc * uc / N) / (2 * N)
    P = {-1: Pm, 0: 1 - Pp - Pm, 1: Pp}
    out = {v: Fraction(0) for v in range(-(2 * N + 1), 2 * N + 2, 2)}
    for seq in itertools.product((-1, 0, 1), repeat=N):
        pr = Fraction(1)
        for s in seq:
            pr *= P[s]
        for b in (-1, 1):
            out[2 * sum(seq) + b] += pr / 2
    return [out[v] for v in sorted(out)]


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_equilibrium_is_dice_plus_coin(N):
    rng = np.random.default_rng(300 + N)
    for _ in range(3):
        u = Fraction(int(rng.integers(-120, 121)), 100)
        exact = _dice_and_coin(N, u)
        np.testing.assert_allclose(orc.eq_axis(N, 1, float(u)), [float(e) for e in exact],
                                   rtol=1e-14, atol=1e-17)


def test_d1q4_rest_weights():
    """N = 1 (four velocities +-1/2 c, +-3/2 c): halves of the D1Q3 weights
    1/6, 2/3, 1/6 summed in neighbouring pairs, 1/12, 5/12, 5/12, 1/12."""
    np.testing.assert_allclose(orc.eq_axis(1, 1, 0.0), [1 / 12, 5 / 12, 5 / 12, 1 / 12],
                               rtol=1e-15)


@pytest.mark.parametrize("N", range(1, 14))
@pytest.mark.parametrize("u", [0.0, 0.11, -0.54, 1.3])
def test_moments_shifted_temperature_and_third(N, u):
    """Sec. 4: mass and momentum exact, second moment u^2 + (4N+3)/3; App. B: the
    third moment is the 2N+1 one at u/2 plus 3/4 c^2 (u/2), all times c^3 = 8."""
    f = orc.eq_axis(N, 1, u)
    v = _axis_v(N, 1)
    assert f.sum() == pytest.approx(1.0, abs=4e-15)
    assert (v * f).sum() == pytest.approx(u, abs=1e-14)
    assert (v * v * f).sum() == pytest.approx(u * u + (4 * N + 3) / 3.0, abs=4e-14)
    uc = u / 2
    m3c = uc ** 3 + 3 * uc * (N / 3.0 + 0.25) - uc ** 3 / N ** 2
    assert (v ** 3 * f).sum() == pytest.approx(8 * m3c, abs=2e-13)


@pytest.mark.parametrize("N", [1, 2, 5, 8, 13])
def test_positive_on_the_positivity_domain(N):
    """Sec. 3 bounds |u/c| by sqrt(2/3) N; on the c/2 lattice that is twice as wide."""
    umax = 2 * np.sqrt(2.0 / 3.0) * N
    for u in np.linspace(-umax, umax, 41) * (1 - 1e-12):
        assert (orc.eq_axis(N, 1, u) >= 0).all()


@pytest.mark.parametrize("zv", [ZV_Y, ZV_X | ZV_Y])
@pytest.mark.parametrize("N", [1, 3])
def test_collision_conserves_mass_and_momentum(N, zv):
    lat = _lat(N, N, 7, 8, zv, tau=0.63)
    F = inputs.random_populations(31, lat.Q, 8, 7)
    X, bad = lat.collide(F)
    assert bad == 0
    nx, ny = _vel(N, N, zv)
    for w in (np.ones_like(nx), nx, ny):
        np.testing.assert_allclose(np.tensordot(w, X, axes=1), np.tensordot(w, F, axes=1),
                                   rtol=0, atol=2e-15)


@pytest.mark.parametrize("zv", [ZV_Y, ZV_X | ZV_Y])
def test_force_injects_exact_momentum_with_theta_x(zv):
    """Sum_i F_i = 0, sum_i xi_x F_i = g: F_i = W_i xi_x g / theta_x needs the
    hierarchy's own theta_x ((4N+3)/3 on the 2N+2 axis)."""
    g = 4.1e-4
    F = inputs.random_populations(32, _lat(2, 3, 5, 8, zv).Q, 8, 5)
    X0, _ = _lat(2, 3, 5, 8, zv, tau=1.2).collide(F)
    Xg, _ = _lat(2, 3, 5, 8, zv, tau=1.2, g=g).collide(F)
    nx, ny = _vel(2, 3, zv)
    np.testing.assert_allclose(np.tensordot(np.ones_like(nx), Xg - X0, axes=1), 0, atol=1e-16)
    np.testing.assert_allclose(np.tensordot(nx, Xg - X0, axes=1), g, rtol=1e-12)
    np.testing.assert_allclose(np.tensordot(ny, Xg - X0, axes=1), 0, atol=1e-16)


@pytest.mark.parametrize("zv", [ZV_Y, ZV_X | ZV_Y])
def test_equilibrium_is_fixed_point_with_lattice_temperature(zv):
    NX, NY = 2, 3
    rho, ux, uy = inputs.random_macro(33, 6, 5)
    lat = _lat(NX, NY, 6, 5, zv, bc=orc.BC_PERIODIC, tau=0.9)
    Feq = lat.equilibrium(rho, ux, uy)
    X, _ = lat.collide(Feq)
    np.testing.assert_allclose(X, Feq, rtol=1e-14, atol=1e-17)
    M = lat.macro(Feq)
    np.testing.assert_allclose(M[1], ux, atol=1e-14)
    np.testing.assert_allclose(M[2], uy, atol=1e-14)
    # the macro temperature is (theta_x + theta_y) / 2 of the equilibrium
    th = 0.5 * (_theta(NX, zv & ZV_X) + _theta(NY, zv & ZV_Y))
    np.testing.assert_allclose(M[3], th, rtol=1e-13)


@pytest.mark.parametrize("zv", [ZV_Y, ZV_X | ZV_Y])
def test_periodic_streaming_is_roll(zv):
    Lx, Ly = 11, 9
    lat = _lat(1, 2, Lx, Ly, zv, bc=orc.BC_PERIODIC)
    X = inputs.random_populations(34, lat.Q, Ly, Lx)
    F = lat.stream(X)
    nx, ny = _vel(1, 2, zv)
    for q in range(lat.Q):
        np.testing.assert_array_equal(
            F[q], np.roll(X[q], shift=(int(ny[q]), int(nx[q])), axis=(0, 1)))


@pytest.mark.parametrize("zv", [ZV_Y, ZV_X | ZV_Y])
@pytest.mark.parametrize("NY", [1, 2, 4])
def test_walls_conserve_mass_and_keep_the_rest_state(NY, zv):
    Ly = 2 * NY + 3
    lat = _lat(2, NY, 6, Ly, zv, uw_lo=-0.06, uw_hi=0.09)
    X = inputs.random_populations(35, lat.Q, Ly, 6)
    F = lat.stream(X)
    assert F.sum() == pytest.approx(X.sum(), rel=1e-14)
    assert (F > 0).all()
    rest = _lat(2, NY, 4, Ly, zv, tau=0.7)
    X = rest.equilibrium(np.ones((Ly, 4)), np.zeros((Ly, 4)), np.zeros((Ly, 4)))
    Y, bad = rest.run(X, 6)
    assert bad == 0
    np.testing.assert_allclose(Y, X, rtol=1e-14)


def test_wall_emits_wall_equilibrium_shape():
    """A diffuse wall re-emits E^x(u_w) W^y into every row a velocity leaving
    it reaches, rows 0..v_y - 1 for the odd v_y = 1..2N+1."""
    NX, NY, Lx, Ly, uw = 1, 2, 3, 7, 0.07
    zv = ZV_Y
    lat = _lat(NX, NY, Lx, Ly, zv, uw_lo=uw)
    X = inputs.random_populations(36, lat.Q, Ly, Lx)
    F = lat.stream(X)
    Ex = orc.eq1d(NX, uw)
    Wy = orc.eq_axis(NY, 1, 0.0)
    vy = _axis_v(NY, 1)
    Qx = 2 * NX + 1
    for x in range(Lx):
        ratios = []
        for iy, v in enumerate(vy):
            if v < 0:
                continue
            for ix in range(Qx):
                for y in range(int(v)):
                    ratios.append(F[iy * Qx + ix, y, x] / (Ex[ix] * Wy[iy]))
        assert len(ratios) == Qx * sum(range(1, 2 * NY + 2, 2))
        np.testing.assert_allclose(ratios, ratios[0], rtol=1e-13)


@pytest.mark.parametrize("NY", [2, 3])
def test_poiseuille_curvature_uses_the_shifted_temperature(NY):
    """Channel models G-D1Q6 x D1Q3 (NY = 2) and G-D1Q8 x D1Q3 (NY = 3) of Sec. 5:
    nu u'' = -g with nu = theta_y tau, theta_y = (4 NY + 3)/3."""
    Ly, g, tau = 28, 1e-5, 0.7
    nu = (4 * NY + 3) / 3.0 * tau
    lat = _lat(1, NY, 1, Ly, ZV_Y, tau=tau, g=g)
    X = lat.equilibrium(np.ones((Ly, 1)), np.zeros((Ly, 1)), np.zeros((Ly, 1)))
    prev = None
    for _ in range(80):
        X, bad = lat.run(X, 500)
        assert bad == 0
        u = lat.observe(X)[1][:, 0]
        if prev is not None and np.abs(u - prev).max() < 1e-11 * np.abs(u).max():
            break
        prev = u
    np.testing.assert_allclose(u, u[::-1], rtol=1e-12)
    y = np.arange(Ly) + 0.5 - Ly / 2.0
    mid = slice(Ly // 4, 3 * Ly // 4)
    a, b, _ = np.polyfit(y[mid], u[mid], 2)
    assert a == pytest.approx(-g / (2 * nu), rel=2e-2)
    # the unshifted temperature NY/3 would give a curvature (4 NY + 3)/NY times larger
    assert abs(a - (-g / (2 * NY / 3.0 * tau))) > 0.5 * abs(a)
    assert abs(b) < 1e-12


def test_couette_is_antisymmetric_with_slip():
    NY, Ly, uw = 2, 20, 0.01
    tau = orc.tau_from_kn(NY, Ly, 0.05, zv=1)
    lat = _lat(1, NY, 1, Ly, ZV_Y, tau=tau, uw_lo=-uw, uw_hi=uw)
    X = lat.equilibrium(np.ones((Ly, 1)), np.zeros((Ly, 1)), np.zeros((Ly, 1)))
    X, bad = lat.run(X, 6000)
    assert bad == 0
    u = lat.observe(X)[1][:, 0]
    np.testing.assert_allclose(u, -u[::-1], atol=1e-14)
    assert np.all(np.diff(u) > 0)
    assert 0 < u[-1] < uw


def test_x_uniform_flow_stays_uniform():
    common = dict(tau=0.85, uw_lo=-0.04, uw_hi=0.03, g=1e-5)
    lat1, lat4 = _lat(2, 2, 1, 9, ZV_X | ZV_Y, **common), _lat(2, 2, 4, 9, ZV_X | ZV_Y, **common)
    rho, ux, uy = inputs.random_macro(37, 1, 9)
    X1 = lat1.equilibrium(rho, ux, uy)
    X4 = lat4.equilibrium(np.repeat(rho, 4, 1), np.repeat(ux, 4, 1), np.repeat(uy, 4, 1))
    X1, _ = lat1.run(X1, 30)
    X4, _ = lat4.run(X4, 30)
    for x in range(4):
        np.testing.assert_array_equal(X4[:, :, x], X1[:, :, 0])


def test_rejected_configurations():
    with pytest.raises(ValueError):
        orc.Lattice(1, 2, 0, 10, 1, orc.BC_PERIODIC, 0.8, zv=ZV_X).stream(np.ones((5, 10)))
    with pytest.raises(ValueError):  # walls need 2 NY + 1 rows for the fastest velocity
        lat = _lat(1, 3, 4, 6, ZV_Y)
        lat.stream(np.ones((lat.Q, 6, 4)))
