"""Pins of the oracle on anisotropic tensor products (Sec. 4 builds a 2D lattice
as the product of two 1D levels): D1Q3 along x times the level-N lattice along
y, the form of the paper's channel models. Each axis keeps its own lattice
units (theta_x = 1/3, theta_y = N/3).

Checked against what the mathematics fixes: the product equilibrium and its
moments, conservation of mass and momentum by the collision, the exact
momentum of the force, the wall rule's mass balance and rest state, and the
Navier-Stokes Poiseuille curvature -g / (2 theta_y tau) (momentum along x
diffuses along y with nu = theta_y tau).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import inputs


def _lat(NY, Lx, Ly, bc=orc.BC_WALLS, tau=0.8, uw_lo=0.0, uw_hi=0.0, g=0.0, NX=1):
    return orc.Lattice(2, NX, NY, Lx, Ly, bc, tau, uw_lo, uw_hi, g)


def _vel(NX, NY):
    nx = np.tile(np.arange(-NX, NX + 1), 2 * NY + 1).astype(float)
    ny = np.repeat(np.arange(-NY, NY + 1), 2 * NX + 1).astype(float)
    return nx, ny


@pytest.mark.parametrize("NY", [2, 4, 8])
def test_equilibrium_is_product_with_exact_moments(NY):
    rho, ux, uy = inputs.random_macro(21, 5, 9)
    lat = _lat(NY, 5, 9)
    X = lat.equilibrium(rho, ux, uy)
    assert X.shape == (3 * (2 * NY + 1), 9, 5)
    for y in range(9):
        for x in range(5):
            want = rho[y, x] * np.outer(orc.eq1d(NY, uy[y, x]), orc.eq1d(1, ux[y, x])).ravel()
            np.testing.assert_allclose(X[:, y, x], want, rtol=1e-14, atol=1e-18)
    nx, ny = _vel(1, NY)
    m = lambda w: np.tensordot(w, X, axes=1)  # noqa: E731
    np.testing.assert_allclose(m(np.ones_like(nx)), rho, rtol=1e-14)
    np.testing.assert_allclose(m(nx), rho * ux, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(m(ny), rho * uy, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(m(nx * nx), rho * (ux ** 2 + 1 / 3), rtol=1e-13)
    np.testing.assert_allclose(m(ny * ny), rho * (uy ** 2 + NY / 3), rtol=1e-13)


@pytest.mark.parametrize("NY", [3, 5])
def test_collision_conserves_mass_and_momentum(NY):
    lat = _lat(NY, 7, 6, tau=0.63)
    F = inputs.random_populations(22, lat.Q, 6, 7)
    X, bad = lat.collide(F)
    assert bad == 0
    nx, ny = _vel(1, NY)
    for w in (np.ones_like(nx), nx, ny):
        np.testing.assert_allclose(np.tensordot(w, X, axes=1), np.tensordot(w, F, axes=1),
                                   rtol=0, atol=1e-15)


def test_force_injects_exact_momentum_with_theta_x():
    g = 2.9e-4
    F = inputs.random_populations(23, 3 * 9, 4, 6)
    X0, _ = _lat(4, 6, 4, tau=1.3).collide(F)
    Xg, _ = _lat(4, 6, 4, tau=1.3, g=g).collide(F)
    nx, ny = _vel(1, 4)
    np.testing.assert_allclose(np.tensordot(np.ones_like(nx), Xg - X0, axes=1), 0, atol=1e-16)
    np.testing.assert_allclose(np.tensordot(nx, Xg - X0, axes=1), g, rtol=1e-12)
    np.testing.assert_allclose(np.tensordot(ny, Xg - X0, axes=1), 0, atol=1e-16)


@pytest.mark.parametrize("NY", [2, 4])
def test_walls_conserve_mass_and_keep_the_rest_state(NY):
    lat = _lat(NY, 6, 9, uw_lo=-0.06, uw_hi=0.04)
    X = inputs.random_populations(24, lat.Q, 9, 6)
    assert lat.stream(X).sum() == pytest.approx(X.sum(), rel=1e-14)
    rest = _lat(NY, 4, 9, tau=0.7)
    X = rest.equilibrium(np.ones((9, 4)), np.zeros((9, 4)), np.zeros((9, 4)))
    Y, bad = rest.run(X, 5)
    assert bad == 0
    np.testing.assert_allclose(Y, X, rtol=1e-14)


def test_poiseuille_curvature_uses_theta_y():
    NY, Ly, g, tau = 3, 24, 1e-5, 0.75
    nu = NY / 3.0 * tau
    lat = _lat(NY, 1, Ly, tau=tau, g=g)
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
    # the isotropic lattice of the same level would give -g / (2 theta tau) with
    # theta = 1/3 along x: a factor NY away, which the fit must exclude
    assert abs(a - (-g / (2 * tau / 3.0))) > 0.5 * abs(a)
    assert abs(b) < 1e-12


def test_x_uniform_flow_stays_uniform():
    common = dict(tau=0.9, uw_lo=-0.03, uw_hi=0.05, g=2e-5)
    lat1, lat4 = _lat(3, 1, 10, **common), _lat(3, 4, 10, **common)
    rho, ux, uy = inputs.random_macro(25, 1, 10)
    X1 = lat1.equilibrium(rho, ux, uy)
    X4 = lat4.equilibrium(np.repeat(rho, 4, 1), np.repeat(ux, 4, 1), np.repeat(uy, 4, 1))
    X1, _ = lat1.run(X1, 40)
    X4, _ = lat4.run(X4, 40)
    for x in range(4):
        np.testing.assert_array_equal(X4[:, :, x], X1[:, :, 0])
