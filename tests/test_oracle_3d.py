"""Pins of the oracle on 3D tensor products (Sec. 4: the product of 1D levels
extends to any number of axes), checked against what the mathematics fixes:

* the D3Q27 weights (N = 1) are the textbook ones, (2/3)^3, (2/3)^2 (1/6),
  (2/3) (1/6)^2, (1/6)^3;
* the product equilibrium has the exact moments of every axis;
* the collision conserves mass and the three momenta; the force injects g;
* periodic streaming is numpy.roll along the three axes;
* the walls conserve mass and keep the rest state;
* a z-uniform 3D state f2 W^z (any f2) steps to (2D step of f2) W^z, which
  ties the 3D oracle to the pinned 2D one;
* on a fully periodic lattice, exchanging the x and z axes commutes with a
  step (no transposed index).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import inputs


def _lat3(N, Lx, Ly, Lz, bc=orc.BC_WALLS, tau=0.8, uw_lo=0.0, uw_hi=0.0, g=0.0):
    return orc.Lattice(3, N, N, Lx, Ly, bc, tau, uw_lo, uw_hi, g, NZ=N, Lz=Lz)


def _vel3(N):
    v = np.arange(-N, N + 1).astype(float)
    Q1 = 2 * N + 1
    nx = np.tile(v, Q1 * Q1)
    ny = np.tile(np.repeat(v, Q1), Q1)
    nz = np.repeat(v, Q1 * Q1)
    return nx, ny, nz


def _fields3(seed, Lx, Ly, Lz, amp=0.03):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, (Lz, Ly, Lx))
    u = [amp * rng.uniform(-1, 1, (Lz, Ly, Lx)) for _ in range(3)]
    return rho, u[0], u[1], u[2]


def test_d3q27_weights():
    lat = _lat3(1, 1, 1, 1, bc=orc.BC_PERIODIC)
    W = lat.equilibrium(np.ones((1, 1, 1)), np.zeros((1, 1, 1)), np.zeros((1, 1, 1)),
                        np.zeros((1, 1, 1))).ravel()
    nx, ny, nz = _vel3(1)
    k = np.abs(nx) + np.abs(ny) + np.abs(nz)
    expect = np.choose(k.astype(int), [8 / 27, 2 / 27, 1 / 54, 1 / 216])
    np.testing.assert_allclose(W, expect, rtol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_equilibrium_moments_per_axis(N):
    rho, ux, uy, uz = _fields3(50 + N, 3, 4, 2)
    lat = _lat3(N, 3, 4, 2, bc=orc.BC_PERIODIC)
    X = lat.equilibrium(rho, ux, uy, uz)
    nx, ny, nz = _vel3(N)
    m = lambda w: np.tensordot(w, X, axes=1)  # noqa: E731
    np.testing.assert_allclose(m(np.ones_like(nx)), rho, rtol=1e-14)
    for v, u in ((nx, ux), (ny, uy), (nz, uz)):
        np.testing.assert_allclose(m(v), rho * u, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(m(v * v), rho * (u * u + N / 3.0), rtol=1e-13)
    np.testing.assert_allclose(m(nx * nz), rho * ux * uz, rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_equilibrium_moment_fields(N):
    """The reducer's fields of a local equilibrium: T = N/3, no shear stress,
    and q_a = half the third central moment of axis a, -rho u_a^3 / N^2 (the
    third moment of Sec. 3); field order rho, ux, uy, T, qx, qy, sxy, uz, qz."""
    rho, ux, uy, uz = _fields3(60 + N, 3, 4, 2)
    lat = _lat3(N, 3, 4, 2, bc=orc.BC_PERIODIC)
    M = lat.macro(lat.equilibrium(rho, ux, uy, uz))
    np.testing.assert_allclose(M[3], N / 3.0, rtol=1e-13)
    np.testing.assert_allclose(M[6], 0.0, rtol=0, atol=1e-14)
    for i, u in ((4, ux), (5, uy), (8, uz)):
        np.testing.assert_allclose(M[i], -rho * u ** 3 / (2 * N ** 2), rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("N", [1, 2])
def test_collision_conserves_mass_and_momenta(N):
    lat = _lat3(N, 5, 4, 3, tau=0.63)
    F = inputs.random_populations(60 + N, lat.Q, 4, 5 * 3).reshape(lat.Q, 3, 4, 5)
    X, bad = lat.collide(F)
    assert bad == 0
    nx, ny, nz = _vel3(N)
    for w in (np.ones_like(nx), nx, ny, nz):
        np.testing.assert_allclose(np.tensordot(w, X, axes=1), np.tensordot(w, F, axes=1),
                                   rtol=0, atol=2e-15)


def test_force_injects_exact_momentum():
    g = 2.3e-4
    F = inputs.random_populations(62, 125, 4, 3 * 4).reshape(125, 3, 4, 4)
    X0, _ = _lat3(2, 4, 4, 3, tau=1.1).collide(F)
    Xg, _ = _lat3(2, 4, 4, 3, tau=1.1, g=g).collide(F)
    nx, ny, nz = _vel3(2)
    d = Xg - X0
    np.testing.assert_allclose(np.tensordot(np.ones_like(nx), d, axes=1), 0, atol=1e-16)
    np.testing.assert_allclose(np.tensordot(nx, d, axes=1), g, rtol=1e-12)
    np.testing.assert_allclose(np.tensordot(ny, d, axes=1), 0, atol=1e-16)
    np.testing.assert_allclose(np.tensordot(nz, d, axes=1), 0, atol=1e-16)


def test_periodic_streaming_is_roll():
    lat = _lat3(1, 5, 4, 3, bc=orc.BC_PERIODIC)
    X = inputs.random_populations(63, 27, 4, 15).reshape(27, 3, 4, 5)
    F = lat.stream(X)
    nx, ny, nz = _vel3(1)
    for q in range(27):
        np.testing.assert_array_equal(
            F[q], np.roll(X[q], shift=(int(nz[q]), int(ny[q]), int(nx[q])), axis=(0, 1, 2)))


@pytest.mark.parametrize("N", [1, 2])
def test_walls_conserve_mass_and_keep_the_rest_state(N):
    lat = _lat3(N, 4, N + 3, 3, uw_lo=-0.04, uw_hi=0.05)
    Q = lat.Q
    X = inputs.random_populations(64, Q, N + 3, 12).reshape(Q, 3, N + 3, 4)
    F = lat.stream(X)
    assert F.sum() == pytest.approx(X.sum(), rel=1e-14)
    assert (F > 0).all()
    rest = _lat3(N, 3, N + 3, 2, tau=0.7)
    ones = np.ones((2, N + 3, 3))
    X = rest.equilibrium(ones, 0 * ones, 0 * ones, 0 * ones)
    Y, bad = rest.run(X, 5)
    assert bad == 0
    np.testing.assert_allclose(Y, X, rtol=1e-14)


@pytest.mark.parametrize("bc", [orc.BC_WALLS, orc.BC_PERIODIC])
@pytest.mark.parametrize("N", [1, 2])
def test_z_uniform_state_steps_like_2d(N, bc):
    """f3 = f2 W^z stays a product under a 3D step, with f2 stepped in 2D."""
    Lx, Ly, Lz = 5, N + 4, 3
    common = dict(tau=0.77, uw_lo=-0.03, uw_hi=0.045, g=3e-5)
    lat2 = orc.Lattice(2, N, N, Lx, Ly, bc, **common)
    lat3 = _lat3(N, Lx, Ly, Lz, bc=bc, **common)
    f2 = inputs.random_populations(65 + N, lat2.Q, Ly, Lx)
    Wz = orc.weights(N)
    Q1 = 2 * N + 1
    f3 = (Wz[:, None, None, None, None] * f2.reshape(1, lat2.Q, 1, Ly, Lx)) * np.ones((1, 1, Lz, 1, 1))
    f3 = f3.reshape(Q1 * lat2.Q, Lz, Ly, Lx)
    y2, _ = lat2.run(f2, 3)
    y3, _ = lat3.run(f3, 3)
    want = (Wz[:, None, None, None, None] * y2.reshape(1, lat2.Q, 1, Ly, Lx)) * np.ones((1, 1, Lz, 1, 1))
    np.testing.assert_allclose(y3, want.reshape(y3.shape), rtol=1e-13, atol=1e-17)


def test_exchanging_x_and_z_commutes_with_a_step():
    N, L = 1, 4
    lat = _lat3(N, L, 5, L, bc=orc.BC_PERIODIC, tau=0.9)
    rho, ux, uy, uz = _fields3(66, L, 5, L, amp=0.05)
    X = lat.equilibrium(rho, ux, uy, uz)
    Q1 = 2 * N + 1
    swap = lambda A: A.reshape(Q1, Q1, Q1, L, 5, L).transpose(2, 1, 0, 5, 4, 3).reshape(A.shape)  # noqa: E731
    a, _ = lat.run(X, 4)
    b, _ = lat.run(swap(X), 4)
    np.testing.assert_allclose(swap(a), b, rtol=1e-13, atol=1e-17)
