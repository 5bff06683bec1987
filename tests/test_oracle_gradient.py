"""Pins of the oracle's forward-mode gradient of the flow rate.

The dual-number tangents (d/dtau, d/dg and d/du_wall of both walls carried
through every stream and collide) are checked against central finite
differences of the oracle's own primal runs, against the linearity of the
flow in the body force (Sec. 5.4: J = g dJ/dg for a slow flow), against the
Navier-Stokes scaling of a force-driven channel at small Knudsen number
(J ~ 1/nu, nu = theta tau), and against a closed form for the walls: in a
steady channel, moving both walls by the same small speed moves the whole gas
with them (a uniform flow at the walls' speed is a steady state of the wall
rule), and the reflection y -> H - 1 - y exchanges the walls, so each wall's
derivative of J = sum_y rho u_x is rho H / 2.
"""
import numpy as np
import pytest

from oracle import oracle as orc


def _poiseuille(N, Ly, tau, g, Lx=1):
    return orc.Lattice(2, N, N, Lx, Ly, orc.BC_WALLS, tau, 0.0, 0.0, g)


def _rest(lat, Ly, Lx=1):
    return lat.equilibrium(np.ones((Ly, Lx)), np.zeros((Ly, Lx)), np.zeros((Ly, Lx)))


@pytest.mark.parametrize("N,tau,uw", [(2, 0.9, 0.0), (3, 2.5, 0.03), (1, 0.7, -0.02)])
def test_tangents_match_central_differences(N, tau, uw):
    Ly, g, steps = 10, 2e-5, 120
    lat = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau, -uw, uw, g)
    rho = 1.0 + 0.01 * np.sin(np.arange(Ly) / 3.0)[:, None] * np.ones((1, 3))
    X = lat.equilibrium(rho, 0.01 * np.ones((Ly, 3)), np.zeros((Ly, 3)))
    J, dtau, dg = lat.flowrate_grad(X, steps)
    assert J == pytest.approx(lat.flowrate(X, steps), rel=1e-13)
    h = 1e-5 * tau
    Jp = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau + h, -uw, uw, g).flowrate(X, steps)
    Jm = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau - h, -uw, uw, g).flowrate(X, steps)
    assert dtau == pytest.approx((Jp - Jm) / (2 * h), rel=1e-6, abs=1e-12)
    hg = 1e-4 * g
    Gp = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau, -uw, uw, g + hg).flowrate(X, steps)
    Gm = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau, -uw, uw, g - hg).flowrate(X, steps)
    assert dg == pytest.approx((Gp - Gm) / (2 * hg), rel=1e-6)
    # the wall speeds, one at a time
    _, _, _, dlo, dhi = lat.flowrate_grad(X, steps, walls=True)
    hu = 1e-5
    for d, lo, hi in ((dlo, (hu, 0.0), (-hu, 0.0)), (dhi, (0.0, hu), (0.0, -hu))):
        Up = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau, -uw + lo[0], uw + lo[1], g).flowrate(X, steps)
        Um = orc.Lattice(2, N, N, 3, Ly, orc.BC_WALLS, tau, -uw + hi[0], uw + hi[1], g).flowrate(X, steps)
        assert d == pytest.approx((Up - Um) / (2 * hu), rel=1e-6)


@pytest.mark.parametrize("N", [1, 3])
def test_wall_speed_tangents_with_unequal_walls(N):
    """Walls at different speeds (not mirror images), a sheared start: each
    wall's tangent against central differences."""
    Ly, tau, steps = 9, 0.8, 150
    ulo, uhi = 0.08, -0.03
    lat = orc.Lattice(2, N, N, 2, Ly, orc.BC_WALLS, tau, ulo, uhi, 1e-5)
    ux = 0.02 * np.linspace(-1, 1, Ly)[:, None] * np.ones((1, 2))
    X = lat.equilibrium(np.ones((Ly, 2)), ux, np.zeros((Ly, 2)))
    _, _, _, dlo, dhi = lat.flowrate_grad(X, steps, walls=True)
    h = 1e-5

    def J(a, b):
        return orc.Lattice(2, N, N, 2, Ly, orc.BC_WALLS, tau, a, b, 1e-5).flowrate(X, steps)

    assert dlo == pytest.approx((J(ulo + h, uhi) - J(ulo - h, uhi)) / (2 * h), rel=1e-7)
    assert dhi == pytest.approx((J(ulo, uhi + h) - J(ulo, uhi - h)) / (2 * h), rel=1e-7)


@pytest.mark.parametrize("N,kn", [(1, 0.05), (2, 0.5)])
def test_wall_speed_derivatives_of_a_steady_channel(N, kn):
    """Steady Couette channel between walls at rest: dJ/du_wall_lo = dJ/du_wall_hi
    = H / 2 (rho = 1), at any Knudsen number."""
    Ly = 8
    tau = orc.tau_from_kn(N, Ly, kn)
    lat = orc.Lattice(2, N, N, 1, Ly, orc.BC_WALLS, tau, 0.0, 0.0, 0.0)
    steps = int(40 * Ly * Ly / (N / 3.0 * tau) + 200 * tau) + 200
    J, _, _, dlo, dhi = lat.flowrate_grad(_rest(lat, Ly), steps, walls=True)
    assert J == pytest.approx(0.0, abs=1e-14)
    assert dlo == pytest.approx(Ly / 2.0, rel=1e-6)
    assert dhi == pytest.approx(Ly / 2.0, rel=1e-6)


def test_wall_speed_derivatives_vanish_without_walls():
    N, L = 2, 6
    lat = orc.Lattice(2, N, N, 3, L, orc.BC_PERIODIC, 0.8, 0.02, -0.01, 1e-5)
    X = lat.equilibrium(np.ones((L, 3)), 0.01 * np.ones((L, 3)), np.zeros((L, 3)))
    _, _, _, dlo, dhi = lat.flowrate_grad(X, 20, walls=True)
    assert dlo == 0.0 and dhi == 0.0


def test_flow_is_linear_in_the_force():
    N, Ly, g = 2, 16, 1e-6
    lat = _poiseuille(N, Ly, 1.1, g)
    J, _, dg = lat.flowrate_grad(_rest(lat, Ly), 3000)
    assert dg * g == pytest.approx(J, rel=1e-6)


def test_small_knudsen_flow_rate_scales_inversely_with_viscosity():
    """Force-driven channel near Navier-Stokes: J = A/tau + B with a small slip part B,
    so -tau dJ/dtau / J lies a little below 1."""
    N, Ly, g = 2, 24, 1e-6
    tau = 0.75
    lat = _poiseuille(N, Ly, tau, g)
    J, dtau, _ = lat.flowrate_grad(_rest(lat, Ly), 12000)
    r = -tau * dtau / J
    assert 0.7 < r < 1.0
