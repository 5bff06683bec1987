"""Pins of the oracle's forward-mode gradient of the flow rate.

The dual-number tangents (d/dtau, d/dg carried through every stream and
collide) are checked against central finite differences of the oracle's own
primal runs, against the linearity of the flow in the body force (Sec. 5.4:
J = g dJ/dg for a slow flow), and against the Navier-Stokes scaling of a
force-driven channel at small Knudsen number (J ~ 1/nu, nu = theta tau).
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
