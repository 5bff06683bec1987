"""Pins of the oracle's channel diagnostics (Sec. 5.3 slip, Sec. 5.4 flow rate
and volumetric flow) against closed forms, and planted mistakes that the pins
must catch.

* A linear Couette profile built with a chosen slip s (gas velocity -U + 2 U s
  at the lower wall plane y = -1/2, U - 2 U s at the upper one) returns s at
  both walls, and the wall-plane velocities exactly.
* The discrete no-slip Poiseuille parabola u(y) = g/(2 nu) s (H - s), s = y + 1/2,
  has sum_y u = g/(2 nu) (H^3/6 + H/12), so J = rho0 times that sum at a
  uniform density rho0, and
  Q Kn = 1/6 + 1/(12 H^2) (Q = 1/(6 Kn) in the continuum, Sec. 5.4 with
  U0 = g H^2 / (8 nu)).
* Averaging over x (and z) removes a zero-mean variation along x.
"""
import types

import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import oracle as orc

SRC = dg.__file__


def couette_fields(s, U, H, nx=4, rho=1.0):
    y = np.arange(H) + 0.5  # distance from the lower wall plane
    u = -U + 2 * U * s + y * (2 * U - 4 * U * s) / H
    ux = np.tile(u[:, None], (1, nx))
    return np.stack([np.full_like(ux, rho), ux])


def poiseuille_fields(g, nu, H, nx=3, rho=1.0):
    s = np.arange(H) + 0.5
    u = g / (2 * nu) * s * (H - s)
    ux = np.tile(u[:, None], (1, nx))
    return np.stack([np.full_like(ux, rho), ux])


def pin_couette(m):
    for s in (0.0, 0.013, 0.2, 0.49):
        for U, H in ((0.05, 256), (0.1, 7)):
            f = couette_fields(s, U, H)
            p = m.velocity_profile(f)
            lo, hi = m.wall_plane_velocities(p)
            assert lo == pytest.approx(-U + 2 * U * s, rel=1e-12, abs=1e-15)
            assert hi == pytest.approx(U - 2 * U * s, rel=1e-12, abs=1e-15)
            slo, shi = m.slip_ratios(p, -U, U)
            assert slo == pytest.approx(s, abs=1e-12)
            assert shi == pytest.approx(s, abs=1e-12)


def pin_poiseuille(m):
    for H, g, tau, theta in ((128, 1e-6, 5.5, 8 / 3), (200, 3e-5, 0.9, 1 / 3), (17, 1e-4, 2.0, 1.0)):
        nu = theta * tau
        f = poiseuille_fields(g, nu, H)
        p = m.velocity_profile(f)
        total = g / (2 * nu) * (H ** 3 / 6 + H / 12)
        assert m.flow_rate(f) == pytest.approx(total, rel=1e-12)
        # J is a momentum: at a uniform density rho0 it is rho0 times the sum
        assert m.flow_rate(poiseuille_fields(g, nu, H, rho=1.3)) == pytest.approx(1.3 * total,
                                                                                   rel=1e-12)
        kn = np.sqrt(2 / theta) * nu / H
        assert m.knudsen(tau, theta, H) == pytest.approx(kn, rel=1e-14)
        Q = m.volumetric_flow(p, g, tau, theta)
        assert Q * kn == pytest.approx(1 / 6 + 1 / (12 * H * H), rel=1e-12)


def pin_averaging(m):
    H, nx = 9, 8
    f = poiseuille_fields(1e-4, 0.5, H, nx=nx)
    base = m.velocity_profile(f)
    wave = 0.01 * np.cos(2 * np.pi * np.arange(nx) / nx)
    g = f.copy()
    g[1] = g[1] + wave[None, :]
    np.testing.assert_allclose(m.velocity_profile(g), base, rtol=0, atol=1e-15)
    # 3D fields [z][y][x]: the mean over z and x
    f3 = np.stack([np.ones((2, H, nx)), np.stack([f[1], f[1] + 2e-3])])
    np.testing.assert_allclose(m.velocity_profile(f3), base + 1e-3, rtol=1e-13)
    assert m.flow_rate(f3) == pytest.approx(m.flow_rate(f) + 1e-3 * H, rel=1e-13)


def all_pins(m):
    pin_couette(m)
    pin_poiseuille(m)
    pin_averaging(m)


def test_pins_hold():
    all_pins(dg)


def test_knudsen_matches_the_oracle_mapping():
    """Eq. (kn) both ways: tau from Kn (the oracle's C mapping), Kn from tau."""
    for N, H, kn in ((4, 256, 0.01), (8, 128, 3.0), (2, 200, 0.5)):
        tau = orc.tau_from_kn(N, H, kn)
        assert dg.knudsen(tau, N / 3, H) == pytest.approx(kn, rel=1e-13)


MUTATIONS = [
    ("lo = p[0] + (p[0] - p[1]) / 2.0", "lo = p[0]"),                        # no extrapolation
    ("hi = p[-1] + (p[-1] - p[-2]) / 2.0", "hi = p[-1] + (p[-1] - p[-2])"),  # a whole node
    ("(ulo - u_wall_lo) / du", "(ulo - u_wall_lo) / (2 * du)"),              # 4 U_w
    ("(u_wall_hi - uhi) / du", "(uhi - u_wall_hi) / du"),                    # sign
    ("return float(j.mean(axis=1).sum())", "return float(j.sum(axis=1).sum())"),  # no 1/nx
    ("U0 = g * H * H / (8.0 * nu)", "U0 = g * H * H / (12.0 * nu)"),
    ("knudsen(tau, theta, H) * 4.0 * U0 * H", "knudsen(tau, theta, H) * 4.0 * U0"),
    ("np.sqrt(2.0 / theta) * theta * tau / H", "np.sqrt(1.0 / theta) * theta * tau / H"),
    ("return ux.mean(axis=(0, 2))", "return ux.mean(axis=(0, 1))"),
    ("rho * ux", "ux"),
]


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistake_is_caught(old, new):
    src = open(SRC).read()
    assert old in src, old
    mod = types.ModuleType("diagnostics_mutant")
    exec(compile(src.replace(old, new), "diagnostics_mutant", "exec"), mod.__dict__)
    with pytest.raises(AssertionError):
        all_pins(mod)
