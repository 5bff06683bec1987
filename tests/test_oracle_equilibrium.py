"""Pins of the oracle's equilibrium against what the paper and mathematics fix.

Each test compares the factorial-sum equilibrium of Sec. 2 (Eq. maineq03,
evaluated by the C oracle) with something computed another way: the paper's
worked example (App. A), the textbook D1Q3 (Sec. 2), exact brute-force
enumeration of the N dice rolls, the moment generating function (Eq. mgf),
the moment identities of Secs. 2-3 and App. B, and the positivity bound of
Sec. 3.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                n, w = line.split()
                rows.append((int(n), Fraction(w)))
    return rows


def test_d1q3_rest_weights_golden():
    w = orc.weights(1)
    for n, frac in _golden("d1q3_weights.txt"):
        assert w[n + 1] == pytest.approx(float(frac), abs=4e-16)


def test_appendix_a_rest_weights_golden():
    w = orc.weights(2)
    for n, frac in _golden("appA_N2_rest_weights.txt"):
        assert w[n + 2] == pytest.approx(float(frac), abs=4e-16)


@pytest.mark.parametrize("u", [0.0, 0.013, -0.2, 0.41, -0.6])
@pytest.mark.parametrize("c", [1.0, math.sqrt(3.0), 0.7])
def test_d1q3_is_textbook(u, c):
    """N = 1 is the root model of Sec. 2: f_{+-1} = rho/6 (1 +- 3u/c + 3u^2/c^2),
    f_0 = 4 rho/6 (1 - 3u^2/(2c^2)), with c_s^2 = c^2/3."""
    f, _ = orc.prob(1, c, c * c / 3.0, u)
    fm = (1 - 3 * u / c + 3 * u * u / c ** 2) / 6
    f0 = 4 * (1 - 1.5 * u * u / c ** 2) / 6
    fp = (1 + 3 * u / c + 3 * u * u / c ** 2) / 6
    np.testing.assert_allclose(f, [fm, f0, fp], rtol=0, atol=2e-16)


@pytest.mark.parametrize("u", [0.0, 0.3, -0.55, 1.1])
def test_appendix_a_worked_example(u):
    """App. A: N = 2 at unit temperature, c = sqrt(3/2),
    P_{2,+-} = (1 +- c u + u^2/2)/(4 c^2), and
    f_{2} = P+^2, f_1 = 2 P0 P+, f_0 = P0^2 + 2 P+ P-, f_{-1} = 2 P0 P-, f_{-2} = P-^2."""
    c = math.sqrt(1.5)
    Pp = (1 + c * u + u * u / 2) / (4 * c * c)
    Pm = (1 - c * u + u * u / 2) / (4 * c * c)
    P0 = 1 - Pp - Pm
    expect = [Pm * Pm, 2 * P0 * Pm, P0 * P0 + 2 * Pp * Pm, 2 * P0 * Pp, Pp * Pp]
    f, _ = orc.prob(2, c, 1.0, u)
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-15)


def _bruteforce(N, Pp, Pm):
    """Exact distribution of the sum of N i.i.d. rolls of {-1, 0, +1}: enumerate
    all 3^N sequences with rational probabilities (the dice problem of Sec. 2)."""
    P0 = 1 - Pp - Pm
    p = {-1: Pm, 0: P0, 1: Pp}
    out = {n: Fraction(0) for n in range(-N, N + 1)}
    for seq in itertools.product((-1, 0, 1), repeat=N):
        pr = Fraction(1)
        for s in seq:
            pr *= p[s]
        out[sum(seq)] += pr
    return [out[n] for n in range(-N, N + 1)]


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_factorial_sum_equals_bruteforce_enumeration(N):
    rng = np.random.default_rng(100 + N)
    for _ in range(3):
        # lattice units: c = 1, c_s^2 = N/3; pick a rational u inside positivity
        u = Fraction(int(rng.integers(-60, 61)), 100)
        Pp = (Fraction(N, 3) + u + u * u / N) / (2 * N)
        Pm = (Fraction(N, 3) - u + u * u / N) / (2 * N)
        exact = _bruteforce(N, Pp, Pm)
        f = orc.eq1d(N, float(u))
        np.testing.assert_allclose(f, [float(e) for e in exact], rtol=1e-14, atol=1e-17)


@pytest.mark.parametrize("N", range(1, 9))
def test_rest_weights_are_powers_of_d1q3(N):
    """At u = 0 the N-fold sum of D1Q3 has weights = coefficients of ((z^-1 + 4 + z)/6)^N
    (App. A for N = 2): exact rational polynomial power."""
    poly = [Fraction(1)]
    for _ in range(N):
        new = [Fraction(0)] * (len(poly) + 2)
        for i, a in enumerate(poly):
            new[i] += a * Fraction(1, 6)
            new[i + 1] += a * Fraction(4, 6)
            new[i + 2] += a * Fraction(1, 6)
        poly = new
    np.testing.assert_allclose(orc.weights(N), [float(p) for p in poly], rtol=4e-15)


@pytest.mark.parametrize("N", range(1, 9))
@pytest.mark.parametrize("u", [0.0, 0.05, -0.27, 0.8])
def test_first_three_moments_exact(N, u):
    """Sec. 2: every level has mean u and variance c_s^2 = N/3 (lattice units)."""
    f = orc.eq1d(N, u)
    n = np.arange(-N, N + 1, dtype=np.float64)
    assert f.sum() == pytest.approx(1.0, abs=2e-15)
    assert (n * f).sum() == pytest.approx(u, abs=2e-15)
    assert (n * n * f).sum() == pytest.approx(u * u + N / 3.0, abs=5e-15)


@pytest.mark.parametrize("N", range(1, 9))
@pytest.mark.parametrize("u", [0.07, -0.3, 0.5])
def test_third_moment_error_appendix_b(N, u):
    """App. B: m_3 = u^3 + 3 u theta_0 - u^3/N^2 (Sec. 3 prints the error's magnitude)."""
    f = orc.eq1d(N, u)
    n = np.arange(-N, N + 1, dtype=np.float64)
    theta = N / 3.0
    assert (n ** 3 * f).sum() == pytest.approx(u ** 3 + 3 * u * theta - u ** 3 / N ** 2,
                                               abs=1e-14)


@pytest.mark.parametrize("N", range(1, 9))
@pytest.mark.parametrize("u", [0.07, -0.3, 0.5])
def test_fourth_moment_error(N, u):
    """Fourth moment (Sec. 3, App. B; the two printed forms disagree, the derived one
    is m_4 - (u^4 + 6u^2 theta + 3 theta^2) = -3 theta u^2/N^2 - (4/N^2 - 3/N^3) u^4)."""
    f = orc.eq1d(N, u)
    n = np.arange(-N, N + 1, dtype=np.float64)
    th = N / 3.0
    maxwell = u ** 4 + 6 * u * u * th + 3 * th * th
    err = -3 * th * u * u / N ** 2 - (4.0 / N ** 2 - 3.0 / N ** 3) * u ** 4
    assert (n ** 4 * f).sum() == pytest.approx(maxwell + err, abs=2e-14)


@pytest.mark.parametrize("N", [1, 2, 4, 8])
@pytest.mark.parametrize("u", [0.0, 0.2, -0.45])
def test_moment_generating_function(N, u):
    """Eq. (mgf): sum_n e^{n c s} f_n = (P- e^{-cs} + P0 + P+ e^{cs})^N; c = 1 here."""
    f = orc.eq1d(N, u)
    n = np.arange(-N, N + 1, dtype=np.float64)
    Pp = (N / 3.0 + u + u * u / N) / (2 * N)
    Pm = (N / 3.0 - u + u * u / N) / (2 * N)
    P0 = 1 - Pp - Pm
    for s in (-0.7, -0.1, 0.3, 1.2):
        lhs = (np.exp(n * s) * f).sum()
        rhs = (Pm * math.exp(-s) + P0 + Pp * math.exp(s)) ** N
        assert lhs == pytest.approx(rhs, rel=1e-13)


def test_moment_errors_decrease_with_level():
    """Sec. 3: the third and fourth moment errors shrink monotonically as N grows."""
    u = 0.4
    e3, e4 = [], []
    for N in range(1, 10):
        f = orc.eq1d(N, u)
        n = np.arange(-N, N + 1, dtype=np.float64)
        th = N / 3.0
        e3.append(abs((n ** 3 * f).sum() - (u ** 3 + 3 * u * th)))
        e4.append(abs((n ** 4 * f).sum() - (u ** 4 + 6 * u * u * th + 3 * th * th)))
    assert all(a > b for a, b in zip(e3, e3[1:]))
    assert all(a > b for a, b in zip(e4, e4[1:]))


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_positivity_domain(N):
    """Sec. 3: the equilibrium is non-negative iff |u| <= sqrt(2/3) N c (c = 1)."""
    umax = math.sqrt(2.0 / 3.0) * N
    for u in (0.0, 0.5 * umax, 0.999 * umax, -0.999 * umax):
        f, flag = orc.prob(N, 1.0, N / 3.0, u)
        assert not flag and (f >= -1e-15).all()
    for u in (1.001 * umax, -1.02 * umax):
        f, flag = orc.prob(N, 1.0, N / 3.0, u)
        assert flag
    # P0 changes sign exactly at the bound
    Pp = (N / 3.0 + umax + umax * umax / N) / (2 * N)
    Pm = (N / 3.0 - umax + umax * umax / N) / (2 * N)
    assert 1 - Pp - Pm == pytest.approx(0.0, abs=1e-15)


def test_physical_units_scale():
    """Eq. maineq06: with c = sqrt(3 theta_0/N) the physical-unit equilibrium at
    velocity u equals the lattice-unit one at u/c (the distribution is a function
    of u/c only)."""
    for N in (2, 5):
        theta0 = 0.37
        c = math.sqrt(3 * theta0 / N)
        for u in (0.01, -0.12):
            fp, _ = orc.prob(N, c, theta0, u)
            np.testing.assert_allclose(fp, orc.eq1d(N, u / c), rtol=1e-13, atol=1e-17)


@pytest.mark.parametrize("N,H,kn", [(4, 256, 0.01), (8, 128, 1.0), (5, 128, 0.1), (2, 1000, 0.01)])
def test_knudsen_mapping(N, H, kn):
    """Eq. (kn): Kn = sqrt(2/theta) nu / H with nu = theta tau (Sec. 5.2)."""
    tau = orc.tau_from_kn(N, H, kn)
    theta = N / 3.0
    assert math.sqrt(2.0 / theta) * theta * tau / H == pytest.approx(kn, rel=1e-14)
