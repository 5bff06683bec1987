"""Channel diagnostics of Sec. 5.3 (Couette slip) and Sec. 5.4 (flow rate,
volumetric flow) computed from the oracle's moment fields, in plain numpy FP64.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the CUDA path never
does.

The fields are those of ``oracle.Lattice.observe`` (rho first, u_x second;
[y][x] in 2D, [z][y][x] in 3D). Lattice units: node spacing 1, walls halfway,
at y = -1/2 and y = ny - 1/2 (channel width H = ny).
"""
from __future__ import annotations

import numpy as np


def velocity_profile(fields):
    """<u_x>(y): the streamwise velocity averaged over x (and z)."""
    ux = np.asarray(fields[1], dtype=np.float64)
    if ux.ndim == 3:  # [z][y][x]
        return ux.mean(axis=(0, 2))
    return ux.mean(axis=1)


def flow_rate(fields):
    """J = sum over y of the x (and z) average of rho u_x: the streamwise
    momentum per unit width, whose gradient the adjoint computes."""
    rho = np.asarray(fields[0], dtype=np.float64)
    ux = np.asarray(fields[1], dtype=np.float64)
    j = rho * ux
    if j.ndim == 3:
        return float(j.mean(axis=(0, 2)).sum())
    return float(j.mean(axis=1).sum())


def wall_plane_velocities(profile):
    """Gas velocity at the wall planes y = -1/2 and y = ny - 1/2: the profile
    continued by the straight line through its two nearest rows (the paper
    evaluates u at the wall, Sec. 5.3; with halfway walls the wall lies half a
    node outside the first row)."""
    p = np.asarray(profile, dtype=np.float64)
    if p.size == 1:
        return float(p[0]), float(p[0])
    lo = p[0] + (p[0] - p[1]) / 2.0
    hi = p[-1] + (p[-1] - p[-2]) / 2.0
    return float(lo), float(hi)


def slip_ratios(profile, u_wall_lo, u_wall_hi):
    """Couette slip of Sec. 5.3, u(0) / (2 U_w), taken in the frame of each
    wall: the gas velocity at the wall plane relative to the wall, over the
    walls' velocity difference (2 U_w for walls at -U_w and +U_w). It is 0
    without slip and 1/2 in the free-molecular limit."""
    ulo, uhi = wall_plane_velocities(profile)
    du = u_wall_hi - u_wall_lo
    return (ulo - u_wall_lo) / du, (u_wall_hi - uhi) / du


def knudsen(tau, theta, H):
    """Eq. (kn): Kn = sqrt(2/theta) nu / H with nu = theta tau."""
    return np.sqrt(2.0 / theta) * theta * tau / H


def volumetric_flow(profile, g, tau, theta):
    """Volumetric flow of Sec. 5.4, Q = delta / (4 U0 H) int_0^H u ds with
    delta = 1/Kn and U0 = g H^2 / (8 nu) the no-slip centreline speed of the
    force g per unit mass (nu = theta tau, H = ny, ds = 1 per row)."""
    p = np.asarray(profile, dtype=np.float64)
    H = float(p.size)
    nu = theta * tau
    U0 = g * H * H / (8.0 * nu)
    return float(p.sum() / (knudsen(tau, theta, H) * 4.0 * U0 * H))
