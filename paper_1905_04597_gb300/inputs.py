"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the lattice Boltzmann method: it draws
random numbers and lays out the workload recipes (sizes, levels, Knudsen
numbers, wall speeds, forces) of the paper's test problems (Sec. 5). Each
consumer turns them into populations with its own code.

Workload recipes (lattice units; k = number of D1Q3 summations, level N = k+1):
  * Sod shock tube (Sec. 5.1): 1D, k = 1, 1000 nodes, density 1 | 0.125, u = 0,
    Kn = 0.01 on the tube length, halfway bounce-back ends.
  * Plane Couette (Sec. 5.3): k = 3 per axis (81 velocities), 512 x 256,
    periodic in x, diffuse walls moving at -0.05 / +0.05, Kn in {0.01, 0.1, 1}.
  * Poiseuille (Sec. 5.4): k = 7 per axis (289 velocities), 1024 x 128,
    stationary diffuse walls, body force 1e-6, Kn log-spaced 0.01 .. 10.
  * Batched channels: 256 instances with Ny ~ U{32..512}, Nx = 64, k ~ U{1..7},
    log10 Kn ~ U[-2, 1], Couette (wall speed ~ U[0, 0.1]) or Poiseuille
    (g ~ U[1e-7, 1e-5]) with probability 1/2 each.
  * Adjoint: Poiseuille k = 4 (121 velocities), 256 x 128, Kn = 0.1, g = 1e-6.
"""
from __future__ import annotations

import numpy as np

SOD = dict(dims=1, k=1, nx=1000, ny=1, kn=0.01, steps=500, rho_left=1.0, rho_right=0.125)
COUETTE = dict(dims=2, k=3, nx=512, ny=256, u_wall_lo=-0.05, u_wall_hi=0.05, g=0.0,
               kn=(0.01, 0.1, 1.0), steps=20000)
POISEUILLE = dict(dims=2, k=7, nx=1024, ny=128, u_wall_lo=0.0, u_wall_hi=0.0, g=1e-6,
                  kn=tuple(float(v) for v in np.logspace(-2, 1, 8)), steps=2000)
ADJOINT = dict(dims=2, k=4, nx=256, ny=128, kn=0.1, g=1e-6, steps=4000, ckpt_every=100)


def smooth_field(seed: int, lx: int, ly: int, amp: float, modes: int = 3) -> np.ndarray:
    """A smooth random field of shape (ly, lx): a sum of a few random sine modes,
    periodic in x, scaled so its largest magnitude is about `amp`."""
    rng = np.random.default_rng(seed)
    x = np.arange(lx)[None, :] / max(lx, 1)
    y = (np.arange(ly)[:, None] + 0.5) / max(ly, 1)
    out = np.zeros((ly, lx))
    for _ in range(modes):
        kx = int(rng.integers(0, 4))
        ky = float(rng.uniform(0.5, 3.0))
        ph = rng.uniform(0, 2 * np.pi, size=2)
        a = rng.uniform(-1, 1)
        out += a * np.sin(2 * np.pi * kx * x + ph[0]) * np.cos(np.pi * ky * y + ph[1])
    m = np.abs(out).max()
    return out * (amp / m if m > 0 else 0.0)


def random_macro(seed: int, lx: int, ly: int, drho: float = 0.02, du: float = 0.03):
    """Seeded smooth (rho, u_x, u_y) fields of shape (ly, lx) around rest."""
    rho = 1.0 + smooth_field(seed, lx, ly, drho)
    ux = smooth_field(seed + 1, lx, ly, du)
    uy = smooth_field(seed + 2, lx, ly, du)
    return rho, ux, uy


def random_populations(seed: int, q: int, ly: int, lx: int, lo: float = 0.5,
                       hi: float = 1.5) -> np.ndarray:
    """Positive random populations f[q][ly][lx] = U(lo, hi)/q (far from equilibrium)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(q, ly, lx)) / q


def sod_density(nx: int = 1000, left: float = 1.0, right: float = 0.125) -> np.ndarray:
    """Step density of the shock tube: `left` on the first half, `right` after."""
    rho = np.full(nx, right)
    rho[: nx // 2] = left
    return rho


# Couette channel on the anisotropic product D1Q3 (x) x D1Q17 (y), the form of
# the paper's channel models (Sec. 5.3) at its Ny = 200
COUETTE_ANISO = dict(nx=1024, ny=200, k=7, x_level=1, kn=(0.01, 0.1, 1.0), u_wall_lo=-0.05,
                     u_wall_hi=0.05)

# Couette channel on the 2N+2 hierarchy (Sec. 4, zero velocity removed): the
# paper's G-D1Q8 x D1Q3 (D1Q3 along x, the 2N+2 axis with N = 3 along y) at
# Ny = 200, long enough in x that the populations exceed the L2 cache
COUETTE_ZV = dict(nx=4096, ny=200, k=2, x_level=1, zv_axes=2, kn=(0.01, 0.1, 1.0),
                  u_wall_lo=-0.05, u_wall_hi=0.05,
                  label="couette_zv_d1q3xd1q8_4096x200_kn{0.01,0.1,1}")
# Couette channel on the 3D product D3Q125 (level 2 on every axis), periodic in
# x and z (Sec. 4's product on three axes; the paper names 3D without a case)
COUETTE_3D = dict(nx=256, ny=64, nz=64, k=1, kn=(0.01, 0.1, 1.0), u_wall_lo=-0.05,
                  u_wall_hi=0.05, label="couette3d_d3q125_256x64x64_kn{0.01,0.1,1}")
# and the fully symmetric 2N+2 lattice of the same level, D2Q64 (8 x 8)
COUETTE_ZV_XY = dict(nx=512, ny=256, k=2, x_level=0, zv_axes=3, kn=(0.01, 0.1, 1.0),
                     u_wall_lo=-0.05, u_wall_hi=0.05,
                     label="couette_zv_d2q64_512x256_kn{0.01,0.1,1}")


def batched_instances(seed: int = 0, n: int = 256, nx: int = 64):
    """Per-instance recipe of the batched channel workload, drawn in a fixed order."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ny = int(rng.integers(32, 513))
        k = int(rng.integers(1, 8))
        kn = float(10.0 ** rng.uniform(-2.0, 1.0))
        couette = bool(rng.integers(0, 2))
        if couette:
            uw = float(rng.uniform(0.0, 0.1))
            out.append(dict(k=k, nx=nx, ny=ny, kn=kn, u_wall_lo=-uw, u_wall_hi=uw, g=0.0))
        else:
            g = float(rng.uniform(1e-7, 1e-5))
            out.append(dict(k=k, nx=nx, ny=ny, kn=kn, u_wall_lo=0.0, u_wall_hi=0.0, g=g))
    return out
