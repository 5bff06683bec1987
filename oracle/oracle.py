"""ctypes binding of the FP64 CPU oracle (``glbm_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It never touches
the CUDA library and the CUDA path never imports it.

Every function follows O. Ilyin, "Gaussian Lattice Boltzmann method and its
applications to rarefied flows" (arXiv:1905.04597); the C source cites the
section and equation behind each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "glbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

BC_WALLS, BC_BOUNCEBACK, BC_PERIODIC = 0, 1, 2
ZV_X, ZV_Y = 1, 2  # axes on the 2N+2 hierarchy (Lattice zv mask)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction).

    ``GLBM_ORACLE_LIB`` names a prebuilt copy to load instead; the mutation
    tests use it to run the pins against an oracle with a planted mistake."""
    override = os.environ.get("GLBM_ORACLE_LIB")
    if override:
        return override
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def build_openmp(force: bool = False) -> str:
    """The same source compiled with -fopenmp: its collision loops over rows run
    on all cores with results identical to the serial build. Used only to time
    the oracle as a CPU baseline on every core of a host."""
    if force or not os.path.exists(LIB_OMP) or os.path.getmtime(LIB_OMP) < os.path.getmtime(SRC):
        tmp = LIB_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
             "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_OMP)
    return LIB_OMP


class Cfg(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("NX", ctypes.c_int), ("NY", ctypes.c_int),
                ("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("bc", ctypes.c_int),
                ("tau", ctypes.c_double), ("uw_lo", ctypes.c_double),
                ("uw_hi", ctypes.c_double), ("g", ctypes.c_double), ("zv", ctypes.c_int),
                ("NZ", ctypes.c_int), ("Lz", ctypes.c_int), ("guo", ctypes.c_int)]


_lib = None


_lib_omp = None


def lib_openmp():
    """The -fopenmp build of the oracle (build_openmp), loaded on first use."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _declare(ctypes.CDLL(build_openmp()))
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    """Argument and result types of the oracle's C functions on handle L."""
    dp = ctypes.POINTER(ctypes.c_double)
    cp = ctypes.POINTER(Cfg)
    L.orc_prob.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    L.orc_prob.restype = ctypes.c_int
    L.orc_eq1d.argtypes = [ctypes.c_int, ctypes.c_double, dp]
    L.orc_weights.argtypes = [ctypes.c_int, dp]
    L.orc_tau_from_kn.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.orc_tau_from_kn.restype = ctypes.c_double
    L.orc_eq_axis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
    L.orc_tau_from_kn_axis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double]
    L.orc_tau_from_kn_axis.restype = ctypes.c_double
    for name in ("orc_stream", "orc_collide", "orc_macro", "orc_observe"):
        getattr(L, name).argtypes = [cp, dp, dp]
        getattr(L, name).restype = ctypes.c_int
    L.orc_equilibrium.argtypes = [cp, dp, dp, dp, dp]
    L.orc_equilibrium.restype = ctypes.c_int
    L.orc_equilibrium3d.argtypes = [cp, dp, dp, dp, dp, dp]
    L.orc_equilibrium3d.restype = ctypes.c_int
    L.orc_run.argtypes = [cp, dp, ctypes.c_long]
    L.orc_run.restype = ctypes.c_long
    L.orc_flowrate_grad.argtypes = [cp, dp, ctypes.c_long, dp]
    L.orc_flowrate_grad.restype = ctypes.c_int
    return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Lattice:
    """One lattice for the oracle: level N per axis (N = k + 1), node counts,
    boundary kind, relaxation time, wall speeds and body force, all in lattice
    units (velocities are the integers -N..N; on an axis that zv selects,
    ZV_X = 1 and/or ZV_Y = 2, the 2N+2 hierarchy's odd integers
    -(2N+1)..2N+1, 2D only). guo=1 takes the force of Guo, Zheng and Shi
    (2002) with the half-force velocity shift instead of the paper's
    linearised force (2D and 3D)."""

    def __init__(self, dims, NX, NY, Lx, Ly, bc, tau, uw_lo=0.0, uw_hi=0.0, g=0.0, zv=0,
                 NZ=0, Lz=1, openmp=False, guo=0):
        self.cfg = Cfg(dims, NX, NY if dims >= 2 else 0, Lx, Ly if dims >= 2 else 1, bc,
                       tau, uw_lo, uw_hi, g, zv, NZ if dims == 3 else 0, Lz if dims == 3 else 1,
                       int(guo))
        self.dims = dims
        # openmp: run on the -fopenmp build (same results, all cores; timing only)
        self._L = lib_openmp() if openmp else lib()
        qx = 2 * NX + (2 if zv & ZV_X else 1)
        qy = 2 * NY + (2 if zv & ZV_Y else 1)
        if dims == 3:
            self.Q = qx * qy * (2 * NZ + 1)
            self.shape = (self.Q, Lz, self.cfg.Ly, Lx)
            self.nfields = 9
        else:
            self.Q = qx * (qy if dims == 2 else 1)
            self.shape = (self.Q, self.cfg.Ly, Lx) if dims == 2 else (self.Q, Lx)
            self.nfields = 7 if dims == 2 else 4

    def _chk(self, rc):
        if rc < 0:
            raise ValueError("oracle rejected the configuration")
        return rc

    def equilibrium(self, rho, ux, uy=None, uz=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        ux = np.ascontiguousarray(ux, dtype=np.float64)
        uy = np.zeros_like(ux) if uy is None else np.ascontiguousarray(uy, dtype=np.float64)
        X = np.empty(self.shape)
        if self.dims == 3:
            uz = np.zeros_like(ux) if uz is None else np.ascontiguousarray(uz, dtype=np.float64)
            self._chk(self._L.orc_equilibrium3d(ctypes.byref(self.cfg), _dp(rho), _dp(ux),
                                              _dp(uy), _dp(uz), _dp(X)))
            return X
        self._chk(self._L.orc_equilibrium(ctypes.byref(self.cfg), _dp(rho), _dp(ux), _dp(uy),
                                        _dp(X)))
        return X

    def stream(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        F = np.empty(self.shape)
        self._chk(self._L.orc_stream(ctypes.byref(self.cfg), _dp(X), _dp(F)))
        return F

    def collide(self, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        X = np.empty(self.shape)
        bad = self._chk(self._L.orc_collide(ctypes.byref(self.cfg), _dp(F), _dp(X)))
        return X, bad

    def macro(self, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.empty((self.nfields,) + self.shape[1:])
        self._chk(self._L.orc_macro(ctypes.byref(self.cfg), _dp(F), _dp(out)))
        return out

    def observe(self, X):
        """Moments at the current time: moments of the streamed state S(X)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        out = np.empty((self.nfields,) + self.shape[1:])
        self._chk(self._L.orc_observe(ctypes.byref(self.cfg), _dp(X), _dp(out)))
        return out

    def flowrate_grad(self, X, steps, walls=False):
        """J = x-momentum of S(X_T) per column after `steps` steps from X, and
        (dJ/dtau, dJ/dg) by forward-mode dual numbers; with walls=True also
        (dJ/du_wall_lo, dJ/du_wall_hi)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        out = np.empty(5)
        self._chk(self._L.orc_flowrate_grad(ctypes.byref(self.cfg), _dp(X), int(steps), _dp(out)))
        return tuple(out) if walls else (out[0], out[1], out[2])

    def flowrate(self, X, steps):
        """J alone from a plain run (no tangents)."""
        Y, _ = self.run(X, steps)
        F = self.stream(Y)
        nx = np.tile(np.arange(-self.cfg.NX, self.cfg.NX + 1), 2 * self.cfg.NY + 1)
        return float(np.tensordot(nx.astype(float), F, axes=1).sum() / self.cfg.Lx)

    def run(self, X, steps):
        """Advance a copy of X by `steps` steps; returns (X, unstable_count)."""
        X = np.array(X, dtype=np.float64, order="C", copy=True)
        bad = self._chk(self._L.orc_run(ctypes.byref(self.cfg), _dp(X), int(steps)))
        return X, bad


def prob(N, c, cs2, u):
    """Eqs. maineq02-05: Prob(sum of N variables = n c), n = -N..N, physical units."""
    out = np.empty(2 * N + 1)
    flag = lib().orc_prob(N, c, cs2, u, _dp(out))
    if flag < 0:
        raise ValueError("level out of range")
    return out, bool(flag)


def eq1d(N, u):
    out = np.empty(2 * N + 1)
    lib().orc_eq1d(N, u, _dp(out))
    return out


def weights(N):
    out = np.empty(2 * N + 1)
    lib().orc_weights(N, _dp(out))
    return out


def tau_from_kn(N, H, kn, zv=0):
    if zv:
        return lib().orc_tau_from_kn_axis(N, zv, H, kn)
    return lib().orc_tau_from_kn(N, H, kn)


def eq_axis(N, zv, u):
    """f^eq / rho of one axis: the 2N+1 hierarchy (zv=0) or the 2N+2 one."""
    out = np.empty(2 * N + (2 if zv else 1))
    lib().orc_eq_axis(N, zv, u, _dp(out))
    return out
