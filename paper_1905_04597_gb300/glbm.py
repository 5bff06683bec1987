"""Python binding of libglbm (argument marshalling only).

Every step of the lattice Boltzmann path runs in the CUDA library; this
module converts numpy arrays / torch tensors to pointers, passes torch's
current CUDA stream, and raises on error statuses. It has no CPU fallback:
if ``libglbm.so`` is missing or no GPU is present, calls fail loudly.

The C functions and their arguments are documented in ``include/glbm.h``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libglbm.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_UNSTABLE, E_TIMEOUT, E_IO, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
BC_WALLS, BC_BOUNCEBACK, BC_PERIODIC = 0, 1, 2
FP64, FP32_DEV = 0, 1
ZV_X, ZV_Y = 1, 2  # axes on the 2N+2 hierarchy (Config.zv_axes)
FORCE_LINEAR, FORCE_GUO = 0, 1  # Config.force: the paper's linearised force, or Guo's
M_RHO, M_UX, M_UY, M_T, M_QX, M_QY, M_SXY, M_ALL = 1, 2, 4, 8, 16, 32, 64, 127
M_UZ, M_QZ, M_ALL3 = 128, 256, 511
FIELDS_2D = ("rho", "ux", "uy", "T", "qx", "qy", "sxy")
FIELDS_3D = FIELDS_2D + ("uz", "qz")
FIELDS_1D = ("rho", "ux", "T", "qx")
# entries of glbm_channel_diagnostics' stats (GLBM_CH_* in glbm.h)
CHANNEL_STATS = ("flow_rate", "volumetric_flow", "u_wall_lo_gas", "u_wall_hi_gas", "slip_lo",
                 "slip_hi")


class GlbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"glbm status {status}: {msg}")
        self.status = status


class UnstableError(GlbmError):
    pass


class Config(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("k", ctypes.c_int), ("x_level", ctypes.c_int), ("tau", ctypes.c_double),
                ("kn", ctypes.c_double),
                ("bc", ctypes.c_int), ("prec", ctypes.c_int), ("u_wall_lo", ctypes.c_double),
                ("u_wall_hi", ctypes.c_double), ("g", ctypes.c_double),
                ("zv_axes", ctypes.c_int), ("nz", ctypes.c_int), ("force", ctypes.c_int)]


_lib = None
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def lib():
    """Load libglbm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1905_04597_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, cp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Config)
    i, i64, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "glbm_create": ([cp, i, vp, ctypes.POINTER(vp)], i),
        "glbm_batch_create": ([cp, i, vp, ctypes.POINTER(vp)], i),
        "glbm_destroy": ([vp], None),
        "glbm_set_allocator": ([ALLOC_FN, FREE_FN, vp], i),
        "glbm_set_equilibrium": ([vp, i, vp, vp, vp, i], i),
        "glbm_set_equilibrium_3d": ([vp, i, vp, vp, vp, vp, i], i),
        "glbm_pack_columns": ([vp, i, i, i, vp, i], i),
        "glbm_unpack_columns": ([vp, i, i, i, vp, i], i),
        "glbm_elem_size": ([vp], ctypes.c_size_t),
        "glbm_set_populations": ([vp, i, vp, i], i),
        "glbm_get_populations": ([vp, i, vp, i], i),
        "glbm_step": ([vp, i64], i),
        "glbm_sync": ([vp], i),
        "glbm_moments": ([vp, i, ctypes.c_uint, vp, sz, i], i),
        "glbm_conservation": ([vp, i, dp, dp, dp], i),
        "glbm_channel_diagnostics": ([vp, i, vp, vp, i], i),
        "glbm_save": ([vp, ctypes.c_char_p], i),
        "glbm_load": ([vp, ctypes.c_char_p], i),
        "glbm_time": ([vp], i64),
        "glbm_kernel_launches": ([vp], i64),
        "glbm_tau": ([vp, i], ctypes.c_double),
        "glbm_eq_table": ([i, dp, sz], i),
        "glbm_conservation_noalloc": ([vp, i, i64, vp, vp], i),
        "glbm_measure_fp64_rate": ([vp, dp], i),
        "glbm_set_dataflow": ([vp, i], i),
        "glbm_get_dataflow": ([vp], i),
        "glbm_adjoint_flowrate": ([vp, i64, i64, dp, dp, dp, dp, dp], i),
        "glbm_tile_count": ([i, i], i),
        "glbm_tile_shape": ([i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "glbm_get_tiles": ([vp, ctypes.POINTER(i)], i),
        "glbm_set_tiles": ([vp, ctypes.POINTER(i)], i),
        "glbm_get_tile_shape": ([vp, i] + [ctypes.POINTER(i)] * 3, i),
        "glbm_autotune": ([vp, i, dp], i),
        "glbm_set_wall_launch": ([vp, i], i),
        "glbm_get_wall_launch": ([vp], i),
        "glbm_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def check(status):
    if status == OK:
        return
    msg = lib().glbm_last_error().decode(errors="replace")
    if status == E_UNSTABLE:
        raise UnstableError(status, msg)
    raise GlbmError(status, msg)


LEVELS = 13     # levels k = 0..12 (k > 7: D1Q3 x D1Q(2k+4) only)
MAX_TILES = 8   # candidate tile shapes per level and precision


def tile_shapes(k: int, prec: int) -> list:
    """Candidate (G, R, V) tile shapes of level k in precision prec (G warps per
    node row, R node rows per CTA, V nodes per thread); entry 0 is the default."""
    L = lib()
    out = []
    for idx in range(L.glbm_tile_count(k, prec)):
        G, R, V = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(L.glbm_tile_shape(k, prec, idx, ctypes.byref(G), ctypes.byref(R), ctypes.byref(V)))
        out.append((G.value, R.value, V.value))
    return out


def eq_table(k: int) -> np.ndarray:
    """Coefficients C[n][j] of E_n(u) = sum_j C[n][j] u^j at level k+1."""
    Q1 = 2 * k + 3
    out = np.empty((Q1, Q1))
    check(lib().glbm_eq_table(k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
    return out


def make_config(dims=2, nx=1, ny=1, k=0, tau=0.0, kn=0.0, bc=None, prec=FP64, u_wall_lo=0.0,
                u_wall_hi=0.0, g=0.0, x_level=0, zv_axes=0, nz=1, force=FORCE_LINEAR) -> Config:
    """One instance; x_level=1 makes the anisotropic product D1Q3 (x) times the
    level-(k+1) lattice (y); 0 keeps level k+1 on both axes. zv_axes (ZV_X,
    ZV_Y) puts axes on the 2N+2 hierarchy (odd velocities, half spacing).
    force=FORCE_GUO takes Guo's force with the half-force velocity shift."""
    if bc is None:
        bc = BC_WALLS if dims >= 2 else BC_BOUNCEBACK
    return Config(dims, nx, ny if dims >= 2 else 1, k, x_level, tau, kn, bc, prec, u_wall_lo,
                  u_wall_hi, g, zv_axes, nz if dims == 3 else 1, force)


_torch_alloc_refs = None


def install_torch_allocator():
    """Back later glbm_create calls with torch's CUDA caching allocator."""
    global _torch_alloc_refs
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    check(lib().glbm_set_allocator(a, f, None))
    _torch_alloc_refs = (a, f)


def uninstall_allocator():
    global _torch_alloc_refs
    check(lib().glbm_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _torch_alloc_refs = None


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(a):
    """(pointer, on_device) of a contiguous float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        return ctypes.c_void_p(a.ctypes.data), 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def _raw_ptr(a, itemsize):
    """(pointer, on_device) of a contiguous numpy array or torch tensor whose
    element size is `itemsize` bytes (the stored population type)."""
    if isinstance(a, np.ndarray):
        if a.itemsize != itemsize or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous array of {itemsize}-byte elements")
        return ctypes.c_void_p(a.ctypes.data), 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.element_size() != itemsize or not a.is_contiguous():
            raise TypeError(f"expected a contiguous tensor of {itemsize}-byte elements")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


class Lattice:
    """One or more lattice instances stepped together by libglbm."""

    def __init__(self, configs, stream=None, hetero=False):
        if isinstance(configs, (Config, dict)):
            configs = [configs]
        cfgs = [c if isinstance(c, Config) else make_config(**c) for c in configs]
        arr = (Config * len(cfgs))(*cfgs)
        self.configs = cfgs
        self.n = len(cfgs)
        self.dims = cfgs[0].dims
        self._stream = stream if stream is not None else _current_stream()
        h = ctypes.c_void_p()
        create = lib().glbm_batch_create if hetero else lib().glbm_create
        check(create(arr, len(cfgs), self._stream, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().glbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def nodes(self, inst=0):
        c = self.configs[inst]
        return c.nx * (c.ny if c.dims >= 2 else 1) * (c.nz if c.dims == 3 else 1)

    def nq(self, inst=0):
        c = self.configs[inst]
        if c.dims == 3:
            return (2 * c.k + 3) ** 3
        if c.dims != 2:
            return 2 * c.k + 3
        q1 = 2 * c.k + 3 + (1 if c.zv_axes & ZV_Y else 0)
        q1x = 2 * (c.x_level if c.x_level > 0 else c.k + 1) + 1 + (1 if c.zv_axes & ZV_X else 0)
        return q1 * q1x

    def shape(self, inst=0):
        c = self.configs[inst]
        if c.dims == 3:
            return (c.nz, c.ny, c.nx)
        return (c.ny, c.nx) if c.dims == 2 else (c.nx,)

    def set_equilibrium(self, inst, rho, ux, uy=None, uz=None):
        pr, dev = _ptr(rho)
        pu, _ = _ptr(ux)
        pv = _ptr(uy)[0] if uy is not None else ctypes.c_void_p()
        if self.dims == 3:
            pw = _ptr(uz)[0] if uz is not None else ctypes.c_void_p()
            check(lib().glbm_set_equilibrium_3d(self.h, inst, pr, pu, pv, pw, dev))
            return
        check(lib().glbm_set_equilibrium(self.h, inst, pr, pu, pv, dev))

    def set_populations(self, inst, f):
        p, dev = _ptr(f)
        check(lib().glbm_set_populations(self.h, inst, p, dev))

    def get_populations(self, inst=0, out=None):
        if out is None:
            out = np.empty((self.nq(inst),) + self.shape(inst))
        p, dev = _ptr(out)
        check(lib().glbm_get_populations(self.h, inst, p, dev))
        return out

    def pack_columns(self, inst, x0, ncols, out):
        """Stored values of x-columns [x0, x0 + ncols) into `out` (numpy or torch,
        host or device, packed [q][(z,)y][ncols], dtype float32 or float64 as
        stored)."""
        p, dev = _raw_ptr(out, self.elem_size)
        check(lib().glbm_pack_columns(self.h, inst, x0, ncols, p, dev))
        return out

    def unpack_columns(self, inst, x0, ncols, src):
        """The inverse of pack_columns: write stored values into the state."""
        p, dev = _raw_ptr(src, self.elem_size)
        check(lib().glbm_unpack_columns(self.h, inst, x0, ncols, p, dev))

    @property
    def elem_size(self):
        return lib().glbm_elem_size(self.h)

    def step(self, n=1):
        check(lib().glbm_step(self.h, int(n)))

    def sync(self):
        check(lib().glbm_sync(self.h))

    def moments(self, inst=0, mask=M_ALL, out=None):
        """Moments of S(X) at the current time; returns a dict of arrays (host) or
        fills `out` (numpy or torch, host or device) packed in field order."""
        if self.dims == 3:
            fields, bits = FIELDS_3D, [1, 2, 4, 8, 16, 32, 64, 128, 256]
            if mask == M_ALL:
                mask = M_ALL3
        elif self.dims == 2:
            fields, bits = FIELDS_2D, [1, 2, 4, 8, 16, 32, 64]
        else:
            fields, bits = FIELDS_1D, [1, 2, 8, 16]
        names = [f for f, b in zip(fields, bits) if mask & b]
        if self.dims == 1:
            mask &= M_RHO | M_UX | M_T | M_QX
        if out is None:
            out = np.empty((len(names),) + self.shape(inst))
        p, dev = _ptr(out)
        n_el = out.size if isinstance(out, np.ndarray) else out.numel()
        check(lib().glbm_moments(self.h, inst, mask, p, n_el, dev))
        if isinstance(out, np.ndarray):
            return {k: out[i] for i, k in enumerate(names)}
        return out

    def conservation(self, inst=0):
        m, jx, jy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().glbm_conservation(self.h, inst, ctypes.byref(m), ctypes.byref(jx),
                                      ctypes.byref(jy)))
        return m.value, jx.value, jy.value

    def channel_diagnostics(self, inst=0, profile=None, stats=None):
        """Channel diagnostics of Sec. 5.3-5.4 at the current time (glbm.h,
        glbm_channel_diagnostics): returns (profile <u_x>(y), dict of the flow
        rate, volumetric flow, wall-plane velocities and slip ratios). With
        torch tensors `profile` and `stats` (float64, device or host), fills
        them and returns them."""
        c = self.configs[inst]
        if profile is None and stats is None:
            prof, st = np.empty(c.ny), np.empty(len(CHANNEL_STATS))
            check(lib().glbm_channel_diagnostics(self.h, inst, ctypes.c_void_p(prof.ctypes.data),
                                                 ctypes.c_void_p(st.ctypes.data), 0))
            return prof, dict(zip(CHANNEL_STATS, st.tolist()))
        pp, dev = _ptr(profile) if profile is not None else (ctypes.c_void_p(), None)
        sp, dev2 = _ptr(stats) if stats is not None else (ctypes.c_void_p(), None)
        on_dev = dev if dev is not None else dev2
        if dev is not None and dev2 is not None and dev != dev2:
            raise TypeError("profile and stats must both be host or both device memory")
        check(lib().glbm_channel_diagnostics(self.h, inst, pp, sp, on_dev))
        return profile, stats

    def save(self, path):
        check(lib().glbm_save(self.h, str(path).encode()))

    def load(self, path):
        check(lib().glbm_load(self.h, str(path).encode()))

    def adjoint_flowrate(self, steps, ckpt_every=100, walls=False):
        """Advance `steps` steps and return per instance (J, dJ/dtau, dJ/dg) of the flow
        rate J = (1/nx) sum of the x-momentum of S(X_T), by the discrete adjoint;
        with walls=True also (dJ/du_wall_lo, dJ/du_wall_hi)."""
        n = self.n
        out = [(ctypes.c_double * n)() for _ in range(5)]
        check(lib().glbm_adjoint_flowrate(self.h, int(steps), int(ckpt_every), *out))
        res = tuple(np.array(o[:]) for o in out)
        return res if walls else res[:3]

    def tiles(self):
        """Tile shape index in use for every level k = 0..LEVELS-1."""
        t = (ctypes.c_int * LEVELS)()
        check(lib().glbm_get_tiles(self.h, t))
        return list(t)

    def tile_shape(self, k):
        """(G, R, V) of the tile this context uses for level k."""
        v = [ctypes.c_int() for _ in range(3)]
        check(lib().glbm_get_tile_shape(self.h, int(k), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_tiles(self, tiles):
        """Set the tile shape index per level (-1 keeps a level's index)."""
        t = (ctypes.c_int * LEVELS)(*[int(v) for v in tiles])
        check(lib().glbm_set_tiles(self.h, t))

    def autotune(self, reps=20):
        """Time every candidate tile shape of the levels this context steps and
        keep the fastest. Returns {k: [us per launch of each candidate]}."""
        us = (ctypes.c_double * (LEVELS * MAX_TILES))()
        check(lib().glbm_autotune(self.h, int(reps), us))
        out = {}
        for k in range(LEVELS):
            row = [us[k * MAX_TILES + j] for j in range(MAX_TILES)]
            if any(v >= 0 for v in row):
                out[k] = [v for v in row if v >= 0]
        return out

    @property
    def wall_launch(self):
        """1: the wall densities get a launch of their own each step; 0: every
        tile near a wall sums them itself; -1: no walls (or a mixed batch, 3D)."""
        return lib().glbm_get_wall_launch(self.h)

    @property
    def dataflow(self):
        """1 when glbm_step runs this context's steps in overlapping dataflow chunks."""
        return lib().glbm_get_dataflow(self.h)

    def set_dataflow(self, on):
        """Overlapping dataflow chunks (1, the default where the context allows
        them) or one launch after another (0); the results are identical."""
        check(lib().glbm_set_dataflow(self.h, int(on)))

    def set_wall_launch(self, mode):
        """Choose how the wall densities are computed (0, 1, or -1 for the
        context's default); the results are identical either way."""
        check(lib().glbm_set_wall_launch(self.h, int(mode)))

    @property
    def time(self):
        return lib().glbm_time(self.h)

    @property
    def kernel_launches(self):
        return lib().glbm_kernel_launches(self.h)

    def tau(self, inst=0):
        return lib().glbm_tau(self.h, inst)


def measure_fp64_rate(stream=None):
    """FP64 FMA thread instructions per second of the current device, measured
    by the library's probe kernel (glbm_measure_fp64_rate)."""
    out = ctypes.c_double()
    s = stream if stream is not None else _current_stream()
    check(lib().glbm_measure_fp64_rate(s, ctypes.byref(out)))
    return out.value


def _flowrate_autograd():
    import torch

    class FlowRate(torch.autograd.Function):
        """J(tau, g, u_wall_lo, u_wall_hi): flow rate of a force-driven (or
        wall-driven) channel after `steps` steps from rest, with gradients from
        the hand-written adjoint.

        config: glbm lattice configuration without tau, g and the wall speeds
        (dims, nx, ny, k, bc, prec); the four parameters are 0-d float64
        tensors or numbers."""

        @staticmethod
        def forward(ctx, tau, g, u_lo, u_hi, config, steps, ckpt_every=100):
            cfg = dict(config, tau=float(tau), kn=0.0, g=float(g), u_wall_lo=float(u_lo),
                       u_wall_hi=float(u_hi))
            dev = tau.device if isinstance(tau, torch.Tensor) else torch.device("cpu")
            f64 = dict(dtype=torch.float64, device=dev)
            if not any(ctx.needs_input_grad[:4]):
                # no gradient wanted: the forward steps and the flow rate only
                with Lattice(cfg) as lat:
                    lat.step(steps)
                    _, stats = lat.channel_diagnostics(0)
                return torch.tensor(stats["flow_rate"], **f64)
            with Lattice(cfg) as lat:
                J, dtau, dg, dlo, dhi = lat.adjoint_flowrate(steps, ckpt_every, walls=True)
            ctx.save_for_backward(*[torch.tensor(v[0], **f64) for v in (dtau, dg, dlo, dhi)])
            return torch.tensor(J[0], **f64)

        @staticmethod
        def backward(ctx, grad):
            d = ctx.saved_tensors  # dJ/dtau, dJ/dg, dJ/du_wall_lo, dJ/du_wall_hi
            return tuple(grad * d[i] if ctx.needs_input_grad[i] else None
                         for i in range(4)) + (None, None, None)

    return FlowRate


def flow_rate(tau, g, config, steps, ckpt_every=100, u_wall_lo=None, u_wall_hi=None):
    """Differentiable flow rate (torch.autograd) through libglbm's adjoint: by
    tau, g and, when given as tensors, the wall speeds (default: those of
    config, else 0)."""
    ulo = config.get("u_wall_lo", 0.0) if u_wall_lo is None else u_wall_lo
    uhi = config.get("u_wall_hi", 0.0) if u_wall_hi is None else u_wall_hi
    base = {k: v for k, v in config.items() if k not in ("u_wall_lo", "u_wall_hi")}
    return _flowrate_autograd().apply(tau, g, ulo, uhi, base, steps, ckpt_every)
