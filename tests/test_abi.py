"""The C-ABI library loads, exports every symbol include/glbm.h declares, and its
host-side pieces (equilibrium-coefficient table, Kn mapping inputs, error
paths) agree with the oracle -- no GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glbm.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glbm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("glbm_create", "glbm_step", "glbm_moments", "glbm_destroy", "glbm_conservation",
                 "glbm_save", "glbm_load", "glbm_batch_create", "glbm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(glbm.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("k", range(0, 13))
def test_coefficient_table_matches_oracle(k):
    """Row a1: the convolution-built polynomial table reproduces the factorial-sum
    equilibrium of the oracle at any velocity (Sec. 2, Eqs. maineq03-05)."""
    N = k + 1
    C = glbm.eq_table(k)
    rng = np.random.default_rng(k)
    for u in np.concatenate([[0.0, 0.05, -0.3], rng.uniform(-0.8, 0.8, 5)]):
        E = np.array([np.polyval(C[i, ::-1], u) for i in range(2 * N + 1)])
        np.testing.assert_allclose(E, orc.eq1d(N, u), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(C[:, 0], orc.weights(N), rtol=1e-9, atol=1e-15)


def test_table_rejects_bad_level():
    with pytest.raises(glbm.GlbmError):
        glbm.eq_table(13)


def test_invalid_config_is_rejected_before_any_device_call():
    cfg = glbm.make_config(dims=2, nx=8, ny=2, k=3, tau=1.0)  # walls need ny >= 4
    h = ctypes.c_void_p()
    st = glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h))
    assert st == glbm.E_INVAL and not h.value
    assert b"ny" in glbm.lib().glbm_last_error()
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=9, tau=1.0)  # k > 7: 2N+2 channels only
    assert glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED
    cfg = glbm.make_config(dims=2, nx=8, ny=32, k=9, tau=1.0, x_level=1)
    assert glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED
    cfg = glbm.make_config(dims=2, nx=8, ny=32, k=13, tau=1.0, x_level=1, zv_axes=glbm.ZV_Y)
    assert glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED
    cfg = glbm.make_config(dims=2, nx=8, ny=20, k=9, tau=1.0, x_level=1, zv_axes=glbm.ZV_Y)
    assert glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL
    assert b"ny >= 21" in glbm.lib().glbm_last_error()
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=1, tau=-1.0)
    assert glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=0, tau=1.0, u_wall_lo=0.9)  # > sqrt(2/3)
    assert glbm.lib().glbm_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL


def test_anisotropic_configs_are_checked_before_any_device_call():
    """x_level: 0 or the level of k (isotropic) or 1 (D1Q3 along x); not in 1D,
    not in heterogeneous batches; the wall speeds are bounded by the x level."""
    h = ctypes.c_void_p()
    create = glbm.lib().glbm_create
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=5, tau=1.0, x_level=3)
    assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=5, tau=1.0, x_level=14)
    assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL
    cfg = glbm.make_config(dims=1, nx=8, k=2, tau=1.0, x_level=1)
    assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL
    # |u_w| < sqrt(2/3) along the D1Q3 axis even at a high y level
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=5, tau=1.0, x_level=1, u_wall_hi=0.9)
    assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL
    cfg = glbm.make_config(dims=2, nx=8, ny=8, k=5, tau=1.0, x_level=1, prec=glbm.FP32_DEV)
    st = glbm.lib().glbm_batch_create(ctypes.byref(cfg), 1, None, ctypes.byref(h))
    assert st == glbm.E_UNSUPPORTED and not h.value
    assert b"isotropic" in glbm.lib().glbm_last_error()
    # a context mixing isotropic and anisotropic instances is not uniform
    two = (glbm.Config * 2)(glbm.make_config(dims=2, nx=8, ny=8, k=5, tau=1.0),
                            glbm.make_config(dims=2, nx=8, ny=8, k=5, tau=1.0, x_level=1))
    assert create(two, 2, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED


def test_2n2_configs_are_checked_before_any_device_call():
    """zv_axes: the 2N+2 hierarchy along y with D1Q3 along x, or along both axes
    of an isotropic lattice; 2D only; walls need ny >= 2N+1; the wall-speed
    bound doubles in the half-spacing units of a 2N+2 x axis; no batches."""
    h = ctypes.c_void_p()
    create = glbm.lib().glbm_create
    zy, zxy = glbm.ZV_Y, glbm.ZV_X | glbm.ZV_Y
    for kw, st in [(dict(dims=1, nx=8, k=2, zv_axes=zy), glbm.E_INVAL),
                   (dict(dims=2, nx=8, ny=16, k=2, zv_axes=4), glbm.E_INVAL),
                   (dict(dims=2, nx=8, ny=16, k=2, zv_axes=glbm.ZV_X), glbm.E_UNSUPPORTED),
                   (dict(dims=2, nx=8, ny=16, k=2, zv_axes=zy), glbm.E_UNSUPPORTED),
                   (dict(dims=2, nx=8, ny=16, k=2, x_level=1, zv_axes=zxy), glbm.E_UNSUPPORTED),
                   (dict(dims=2, nx=8, ny=6, k=2, x_level=1, zv_axes=zy), glbm.E_INVAL),
                   (dict(dims=2, nx=8, ny=6, k=2, zv_axes=zxy), glbm.E_INVAL),
                   (dict(dims=2, nx=8, ny=8, k=0, zv_axes=zxy, u_wall_lo=1.7), glbm.E_INVAL),
                   (dict(dims=2, nx=8, ny=8, k=0, x_level=1, zv_axes=zy, u_wall_lo=0.9),
                    glbm.E_INVAL)]:
        cfg = glbm.make_config(tau=1.0, **kw)
        assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == st, kw
        assert not h.value
    cfg = glbm.make_config(dims=2, nx=8, ny=16, k=2, tau=1.0, zv_axes=zxy, prec=glbm.FP32_DEV)
    assert glbm.lib().glbm_batch_create(ctypes.byref(cfg), 1, None,
                                        ctypes.byref(h)) == glbm.E_UNSUPPORTED
    # instances on different hierarchies are not one uniform context
    two = (glbm.Config * 2)(glbm.make_config(dims=2, nx=8, ny=16, k=2, tau=1.0),
                            glbm.make_config(dims=2, nx=8, ny=16, k=2, tau=1.0, zv_axes=zxy))
    assert create(two, 2, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED


def test_guo_configs_are_checked_before_any_device_call():
    """force: GLBM_FORCE_LINEAR or GLBM_FORCE_GUO; Guo's form is compiled for 2D
    lattices with k <= 7 (isotropic, D1Q3 x level N, D1Q3 x the 2N+2 axis), not
    for heterogeneous batches, and every instance of a context takes one form."""
    h = ctypes.c_void_p()
    create = glbm.lib().glbm_create
    G = glbm.FORCE_GUO
    zy, zxy = glbm.ZV_Y, glbm.ZV_X | glbm.ZV_Y
    for kw, st in [(dict(dims=2, nx=8, ny=16, k=2, force=2), glbm.E_INVAL),
                   (dict(dims=2, nx=8, ny=16, k=2, force=-1), glbm.E_INVAL),
                   (dict(dims=1, nx=8, k=2, force=G), glbm.E_UNSUPPORTED),
                   (dict(dims=3, nx=8, ny=8, nz=8, k=1, force=G), glbm.E_UNSUPPORTED),
                   (dict(dims=2, nx=8, ny=32, k=8, x_level=1, zv_axes=zy, force=G),
                    glbm.E_UNSUPPORTED),
                   (dict(dims=2, nx=8, ny=16, k=2, zv_axes=zxy, force=G), glbm.E_UNSUPPORTED)]:
        cfg = glbm.make_config(tau=1.0, **kw)
        assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == st, kw
        assert not h.value
    cfg = glbm.make_config(dims=2, nx=8, ny=16, k=2, tau=1.0, prec=glbm.FP32_DEV, force=G)
    assert glbm.lib().glbm_batch_create(ctypes.byref(cfg), 1, None,
                                        ctypes.byref(h)) == glbm.E_UNSUPPORTED
    two = (glbm.Config * 2)(glbm.make_config(dims=2, nx=8, ny=16, k=2, tau=1.0),
                            glbm.make_config(dims=2, nx=8, ny=16, k=2, tau=1.0, force=G))
    assert create(two, 2, None, ctypes.byref(h)) == glbm.E_UNSUPPORTED


def test_3d_configs_are_checked_before_any_device_call():
    """3D: levels k <= 2, the level of k on every axis, ny * nz <= 65535, no
    heterogeneous batches; invalid configurations fail before any CUDA call."""
    h = ctypes.c_void_p()
    create = glbm.lib().glbm_create
    for kw, st in [(dict(k=3, nx=8, ny=8, nz=8), glbm.E_UNSUPPORTED),
                   (dict(k=1, nx=8, ny=8, nz=8, x_level=1), glbm.E_UNSUPPORTED),
                   (dict(k=1, nx=8, ny=8, nz=8, zv_axes=glbm.ZV_Y), glbm.E_UNSUPPORTED),
                   (dict(k=1, nx=8, ny=300, nz=300), glbm.E_UNSUPPORTED),
                   (dict(k=2, nx=8, ny=2, nz=8), glbm.E_INVAL),
                   (dict(k=1, nx=8, ny=8, nz=0), glbm.E_INVAL),
                   (dict(k=0, nx=8, ny=8, nz=8, u_wall_lo=0.9), glbm.E_INVAL)]:
        cfg = glbm.make_config(dims=3, tau=1.0, **kw)
        assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == st, kw
        assert not h.value
    cfg = glbm.make_config(dims=3, nx=8, ny=8, nz=8, k=1, tau=1.0, prec=glbm.FP32_DEV)
    assert glbm.lib().glbm_batch_create(ctypes.byref(cfg), 1, None,
                                        ctypes.byref(h)) == glbm.E_UNSUPPORTED
    cfg = glbm.make_config(dims=4, nx=8, ny=8, k=1, tau=1.0)
    assert create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == glbm.E_INVAL


def test_tile_shape_candidates():
    """Every level has 1..MAX_TILES candidate shapes in each precision, each
    with 1 <= G <= 2k+3 warp groups, at most 512 threads per CTA and one or
    two nodes per thread (pairs in FP32 only); invalid levels have none."""
    for prec in (glbm.FP64, glbm.FP32_DEV):
        for k in range(8):
            shapes = glbm.tile_shapes(k, prec)
            assert 1 <= len(shapes) <= glbm.MAX_TILES
            assert len(set(shapes)) == len(shapes)
            for G, R, V in shapes:
                assert 1 <= G <= 2 * k + 3 and R >= 1 and 32 * G * R <= 512
                assert V == 1 or (V == 2 and prec == glbm.FP32_DEV)
        assert glbm.tile_shapes(8, prec) == [] and glbm.tile_shapes(-1, prec) == []
    with pytest.raises(glbm.GlbmError):
        glbm.check(glbm.lib().glbm_tile_shape(0, glbm.FP64, 99, None, None, None))


def test_wall_launch_mode_rejects_null_context():
    """The wall-density mode calls check their arguments before touching a
    device: a null context is GLBM_E_INVAL (set) or -1 (get)."""
    assert glbm.lib().glbm_set_wall_launch(None, 0) == glbm.E_INVAL
    assert glbm.lib().glbm_set_wall_launch(None, 1) == glbm.E_INVAL
    assert glbm.lib().glbm_get_wall_launch(None) == -1
