"""GPU parity of the Guo forcing option (Guo, Zheng and Shi 2002; the paper's
own force is the linearised one of Sec. 5.4) against the FP64 oracle's Guo
form, through the C ABI: FP64 storage to 1e-12 and FP32 deviations to 1e-5 in
every moment, on the Poiseuille channel configuration and on random states
of the isotropic, anisotropic (D1Q3 x level N) and 2N+2 (D1Q3 x D1Q(2N+2))
lattices with moving walls, spanning several tiles with ragged edges. The
error metric is that of the other parity tests (parity_helpers)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs
from parity_helpers import oracle_moments, rel_errors

pytestmark = pytest.mark.gpu

TOL = {glbm.FP64: 1e-12, glbm.FP32_DEV: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_guo_poiseuille_config(prec):
    """D2Q289 (k = 7), 1024 x 128 channel, g = 1e-6, the 8 Knudsen numbers
    0.01..10 as one batch, 2000 steps from rest (x-uniform: the oracle runs
    one column and every GPU column is compared with it)."""
    c = inputs.POISEUILLE
    N = c["k"] + 1
    ny, steps = c["ny"], c["steps"]
    cfgs = [dict(dims=2, nx=c["nx"], ny=ny, k=c["k"], kn=kn, prec=prec, g=c["g"],
                 force=glbm.FORCE_GUO) for kn in c["kn"]]
    lat = glbm.Lattice(cfgs)
    lat.step(steps)
    lat.sync()
    for i, kn in enumerate(c["kn"]):
        got = lat.moments(i)
        o = orc.Lattice(2, N, N, 1, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, kn), g=c["g"],
                        guo=1)
        X = o.equilibrium(np.ones((ny, 1)), np.zeros((ny, 1)), np.zeros((ny, 1)))
        X, _ = o.run(X, steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(got, want, F=F)
        if prec == glbm.FP64:
            # u_y is identically zero in exact arithmetic here (an x-uniform
            # channel from rest keeps a uniform density, so mass conservation
            # leaves no y flux), and both sides hold FP64 rounding noise of a
            # few 1e-15 after 2000 steps; its ratio to max |u| (1e-3 in this
            # slow channel) says nothing. Checked instead: it stays at that
            # noise level on both sides.
            assert np.abs(got["uy"]).max() < 1e-13 and np.abs(want[2]).max() < 1e-13
            errs.pop("uy")
        assert max(errs.values()) < TOL[prec], (kn, errs)
        # the reported velocity carries the half-force shift: at the wall-
        # adjacent rows of a slow channel it is far from j / rho
        assert got["ux"].min() > 0.0
    lat.close()


# (k, x_level, zv_axes): isotropic levels, D1Q3 x level N, D1Q3 x D1Q(2N+2)
LATTICES = [(0, 0, 0), (3, 0, 0), (6, 0, 0), (3, 1, 0), (7, 1, 0), (2, 1, glbm.ZV_Y),
            (5, 1, glbm.ZV_Y)]


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("k,x_level,zv", LATTICES)
def test_guo_random_state_moving_walls(k, x_level, zv, prec):
    N = k + 1
    NX = 1 if x_level == 1 else N
    vmax = 2 * N + 1 if zv else N
    nx, ny, steps = 70, 2 * vmax + 9, 30
    kn, uw, g = 0.07, 0.04, 3e-5
    rho, ux, uy = inputs.random_macro(80 + k + 10 * x_level + zv, nx, ny)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, x_level=x_level, zv_axes=zv, kn=kn,
                            prec=prec, u_wall_lo=-uw, u_wall_hi=uw, g=g, force=glbm.FORCE_GUO))
    lat.set_equilibrium(0, rho, ux, uy)
    lat.step(steps)
    lat.sync()
    got = lat.moments(0)
    tau = orc.tau_from_kn(N, ny, kn, zv=zv)
    assert lat.tau(0) == pytest.approx(tau, rel=1e-15)
    o = orc.Lattice(2, NX, N, nx, ny, orc.BC_WALLS, tau, -uw, uw, g, zv=zv, guo=1)
    X, _ = o.run(o.equilibrium(rho, ux, uy), steps)
    want, F = oracle_moments(o, X)
    q1x = 3 if x_level == 1 else 2 * N + 1
    errs = rel_errors(got, want, F=F, q1x=q1x, zv=zv)
    assert max(errs.values()) < TOL[prec], errs
    lat.close()


@pytest.mark.parametrize("prec,tol", [(glbm.FP64, 1e-12), (glbm.FP32_DEV, 1e-6)])
def test_guo_periodic_box_gains_g_per_node_and_step(prec, tol):
    """Fully periodic box from rest: the x momentum grows by exactly g per node
    and step, and the reported velocity is (t + 1/2) g / rho (the half-force
    shift). The conservation sums add rho u, the reported (shifted) momentum,
    so they read (t + 1/2) g per node. The populations' momentum starts at the
    rounding of a sum of O(1) terms (1e-17 in FP64), which bounds the absolute
    agreement of u at t = 0."""
    k, nx, ny, g, steps = 2, 48, 20, 2e-5, 64
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.8, prec=prec, bc=glbm.BC_PERIODIC,
                            g=g, force=glbm.FORCE_GUO))
    lat.set_equilibrium(0, np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    u0 = lat.moments(0)["ux"]
    np.testing.assert_allclose(u0, 0.5 * g, rtol=0, atol=tol * g)
    lat.step(steps)
    lat.sync()
    mass, jx, jy = lat.conservation(0)
    assert jx == pytest.approx((steps + 0.5) * g * nx * ny, rel=tol)
    assert abs(jy) < tol * steps * g * nx * ny
    np.testing.assert_allclose(lat.moments(0)["ux"], (steps + 0.5) * g, rtol=tol)
    lat.close()


def test_guo_and_linear_share_the_poiseuille_profile_up_to_g_over_2():
    """A unidirectional steady channel flow is the same under both force forms
    except for the half-force shift of the reported velocity (the oracle's pin,
    here through the GPU path in FP64)."""
    k, nx, ny, g = 1, 32, 24, 1e-5
    out = []
    for force in (glbm.FORCE_LINEAR, glbm.FORCE_GUO):
        lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, kn=0.05, prec=glbm.FP64, g=g,
                                force=force))
        lat.step(20000)
        lat.sync()
        out.append(lat.moments(0)["ux"])
        lat.close()
    np.testing.assert_allclose(out[1] - out[0], 0.5 * g, rtol=1e-6)


def test_guo_tile_shape_is_fixed():
    lat = glbm.Lattice(dict(dims=2, nx=64, ny=32, k=4, kn=0.1, prec=glbm.FP32_DEV, g=1e-5,
                            force=glbm.FORCE_GUO))
    assert lat.tile_shape(4)[2] == 1  # one-node tile
    lat.close()
