"""3D tensor products (Sec. 4 on three axes, D3Q27 / D3Q125 / D3Q343) on the
GPU against the oracle: every population after one step at every level in
both precisions with walls (moving, with the force) and periodic, moments
after steps from smooth fields, every tile shape, a z-uniform channel equal
to the 2D one, and checkpoints."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs
from paper_1905_04597_gb300.metrics import rel_errors

pytestmark = pytest.mark.gpu

TOL = {glbm.FP64: 1e-12, glbm.FP32_DEV: 1e-5}
POP_TOL = {glbm.FP64: 1e-13, glbm.FP32_DEV: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _oracle(k, nx, ny, nz, bc, tau, uw_lo=0.0, uw_hi=0.0, g=0.0):
    N = k + 1
    return orc.Lattice(3, N, N, nx, ny, bc, tau, uw_lo, uw_hi, g, NZ=N, Lz=nz)


def _cfg(k, nx, ny, nz, prec, **kw):
    return dict(dims=3, nx=nx, ny=ny, nz=nz, k=k, prec=prec, **kw)


def _fields(seed, nx, ny, nz, amp=0.03):
    rng = np.random.default_rng(seed)
    x = np.arange(nx)[None, None, :] / nx
    y = (np.arange(ny)[None, :, None] + 0.5) / ny
    z = np.arange(nz)[:, None, None] / nz
    out = []
    for i in range(4):
        a, b, c = rng.uniform(0, 2 * np.pi, 3)
        f = np.sin(2 * np.pi * x + a) * np.cos(np.pi * y + b) * np.cos(2 * np.pi * z + c)
        out.append((0.02 if i == 0 else amp) * f)
    return 1.0 + out[0], out[1], out[2], out[3]


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("bc", [glbm.BC_WALLS, glbm.BC_PERIODIC])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_one_step_all_populations(k, bc, prec):
    N = k + 1
    nx, ny, nz = 37, 2 * N + 5, 5
    tau, uw_lo, uw_hi, g = 0.83, -0.04, 0.06, 2e-4
    Q = (2 * N + 1) ** 3
    f0 = inputs.random_populations(1000 + k, Q, ny, nx * nz).reshape(Q, ny, nz, nx)
    f0 = np.ascontiguousarray(f0.transpose(0, 2, 1, 3))
    lat = glbm.Lattice(_cfg(k, nx, ny, nz, prec, tau=tau, bc=bc, u_wall_lo=uw_lo, u_wall_hi=uw_hi,
                            g=g))
    assert lat.nq() == Q and lat.shape() == (nz, ny, nx)
    lat.set_populations(0, f0)
    lat.step(1)
    lat.sync()
    got = lat.get_populations(0)
    want, _ = _oracle(k, nx, ny, nz, bc, tau, uw_lo, uw_hi, g).run(f0, 1)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < POP_TOL[prec], err
    lat.close()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_moments_after_steps(k, prec):
    N = k + 1
    nx, ny, nz, steps = 40, 2 * N + 10, 6, 40
    kw = dict(kn=0.15, u_wall_lo=-0.05, u_wall_hi=0.05, g=1e-5)
    rho, ux, uy, uz = _fields(1010 + k, nx, ny, nz)
    lat = glbm.Lattice(_cfg(k, nx, ny, nz, prec, **kw))
    lat.set_equilibrium(0, rho, ux, uy, uz)
    lat.step(steps)
    lat.sync()
    tau = orc.tau_from_kn(N, ny, 0.15)
    assert lat.tau(0) == pytest.approx(tau, rel=1e-14)
    o = _oracle(k, nx, ny, nz, orc.BC_WALLS, tau, -0.05, 0.05, 1e-5)
    X, _ = o.run(o.equilibrium(rho, ux, uy, uz), steps)
    F = o.stream(X)
    want = o.macro(F)
    got = lat.moments(0)
    assert set(got) == {"rho", "ux", "uy", "T", "qx", "qy", "sxy", "uz", "qz"}
    errs = rel_errors(got, want, dims=3, F=F)
    assert max(errs.values()) < TOL[prec], errs
    m, jx, jy = lat.conservation(0)
    assert m == pytest.approx(want[0].sum(), rel=1e-12 if prec == glbm.FP64 else 1e-7)
    lat.close()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_every_tile_shape_one_step(prec):
    for k in (0, 2):
        N = k + 1
        nx, ny, nz = 45, 2 * N + 3, 4
        Q = (2 * N + 1) ** 3
        f0 = inputs.random_populations(1020 + k, Q, nz * ny, nx).reshape(Q, nz, ny, nx)
        kw = dict(tau=0.9, u_wall_lo=0.03, u_wall_hi=-0.02, g=1e-4)
        want, _ = _oracle(k, nx, ny, nz, orc.BC_WALLS, 0.9, 0.03, -0.02, 1e-4).run(f0, 1)
        base = glbm.Lattice(_cfg(k, nx, ny, nz, prec, **kw))
        times = base.autotune(reps=2)
        assert set(times) == {k} and len(times[k]) >= 2
        n_shapes = len(times[k])
        base.close()
        for idx in range(n_shapes):
            lat = glbm.Lattice(_cfg(k, nx, ny, nz, prec, **kw))
            t = [-1] * glbm.LEVELS
            t[k] = idx
            lat.set_tiles(t)
            lat.set_populations(0, f0)
            lat.step(1)
            lat.sync()
            err = np.abs(lat.get_populations(0) - want).max() / np.abs(want).max()
            assert err < POP_TOL[prec], (k, idx, err)
            lat.close()


def test_z_uniform_channel_equals_2d_fp64():
    """A z-uniform 3D Couette-Poiseuille channel has the 2D channel's moments."""
    k, nx, ny, nz, steps = 1, 8, 20, 3, 300
    kw = dict(kn=0.1, u_wall_lo=-0.04, u_wall_hi=0.04, g=2e-5, prec=glbm.FP64)
    l3 = glbm.Lattice(_cfg(k, nx, ny, nz, **kw))
    l2 = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, **kw))
    l3.step(steps)
    l2.step(steps)
    m3, m2 = l3.moments(0), l2.moments(0)
    # the same sums in another order: agreement to FP64 rounding of each field's scale
    for name in ("rho", "ux", "uy", "sxy"):
        scale = max(np.abs(m2[name]).max(), np.abs(m2["ux"]).max())
        for z in range(nz):
            np.testing.assert_allclose(m3[name][z], m2[name], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(m3["uz"], 0, atol=1e-12 * np.abs(m2["ux"]).max())
    for x in (l3, l2):
        x.close()


def test_checkpoint_and_unsupported_operations(tmp_path):
    cfg = _cfg(1, 24, 12, 4, glbm.FP32_DEV, tau=0.7, u_wall_lo=-0.03, u_wall_hi=0.03)
    a = glbm.Lattice(cfg)
    a.set_equilibrium(0, *_fields(1030, 24, 12, 4))
    a.step(10)
    path = str(tmp_path / "d3.ckpt")
    a.save(path)
    b = glbm.Lattice(cfg)
    b.load(path)
    a.step(15)
    b.step(15)
    np.testing.assert_array_equal(a.get_populations(0), b.get_populations(0))
    other = glbm.Lattice(dict(cfg, nz=5))
    with pytest.raises(glbm.GlbmError):
        other.load(path)
    with pytest.raises(glbm.GlbmError):
        a.adjoint_flowrate(10, 5)
    for x in (a, b, other):
        x.close()
