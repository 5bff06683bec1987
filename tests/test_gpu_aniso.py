"""Anisotropic tensor products on the GPU against the oracle: D1Q3 along x times
the level-(k+1) lattice along y (x_level = 1), the 2D form of Sec. 4 that the
paper uses for its channel flows. Every population after one step at every
level in both precisions, moments after many steps from smooth fields, every
tile shape, a Poiseuille channel, checkpoints and the operations that take
isotropic lattices only."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs
from parity_helpers import oracle_moments, rel_errors

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


def _oracle(k, nx, ny, bc, tau, uw_lo=0.0, uw_hi=0.0, g=0.0):
    return orc.Lattice(2, 1, k + 1, nx, ny, bc, tau, uw_lo, uw_hi, g)


def _cfg(k, nx, ny, prec, **kw):
    return dict(dims=2, nx=nx, ny=ny, k=k, x_level=1, prec=prec, **kw)


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("bc", [glbm.BC_WALLS, glbm.BC_PERIODIC])
@pytest.mark.parametrize("k", range(8))
def test_one_step_all_populations(k, bc, prec):
    N = k + 1
    nx, ny = 37, 2 * N + 5
    tau, uw_lo, uw_hi, g = 0.83, -0.04, 0.06, 2e-4
    Q = 3 * (2 * N + 1)
    f0 = inputs.random_populations(800 + k, Q, ny, nx)
    lat = glbm.Lattice(_cfg(k, nx, ny, prec, tau=tau, bc=bc, u_wall_lo=uw_lo, u_wall_hi=uw_hi, g=g))
    assert lat.nq() == Q
    lat.set_populations(0, f0)
    lat.step(1)
    lat.sync()
    got = lat.get_populations(0)
    want, _ = _oracle(k, nx, ny, bc, tau, uw_lo, uw_hi, g).run(f0, 1)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < POP_TOL[prec], err
    lat.close()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("k", [1, 4, 7])
def test_moments_after_steps(k, prec):
    N = k + 1
    nx, ny, steps = 48, 3 * N + 6, 60
    kw = dict(kn=0.15, u_wall_lo=-0.05, u_wall_hi=0.05, g=1e-5)
    fields = inputs.random_macro(820 + k, nx, ny)
    lat = glbm.Lattice(_cfg(k, nx, ny, prec, **kw))
    lat.set_equilibrium(0, *fields)
    lat.step(steps)
    lat.sync()
    o = _oracle(k, nx, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, 0.15), -0.05, 0.05, 1e-5)
    assert lat.tau(0) == pytest.approx(orc.tau_from_kn(N, ny, 0.15), rel=1e-14)
    X, _ = o.run(o.equilibrium(*fields), steps)
    want, F = oracle_moments(o, X)
    errs = rel_errors(lat.moments(0), want, F=F, q1x=3)
    assert max(errs.values()) < TOL[prec], errs
    lat.close()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_every_tile_shape_one_step(prec):
    for k in (2, 7):
        N = k + 1
        nx, ny = 45, 2 * N + 3
        f0 = inputs.random_populations(830 + k, 3 * (2 * N + 1), ny, nx)
        want, _ = _oracle(k, nx, ny, orc.BC_WALLS, 0.9, 0.03, -0.02, 1e-4).run(f0, 1)
        base = glbm.Lattice(_cfg(k, nx, ny, prec, tau=0.9, u_wall_lo=0.03, u_wall_hi=-0.02, g=1e-4))
        times = base.autotune(reps=2)
        assert set(times) == {k} and len(times[k]) >= 2
        G, R, V = base.tile_shape(k)
        assert G >= 1 and R >= 1 and (V == 1 or prec == glbm.FP32_DEV)
        n_shapes = len(times[k])
        base.close()
        for idx in range(n_shapes):
            lat = glbm.Lattice(_cfg(k, nx, ny, prec, tau=0.9, u_wall_lo=0.03, u_wall_hi=-0.02,
                                    g=1e-4))
            t = [-1] * glbm.LEVELS
            t[k] = idx
            lat.set_tiles(t)
            lat.set_populations(0, f0)
            lat.step(1)
            lat.sync()
            err = np.abs(lat.get_populations(0) - want).max() / np.abs(want).max()
            assert err < POP_TOL[prec], (k, idx, err)
            lat.close()


def test_poiseuille_channel_d1q3_by_d1q11_fp32():
    """The paper's channel form: x-uniform Poiseuille flow between diffuse walls,
    D1Q3 x D1Q11, 2000 steps in FP32 deviations against the FP64 oracle."""
    k, ny, steps, g = 4, 40, 2000, 1e-5
    N = k + 1
    for kn in (0.05, 0.5):
        lat = glbm.Lattice(_cfg(k, 1, ny, glbm.FP32_DEV, kn=kn, g=g))
        lat.step(steps)
        lat.sync()
        o = _oracle(k, 1, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, kn), g=g)
        X, _ = o.run(o.equilibrium(np.ones((ny, 1)), np.zeros((ny, 1)), np.zeros((ny, 1))), steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(lat.moments(0), want, F=F, q1x=3)
        assert max(errs.values()) < TOL[glbm.FP32_DEV], (kn, errs)
        u = lat.moments(0)["ux"][:, 0]
        assert u.max() > 0 and np.allclose(u, u[::-1], rtol=1e-4)
        lat.close()


def test_conservation_checkpoint_and_isotropic_only_operations(tmp_path):
    k, nx, ny = 3, 40, 14
    cfg = _cfg(k, nx, ny, glbm.FP32_DEV, tau=0.7, u_wall_lo=-0.03, u_wall_hi=0.03)
    a = glbm.Lattice(cfg)
    a.set_equilibrium(0, *inputs.random_macro(840, nx, ny))
    m0, _, _ = a.conservation(0)
    a.step(30)
    m1, _, _ = a.conservation(0)
    assert m1 == pytest.approx(m0, rel=1e-6)
    path = str(tmp_path / "aniso.ckpt")
    a.save(path)
    b = glbm.Lattice(cfg)
    b.load(path)
    a.step(20)
    b.step(20)
    np.testing.assert_array_equal(a.get_populations(0), b.get_populations(0))
    iso = glbm.Lattice(dict(cfg, x_level=0))
    with pytest.raises(glbm.GlbmError):
        iso.load(path)  # another lattice: the checkpoint's configuration check refuses it
    with pytest.raises(glbm.GlbmError):
        a.adjoint_flowrate(10, 5)
    for x in (a, b, iso):
        x.close()


@pytest.mark.parametrize("k", [1, 3, 6, 7])
def test_pair_tiles_bitwise_equal_one_node_tiles(k):
    """On the anisotropic lattices too, pair and one-node tiles of the same
    warp-group split give bit-identical populations."""
    N = k + 1
    nx, ny = 100, 3 * N + 4
    cfg = _cfg(k, nx, ny, glbm.FP32_DEV, kn=0.2, u_wall_lo=-0.03, u_wall_hi=0.05, g=2e-5)
    fields = inputs.random_macro(850 + k, nx, ny)
    probe = glbm.Lattice(cfg)
    n = len(probe.autotune(reps=1)[k])
    shapes = []
    for idx in range(n):
        t = [-1] * glbm.LEVELS
        t[k] = idx
        probe.set_tiles(t)
        shapes.append(probe.tile_shape(k))
    probe.close()
    pairs = [(i, j) for i, a in enumerate(shapes) for j, b in enumerate(shapes)
             if a[2] == 1 and b[2] == 2 and a[0] == b[0]]
    assert pairs, shapes
    i, j = pairs[0]
    out = []
    for idx in (i, j):
        lat = glbm.Lattice(cfg)
        t = [-1] * glbm.LEVELS
        t[k] = idx
        lat.set_tiles(t)
        lat.set_equilibrium(0, *fields)
        lat.step(9)
        lat.sync()
        out.append(lat.get_populations(0))
        lat.close()
    np.testing.assert_array_equal(out[0], out[1])
