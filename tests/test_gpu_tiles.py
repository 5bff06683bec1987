"""Tile shapes of the fused 2D step and the autotuner: every candidate shape of
every level gives the oracle's populations, autotuning leaves the state, the
step clock and the dither sequence unchanged, and an autotuned batch still
matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs
from parity_helpers import oracle_moments, rel_errors

pytestmark = pytest.mark.gpu

POP_TOL = {glbm.FP64: 1e-13, glbm.FP32_DEV: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("k", range(8))
def test_every_tile_shape_one_step(k, prec):
    """One step from random populations with walls, a moving wall pair and a
    force, ragged in x (37 columns) and in y, for each candidate shape."""
    N = k + 1
    nx, ny = 37, 2 * N + 5
    tau, uw_lo, uw_hi, g = 0.9, -0.04, 0.03, 1e-4
    f0 = inputs.random_populations(700 + k, (2 * N + 1) ** 2, ny, nx)
    o = orc.Lattice(2, N, N, nx, ny, orc.BC_WALLS, tau, uw_lo, uw_hi, g)
    want, _ = o.run(f0, 1)
    shapes = glbm.tile_shapes(k, prec)
    assert shapes
    for idx, (G, R, V) in enumerate(shapes):
        lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=tau, prec=prec, u_wall_lo=uw_lo,
                                u_wall_hi=uw_hi, g=g))
        tiles = [-1] * glbm.LEVELS
        tiles[k] = idx
        lat.set_tiles(tiles)
        assert lat.tiles()[k] == idx
        lat.set_populations(0, f0)
        lat.step(1)
        lat.sync()
        got = lat.get_populations(0)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < POP_TOL[prec], (idx, G, R, V, err)
        lat.close()


def test_autotune_keeps_state_clock_and_dither_sequence():
    cfg = dict(dims=2, nx=96, ny=40, k=3, kn=0.1, prec=glbm.FP32_DEV, u_wall_lo=-0.05,
               u_wall_hi=0.05)
    fields = inputs.random_macro(11, 96, 40)
    a = glbm.Lattice([cfg, cfg])
    b = glbm.Lattice([cfg, cfg])
    for lat in (a, b):
        for i in range(2):
            lat.set_equilibrium(i, *fields)
        lat.step(7)
    before = a.get_populations(1)
    times = a.autotune(reps=3)
    assert set(times) == {3} and len(times[3]) == len(glbm.tile_shapes(3, glbm.FP32_DEV))
    assert all(t > 0 for t in times[3])
    chosen = a.tiles()[3]
    assert times[3][chosen] == min(times[3])
    np.testing.assert_array_equal(a.get_populations(1), before)
    assert a.time == 7
    b.set_tiles(a.tiles())
    for lat in (a, b):
        lat.step(70)  # one graph chunk and six single launches
        lat.sync()
    for i in range(2):
        np.testing.assert_array_equal(a.get_populations(i), b.get_populations(i))
    a.close()
    b.close()


def test_autotuned_batch_matches_oracle():
    mixed = [
        dict(k=1, nx=64, ny=21, kn=0.05, u_wall_lo=-0.03, u_wall_hi=0.04, g=0.0),
        dict(k=4, nx=64, ny=33, kn=0.3, u_wall_lo=0.0, u_wall_hi=0.0, g=2e-5),
        dict(k=7, nx=64, ny=19, kn=2.0, u_wall_lo=-0.05, u_wall_hi=0.05, g=0.0),
        dict(k=4, nx=64, ny=10, kn=0.02, u_wall_lo=0.02, u_wall_hi=-0.01, g=0.0),
    ]
    steps = 20
    lat = glbm.Lattice([dict(dims=2, prec=glbm.FP32_DEV, **c) for c in mixed], hetero=True)
    fields = [inputs.random_macro(900 + i, c["nx"], c["ny"]) for i, c in enumerate(mixed)]
    for i, f in enumerate(fields):
        lat.set_equilibrium(i, *f)
    times = lat.autotune(reps=2)
    assert set(times) == {1, 4, 7}
    launches = lat.kernel_launches
    lat.step(steps)
    lat.sync()
    assert lat.kernel_launches - launches == 3 * steps  # one launch per level present
    for i, c in enumerate(mixed):
        N = c["k"] + 1
        o = orc.Lattice(2, N, N, c["nx"], c["ny"], orc.BC_WALLS,
                        orc.tau_from_kn(N, c["ny"], c["kn"]), c["u_wall_lo"], c["u_wall_hi"],
                        c["g"])
        X, _ = o.run(o.equilibrium(*fields[i]), steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(lat.moments(i), want, F=F)
        assert max(errs.values()) < 1e-5, (i, errs)
    lat.close()


def test_set_tiles_rejects_out_of_range_index():
    lat = glbm.Lattice(dict(dims=2, nx=32, ny=8, k=2, tau=0.8, prec=glbm.FP32_DEV))
    bad = [-1] * glbm.LEVELS
    bad[2] = len(glbm.tile_shapes(2, glbm.FP32_DEV))
    before = lat.tiles()
    with pytest.raises(glbm.GlbmError):
        lat.set_tiles(bad)
    assert lat.tiles() == before
    lat.close()


@pytest.mark.parametrize("k", range(8))
def test_pair_tiles_bitwise_equal_one_node_tiles_of_same_split(k):
    """A packed pair tile rounds every lane like the one-node tile: with the same
    warp-group split G they give bit-identical populations (walls, force, a
    ragged width that is not a multiple of the 64-column pair tile)."""
    shapes = glbm.tile_shapes(k, glbm.FP32_DEV)
    pairs = [(i, j) for i, a in enumerate(shapes) for j, b in enumerate(shapes)
             if a[2] == 1 and b[2] == 2 and a[0] == b[0]]
    if not pairs:
        pytest.skip("no pair tile with a one-node tile of the same G at this level")
    N = k + 1
    nx, ny = 100, 3 * N + 4
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, kn=0.2, prec=glbm.FP32_DEV, u_wall_lo=-0.03,
               u_wall_hi=0.05, g=2e-5)
    fields = inputs.random_macro(40 + k, nx, ny)
    for i, j in pairs[:2]:
        out = []
        for idx in (i, j):
            lat = glbm.Lattice(cfg)
            tiles = [-1] * glbm.LEVELS
            tiles[k] = idx
            lat.set_tiles(tiles)
            lat.set_equilibrium(0, *fields)
            lat.step(9)
            lat.sync()
            out.append(lat.get_populations(0))
            lat.close()
        np.testing.assert_array_equal(out[0], out[1])
