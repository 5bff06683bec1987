"""Wall densities of the diffuse walls (Sec. 5.3): summed by every tile within
reach of a wall (mode 0) or by a launch of their own before the stream-collide
kernel (mode 1). The two modes give bit-identical populations for every tile
shape, hierarchy and precision; the default mode follows the share of repeated
wall sums; the extra launch is counted; the adjoint does not depend on it."""
import numpy as np
import pytest

from paper_1905_04597_gb300 import glbm, inputs

pytestmark = pytest.mark.gpu

KINDS = {"iso": (0, 0), "x1": (1, glbm.ZV_Y), "xy": (0, glbm.ZV_X | glbm.ZV_Y), "aniso": (1, 0)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _cfg(kind, k, nx, ny, prec, **kw):
    x_level, zv = KINDS[kind]
    return dict(dims=2, nx=nx, ny=ny, k=k, x_level=x_level, zv_axes=zv, prec=prec, **kw)


def _shape_count(cfg, k):
    probe = glbm.Lattice(cfg)
    n = len(probe.autotune(reps=1)[k])
    probe.close()
    return n


def _run(cfg, k, idx, mode, fields, steps):
    lat = glbm.Lattice(cfg)
    t = [-1] * glbm.LEVELS
    t[k] = idx
    lat.set_tiles(t)
    lat.set_wall_launch(mode)
    assert lat.wall_launch == mode
    lat.set_equilibrium(0, *fields)
    lat.step(steps)
    lat.sync()
    out = lat.get_populations(0)
    lat.close()
    return out


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("kind,k", [("iso", 0), ("iso", 3), ("iso", 7), ("x1", 2), ("x1", 9),
                                    ("xy", 2), ("aniso", 3)])
def test_modes_bitwise_equal_every_tile_shape(kind, k, prec):
    """Walls moving both ways, a force, a ragged width (not a multiple of the
    64-column pair tile) and a channel of 3N + 4 rows, 9 steps per shape."""
    N = k + 1
    nx, ny = 100, 3 * N + 4
    cfg = _cfg(kind, k, nx, ny, prec, kn=0.2, u_wall_lo=-0.03, u_wall_hi=0.05, g=2e-5)
    fields = inputs.random_macro(1300 + k, nx, ny)
    for idx in range(_shape_count(cfg, k)):
        a = _run(cfg, k, idx, 0, fields, 9)
        b = _run(cfg, k, idx, 1, fields, 9)
        np.testing.assert_array_equal(a, b, err_msg=f"shape {idx}")


def test_default_mode_follows_repeated_share():
    """Mode 1 where the tiles of one node row within reach of the walls would
    repeat the wall sums for more than a tenth of a step's loads."""
    def mode(**kw):
        lat = glbm.Lattice(dict(dims=2, nx=32, prec=glbm.FP32_DEV, kn=0.1, **kw))
        m = lat.wall_launch
        lat.close()
        return m
    # D2Q289, 128 rows: 2 * 8 * 36 * 17 repeated loads per column, 128 * 289 own
    assert mode(ny=128, k=7) == 1
    # D2Q81, 256 rows: 720 against 20736
    assert mode(ny=256, k=3) == 0
    # D2Q81, 24 rows: 720 against 1944
    assert mode(ny=24, k=3) == 1
    # 2N+2 along y, level 13, the paper's 200 rows
    assert mode(ny=200, k=12, x_level=1, zv_axes=glbm.ZV_Y) == 1
    assert mode(ny=64, k=3, bc=glbm.BC_PERIODIC) == -1


def test_mode_rejected_without_walls():
    lat = glbm.Lattice(dict(dims=2, nx=32, ny=16, k=1, kn=0.1, prec=glbm.FP64,
                            bc=glbm.BC_PERIODIC))
    with pytest.raises(glbm.GlbmError):
        lat.set_wall_launch(1)
    lat.close()
    lat = glbm.Lattice(dict(dims=2, nx=32, ny=16, k=1, kn=0.1, prec=glbm.FP64))
    with pytest.raises(glbm.GlbmError):
        lat.set_wall_launch(2)
    lat.set_wall_launch(-1)
    assert lat.wall_launch == 1  # 2 * 2 * 3 * 5 repeated against 16 * 25 own loads
    lat.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_launch_count(mode):
    lat = glbm.Lattice(dict(dims=2, nx=64, ny=20, k=2, kn=0.1, prec=glbm.FP32_DEV,
                            u_wall_lo=-0.05, u_wall_hi=0.05))
    lat.set_wall_launch(mode)
    n0 = lat.kernel_launches
    lat.step(5)    # single launches
    lat.step(128)  # two captured chunks of 64 steps
    lat.sync()
    # in dataflow mode (wall densities from the tiles) each of the three
    # chunks also launches the kernel that resets its counters
    assert lat.kernel_launches - n0 == (1 + mode) * 133 + (3 if lat.dataflow else 0)
    lat.close()


def test_adjoint_independent_of_mode():
    cfg = dict(dims=2, nx=48, ny=24, k=3, kn=0.1, prec=glbm.FP32_DEV, g=1e-5)
    out = []
    for mode in (0, 1):
        lat = glbm.Lattice(cfg)
        lat.set_wall_launch(mode)
        out.append(lat.adjoint_flowrate(60, ckpt_every=20))
        lat.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


def test_autotune_picks_a_mode():
    lat = glbm.Lattice(dict(dims=2, nx=64, ny=40, k=4, kn=0.1, prec=glbm.FP32_DEV,
                            u_wall_lo=-0.05, u_wall_hi=0.05))
    lat.autotune(reps=2)
    assert lat.wall_launch in (0, 1)
    lat.close()
