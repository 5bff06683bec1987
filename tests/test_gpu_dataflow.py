"""Dataflow stepping (overlapping launches within a chunk of steps, glbm.h
glbm_set_dataflow) against stepping one launch after another: the same
arithmetic and the same dither, so the populations must agree bit for bit,
for every tile kind, both precisions, walls and periodic boundaries, several
instances, and step counts that leave a partial chunk. Also the failure
contract: a node leaving the positivity domain partway through a dataflow call
stops the run exactly where the one-after-another run stops."""
import numpy as np
import pytest

from paper_1905_04597_gb300 import glbm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _pair(cfgs, tiles=None, seed=0):
    """Two contexts of the same instances from the same random state, one in
    dataflow mode and one stepping launch after launch."""
    out = []
    for df in (1, 0):
        lat = glbm.Lattice(cfgs)
        if tiles is not None:
            lat.set_tiles(tiles)
        if cfgs[0].get("bc", glbm.BC_WALLS) == glbm.BC_WALLS:
            lat.set_wall_launch(0)  # the wall densities from the tiles
        lat.set_dataflow(df)
        for i, c in enumerate(cfgs):
            lat.set_equilibrium(i, *inputs.random_macro(seed + i, c["nx"], c["ny"]))
        out.append(lat)
    assert out[0].dataflow == 1 and out[1].dataflow == 0
    return out


def _same(a, b, n):
    for i in range(n):
        np.testing.assert_array_equal(a.get_populations(i), b.get_populations(i))


CASES = [
    # (k, x_level, zv, prec, bc, nx, ny, instances)
    (3, 0, 0, glbm.FP32_DEV, glbm.BC_WALLS, 200, 70, 3),
    (3, 0, 0, glbm.FP64, glbm.BC_WALLS, 96, 40, 2),
    (0, 0, 0, glbm.FP32_DEV, glbm.BC_PERIODIC, 130, 33, 2),
    (7, 0, 0, glbm.FP32_DEV, glbm.BC_WALLS, 70, 50, 1),
    (4, 1, 0, glbm.FP32_DEV, glbm.BC_WALLS, 150, 45, 2),
    (2, 1, glbm.ZV_Y, glbm.FP32_DEV, glbm.BC_WALLS, 100, 30, 2),
    (1, 0, glbm.ZV_X | glbm.ZV_Y, glbm.FP32_DEV, glbm.BC_PERIODIC, 64, 20, 1),
]


@pytest.mark.parametrize("k,x_level,zv,prec,bc,nx,ny,n", CASES)
def test_dataflow_equals_launch_after_launch(k, x_level, zv, prec, bc, nx, ny, n):
    cfgs = [dict(dims=2, nx=nx, ny=ny, k=k, x_level=x_level, zv_axes=zv, kn=0.05 * (i + 1),
                 prec=prec, bc=bc, u_wall_lo=-0.03, u_wall_hi=0.04, g=2e-5) for i in range(n)]
    a, b = _pair(cfgs, seed=10 * k + n)
    for steps in (64, 37, 130):  # whole chunks, a partial one, both
        a.step(steps)
        b.step(steps)
        assert a.time == b.time
        _same(a, b, n)
    a.close()
    b.close()


@pytest.mark.parametrize("idx", range(3))
def test_dataflow_every_couette_tile_shape(idx):
    """The first three candidate tile shapes of Couette D2Q81 (pair and one-node
    tiles of several row counts)."""
    cfgs = [dict(dims=2, nx=160, ny=48, k=3, kn=kn, prec=glbm.FP32_DEV, u_wall_lo=-0.05,
                 u_wall_hi=0.05) for kn in (0.01, 0.1, 1.0)]
    tiles = [-1] * glbm.LEVELS
    tiles[3] = idx
    a, b = _pair(cfgs, tiles=tiles, seed=40 + idx)
    a.step(200)
    b.step(200)
    _same(a, b, 3)
    a.close()
    b.close()


def test_dataflow_guo_force():
    cfgs = [dict(dims=2, nx=90, ny=36, k=5, kn=0.1, prec=glbm.FP32_DEV, g=3e-5,
                 force=glbm.FORCE_GUO)]
    a, b = _pair(cfgs, seed=77)
    a.step(100)
    b.step(100)
    _same(a, b, 1)
    a.close()
    b.close()


def test_dataflow_calls_of_every_length():
    """Calls of 1 to 130 steps one after another: a dataflow call leaves the
    buffer of its starting state unwritten and rotates three state buffers, so
    its chunks replay graphs captured for several bindings of them. Populations
    and moments stay equal to launch-after-launch stepping after every call,
    also across a state set in between."""
    cfgs = [dict(dims=2, nx=120, ny=40, k=3, kn=kn, prec=glbm.FP32_DEV, u_wall_lo=-0.05,
                 u_wall_hi=0.05, g=1e-5) for kn in (0.05, 0.5)]
    a, b = _pair(cfgs, seed=91)
    for j, n in enumerate((1, 2, 3, 64, 65, 1, 128, 7, 64, 64, 129, 2)):
        a.step(n)
        b.step(n)
        assert a.time == b.time
        _same(a, b, 2)
        for i in range(2):
            ma, mb = a.moments(i), b.moments(i)
            for key in ma:
                np.testing.assert_array_equal(ma[key], mb[key])
        if j == 5:
            f = a.get_populations(1)
            for lat in (a, b):
                lat.set_populations(1, f)
    a.close()
    b.close()


@pytest.mark.parametrize("before", [0, 40])
def test_dataflow_failure_stops_at_the_failing_step(before):
    """A uniform periodic flow driven from rest by g = 0.01 on D2Q9 leaves the
    positivity domain at step 82 (u = g t), inside the second chunk of a
    200-step call (started at rest, or after a successful 40-step call that
    rotated the state buffers): the dataflow context reports the same error,
    the same completed steps and the same state as the launch-after-launch one
    (it binds the call's starting buffer again and replays the call)."""
    nx, ny = 32, 8
    cfg = dict(dims=2, nx=nx, ny=ny, k=0, tau=0.8, prec=glbm.FP32_DEV, bc=glbm.BC_PERIODIC,
               g=0.01)
    res = []
    for df in (1, 0):
        lat = glbm.Lattice(cfg)
        lat.set_dataflow(df)
        assert lat.dataflow == df
        if before:
            lat.step(before)
        err = None
        try:
            lat.step(200)
        except glbm.GlbmError as e:
            err = str(e)
        res.append((err, lat.time, lat.get_populations(0)))
        # the context stays stopped, in either mode
        with pytest.raises(glbm.UnstableError, match="0 of 10 steps completed"):
            lat.step(10)
        lat.close()
    (e1, t1, f1), (e0, t0, f0) = res
    assert e0 is not None and f"{83 - before} of 200 steps completed" in e0
    assert e1 == e0 and t1 == t0 == 83
    np.testing.assert_array_equal(f1, f0)


def test_dataflow_wait_that_runs_out_reports_a_timeout():
    """Test mode 2 makes every wait of a chunk's later steps unsatisfiable: the
    first wait gives up after 0.5 s and sets the timeout flag, no later wait
    goes on (the halt word), and glbm_step returns GLBM_E_TIMEOUT with the state
    and the clock of the call's start. The context then steps normally."""
    import time
    nx, ny = 96, 32
    cfg = dict(dims=2, nx=nx, ny=ny, k=2, kn=0.1, prec=glbm.FP32_DEV, u_wall_lo=-0.05,
               u_wall_hi=0.05)
    lat = glbm.Lattice(cfg)
    lat.set_wall_launch(0)
    lat.set_equilibrium(0, *inputs.random_macro(5, nx, ny))
    lat.step(3)
    before = lat.get_populations(0)
    lat.set_dataflow(2)
    t0 = time.perf_counter()
    with pytest.raises(glbm.GlbmError) as err:
        lat.step(64)
    assert err.value.status == glbm.E_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert lat.time == 3
    np.testing.assert_array_equal(lat.get_populations(0), before)
    lat.set_dataflow(1)
    lat.step(64)
    ref = glbm.Lattice(cfg)
    ref.set_wall_launch(0)
    ref.set_dataflow(0)
    ref.set_equilibrium(0, *inputs.random_macro(5, nx, ny))
    ref.step(67)
    np.testing.assert_array_equal(lat.get_populations(0), ref.get_populations(0))
    lat.close()
    ref.close()


def test_checkpoint_and_adjoint_after_rotated_buffers(tmp_path):
    """After dataflow calls have rotated the three state buffers, a checkpoint
    written by the dataflow context and loaded into a fresh one continues
    identically, and the adjoint starts from the same state as in a context
    stepped launch after launch."""
    cfg = dict(dims=2, nx=64, ny=30, k=2, kn=0.1, prec=glbm.FP32_DEV, u_wall_lo=-0.04,
               u_wall_hi=0.05, g=1e-5)
    a, b = _pair([cfg], seed=123)
    for n in (3, 64, 5):
        a.step(n)
        b.step(n)
    path = tmp_path / "ck.glbm"
    a.save(path)
    c = glbm.Lattice(cfg)
    c.set_wall_launch(0)
    c.load(path)
    assert c.time == a.time
    for lat in (a, c):
        lat.step(33)
    _same(a, c, 1)
    b.step(33)
    ja = a.adjoint_flowrate(40, ckpt_every=8, walls=True)
    jb = b.adjoint_flowrate(40, ckpt_every=8, walls=True)
    np.testing.assert_array_equal(np.asarray(ja), np.asarray(jb))
    for lat in (a, b, c):
        lat.close()


def test_dataflow_falls_back_when_its_buffers_cannot_be_allocated():
    """An allocator that refuses the third state buffer (and the dataflow
    counters): glbm_step runs the call launch after launch, switches the
    context's dataflow off, and the results are those of stepping launch after
    launch from the start."""
    import torch
    refuse = {"on": False}

    def _alloc(nbytes, stream, user):
        if refuse["on"]:
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  stream or 0)

    def _free(ptr, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (glbm.ALLOC_FN(_alloc), glbm.FREE_FN(_free))
    had_torch = glbm._torch_alloc_refs is not None
    glbm.check(glbm.lib().glbm_set_allocator(hooks[0], hooks[1], None))
    nx, ny = 96, 32
    cfg = dict(dims=2, nx=nx, ny=ny, k=2, kn=0.1, prec=glbm.FP32_DEV, u_wall_lo=-0.05,
               u_wall_hi=0.05)
    fields = inputs.random_macro(8, nx, ny)
    try:
        lat = glbm.Lattice(cfg)
        lat.set_wall_launch(0)
        lat.set_equilibrium(0, *fields)
        assert lat.dataflow == 1
        refuse["on"] = True
        lat.step(40)
        refuse["on"] = False
        assert lat.dataflow == 0 and lat.time == 40
        got = lat.get_populations(0)
        lat.close()
    finally:
        refuse["on"] = False
        if had_torch:
            glbm.install_torch_allocator()
        else:
            glbm.uninstall_allocator()
    ref = glbm.Lattice(cfg)
    ref.set_wall_launch(0)
    ref.set_dataflow(0)
    ref.set_equilibrium(0, *fields)
    ref.step(40)
    np.testing.assert_array_equal(got, ref.get_populations(0))
    ref.close()
