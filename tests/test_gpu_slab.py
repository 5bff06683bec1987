"""The x-slab decomposition on the GPU library: slabs of Ls + 2H columns with
their halos refilled after every step, or H = m x reach refilled after every
m steps, reproduce the undivided lattice on
their owned columns (FP64 bit for bit; FP32 within the dithered rounding,
whose random words follow the local node index). Every call of this run has
one GPU, so the multi-slab case runs its slabs as separate contexts on that
GPU, exchanging columns through the library's pack/unpack calls from the
host (no kernel waits on another)."""
import numpy as np
import pytest

from paper_1905_04597_gb300 import glbm, inputs, slab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _cfg(prec, **kw):
    c = dict(dims=2, nx=96, ny=20, k=2, kn=0.2, u_wall_lo=-0.04, u_wall_hi=0.05, g=2e-5, prec=prec)
    c.update(kw)
    return c


def _reference(cfg, f0, steps):
    lat = glbm.Lattice(cfg)
    lat.set_populations(0, f0)
    lat.step(steps)
    out = lat.get_populations(0)
    lat.close()
    return out


def _exchange_in_process(slabs):
    """Halo exchange between the slabs of one process (ring along x)."""
    W = len(slabs)
    firsts = [s.pack(s.H, s.H) for s in slabs]
    lasts = [s.pack(s.Ls, s.H) for s in slabs]
    for r, s in enumerate(slabs):
        s.unpack(0, s.H, lasts[(r - 1) % W])
        s.unpack(s.Ls + s.H, s.H, firsts[(r + 1) % W])


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("world", [1, 2, 3])
def test_slabs_reproduce_the_undivided_lattice(world, prec):
    cfg = _cfg(prec)
    Q = (2 * cfg["k"] + 3) ** 2
    f0 = inputs.random_populations(1100, Q, cfg["ny"], cfg["nx"])
    steps = 12
    want = _reference(cfg, f0, steps)
    slabs = [slab.SlabLattice(cfg, r, world, sendrecv=lambda *a: None) for r in range(world)]
    for s in slabs:
        s.set_populations_global(f0)
    for _ in range(steps):
        for s in slabs:
            s.step(1)
        if world == 1:
            slabs[0].exchange()
        else:
            _exchange_in_process(slabs)
    got = np.concatenate([s.owned_populations() for s in slabs], axis=-1)
    if prec == glbm.FP64:
        np.testing.assert_array_equal(got, want)
    else:
        assert np.abs(got - want).max() / np.abs(want).max() < 1e-6
    for s in slabs:
        s.lat.close()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("world,depth", [(1, 4), (2, 5), (3, 3)])
def test_deep_halos_reproduce_the_undivided_lattice(world, depth, prec):
    """Halos of depth x reach columns refilled once every `depth` steps (13
    steps: a ragged last block); the slabs' steps of several steps per call
    run in dataflow chunks."""
    cfg = _cfg(prec)
    Q = (2 * cfg["k"] + 3) ** 2
    f0 = inputs.random_populations(1200 + depth, Q, cfg["ny"], cfg["nx"])
    steps = 13
    want = _reference(cfg, f0, steps)
    slabs = [slab.SlabLattice(cfg, r, world, sendrecv=lambda *a: None, depth=depth)
             for r in range(world)]
    assert all(s.H == depth * 3 for s in slabs)
    for s in slabs:
        s.set_populations_global(f0)
    if world == 1:
        slabs[0].advance(steps)
    else:
        left = steps
        while left > 0:
            n = min(depth, left)
            for s in slabs:
                s.step(n)
            _exchange_in_process(slabs)
            left -= n
    got = np.concatenate([s.owned_populations() for s in slabs], axis=-1)
    if prec == glbm.FP64:
        np.testing.assert_array_equal(got, want)
    else:
        assert np.abs(got - want).max() / np.abs(want).max() < 1e-6
    for s in slabs:
        s.lat.close()


def test_pack_unpack_round_trip_and_bounds():
    lat = glbm.Lattice(_cfg(glbm.FP32_DEV, nx=40))
    import torch
    buf = torch.empty((lat.nq(), 20, 5), dtype=torch.float32, device="cuda")
    lat.pack_columns(0, 7, 5, buf)
    before = lat.get_populations(0)
    lat.unpack_columns(0, 30, 5, buf)
    after = lat.get_populations(0)
    np.testing.assert_array_equal(after[..., 30:35], before[..., 7:12])
    np.testing.assert_array_equal(after[..., :30], before[..., :30])
    host = np.empty((lat.nq(), 20, 5), dtype=np.float32)
    lat.pack_columns(0, 7, 5, host)
    np.testing.assert_array_equal(host, buf.cpu().numpy())
    with pytest.raises(glbm.GlbmError):
        lat.pack_columns(0, 38, 5, buf)
    with pytest.raises(TypeError):
        lat.pack_columns(0, 0, 5, np.empty((lat.nq(), 20, 5)))  # FP64 buffer for FP32 storage
    lat.close()
