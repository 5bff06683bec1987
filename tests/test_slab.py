"""The x-slab decomposition's exchange on CPU ranks (gloo, world sizes 2 and
3) with the oracle as each rank's local stepper: the owned columns of the
slabs, stepped with one halo exchange per step, equal the undivided
lattice's run bit for bit (FP64), with walls, moving walls and the force, on
the isotropic, anisotropic, 2N+2 and 3D lattices (halo width H = the largest
x speed: N_x, or 2N_x + 1 with the 2N+2 hierarchy along x). Deep halos
(H = m x that reach, one exchange per m steps, a ragged last block) give the
same bits."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = {
    "d2q25_walls": dict(N=2, nx=24, ny=9, bc=0, tau=0.8, uw=(-0.04, 0.05), g=3e-5, steps=12),
    "d2q49_periodic": dict(N=3, nx=18, ny=7, bc=2, tau=0.7, uw=(0.0, 0.0), g=0.0, steps=9),
    # D1Q3 along x, D1Q9 along y: H = 1
    "d1q3xd1q9_walls": dict(N=4, NX=1, nx=24, ny=11, bc=0, tau=0.9, uw=(-0.03, 0.04), g=2e-5,
                            steps=10),
    # the 2N+2 hierarchy on both axes (D2Q36): odd x speeds up to 5, H = 5
    "d2q36_zv_walls": dict(N=2, zv=3, nx=30, ny=7, bc=0, tau=0.75, uw=(-0.05, 0.03), g=1e-5,
                           steps=8),
    # D3Q27 channel, 4 z-slices: H = 1
    "d3q27_walls": dict(N=1, dims=3, Lz=4, nx=18, ny=5, bc=0, tau=0.8, uw=(-0.04, 0.04), g=2e-5,
                        steps=8),
}


def _oracle(c, nx):
    from oracle import oracle as orc
    dims = c.get("dims", 2)
    return orc.Lattice(dims, c.get("NX", c["N"]), c["N"], nx, c["ny"], c["bc"], c["tau"],
                       c["uw"][0], c["uw"][1], c["g"], zv=c.get("zv", 0),
                       NZ=c["N"] if dims == 3 else 0, Lz=c.get("Lz", 1))


def _halo(c):
    NX = c.get("NX", c["N"])
    return 2 * NX + 1 if c.get("zv", 0) & 1 else NX


class OracleSlab:
    """A rank's slab stepped by the oracle (periodic over the padded width)."""

    def __init__(self, c, X):
        self.o = _oracle(c, X.shape[-1])
        self.X = X

    def step(self, n=1):
        self.X, _ = self.o.run(self.X, n)

    def pack(self, x0, n):
        return torch.from_numpy(np.ascontiguousarray(self.X[..., x0:x0 + n]))

    def unpack(self, x0, n, buf):
        self.X[..., x0:x0 + n] = buf.numpy()


def _initial(c):
    shape = _oracle(c, c["nx"]).shape
    rng = np.random.default_rng(7)
    return rng.uniform(0.5, 1.5, size=shape) / shape[0]


def _rank_main(rank, world, port, name, out, depth=1):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1905_04597_gb300 import slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = CASES[name]
    Ls, H = c["nx"] // world, depth * _halo(c)
    cols = [(rank * Ls + j - H) % c["nx"] for j in range(Ls + 2 * H)]
    st = OracleSlab(c, np.ascontiguousarray(_initial(c)[..., cols]))
    slab.step_slab(st, c["steps"], Ls, H, rank, world, slab.torch_sendrecv(), per=depth)
    np.save(os.path.join(out, f"rank{rank}.npy"), st.X[..., H:H + Ls])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_slabs_equal_the_undivided_lattice(name, world, tmp_path):
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    orc.build()
    c = CASES[name]
    mp.spawn(_rank_main, args=(world, _free_port(), name, str(tmp_path)), nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)], axis=-1)
    want, _ = _oracle(c, c["nx"]).run(_initial(c), c["steps"])
    np.testing.assert_array_equal(got, want)


# (case, world, steps per exchange): H = depth x reach fits the owned columns
DEEP = [("d2q25_walls", 2, 5), ("d1q3xd1q9_walls", 2, 4), ("d2q36_zv_walls", 2, 3),
        ("d3q27_walls", 3, 3)]


@pytest.mark.parametrize("name,world,depth", DEEP)
def test_deep_halos_equal_the_undivided_lattice(name, world, depth, tmp_path):
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    orc.build()
    c = CASES[name]
    assert c["steps"] % depth != 0  # a ragged last block
    assert depth * _halo(c) <= c["nx"] // world
    mp.spawn(_rank_main, args=(world, _free_port(), name, str(tmp_path), depth), nprocs=world,
             join=True)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)], axis=-1)
    want, _ = _oracle(c, c["nx"]).run(_initial(c), c["steps"])
    np.testing.assert_array_equal(got, want)


def test_default_depth():
    from paper_1905_04597_gb300 import slab
    assert slab.default_depth(4096, 4) == 16   # 2 * 16 * 4 = 128 = 4096 / 32
    assert slab.default_depth(512, 4) == 2     # 16 <= 16
    assert slab.default_depth(96, 3) == 1
    for Ls, reach in ((4096, 4), (512, 4), (2048, 9), (100, 1)):
        m = slab.default_depth(Ls, reach)
        assert m == 1 or 2 * m * reach * 32 <= Ls
        assert m == 16 or 2 * (m + 1) * reach * 32 > Ls


def test_single_rank_exchange_wraps_onto_itself():
    """world = 1: the halos are the slab's own opposite columns."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_1905_04597_gb300 import slab
    c = CASES["d2q25_walls"]
    H, nx = _halo(c), c["nx"]
    cols = [(j - H) % nx for j in range(nx + 2 * H)]
    st = OracleSlab(c, np.ascontiguousarray(_initial(c)[..., cols]))
    slab.step_slab(st, c["steps"], nx, H, 0, 1, None)
    want, _ = _oracle(c, nx).run(_initial(c), c["steps"])
    np.testing.assert_array_equal(st.X[..., H:H + nx], want)
