"""x-slab decomposition of one lattice over several ranks (one GPU each).

The lattice is periodic along x, so it can be cut into slabs of consecutive
columns. Rank r of W owns the global columns [r Ls, (r+1) Ls) and stores them
with H halo columns on each side (local width Ls + 2H): local column H + i is
global column r Ls + i. A step of the fused kernel pulls each population from
at most `reach` columns away (the largest x speed: N_x, or 2 N_x + 1 on a 2N+2
x axis), so a column whose neighbourhood within `reach` held exact values
before a step holds an exact value after it. With H = m reach, m steps after
an exchange the exact columns have shrunk from [0, Ls + 2H) to exactly the
owned ones [H, Ls + H): the halos are refilled once every m steps (deep halos:
m times fewer, m times larger messages, at 2H / Ls redundant work), the left
halo [0, H) from the left neighbour's last H owned columns and the right halo
[Ls + H, Ls + 2H) from the right neighbour's first H owned columns. Halo nodes
are stepped too (their pulls wrap around the local array) but are overwritten
by the next exchange; the owned nodes see exactly the populations the
undivided lattice would give them, so in FP64 the slabs reproduce the
undivided run bit for bit. The walls are along y and stay local; the wall
density is per column.

The exchange works on any local stepper with step(), pack(x0, n) and
unpack(x0, n, buf) and any pair of send/recv callables, so the same code runs
on the GPU library (SlabLattice, NCCL or a single rank's own columns) and,
in the tests, on CPU ranks over gloo.
"""
from __future__ import annotations


def exchange_halos(stepper, Ls: int, H: int, rank: int, world: int, sendrecv):
    """Refill both halos of this rank's slab from its neighbours' owned columns.

    sendrecv(send_buf, dst, src) sends send_buf to rank dst and returns the
    buffer received from rank src (with world == 1 the neighbour is the rank
    itself: the owned columns are copied across locally)."""
    left, right = (rank - 1) % world, (rank + 1) % world
    first = stepper.pack(H, H)         # owned columns [H, 2H): the left neighbour's right halo
    last = stepper.pack(Ls, H)         # owned columns [Ls, Ls + H): the right neighbour's left halo
    if world == 1:
        stepper.unpack(0, H, last)
        stepper.unpack(Ls + H, H, first)
        return
    from_right = sendrecv(first, left, right)   # our right halo comes from the right neighbour
    from_left = sendrecv(last, right, left)    # our left halo from the left neighbour
    stepper.unpack(Ls + H, H, from_right)
    stepper.unpack(0, H, from_left)


def step_slab(stepper, steps: int, Ls: int, H: int, rank: int, world: int, sendrecv,
              per: int = 1):
    """Advance a slab by `steps` steps, exchanging the halos (H >= per x the
    reach of a step) after every `per` steps and after the last."""
    left = steps
    while left > 0:
        n = min(per, left)
        stepper.step(n)
        exchange_halos(stepper, Ls, H, rank, world, sendrecv)
        left -= n


def default_depth(Ls: int, reach: int) -> int:
    """Steps per exchange: the largest m <= 16 whose redundant halo work
    2 m reach / Ls stays within 1/32 of the owned columns' (at least 1)."""
    m = 16
    while m > 1 and 2 * m * reach * 32 > Ls:
        m -= 1
    return m


def torch_sendrecv(group=None):
    """A sendrecv over torch.distributed (NCCL for GPU tensors, gloo for CPU):
    non-blocking send and receive of equally shaped buffers, in an order that
    cannot deadlock."""
    import torch
    import torch.distributed as dist

    def sendrecv(buf, dst, src):
        out = torch.empty_like(buf)
        reqs = [dist.isend(buf.contiguous(), dst, group=group), dist.irecv(out, src, group=group)]
        for r in reqs:
            r.wait()
        return out

    return sendrecv


class SlabLattice:
    """The slab of one rank on the GPU library: a glbm.Lattice of Ls + 2H
    columns, H = depth x reach, whose halos are exchanged after every `depth`
    steps (default_depth unless given). cfg is the undivided lattice's
    configuration with nx = W Ls."""

    def __init__(self, cfg: dict, rank: int = 0, world: int = 1, sendrecv=None,
                 depth: int | None = None):
        import torch
        from . import glbm
        nx = cfg["nx"]
        if nx % world:
            raise ValueError("nx must divide among the ranks")
        if cfg.get("dims", 2) != 2:
            raise ValueError("x slabs are implemented for 2D lattices")
        self.Ls = nx // world
        NX = cfg.get("x_level") or (cfg["k"] + 1)
        # the largest x speed: N_x, or 2 N_x + 1 on a 2N+2 x axis
        self.reach = 2 * NX + 1 if cfg.get("zv_axes", 0) & 1 else NX
        self.depth = default_depth(self.Ls, self.reach) if depth is None else int(depth)
        if self.depth < 1:
            raise ValueError("depth must be at least 1")
        self.H = self.depth * self.reach
        if self.Ls < self.H:
            raise ValueError("each slab needs at least H = depth x reach owned columns")
        self.rank, self.world = rank, world
        self.lat = glbm.Lattice(dict(cfg, nx=self.Ls + 2 * self.H))
        self.sendrecv = sendrecv or torch_sendrecv()
        self._dtype = torch.float32 if self.lat.elem_size == 4 else torch.float64
        self._shape = (self.lat.nq(), cfg["ny"])

    def pack(self, x0, n):
        import torch
        buf = torch.empty(self._shape + (n,), dtype=self._dtype, device="cuda")
        return self.lat.pack_columns(0, x0, n, buf)

    def unpack(self, x0, n, buf):
        self.lat.unpack_columns(0, x0, n, buf)

    def step(self, n=1):
        self.lat.step(n)

    def exchange(self):
        exchange_halos(self, self.Ls, self.H, self.rank, self.world, self.sendrecv)

    def advance(self, steps):
        """steps steps of the undivided lattice (one halo exchange per `depth`
        steps and one after the last)."""
        step_slab(self, steps, self.Ls, self.H, self.rank, self.world, self.sendrecv, self.depth)

    def local_columns(self):
        """Global column of every local column (halos wrap around)."""
        nx = self.Ls * self.world
        return [(self.rank * self.Ls + j - self.H) % nx for j in range(self.Ls + 2 * self.H)]

    def set_equilibrium_global(self, rho, ux, uy):
        """Initial equilibrium from the undivided lattice's fields [ny][nx]."""
        import numpy as np
        cols = self.local_columns()
        self.lat.set_equilibrium(0, *(np.ascontiguousarray(a[:, cols]) for a in (rho, ux, uy)))

    def set_populations_global(self, f):
        """Initial populations from the undivided lattice's X [q][ny][nx]."""
        import numpy as np
        self.lat.set_populations(0, np.ascontiguousarray(f[..., self.local_columns()]))

    def owned_populations(self):
        """X_t of the owned columns, [q][y][Ls] (FP64 logical values)."""
        f = self.lat.get_populations(0)
        return f[..., self.H:self.H + self.Ls]
