"""Heterogeneous batches (one persistent launch per step over many instances of
different level, size, Knudsen number, walls and force) against the oracle,
instance by instance, in FP32 deviations."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs
from parity_helpers import oracle_moments, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


MIXED = [
    dict(k=0, nx=40, ny=9, kn=0.05, u_wall_lo=-0.03, u_wall_hi=0.04, g=0.0),
    dict(k=3, nx=64, ny=33, kn=0.2, u_wall_lo=0.0, u_wall_hi=0.0, g=2e-5),
    dict(k=7, nx=37, ny=20, kn=1.0, u_wall_lo=-0.05, u_wall_hi=0.05, g=0.0),
    dict(k=2, nx=96, ny=14, kn=0.02, u_wall_lo=0.01, u_wall_hi=-0.02, g=1e-5),
    dict(k=5, nx=33, ny=40, kn=3.0, u_wall_lo=0.0, u_wall_hi=0.0, g=5e-6),
    dict(k=4, nx=70, ny=12, kn=0.1, u_wall_lo=-0.02, u_wall_hi=0.06, g=0.0),
    dict(k=6, nx=32, ny=15, kn=0.5, u_wall_lo=0.03, u_wall_hi=0.03, g=3e-6),
    dict(k=1, nx=50, ny=25, kn=0.01, u_wall_lo=0.0, u_wall_hi=0.0, g=0.0, bc=glbm.BC_PERIODIC),
]


def test_mixed_batch_matches_oracle_per_instance():
    steps = 30
    cfgs = [dict(dims=2, prec=glbm.FP32_DEV, **c) for c in MIXED]
    lat = glbm.Lattice(cfgs, hetero=True)
    fields = []
    for i, c in enumerate(MIXED):
        rho, ux, uy = inputs.random_macro(300 + i, c["nx"], c["ny"])
        lat.set_equilibrium(i, rho, ux, uy)
        fields.append((rho, ux, uy))
    lat.step(steps)
    lat.sync()
    for i, c in enumerate(MIXED):
        N = c["k"] + 1
        bc = c.get("bc", glbm.BC_WALLS)
        o = orc.Lattice(2, N, N, c["nx"], c["ny"], bc, orc.tau_from_kn(N, c["ny"], c["kn"]),
                        c["u_wall_lo"], c["u_wall_hi"], c["g"])
        X, _ = o.run(o.equilibrium(*fields[i]), steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(lat.moments(i), want, F=F)
        assert max(errs.values()) < 1e-5, (i, c, errs)
    lat.close()


def test_batch_of_one_equals_single_instance_context():
    """The batched launch and the uniform launch run the same tile code with the same
    tile shape and dither seed: one FP32 instance is bitwise equal after 64 steps."""
    c = dict(dims=2, prec=glbm.FP32_DEV, k=3, nx=64, ny=24, kn=0.1, u_wall_lo=-0.05,
             u_wall_hi=0.05, g=1e-5)
    rho, ux, uy = inputs.random_macro(5, 64, 24)
    a = glbm.Lattice(c, hetero=True)
    b = glbm.Lattice(c)
    for lat in (a, b):
        lat.set_equilibrium(0, rho, ux, uy)
        lat.step(64)
    fa, fb = a.get_populations(0), b.get_populations(0)
    np.testing.assert_array_equal(fa, fb)
    a.close()
    b.close()


def test_batched_workload_sample_matches_oracle():
    """The 256-instance batched workload (Ny 32..512, Nx 64, k 1..7, Kn 0.01..10,
    Couette or Poiseuille) after 2000 steps: 12 instances spread over the levels are
    checked against one-column oracle runs (the flows stay x-uniform)."""
    recipe = inputs.batched_instances(seed=0)
    cfgs = [dict(dims=2, prec=glbm.FP32_DEV, **r) for r in recipe]
    lat = glbm.Lattice(cfgs, hetero=True)
    steps = 2000
    lat.step(steps)
    lat.sync()
    picks = []
    for k in range(1, 8):
        idx = [i for i, r in enumerate(recipe) if r["k"] == k]
        picks += sorted(idx, key=lambda i: recipe[i]["ny"])[:1] + sorted(idx, key=lambda i: recipe[i]["kn"])[-1:]
    failures = []
    for i in sorted(set(picks))[:12]:
        r = recipe[i]
        N = r["k"] + 1
        o = orc.Lattice(2, N, N, 1, r["ny"], orc.BC_WALLS, orc.tau_from_kn(N, r["ny"], r["kn"]),
                        r["u_wall_lo"], r["u_wall_hi"], r["g"])
        X = o.equilibrium(np.ones((r["ny"], 1)), np.zeros((r["ny"], 1)), np.zeros((r["ny"], 1)))
        X, _ = o.run(X, steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(lat.moments(i), want, F=F)
        print(i, r["k"], r["ny"], round(r["kn"], 3), {n: f"{e:.1e}" for n, e in errs.items()})
        if max(errs.values()) >= 1e-5:
            failures.append((i, r, errs))
    lat.close()
    assert not failures, failures


def test_every_instance_of_the_256_batch_equals_its_own_context():
    """Every instance of the 256-instance batch, from its own random state, after 6
    steps against the same instance stepped alone in a uniform context: a tile or
    work-list boundary that mixed instances would show as an O(1) error somewhere.
    The two runs differ only in the dither seed (the instance index enters it), so
    they agree to FP32 rounding, not bit for bit (a batch of one is bitwise equal,
    above)."""
    recipe = inputs.batched_instances(seed=0)
    cfgs = [dict(dims=2, prec=glbm.FP32_DEV, **r) for r in recipe]
    lat = glbm.Lattice(cfgs, hetero=True)
    fields = []
    for i, r in enumerate(recipe):
        f = inputs.random_macro(1000 + i, r["nx"], r["ny"])
        lat.set_equilibrium(i, *f)
        fields.append(f)
    steps = 6
    lat.step(steps)
    lat.sync()
    worst = (0.0, None)
    for i, r in enumerate(recipe):
        one = glbm.Lattice(cfgs[i])
        one.set_equilibrium(0, *fields[i])
        one.step(steps)
        m = one.moments(0)
        want = np.stack([m[n] for n in glbm.FIELDS_2D])
        F = one.get_populations(0)  # term scales of the metric (post-collision state)
        one.close()
        errs = rel_errors(lat.moments(i), want, F=F)
        n = max(errs, key=errs.get)
        if errs[n] > worst[0]:
            worst = (errs[n], (i, n))
    lat.close()
    assert worst[0] < 1e-5, worst


def test_batched_rejects_fp64_and_1d():
    with pytest.raises(glbm.GlbmError):
        glbm.Lattice([dict(dims=2, nx=32, ny=8, k=1, tau=1.0, prec=glbm.FP64)], hetero=True)
    with pytest.raises(glbm.GlbmError):
        glbm.Lattice([dict(dims=1, nx=32, k=1, tau=1.0, prec=glbm.FP32_DEV)], hetero=True)
