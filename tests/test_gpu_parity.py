"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 storage 1e-12 relative, FP32-deviation storage 1e-5 relative
in every moment, after the stated step counts. A field's error is
max |got - want| divided by max(max |want|, 1e-3 * S), where S is the largest
per-node sum of the absolute terms of that moment (for the heat flux
(1/2) sum |xi-u|^3 f): a moment that cancels to below a thousandth of its own
terms (the heat flux of a slow flow) cannot be reproduced to 1e-12 of its value
by FP64 sums taken in another order, so it is judged against that floor. The two
velocity and the two heat-flux components are normalised jointly. One-step
population checks compare every population (FP64 1e-13, FP32 1e-6 of the
largest population).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs
from parity_helpers import oracle_moments, rel_errors  # noqa: F401

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
    yield
    torch.cuda.synchronize()


def oracle_lattice(dims, k, nx, ny, bc, tau, uw_lo=0.0, uw_hi=0.0, g=0.0):
    N = k + 1
    return orc.Lattice(dims, N, N, nx, ny, bc, tau, uw_lo, uw_hi, g)


# --------------------------------------------------------------------------
# one step, every population, every level, both precisions and boundaries
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("bc", [glbm.BC_WALLS, glbm.BC_PERIODIC])
@pytest.mark.parametrize("k", range(0, 8))
def test_one_step_all_populations(k, bc, prec):
    N = k + 1
    nx, ny = 37, max(2 * N + 1, 9)      # ragged: two 32-wide tiles, partial row tiles
    tau, uw_lo, uw_hi, g = 0.83, -0.04, 0.07, 3e-4
    f0 = inputs.random_populations(20 + k, (2 * N + 1) ** 2, ny, nx)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=tau, bc=bc, prec=prec,
                            u_wall_lo=uw_lo, u_wall_hi=uw_hi, g=g))
    lat.set_populations(0, f0)
    lat.step(1)
    lat.sync()
    got = lat.get_populations(0)
    o = oracle_lattice(2, k, nx, ny, bc, tau, uw_lo, uw_hi, g)
    want, _ = o.run(f0, 1)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < POP_TOL[prec], err
    lat.close()


@pytest.mark.parametrize("nx", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 3, 7])
def test_one_step_narrow_periodic_x(k, nx):
    """Fewer columns than the largest shift: the periodic wrap goes round repeatedly."""
    N = k + 1
    ny = N + 1
    f0 = inputs.random_populations(40 + k, (2 * N + 1) ** 2, ny, nx)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.7, prec=glbm.FP64,
                            u_wall_lo=0.02, u_wall_hi=-0.03, g=1e-4))
    lat.set_populations(0, f0)
    lat.step(1)
    got = lat.get_populations(0)
    o = oracle_lattice(2, k, nx, ny, orc.BC_WALLS, 0.7, 0.02, -0.03, 1e-4)
    want, _ = o.run(f0, 1)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-13


# --------------------------------------------------------------------------
# moments after many steps
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
@pytest.mark.parametrize("k", [0, 1, 3, 4, 7])
def test_moments_after_steps(k, prec):
    N = k + 1
    nx, ny, steps = 70, 3 * N + 5, 40
    kn, uw, g = 0.05, 0.05, 2e-5
    rho, ux, uy = inputs.random_macro(60 + k, nx, ny)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, kn=kn, prec=prec, u_wall_lo=-uw,
                            u_wall_hi=uw, g=g))
    lat.set_equilibrium(0, rho, ux, uy)
    lat.step(steps)
    lat.sync()
    got = lat.moments(0)
    tau = orc.tau_from_kn(N, ny, kn)
    assert lat.tau(0) == pytest.approx(tau, rel=1e-15)
    o = oracle_lattice(2, k, nx, ny, orc.BC_WALLS, tau, -uw, uw, g)
    X, _ = o.run(o.equilibrium(rho, ux, uy), steps)
    want, F = oracle_moments(o, X)
    errs = rel_errors(got, want, F=F)
    assert max(errs.values()) < TOL[prec], errs
    lat.close()


def test_moments_at_time_zero_are_the_initial_fields():
    k, nx, ny = 2, 33, 12
    rho, ux, uy = inputs.random_macro(5, nx, ny)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.9, bc=glbm.BC_PERIODIC))
    lat.set_equilibrium(0, rho, ux, uy)
    m = lat.moments(0)
    o = oracle_lattice(2, k, nx, ny, orc.BC_PERIODIC, 0.9)
    want, F = oracle_moments(o, o.equilibrium(rho, ux, uy))
    errs = rel_errors(m, want, F=F)
    assert max(errs.values()) < 1e-13, errs


# --------------------------------------------------------------------------
# the workloads of the paper's test problems (Sec. 5), at their sizes
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_sod_shock_tube_full_config(prec):
    """1D, k = 1 (D1Q5), 1000 nodes, density 1 | 0.125, Kn = 0.01, 500 steps, bounce-back."""
    cfg = inputs.SOD
    N = cfg["k"] + 1
    L = cfg["nx"]
    rho = inputs.sod_density(L, cfg["rho_left"], cfg["rho_right"])
    lat = glbm.Lattice(dict(dims=1, nx=L, k=cfg["k"], kn=cfg["kn"], bc=glbm.BC_BOUNCEBACK,
                            prec=prec))
    lat.set_equilibrium(0, rho, np.zeros(L))
    l0 = lat.kernel_launches
    lat.step(cfg["steps"])
    lat.sync()
    launches = lat.kernel_launches - l0
    got = lat.moments(0)
    tau = orc.tau_from_kn(N, L, cfg["kn"])
    o = orc.Lattice(1, N, 0, L, 1, orc.BC_BOUNCEBACK, tau)
    X, bad = o.run(o.equilibrium(rho, np.zeros(L)), cfg["steps"])
    assert bad == 0
    want, F = oracle_moments(o, X)
    errs = rel_errors(got, want, dims=1, F=F)
    assert max(errs.values()) < TOL[prec], errs
    assert launches == 1  # the whole run is one resident launch
    lat.close()


_couette_ref = {}


def _couette_oracle(kn, steps):
    """x-uniform Couette from rest: the oracle runs one column (Nx = 1)."""
    key = (kn, steps)
    if key not in _couette_ref:
        c = inputs.COUETTE
        N = c["k"] + 1
        ny = c["ny"]
        o = oracle_lattice(2, c["k"], 1, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, kn),
                           c["u_wall_lo"], c["u_wall_hi"])
        X = o.equilibrium(np.ones((ny, 1)), np.zeros((ny, 1)), np.zeros((ny, 1)))
        X, bad = o.run(X, steps)
        assert bad == 0
        _couette_ref[key] = oracle_moments(o, X)
    return _couette_ref[key]


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_couette_full_config_20000_steps(prec):
    """D2Q81 (k = 3), 512 x 256, walls -+0.05, Kn in {0.01, 0.1, 1}, 20000 steps; the three
    Knudsen numbers are three instances of one batched launch."""
    c = inputs.COUETTE
    cfgs = [dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], kn=kn, prec=prec,
                 u_wall_lo=c["u_wall_lo"], u_wall_hi=c["u_wall_hi"]) for kn in c["kn"]]
    lat = glbm.Lattice(cfgs)
    lat.step(c["steps"])
    lat.sync()
    for i, kn in enumerate(c["kn"]):
        got = lat.moments(i)
        if prec == glbm.FP64:
            # x-uniform and no dither: every column bitwise identical
            for name, fld in got.items():
                assert (fld == fld[:, :1]).all(), name
        # every column against the oracle's single column
        want, F = _couette_oracle(kn, c["steps"])
        errs = rel_errors(got, want, F=F)
        for name, e in errs.items():
            assert e < TOL[prec], (kn, name, errs)
    lat.close()


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_couette_full_size_random_state(prec):
    """512 x 256 D2Q81 from a random non-uniform state: every node after 3 steps."""
    c = inputs.COUETTE
    N = c["k"] + 1
    nx, ny, steps, kn = c["nx"], c["ny"], 3, 0.1
    rho, ux, uy = inputs.random_macro(77, nx, ny)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=c["k"], kn=kn, prec=prec,
                            u_wall_lo=c["u_wall_lo"], u_wall_hi=c["u_wall_hi"]))
    lat.set_equilibrium(0, rho, ux, uy)
    lat.step(steps)
    got = lat.moments(0)
    o = oracle_lattice(2, c["k"], nx, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, kn),
                       c["u_wall_lo"], c["u_wall_hi"])
    X, _ = o.run(o.equilibrium(rho, ux, uy), steps)
    want, F = oracle_moments(o, X)
    errs = rel_errors(got, want, F=F)
    assert max(errs.values()) < TOL[prec], errs
    lat.close()


def test_poiseuille_full_config_fp32():
    """D2Q289 (k = 7), 1024 x 128, g = 1e-6, 8 Knudsen numbers 0.01..10 as one batch,
    FP32 deviations against the FP64 oracle after 2000 steps (x-uniform: one column)."""
    c = inputs.POISEUILLE
    N = c["k"] + 1
    ny, steps = c["ny"], c["steps"]
    cfgs = [dict(dims=2, nx=c["nx"], ny=ny, k=c["k"], kn=kn, prec=glbm.FP32_DEV, g=c["g"])
            for kn in c["kn"]]
    lat = glbm.Lattice(cfgs)
    lat.step(steps)
    lat.sync()
    for i, kn in enumerate(c["kn"]):
        got = lat.moments(i)
        o = oracle_lattice(2, c["k"], 1, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, kn),
                           0.0, 0.0, c["g"])
        X = o.equilibrium(np.ones((ny, 1)), np.zeros((ny, 1)), np.zeros((ny, 1)))
        X, _ = o.run(X, steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(got, want, F=F)  # every column against the oracle column
        assert max(errs.values()) < TOL[glbm.FP32_DEV], (kn, errs)
    lat.close()


# --------------------------------------------------------------------------
# invariants and runtime behaviour
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec,tol", [(glbm.FP64, 1e-13), (glbm.FP32_DEV, 1e-6)])
def test_mass_conserved_with_walls(prec, tol):
    """Streaming with diffuse walls and the collision both conserve mass: drift over
    1000 steps stays at rounding level (FP64) or FP32-storage level."""
    k, nx, ny = 3, 64, 40
    rho, ux, uy = inputs.random_macro(9, nx, ny)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.6, prec=prec, u_wall_lo=-0.05,
                            u_wall_hi=0.05))
    lat.set_equilibrium(0, rho, ux, uy)
    m0, _, _ = lat.conservation(0)
    lat.step(1000)
    m1, _, _ = lat.conservation(0)
    # the initial state's mass is rounded once into the storage precision
    assert m0 == pytest.approx(rho.sum(), rel=1e-13 if prec == glbm.FP64 else 1e-9)
    assert abs(m1 - m0) / m0 < tol
    lat.close()


def test_periodic_momentum_conserved_and_force_adds_momentum():
    k, nx, ny, g = 2, 40, 24, 1e-5
    rho, ux, uy = inputs.random_macro(12, nx, ny)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.8, bc=glbm.BC_PERIODIC, g=g))
    lat.set_equilibrium(0, rho, ux, uy)
    m0, jx0, jy0 = lat.conservation(0)
    lat.step(50)
    m1, jx1, jy1 = lat.conservation(0)
    assert m1 == pytest.approx(m0, rel=1e-14)
    assert jx1 - jx0 == pytest.approx(50 * g * nx * ny, rel=1e-9)
    assert jy1 == pytest.approx(jy0, abs=1e-13)
    lat.close()


def test_deterministic_and_checkpoint_resume(tmp_path):
    k, nx, ny = 4, 48, 20
    rho, ux, uy = inputs.random_macro(3, nx, ny)
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, tau=0.7, prec=glbm.FP32_DEV, u_wall_lo=-0.03,
               u_wall_hi=0.03, g=1e-5)
    a = glbm.Lattice(cfg)
    a.set_equilibrium(0, rho, ux, uy)
    a.step(130)
    path = tmp_path / "ck.bin"
    a.save(path)
    a.step(70)
    fa = a.get_populations(0)
    b = glbm.Lattice(cfg)
    b.set_equilibrium(0, rho, ux, uy)
    b.step(200)
    np.testing.assert_array_equal(b.get_populations(0), fa)
    c = glbm.Lattice(cfg)
    c.load(path)
    assert c.time == 130
    c.step(70)
    np.testing.assert_array_equal(c.get_populations(0), fa)
    # a corrupted checkpoint is refused
    raw = bytearray(path.read_bytes())
    raw[100] ^= 0xFF
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(glbm.GlbmError):
        c.load(bad)
    for x in (a, b, c):
        x.close()


def test_graph_chunks_match_single_launches():
    """Replay of the captured 64-step graph equals 64 individual launches."""
    k, nx, ny = 1, 40, 10
    rho, ux, uy = inputs.random_macro(4, nx, ny)
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, tau=0.9, u_wall_lo=0.01, u_wall_hi=-0.02)
    a = glbm.Lattice(cfg)
    a.set_equilibrium(0, rho, ux, uy)
    a.step(1)          # odd offset: the graph for the other starting buffer
    a.step(130)        # two graph replays + 2 single launches
    b = glbm.Lattice(cfg)
    b.set_equilibrium(0, rho, ux, uy)
    for _ in range(131):
        b.step(1)
    np.testing.assert_array_equal(a.get_populations(0), b.get_populations(0))
    a.close()
    b.close()


def test_column_invariance_nx1_vs_nx64():
    k, ny = 3, 16
    cfg = dict(dims=2, ny=ny, k=k, tau=0.75, u_wall_lo=-0.05, u_wall_hi=0.05, g=1e-5)
    a = glbm.Lattice(dict(cfg, nx=1))
    b = glbm.Lattice(dict(cfg, nx=64))
    a.step(300)
    b.step(300)
    ma, mb = a.moments(0), b.moments(0)
    for n in ma:
        assert (mb[n] == ma[n]).all(), n
    a.close()
    b.close()


def test_instability_flag_is_reported():
    """A state outside the positivity domain (|u| > sqrt(2/3) N, Sec. 3): the
    first step flags it, glbm_step reports one completed step, and the flag
    stays visible to glbm_sync."""
    k, nx, ny = 0, 32, 8
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.8, bc=glbm.BC_PERIODIC))
    ux = np.full((ny, nx), 1.2 * np.sqrt(2 / 3))
    lat.set_equilibrium(0, np.ones((ny, nx)), ux, np.zeros((ny, nx)))
    with pytest.raises(glbm.UnstableError, match="1 of 2 steps completed"):
        lat.step(2)
    assert lat.time == 1
    with pytest.raises(glbm.UnstableError):
        lat.sync()
    lat.close()


def test_device_pointers_and_torch_allocator():
    import torch
    k, nx, ny = 2, 32, 10
    rho, ux, uy = inputs.random_macro(21, nx, ny)
    glbm.install_torch_allocator()
    try:
        lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.9))
        t = [torch.from_numpy(a).cuda() for a in (rho, ux, uy)]
        lat.set_equilibrium(0, *t)
        lat.step(10)
        out = torch.empty((7, ny, nx), dtype=torch.float64, device="cuda")
        lat.moments(0, out=out)
        host = lat.moments(0)
        np.testing.assert_array_equal(out[0].cpu().numpy(), host["rho"])
        lat.close()
    finally:
        glbm.uninstall_allocator()


# --------------------------------------------------------------------------
# high levels: narrow and ragged widths, several instances in one launch
# --------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [glbm.BC_WALLS, glbm.BC_PERIODIC])
@pytest.mark.parametrize("nx", [64, 100, 36, 4])
@pytest.mark.parametrize("k", [3, 4, 5, 6, 7])
def test_high_level_one_step(k, nx, bc):
    """Pulls that wrap the periodic x edge once (nx = 36, 100) or several times
    (nx = 4 < the largest shift), walls and periodic rows, one step."""
    N = k + 1
    ny = 2 * N + 3
    tau, uw_lo, uw_hi, g = 0.77, 0.03, -0.05, 2e-4
    f0 = inputs.random_populations(500 + k + nx, (2 * N + 1) ** 2, ny, nx)
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=tau, bc=bc, prec=glbm.FP32_DEV,
                            u_wall_lo=uw_lo, u_wall_hi=uw_hi, g=g))
    lat.set_populations(0, f0)
    lat.step(1)
    lat.sync()
    got = lat.get_populations(0)
    o = oracle_lattice(2, k, nx, ny, bc, tau, uw_lo, uw_hi, g)
    want, _ = o.run(f0, 1)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < POP_TOL[glbm.FP32_DEV], err
    lat.close()


@pytest.mark.parametrize("k", [3, 7])
def test_high_level_many_steps_batch(k):
    """Three instances in one launch, 50 steps, moments against the oracle."""
    N = k + 1
    nx, ny, steps = 68, 3 * N + 4, 50
    cfgs, fields = [], []
    for i, kn in enumerate((0.05, 0.3, 2.0)):
        cfgs.append(dict(dims=2, nx=nx, ny=ny, k=k, kn=kn, prec=glbm.FP32_DEV,
                         u_wall_lo=-0.04 * i, u_wall_hi=0.03, g=1e-5 * i))
        fields.append(inputs.random_macro(600 + 10 * k + i, nx, ny))
    lat = glbm.Lattice(cfgs)
    for i, f in enumerate(fields):
        lat.set_equilibrium(i, *f)
    lat.step(steps)
    lat.sync()
    for i, c in enumerate(cfgs):
        o = oracle_lattice(2, k, nx, ny, orc.BC_WALLS, orc.tau_from_kn(N, ny, c["kn"]),
                           c["u_wall_lo"], c["u_wall_hi"], c["g"])
        X, _ = o.run(o.equilibrium(*fields[i]), steps)
        want, F = oracle_moments(o, X)
        errs = rel_errors(lat.moments(i), want, F=F)
        assert max(errs.values()) < TOL[glbm.FP32_DEV], (i, errs)
    lat.close()
