"""GPU channel diagnostics (glbm_channel_diagnostics: profile <u_x>(y), flow
rate, volumetric flow of Sec. 5.4, wall-plane velocities and Couette slip of
Sec. 5.3) against the oracle's diagnostics of the oracle's own run, element
by element: 1e-12 relative in FP64 storage, 1e-5 in FP32 deviations.
"""
import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    yield
    torch.cuda.synchronize()


def theta_y(k, zv_y=False):
    N = k + 1
    return (4 * N + 3) / 3 if zv_y else N / 3


def oracle_diag(o, X, u_lo, u_hi, g, tau, th, walls=True):
    f = o.observe(X)
    p = dg.velocity_profile(f)
    lo, hi = dg.wall_plane_velocities(p)
    nan = float("nan")
    slo, shi = dg.slip_ratios(p, u_lo, u_hi) if (walls and u_hi != u_lo) else (nan, nan)
    return p, {"flow_rate": dg.flow_rate(f),
               "volumetric_flow": dg.volumetric_flow(p, g, tau, th) if g != 0 else nan,
               "u_wall_lo_gas": lo if walls else nan, "u_wall_hi_gas": hi if walls else nan,
               "slip_lo": slo, "slip_hi": shi}


def compare(got_p, got_s, want_p, want_s, tol):
    """Profile to tol of its largest value; each scalar to tol of itself, but
    the flow rate (which cancels in a Couette flow) to tol of sum |<u_x>|, the
    wall-plane velocities to tol of max |<u_x>|, and the slip ratios (a
    difference of nearly equal velocities over the walls' speed difference)
    to tol absolute."""
    pmax = max(np.abs(want_p).max(), 1e-300)
    assert np.abs(got_p - want_p).max() / pmax < tol
    floor = {"flow_rate": np.abs(want_p).sum(), "u_wall_lo_gas": pmax, "u_wall_hi_gas": pmax,
             "slip_lo": 1.0, "slip_hi": 1.0, "volumetric_flow": 0.0}
    for key, w in want_s.items():
        g = got_s[key]
        if np.isnan(w):
            assert np.isnan(g), key
        else:
            assert abs(g - w) <= tol * max(abs(w), floor[key], 1e-300), (key, g, w)


CASES = {
    # name: (lattice config, oracle level along x (0: same as y), zv mask, steps)
    "couette_d2q49": (dict(dims=2, nx=48, ny=24, k=2, kn=0.1, u_wall_lo=-0.05, u_wall_hi=0.05),
                      0, 0, 400),
    # (flows fast enough that u is not a sum cancelling to near FP64 rounding)
    "poiseuille_d2q25": (dict(dims=2, nx=32, ny=20, k=1, kn=0.1, g=1e-4), 0, 0, 500),
    "couette_poiseuille_d2q81": (dict(dims=2, nx=40, ny=16, k=3, kn=0.3, u_wall_lo=0.0,
                                      u_wall_hi=0.04, g=2e-5), 0, 0, 300),
    # (g = 1e-4: the profile, about 1e-3, stands well above the FP64 rounding of
    # the O(1) population sums, about 1e-16, that a 1e-12 relative check sees)
    "channel_d1q3xd1q8_zv": (dict(dims=2, nx=16, ny=24, k=2, x_level=1, zv_axes=glbm.ZV_Y,
                                  kn=0.5, g=1e-4), 1, orc.ZV_Y, 300),
    "periodic_d2q9": (dict(dims=2, nx=20, ny=12, k=0, tau=0.7, bc=glbm.BC_PERIODIC, g=1e-4),
                      0, 0, 50),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_channel_diagnostics_fp64_against_oracle(name):
    cfg, xl, zv, steps = CASES[name]
    lat = glbm.Lattice(dict(cfg, prec=glbm.FP64))
    lat.step(steps)
    gp, gs = lat.channel_diagnostics(0)
    N = cfg["k"] + 1
    tau = lat.tau(0)
    walls = cfg.get("bc", glbm.BC_WALLS) == glbm.BC_WALLS
    o = orc.Lattice(2, xl or N, N, cfg["nx"], cfg["ny"],
                    orc.BC_WALLS if walls else orc.BC_PERIODIC, tau, cfg.get("u_wall_lo", 0.0),
                    cfg.get("u_wall_hi", 0.0), cfg.get("g", 0.0), zv=zv)
    X, bad = o.run(o.equilibrium(np.ones((cfg["ny"], cfg["nx"])),
                                 np.zeros((cfg["ny"], cfg["nx"]))), steps)
    assert bad == 0
    wp, ws = oracle_diag(o, X, cfg.get("u_wall_lo", 0.0), cfg.get("u_wall_hi", 0.0),
                         cfg.get("g", 0.0), tau, theta_y(cfg["k"], zv & orc.ZV_Y), walls)
    compare(gp, gs, wp, ws, 1e-12)
    lat.close()


def test_channel_diagnostics_3d_against_oracle():
    """D3Q27 channel, walls moving, force, averaged over x and z."""
    k, nx, ny, nz, steps, g = 1, 8, 10, 4, 120, 2e-5
    lat = glbm.Lattice(dict(dims=3, nx=nx, ny=ny, nz=nz, k=k, kn=0.2, u_wall_lo=-0.03,
                            u_wall_hi=0.03, g=g))
    lat.step(steps)
    gp, gs = lat.channel_diagnostics(0)
    N, tau = k + 1, lat.tau(0)
    o = orc.Lattice(3, N, N, nx, ny, orc.BC_WALLS, tau, -0.03, 0.03, g, NZ=N, Lz=nz)
    X, bad = o.run(o.equilibrium(np.ones((nz, ny, nx)), np.zeros((nz, ny, nx))), steps)
    assert bad == 0
    wp, ws = oracle_diag(o, X, -0.03, 0.03, g, tau, N / 3)
    compare(gp, gs, wp, ws, 1e-12)
    lat.close()


@pytest.mark.parametrize("kind", ["couette", "poiseuille"])
def test_channel_diagnostics_fp32_against_oracle(kind):
    """FP32 deviations on the Couette workload's lattice (D2Q81), narrow
    channel, 2000 steps: every diagnostic to 1e-5 (scales as in compare)."""
    ny, steps, N = 48, 2000, 4
    extra = (dict(u_wall_lo=-0.05, u_wall_hi=0.05) if kind == "couette" else dict(g=1e-5))
    cfg = dict(dims=2, nx=32, ny=ny, k=N - 1, kn=0.05, prec=glbm.FP32_DEV, **extra)
    lat = glbm.Lattice(cfg)
    lat.step(steps)
    gp, gs = lat.channel_diagnostics(0)
    tau = lat.tau(0)
    ulo, uhi, g = extra.get("u_wall_lo", 0.0), extra.get("u_wall_hi", 0.0), extra.get("g", 0.0)
    o = orc.Lattice(2, N, N, 1, ny, orc.BC_WALLS, tau, ulo, uhi, g)
    X, _ = o.run(o.equilibrium(np.ones((ny, 1)), np.zeros((ny, 1))), steps)
    wp, ws = oracle_diag(o, X, ulo, uhi, g, tau, N / 3)
    compare(gp, gs, wp, ws, 1e-5)
    lat.close()


def test_device_outputs_equal_host_outputs():
    import torch
    cfg = dict(dims=2, nx=40, ny=16, k=3, kn=0.3, u_wall_lo=0.0, u_wall_hi=0.04, g=2e-5)
    lat = glbm.Lattice(cfg)
    lat.step(100)
    hp, hs = lat.channel_diagnostics(0)
    dp = torch.empty(16, dtype=torch.float64, device="cuda")
    ds = torch.empty(len(glbm.CHANNEL_STATS), dtype=torch.float64, device="cuda")
    lat.channel_diagnostics(0, profile=dp, stats=ds)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dp.cpu().numpy(), hp)
    np.testing.assert_array_equal(ds.cpu().numpy(), np.array([hs[k] for k in glbm.CHANNEL_STATS]))
    # repeated calls agree bit for bit (fixed-order sums)
    hp2, hs2 = lat.channel_diagnostics(0)
    np.testing.assert_array_equal(hp2, hp)
    assert hs2 == hs
    lat.close()


def test_diagnostics_reject_1d():
    lat = glbm.Lattice(dict(dims=1, nx=64, k=1, tau=0.8))
    with pytest.raises(glbm.GlbmError):
        lat.channel_diagnostics(0)
    lat.close()
