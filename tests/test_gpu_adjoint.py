"""Gradient of the flow rate by the hand-written adjoint (glbm_adjoint_flowrate):
by tau, g and both wall speeds, against the oracle's forward-mode dual numbers
and against central finite differences of GPU forward runs."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1905_04597_gb300 import glbm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _compare(cfg, steps, ckpt, fields, rtol):
    N = cfg["k"] + 1
    lat = glbm.Lattice(cfg)
    lat.set_equilibrium(0, *fields)
    J, dtau, dg, dlo, dhi = lat.adjoint_flowrate(steps, ckpt, walls=True)
    assert lat.time == steps
    lat.close()
    o = orc.Lattice(2, N, N, cfg["nx"], cfg["ny"], cfg.get("bc", orc.BC_WALLS), cfg["tau"],
                    cfg.get("u_wall_lo", 0.0), cfg.get("u_wall_hi", 0.0), cfg.get("g", 0.0))
    oJ, otau, og, olo, ohi = o.flowrate_grad(o.equilibrium(*fields), steps, walls=True)
    assert J[0] == pytest.approx(oJ, rel=rtol, abs=1e-300)
    assert dtau[0] == pytest.approx(otau, rel=rtol)
    assert dg[0] == pytest.approx(og, rel=rtol)
    if cfg.get("bc", orc.BC_WALLS) == orc.BC_WALLS:
        assert dlo[0] == pytest.approx(olo, rel=rtol)
        assert dhi[0] == pytest.approx(ohi, rel=rtol)
    else:
        assert dlo[0] == 0.0 and dhi[0] == 0.0 and olo == 0.0 and ohi == 0.0
    return J[0], dtau[0], dg[0]


@pytest.mark.parametrize("k", [0, 2, 4])
def test_adjoint_fp64_matches_dual_numbers(k):
    """Random initial fields, force and moving walls; 61 steps with checkpoints every
    16 (a short last segment)."""
    nx, ny = 20, 3 * (k + 1) + 5
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, tau=0.8, prec=glbm.FP64, u_wall_lo=-0.02,
               u_wall_hi=0.04, g=3e-5)
    _compare(cfg, 61, 16, inputs.random_macro(70 + k, nx, ny), 1e-9)


def test_adjoint_periodic_fp64():
    nx, ny, k = 16, 10, 1
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, tau=1.3, prec=glbm.FP64, bc=glbm.BC_PERIODIC, g=1e-5)
    _compare(cfg, 40, 7, inputs.random_macro(81, nx, ny), 1e-9)


def test_adjoint_fp32_forward_matches_dual_numbers():
    nx, ny, k = 24, 16, 3
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, tau=0.9, prec=glbm.FP32_DEV, u_wall_lo=-0.03,
               u_wall_hi=0.03, g=2e-5)
    _compare(cfg, 80, 20, inputs.random_macro(90, nx, ny), 1e-4)


def test_adjoint_config_poiseuille_d2q121():
    """The adjoint workload: D2Q121 (k = 4), 256 x 128, Kn = 0.1, g = 1e-6, 4000 FP32
    steps with checkpoints every 100. The flow stays x-uniform, so the oracle's
    dual-number gradient runs on one column. Also checked against central finite
    differences (h = 1e-4 relative) of FP64 GPU forward runs."""
    c = inputs.ADJOINT
    N = c["k"] + 1
    tau = orc.tau_from_kn(N, c["ny"], c["kn"])
    cfg = dict(dims=2, nx=c["nx"], ny=c["ny"], k=c["k"], tau=tau, prec=glbm.FP32_DEV, g=c["g"])
    lat = glbm.Lattice(cfg)
    J, dtau, dg = lat.adjoint_flowrate(c["steps"], c["ckpt_every"])
    lat.close()
    o = orc.Lattice(2, N, N, 1, c["ny"], orc.BC_WALLS, tau, 0.0, 0.0, c["g"])
    X0 = o.equilibrium(np.ones((c["ny"], 1)), np.zeros((c["ny"], 1)), np.zeros((c["ny"], 1)))
    oJ, otau, og = o.flowrate_grad(X0, c["steps"])
    assert J[0] == pytest.approx(oJ, rel=1e-4)
    assert dtau[0] == pytest.approx(otau, rel=1e-4)
    assert dg[0] == pytest.approx(og, rel=1e-4)

    def J64(t, g):
        with glbm.Lattice(dict(cfg, prec=glbm.FP64, tau=t, g=g)) as L:
            L.step(c["steps"])
            return L.conservation(0)[1] / c["nx"]
    h = 1e-4
    fd_tau = (J64(tau * (1 + h), c["g"]) - J64(tau * (1 - h), c["g"])) / (2 * h * tau)
    fd_g = (J64(tau, c["g"] * (1 + h)) - J64(tau, c["g"] * (1 - h))) / (2 * h * c["g"])
    assert dtau[0] == pytest.approx(fd_tau, rel=1e-4)
    assert dg[0] == pytest.approx(fd_g, rel=1e-4)


@pytest.mark.parametrize("prec,rtol", [(glbm.FP64, 1e-9), (glbm.FP32_DEV, 1e-4)])
def test_adjoint_wall_speeds_couette(prec, rtol):
    """Couette channel D2Q81 (k = 3), walls at -0.03 and +0.05, Kn 0.1, from a
    sheared random state, 200 steps with checkpoints every 64: every derivative
    against the oracle's dual numbers, and the wall speeds' against central
    differences of FP64 GPU forward runs."""
    nx, ny, k = 24, 20, 3
    N = k + 1
    tau = orc.tau_from_kn(N, ny, 0.1)
    cfg = dict(dims=2, nx=nx, ny=ny, k=k, tau=tau, prec=prec, u_wall_lo=-0.03, u_wall_hi=0.05)
    fields = inputs.random_macro(95, nx, ny)
    steps = 200
    _compare(cfg, steps, 64, fields, rtol)
    if prec != glbm.FP64:
        return
    with glbm.Lattice(cfg) as lat:
        lat.set_equilibrium(0, *fields)
        _, _, _, dlo, dhi = lat.adjoint_flowrate(steps, 64, walls=True)

    def J64(ulo, uhi):
        with glbm.Lattice(dict(cfg, u_wall_lo=ulo, u_wall_hi=uhi)) as L:
            L.set_equilibrium(0, *fields)
            L.step(steps)
            return L.conservation(0)[1] / nx
    h = 1e-5
    fd_lo = (J64(-0.03 + h, 0.05) - J64(-0.03 - h, 0.05)) / (2 * h)
    fd_hi = (J64(-0.03, 0.05 + h) - J64(-0.03, 0.05 - h)) / (2 * h)
    assert dlo[0] == pytest.approx(fd_lo, rel=1e-6)
    assert dhi[0] == pytest.approx(fd_hi, rel=1e-6)


def test_autograd_function_wall_speeds():
    import torch
    nx, ny, k = 16, 12, 1
    config = dict(dims=2, nx=nx, ny=ny, k=k, prec=glbm.FP64)
    tau = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(0.0, dtype=torch.float64)
    ulo = torch.tensor(-0.02, dtype=torch.float64, requires_grad=True)
    uhi = torch.tensor(0.04, dtype=torch.float64, requires_grad=True)
    J = glbm.flow_rate(tau, g, config, steps=60, ckpt_every=20, u_wall_lo=ulo, u_wall_hi=uhi)
    J.backward()
    N = k + 1
    o = orc.Lattice(2, N, N, nx, ny, orc.BC_WALLS, 0.9, -0.02, 0.04, 0.0)
    X0 = o.equilibrium(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    oJ, otau, _, olo, ohi = o.flowrate_grad(X0, 60, walls=True)
    assert J.item() == pytest.approx(oJ, rel=1e-10)
    assert tau.grad.item() == pytest.approx(otau, rel=1e-9)
    assert ulo.grad.item() == pytest.approx(olo, rel=1e-9)
    assert uhi.grad.item() == pytest.approx(ohi, rel=1e-9)


def test_autograd_function():
    import torch
    nx, ny, k = 16, 12, 1
    config = dict(dims=2, nx=nx, ny=ny, k=k, prec=glbm.FP64)
    tau = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(2e-5, dtype=torch.float64, requires_grad=True)
    J = glbm.flow_rate(tau, g, config, steps=50, ckpt_every=10)
    (3.0 * J).backward()
    N = k + 1
    o = orc.Lattice(2, N, N, nx, ny, orc.BC_WALLS, 0.9, 0.0, 0.0, 2e-5)
    X0 = o.equilibrium(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    oJ, otau, og = o.flowrate_grad(X0, 50)
    assert J.item() == pytest.approx(oJ, rel=1e-10)
    assert tau.grad.item() == pytest.approx(3 * otau, rel=1e-9)
    assert g.grad.item() == pytest.approx(3 * og, rel=1e-9)


def test_autograd_function_without_gradients_runs_forward_only():
    """With no input requiring a gradient the Function runs the forward steps
    only (no adjoint sweep) and returns the same flow rate, on the device of
    tau."""
    import torch
    nx, ny, k = 16, 12, 1
    config = dict(dims=2, nx=nx, ny=ny, k=k, prec=glbm.FP64)
    tau = torch.tensor(0.9, dtype=torch.float64, device="cuda")
    g = torch.tensor(2e-5, dtype=torch.float64, device="cuda")
    J = glbm.flow_rate(tau, g, config, steps=50, ckpt_every=10)
    assert J.device == tau.device and not J.requires_grad
    N = k + 1
    o = orc.Lattice(2, N, N, nx, ny, orc.BC_WALLS, 0.9, 0.0, 0.0, 2e-5)
    X0 = o.equilibrium(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    oJ, _, _ = o.flowrate_grad(X0, 50)
    assert J.item() == pytest.approx(oJ, rel=1e-10)
    with torch.no_grad():
        tau2 = tau.clone().requires_grad_(True)
        J2 = glbm.flow_rate(tau2, g, config, steps=50, ckpt_every=10)
    assert J2.item() == pytest.approx(oJ, rel=1e-10)
