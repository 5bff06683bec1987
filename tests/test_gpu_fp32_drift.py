"""Long-run momentum of the FP32-deviation step on periodic lattices.

The collision conserves mass and momentum exactly (Sec. 2: the equilibrium
reproduces rho and rho u). In FP32 deviations the rest weights are floats;
if one axis's float weights summed to 1 + eps, the deviation equilibrium
delta f^eq = d^x rho e^y + W^x (...) would scale the other axis's momentum
by 1 + eps at every collision: a uniform flow, which stays at equilibrium,
would drift by omega eps per step (3e-8 for D1Q3 weights rounded to nearest,
5e-4 over 2e4 steps). The table builder balances the float weights so that
their exact sum is 1; a uniform periodic flow then keeps its momentum over
2e4 steps to 1e-5 (measured: below 4e-6)."""
import numpy as np
import pytest

from paper_1905_04597_gb300 import glbm

pytestmark = pytest.mark.gpu

LATTICES = {
    "d2q81": dict(k=3),
    "d2q289": dict(k=7),
    "d1q3xd1q17": dict(k=7, x_level=1),
    "d1q3xd1q8": dict(k=2, x_level=1, zv_axes=glbm.ZV_Y),
    "d2q64": dict(k=2, zv_axes=glbm.ZV_X | glbm.ZV_Y),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name", sorted(LATTICES))
def test_uniform_flow_keeps_its_momentum(name):
    nx, ny, steps = 64, 32, 20000
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, tau=0.75, bc=glbm.BC_PERIODIC,
                            prec=glbm.FP32_DEV, **LATTICES[name]))
    ux, uy = 0.05, -0.02
    lat.set_equilibrium(0, np.ones((ny, nx)), np.full((ny, nx), ux), np.full((ny, nx), uy))
    m0, jx0, jy0 = lat.conservation(0)
    assert jx0 == pytest.approx(ux * nx * ny, rel=1e-6)
    lat.step(steps)
    m1, jx1, jy1 = lat.conservation(0)
    assert abs(m1 - m0) / m0 < 1e-6
    assert abs(jx1 - jx0) / abs(jx0) < 1e-5, (jx0, jx1)
    assert abs(jy1 - jy0) / abs(jy0) < 1e-5, (jy0, jy1)
    lat.close()
