"""The Knudsen paradox of force-driven Poiseuille flow (Sec. 5.4) on the GPU.

The paper reports, for single-relaxation-time models between diffuse walls:
the 2N+1 hierarchy suffers runaway effects in the ballistic regime (the flow
rate grows without bound as Kn grows); the low levels of the 2N+2 hierarchy
(no wall-parallel velocities, G-D1Q6 x D1Q3, G-D1Q8 x D1Q3) are free of them
but their flow rate has no minimum; the Knudsen minimum appears in the 2N+2
hierarchy from N = 10 on, and G-D1Q28 x D1Q3 (N = 13) is the model it shows.

Each case runs x-uniform channels of H = 200 nodes (the paper's node count)
to a steady state in FP64 and compares the dimensionless flow rate
G(Kn) = sum_y u_x / (g H^2 / sqrt(2 theta_x)), which is the paper's volumetric
flow Q up to a factor that does not depend on Kn (its delta / U0 is constant
in Kn)."""
import math

import numpy as np
import pytest

from paper_1905_04597_gb300 import glbm

pytestmark = pytest.mark.gpu

KN = (0.1, 0.316, 1.0, 3.16, 10.0)
H, G_FORCE = 200, 1e-7


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def flow_rates(k, zv_axes):
    out = []
    for kn in KN:
        lat = glbm.Lattice(dict(dims=2, nx=1, ny=H, k=k, x_level=1, zv_axes=zv_axes, kn=kn,
                                g=G_FORCE, prec=glbm.FP64))
        prev = None
        for _ in range(200):
            lat.step(500)
            J = float(lat.moments(0)["ux"][:, 0].sum())
            if prev is not None and abs(J - prev) < 1e-7 * abs(J):
                break
            prev = J
        else:
            raise AssertionError(f"no steady state at Kn={kn}")
        lat.close()
        out.append(J / (G_FORCE * H * H / math.sqrt(2.0 / 3.0)))
    return np.array(out)


def test_2n2_hierarchy_n13_has_the_knudsen_minimum():
    G = flow_rates(12, glbm.ZV_Y)  # G-D1Q28 x D1Q3
    i = int(np.argmin(G))
    assert 0 < i < len(KN) - 1, G
    assert KN[i] == pytest.approx(1.0), G
    assert G[-1] > 1.02 * G[i], G


def test_2n2_hierarchy_low_level_has_no_minimum():
    G = flow_rates(2, glbm.ZV_Y)  # G-D1Q8 x D1Q3
    assert np.all(np.diff(G) < 0), G


def test_2n1_hierarchy_runs_away_in_the_ballistic_regime():
    G = flow_rates(4, 0)  # G-D1Q11 x D1Q3
    i = int(np.argmin(G))
    assert 0 < i < len(KN) - 1, G
    assert G[-1] > 2.0 * G[i], G
