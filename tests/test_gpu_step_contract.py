"""glbm_step's failure contract: a step in which a node leaves the positivity
domain of Sec. 3 (|u| <= sqrt(2/3) N per axis) completes, every later step of
the call is skipped on the device, and the call reports the steps completed
(glbm_last_error, glbm_time). The failure is made by the physics, not by a
fault: a uniform periodic flow driven by the body force g from rest has
u = g t in the moments at time t (the force of Sec. 5.4 adds g of momentum per
unit mass and step), so the step that leaves the domain is known exactly.
"""
import numpy as np
import pytest

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


def _failing_step(g, N):
    """First t with g t > sqrt(2/3) N: the step from X_t to X_{t+1} flags."""
    return int(np.floor(np.sqrt(2.0 / 3.0) * N / g)) + 1


@pytest.mark.parametrize("prec", [glbm.FP64, glbm.FP32_DEV])
def test_step_stops_after_the_failing_step(prec):
    """k = 0 (D2Q9), g = 0.01: u(82) = 0.82 > sqrt(2/3); glbm_step(200) (three
    64-step graph chunks and 8 single launches) completes 83 steps."""
    k, nx, ny, g = 0, 32, 8, 0.01
    t_bad = _failing_step(g, k + 1)
    assert t_bad == 82
    lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.8, bc=glbm.BC_PERIODIC, g=g,
                            prec=prec))
    with pytest.raises(glbm.UnstableError, match=f"{t_bad + 1} of 200 steps completed"):
        lat.step(200)
    assert lat.time == t_bad + 1
    m = lat.moments(0)  # the state X_83: u = 0.83 everywhere
    # (FP32 deviations at the edge of the domain, where f - W is of order 1)
    np.testing.assert_allclose(m["ux"], g * (t_bad + 1), rtol=1e-6 if prec == glbm.FP64 else 1e-4)
    np.testing.assert_allclose(m["uy"], 0.0, atol=1e-9 if prec == glbm.FP64 else 1e-6)
    # the context stays stopped: no step completes, the clock and state stay
    with pytest.raises(glbm.UnstableError, match="0 of 10 steps completed"):
        lat.step(10)
    assert lat.time == t_bad + 1
    np.testing.assert_array_equal(lat.moments(0)["ux"], m["ux"])
    # a new state clears the failure
    lat.set_equilibrium(0, np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    lat.step(10)
    assert lat.time == 10
    np.testing.assert_allclose(lat.moments(0)["ux"], 10 * g, rtol=1e-6 if prec == glbm.FP64 else 1e-5)
    lat.close()


def test_step_stops_at_the_failing_step_with_a_wall_launch():
    """The same in a force-driven channel whose wall densities have a launch of
    their own (two launches per step): the run stops whole after the flagged
    step, in the state a second context reaches by t - 1 steps and then the
    one step that flags."""
    cfg = dict(dims=2, nx=64, ny=24, k=1, tau=0.8, g=0.02)
    lat = glbm.Lattice(cfg)
    lat.set_wall_launch(1)
    assert lat.wall_launch == 1
    with pytest.raises(glbm.UnstableError) as ei:
        lat.step(500)
    t = lat.time
    assert 0 < t < 500
    assert f"{t} of 500 steps completed" in str(ei.value)
    ref = glbm.Lattice(cfg)
    ref.set_wall_launch(1)
    ref.step(t - 1)  # inside the domain up to here: no error
    with pytest.raises(glbm.UnstableError, match="1 of 1 steps completed"):
        ref.step(1)
    assert ref.time == t
    np.testing.assert_array_equal(ref.get_populations(0), lat.get_populations(0))
    lat.close()
    ref.close()


def test_batch_stops_every_instance_at_the_failing_step():
    """A heterogeneous batch (one launch per level): instance 0 (k = 1,
    g = 0.02) leaves the domain in step 82; instance 1 (k = 2, at rest with
    moving walls) stops with it, at time 83, equal to its own run of 83 steps."""
    g = 0.02
    a = dict(dims=2, nx=64, ny=16, k=1, tau=0.8, bc=glbm.BC_PERIODIC, g=g, prec=glbm.FP32_DEV)
    b = dict(dims=2, nx=64, ny=40, k=2, kn=0.1, u_wall_lo=-0.05, u_wall_hi=0.05,
             prec=glbm.FP32_DEV)
    t_bad = _failing_step(g, 2)
    lat = glbm.Lattice([a, b], hetero=True)
    with pytest.raises(glbm.UnstableError, match=f"{t_bad + 1} of 300 steps completed"):
        lat.step(300)
    assert lat.time == t_bad + 1
    np.testing.assert_allclose(lat.moments(0)["ux"], g * (t_bad + 1), rtol=1e-5)
    solo = glbm.Lattice([b])
    solo.step(t_bad + 1)
    mb, ms = lat.moments(1), solo.moments(0)
    for name in ("rho", "ux", "sxy"):
        scale = max(np.abs(ms[name]).max(), 1e-12)
        assert np.abs(mb[name] - ms[name]).max() / scale < 1e-5, name
    lat.close()
    solo.close()


def test_1d_resident_run_stops_at_the_failing_step():
    """1D (one resident launch): a state already outside the domain
    (|u| > sqrt(2/3) N) flags in its first step; 1 of 10 steps completes."""
    k, L = 1, 64
    lat = glbm.Lattice(dict(dims=1, nx=L, k=k, tau=0.8))
    umax = np.sqrt(2.0 / 3.0) * (k + 1)
    lat.set_equilibrium(0, np.ones(L), np.full(L, 1.1 * umax))
    with pytest.raises(glbm.UnstableError, match="1 of 10 steps completed"):
        lat.step(10)
    assert lat.time == 1
    with pytest.raises(glbm.UnstableError, match="0 of 5 steps completed"):
        lat.step(5)
    assert lat.time == 1
    lat.close()


def test_steps_inside_the_domain_report_nothing():
    """A stable run returns OK with the full step count on the clock, also
    after an autotune (whose trial launches leave the status words alone)."""
    lat = glbm.Lattice(dict(dims=2, nx=64, ny=32, k=3, kn=0.1, u_wall_lo=-0.05, u_wall_hi=0.05,
                            prec=glbm.FP32_DEV))
    lat.autotune(reps=2)
    lat.step(130)
    assert lat.time == 130
    lat.sync()
    lat.close()
