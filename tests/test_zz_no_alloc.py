"""The allocation-free conservation sums against the context-owned ones.

glbm_conservation_noalloc serves callers that may not allocate device memory
(real-time loops that cannot take the allocator's synchronisation,
applications whose pool owns all device memory, code inside such a pool's
callbacks). Its block partials live in a static array in the library's device
memory that every call shares. This test calls it through the C ABI several
times in a row, from large to small, so that each later call runs over the
partials the earlier ones left behind; the first call is near the size cap
and uses many blocks. Each result must equal glbm_conservation on the same
fields, and the 1D call must write 0 for the y-momentum.
"""
import ctypes

import numpy as np
import pytest

from paper_1905_04597_gb300 import glbm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()


def test_noalloc_sums_match_context_sums_twice():
    import torch
    L = glbm.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # largest first: 2048 x 2000 nodes (near GLBM_NOALLOC_MAX_NODES = 4096 x 1024)
    for call, (k, nx, ny, seed) in enumerate(((0, 2048, 2000, 3), (3, 96, 40, 1), (1, 333, 17, 2))):
        lat = glbm.Lattice(dict(dims=2, nx=nx, ny=ny, k=k, tau=0.8, u_wall_lo=-0.04,
                                u_wall_hi=0.03, g=1e-5))
        rho, ux, uy = inputs.random_macro(seed, nx, ny)
        lat.set_equilibrium(0, rho, ux, uy)
        lat.step(7)
        mass, jx, jy = lat.conservation(0)
        fields = torch.empty((3, ny, nx), dtype=torch.float64, device="cuda")
        lat.moments(0, mask=glbm.M_RHO | glbm.M_UX | glbm.M_UY, out=fields)
        sums = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.glbm_conservation_noalloc(ctypes.c_void_p(fields.data_ptr()), 2, nx * ny,
                                         ctypes.c_void_p(sums.data_ptr()), stream)
        glbm.check(st)
        torch.cuda.synchronize()
        got = sums.cpu().numpy()
        np.testing.assert_allclose(got, [mass, jx, jy], rtol=1e-12, atol=1e-14,
                                   err_msg=f"call {call}")
        lat.close()


def test_noalloc_1d_writes_zero_y_momentum():
    """dims = 1: two fields (rho, u_x); sums[2] is written as 0, after a 2D
    call that left a nonzero y-momentum in the same scratch."""
    import torch
    L = glbm.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lat2 = glbm.Lattice(dict(dims=2, nx=64, ny=32, k=2, tau=0.8, bc=glbm.BC_PERIODIC))
    rho, ux, uy = inputs.random_macro(5, 64, 32)
    lat2.set_equilibrium(0, rho, ux, uy + 0.01)
    f2 = torch.empty((3, 32, 64), dtype=torch.float64, device="cuda")
    lat2.moments(0, mask=glbm.M_RHO | glbm.M_UX | glbm.M_UY, out=f2)
    s2 = torch.empty(3, dtype=torch.float64, device="cuda")
    glbm.check(L.glbm_conservation_noalloc(ctypes.c_void_p(f2.data_ptr()), 2, 64 * 32,
                                           ctypes.c_void_p(s2.data_ptr()), stream))
    torch.cuda.synchronize()
    assert abs(float(s2[2])) > 1.0  # a y-momentum sum is left in the scratch
    lat2.close()
    L1 = 1000
    lat = glbm.Lattice(dict(dims=1, nx=L1, k=1, tau=0.9))
    x = np.arange(L1)
    lat.set_equilibrium(0, 1.0 + 0.1 * np.sin(2 * np.pi * x / L1), 0.05 * np.cos(2 * np.pi * x / L1))
    lat.step(5)
    mass, jx, _ = lat.conservation(0)
    fields = torch.empty((2, L1), dtype=torch.float64, device="cuda")
    lat.moments(0, mask=glbm.M_RHO | glbm.M_UX, out=fields)
    sums = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    glbm.check(L.glbm_conservation_noalloc(ctypes.c_void_p(fields.data_ptr()), 1, L1,
                                           ctypes.c_void_p(sums.data_ptr()), stream))
    torch.cuda.synchronize()
    got = sums.cpu().numpy()
    np.testing.assert_allclose(got[:2], [mass, jx], rtol=1e-12, atol=1e-14)
    assert got[2] == 0.0
    lat.close()


def test_noalloc_rejects_oversize_without_launching():
    L = glbm.lib()
    big = glbm.lib().glbm_conservation_noalloc(ctypes.c_void_p(16), 2, 4096 * 1024 + 1,
                                               ctypes.c_void_p(16), None)
    assert big == glbm.E_INVAL
    assert b"static scratch" in L.glbm_last_error()
