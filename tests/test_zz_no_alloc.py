"""The allocation-free conservation sums against the context-owned ones.

glbm_conservation_noalloc serves callers that may not allocate device memory
(code under CUDA-graph capture, real-time loops, applications whose pool owns
all device memory). Its block partials live in a static array in the
library's device memory. This test calls it through the C ABI twice in a row,
on different inputs, so the second call runs over the first call's leftovers.
Each result must equal glbm_conservation on the same fields.
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
    for call, (k, nx, ny, seed) in enumerate(((3, 96, 40, 1), (1, 333, 17, 2))):
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


def test_noalloc_rejects_oversize_without_launching():
    L = glbm.lib()
    big = glbm.lib().glbm_conservation_noalloc(ctypes.c_void_p(16), 2, 4096 * 1024 + 1,
                                               ctypes.c_void_p(16), None)
    assert big == glbm.E_INVAL
    assert b"static scratch" in L.glbm_last_error()
