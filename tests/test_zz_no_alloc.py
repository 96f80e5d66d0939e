"""lbm_plane_average_static: plane averages for callers that cannot allocate
device memory (an application whose pool allocator owns all device memory, or a
loop that must not stall on cudaMalloc/cudaFree).  Its scratch is a fixed array
inside the library.  Checked through the C ABI against lbm_plane_average on two
calls in a row (the shared scratch must not carry state from call to call).
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu


def _static_planes(lib, ux, solid, nx, ny, nz, stream):
    out = np.full((nz, 3), np.nan)
    rc = lib.lbm_plane_average_static(ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(solid.data_ptr()), nx, ny, nz,
                                      out.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(stream))
    return rc, out


def test_static_scratch_matches_workspace_entry_point():
    import torch

    assert torch.cuda.is_available()
    build()
    lib = L.load_library()
    case = W.W1
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=21, amplitude=1e-2)
    solver = L.Solver(geom, case.tau, case.lam, (2e-5, 0.0, 0.0), u0=torch.from_numpy(u0).cuda())
    solid = torch.from_numpy(geom.mask()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for nsteps in (7, 30):   # two calls in a row, different states
        solver.step(nsteps)
        want = solver.plane_average()
        _, u = solver.moments()
        ux = u[0].contiguous()
        torch.cuda.synchronize()
        rc, got = _static_planes(lib, ux, solid, case.nx, case.ny, case.nz, stream)
        assert rc == L.LBM_OK
        assert np.array_equal(got[:, 2], want[:, 2])
        assert np.max(np.abs(got[:, :2] - want[:, :2])) <= 1e-12 * np.max(np.abs(want[:, :2]))


def test_static_scratch_rejects_oversize():
    import torch

    build()
    lib = L.load_library()
    nz = 4097
    ux = torch.zeros((nz, 1, 1), dtype=torch.float32, device="cuda")
    solid = torch.zeros((nz, 1, 1), dtype=torch.uint8, device="cuda")
    rc, _ = _static_planes(lib, ux, solid, 1, 1, nz, torch.cuda.current_stream().cuda_stream)
    assert rc == L.LBM_EINVAL
