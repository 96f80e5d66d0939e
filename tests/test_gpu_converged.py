"""Converged permeability in FP32 storage at the paper's driving force.

Sec. 3.1 drives every pore-scale run with a pressure drop of 1e-6 (here the
equivalent body force g_x = 1e-6) and reads the Darcy permeability (Eq. (Darcy))
from the steady state.  The GPU runs in FP32 storage to a plane-profile
residual of 1e-8; the FP64 oracle then takes the same number of steps from the
same start (step-exact parity at the steady state), and the two permeabilities
must agree to 1e-4 relative.  A second GPU run from another initial field must
reach the same permeability to 1e-4 (the steady Stokes state is unique, so the
start may only change how many steps it takes).
"""
import numpy as np
import pytest

import oracle as O
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu

TOL_K = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    L.load_library()
    return torch


def _converge(torch, geom, case, u0=None, flags=0):
    u0_t = None if u0 is None else torch.from_numpy(np.ascontiguousarray(u0, np.float32)).cuda()
    solver = L.Solver(geom, case.tau, case.lam, case.g, "f32", u0=u0_t, flags=flags)
    rc, n, res = solver.run_until(1e-8, 100, 2_000_000, criterion="profile")
    assert rc == L.LBM_OK, (rc, n, res)
    return solver, n


def _window_k(pa, nu, g, lo, hi):
    return nu * pa[lo:hi + 1, 0].mean() / g


CASES = {
    # the 32x32x64 channel of the first configuration: K over the whole box
    # and over the porous layer's interior z in [5, 27]
    "W1": (W.W1, [(-1, -1), (5, 27)]),
    # the smallest porous REV cube of the batched sweep (51^3, porosity 0.61)
    "W4 cube 59": (W.W4_cube(59), [(-1, -1)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_permeability_at_paper_force(torch_cuda, name):
    case, windows = CASES[name]
    assert case.g == (1e-6, 0.0, 0.0)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    cold, n = _converge(torch_cuda, geom, case)
    lat = O.Lattice(case.nx, case.ny, case.nz, case.periodic_z, geom.spheres(), case.tau, case.lam, case.g,
                    case.q_lo, case.q_hi).init()
    lat.step(n)
    pa, pa_o = cold.plane_average(), lat.plane_average()
    # a start far from the steady state: half the converged field plus smooth
    # random modes of a tenth of its peak
    _, u = cold.moments()
    u = u.cpu().numpy()
    u0 = 0.5 * u + W.velocity_field(u.shape[1:], seed=59, amplitude=0.1 * float(np.abs(u).max()))
    u0[:, geom.mask().astype(bool)] = 0.0
    warm, n_warm = _converge(torch_cuda, geom, case, u0=u0)
    pa_w = warm.plane_average()
    report = []
    for lo, hi in windows:
        lo_, hi_ = (0, case.nz - 1) if lo < 0 else (lo, hi)
        k = _window_k(pa, cold.nu, case.g[0], lo_, hi_)
        k_o = _window_k(pa_o, lat.nu, case.g[0], lo_, hi_)
        k_w = _window_k(pa_w, warm.nu, case.g[0], lo_, hi_)
        report.append((lo_, hi_, k, k_o, k_w, k / k_o - 1, k_w / k - 1))
    print(f"\n{name}: cold {n} steps, warm {n_warm} steps")
    for lo_, hi_, k, k_o, k_w, e, ew in report:
        print(f"  z {lo_}..{hi_}: K gpu {k:.9g} oracle {k_o:.9g} warm {k_w:.9g}  rel err {e:.2e}  warm-cold {ew:.2e}")
    for lo_, hi_, k, k_o, k_w, e, ew in report:
        assert abs(e) <= TOL_K, (lo_, hi_, e)
        assert abs(ew) <= TOL_K, (lo_, hi_, ew)
