"""Resolution and Reynolds-number studies of the pore-scale profile (Sec. 3.1).

The paper checks that its channel profile is grid-converged by refining the
same packing (sphere diameters 16 to 48 cells) and that it changes with the
Reynolds number of the flow.  Its packing is not available; these helpers
build the synthetic counterpart: one seeded packing of a 16x16x32 channel
(walls z = 0/31, overlapping spheres of diameter 4 in the lower half at
porosity 0.6) with every length multiplied by an integer scale, so that the
geometry is the same at every resolution, and run it to a steady profile.
Host-side orchestration only; every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

# the packing of the study at scale 1 (sphere diameter 4)
BASE = W.Channel("study base", 16, 16, 32, 1.0, 16.0, 2.0, 2.0, 0.6, True, 2060)
# force of the coarsest case: a free layer of ~15 cells with nu = 0.1 peaks
# near g L^2 / (8 nu) = 0.05, i.e. Re_D = u_max D / nu ~ 2 at D = 4
G1 = 1.8e-4


def scaled_spheres(scale: int) -> tuple[tuple[int, int, int], np.ndarray]:
    """Box (nx, ny, nz) and sphere list of the study packing at `scale`:
    centres scaled about the bottom wall surface z = 1/2, radii and the box
    scaled by the same factor (the wall layers stay one cell thick)."""
    from . import lbm_geometry_from_spheres

    sp = lbm_geometry_from_spheres(*BASE.sphere_args()).spheres()
    sc = sp.copy()
    sc[:, 0] *= scale
    sc[:, 1] *= scale
    sc[:, 2] = 0.5 + scale * (sp[:, 2] - 0.5)
    sc[:, 3] *= scale
    return (16 * scale, 16 * scale, 30 * scale + 2), sc


def layer_porosity(scale: int) -> float:
    """Voxel porosity of the scaled packing over the lower half of the fluid
    height (the layer the spheres fill), from the library's voxelisation."""
    from . import lbm_geometry_from_list

    (nx, ny, nz), sc = scaled_spheres(scale)
    mask = lbm_geometry_from_list(nx, ny, nz, False, sc).mask()
    h = nz - 2
    return float(1.0 - mask[1:1 + h // 2].mean())


def run_case(scale: int, g: float, tol: float, interval: int, max_steps: int, flags: int = 0):
    """Run the scaled packing to the profile tolerance.  Returns (normalised
    height of the fluid planes, u / u_max, steps, u_max, Re_D, status)."""
    from . import Solver, lbm_geometry_from_list, status_string

    (nx, ny, nz), sc = scaled_spheres(scale)
    geom = lbm_geometry_from_list(nx, ny, nz, False, sc)
    solver = Solver(geom, BASE.tau, BASE.lam, (g, 0.0, 0.0), flags=flags)
    rc, n, _ = solver.run_until(tol, interval, max_steps, criterion="profile")
    u = solver.plane_average()[1:-1, 0]
    h = (np.arange(1, nz - 1) - 0.5) / (nz - 2)
    nu = (BASE.tau - 0.5) / 3.0
    return h, u / u.max(), n, float(u.max()), float(u.max() * 4 * scale / nu), status_string(rc)


def profile_change(a, b, h_ref) -> float:
    """Relative L2 difference of two normalised profiles (h, u) sampled at
    the heights h_ref."""
    ua = np.interp(h_ref, *a)
    ub = np.interp(h_ref, *b)
    return float(np.linalg.norm(ua - ub) / np.linalg.norm(ub))
