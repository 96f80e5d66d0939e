"""Parity at the benchmark's full sizes and launch configuration: the
256x256x512 channel (26.7 M fluid cells, porosity 0.6) with the tuned grid and
CUDA-graph replay that bench.py times, against the FP64 oracle run on the
whole box on the host; FP16/BF16 storage on the same box with its error
stated; and cubes of the 64-cube REV batch against the oracle cube by cube.

The oracle needs ~10 GB of host memory and ~0.4 s per step on 16 cores here."""
import numpy as np
import pytest

import oracle as O
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu

TOL_U = 1e-5
G = (3e-5, 0.0, 0.0)
# 24 tuning launches (4 grids x 3 repetitions x 2 parities), one 32-step graph
# replay, one more single launch: every launch path of the timed run
NSTEPS = 57


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available()
    build()
    L.load_library()
    return torch


@pytest.fixture(scope="module")
def channel(torch_cuda):
    """The porosity-0.6 channel of the benchmark sweep, a warm start, and the
    oracle's state after NSTEPS steps."""
    case = W.W2(0.6)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=11, amplitude=1e-2)
    lat = O.Lattice(case.nx, case.ny, case.nz, False, geom.spheres(), case.tau, case.lam, G).init(
        u0.astype(np.float64))
    lat.step(NSTEPS)
    rho_o, u_o = lat.moments()
    pa_o = lat.plane_average()
    k_o = lat.permeability(*case.perm_window)
    _, w = O.velocity_set()
    f = lat.get_f().reshape(19, -1)
    del lat
    return {"case": case, "geom": geom, "u0": u0, "f": f, "w": w, "u": u_o, "pa": pa_o, "k": k_o}


def _solver(torch, ch, storage):
    c = ch["case"]
    return L.Solver(ch["geom"], c.tau, c.lam, G, storage, u0=torch.from_numpy(ch["u0"]).cuda())


def test_full_size_fp32_every_population(torch_cuda, channel):
    s = _solver(torch_cuda, channel, "f32")
    s.step(NSTEPS)
    sched = s.schedule()
    assert sched["tuned"] and sched["graph_steps"] == 32
    fluid = s.export_lists()["fluid_cell"]
    got = s.populations().cpu().numpy()
    want = channel["f"][:, fluid] - channel["w"][:, None]
    assert np.max(np.abs(got - want)) <= TOL_U * np.max(np.abs(want))
    pa = s.plane_average()
    umax = np.max(np.abs(channel["u"]))
    assert np.array_equal(pa[:, 2], channel["pa"][:, 2])
    assert np.max(np.abs(pa[:, :2] - channel["pa"][:, :2])) <= TOL_U * umax
    k = s.permeability(*channel["case"].perm_window)
    assert abs(k / channel["k"] - 1) <= 1e-4


# Bound on the velocity error of 16-bit storage after NSTEPS steps, relative
# to u_max: each step rounds every stored population to half an ulp of the
# format (FP16 stores h * 2^14 with an 11-bit significand: 2^-12; BF16 an
# 8-bit significand: 2^-9), u sums about ten populations with |h| <= u_max/4,
# and independent roundings add like a random walk over the steps:
# 10 * 2^-p / 4 * sqrt(NSTEPS) * (safety 2).
@pytest.mark.parametrize("storage,p", [("f16", 12), ("bf16", 9)])
def test_full_size_reduced_precision_error(torch_cuda, channel, storage, p):
    s = _solver(torch_cuda, channel, storage)
    s.step(NSTEPS)
    _, u = s.moments()
    umax = np.max(np.abs(channel["u"]))
    err = np.max(np.abs(u.cpu().numpy() - channel["u"])) / umax
    bound = 2 * 10 * 2.0 ** -p / 4 * np.sqrt(NSTEPS)
    print(f"{storage}: max |u - u_oracle| / u_max = {err:.3e} (bound {bound:.3e})")
    assert err <= bound
    k = s.permeability(*channel["case"].perm_window)
    print(f"{storage}: permeability relative error {abs(k / channel['k'] - 1):.3e}")


def test_rev_batch_cubes_match_oracle(torch_cuda):
    """The 64-cube REV batch of the benchmark in its launch configuration; the
    four smallest cubes against the oracle cube by cube."""
    torch = torch_cuda
    cubes = [W.W4_cube(i) for i in range(64)]
    geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cubes]
    small = sorted(range(64), key=lambda i: cubes[i].nx)[:4]
    u0s = [W.velocity_field((c.nz, c.ny, c.nx), seed=900 + i, amplitude=1e-2) if i in small else
           np.zeros((3, c.nz, c.ny, c.nx), np.float32) for i, c in enumerate(cubes)]
    u0 = torch.from_numpy(np.concatenate([u.reshape(3, -1) for u in u0s], axis=1)).cuda()
    bs = L.BatchSolver(geoms, cubes[0].tau, cubes[0].lam, G, u0=u0)
    del u0
    bs.step(NSTEPS)
    h = bs.populations().cpu().numpy()
    fluid_all = bs.export_lists()["fluid_cell"]
    _, w = O.velocity_set()
    for i in small:
        c = cubes[i]
        inf = bs.part_info(i)
        fo, co, nf = inf["fluid_offset"], inf["cell_offset"], inf["n_fluid"]
        fluid = fluid_all[fo:fo + nf] - co
        lat = O.Lattice(c.nx, c.ny, c.nz, True, geoms[i].spheres(), c.tau, c.lam, G).init(u0s[i].astype(np.float64))
        lat.step(NSTEPS)
        want = lat.get_f().reshape(19, -1)[:, fluid] - w[:, None]
        got = h[:, fo:fo + nf]
        assert np.max(np.abs(got - want)) <= TOL_U * np.max(np.abs(want)), c.name
