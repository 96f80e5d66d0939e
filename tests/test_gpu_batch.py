"""Batched REV cubes (independent periodic boxes advanced in one launch per
step) and the launch schedule (autotuned tile-loop grid, CUDA-graph replay),
against the FP64 oracle run cube by cube."""
import numpy as np
import pytest

import oracle as O
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu

TOL_U = 1e-5
TOL_K = 1e-4


def small_cubes():
    """Periodic sphere cubes of uneven size (the REV sweep's shape, small
    enough for the oracle)."""
    out = []
    for i, (edge, phi) in enumerate([(16, 0.6), (22, 0.45), (19, 0.8), (26, 0.7)]):
        out.append(W.Channel(f"cube {edge}", edge, edge, edge, 0.0, float(edge), 2.0, 4.0, phi, True, 700 + i,
                             periodic_z=True))
    return out


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available()
    build()
    L.load_library()
    return torch


def _batch(cubes, g=(1e-4, 0.0, 0.0), flags=0, u0=None):
    import torch

    geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cubes]
    u0_t = None if u0 is None else torch.from_numpy(np.concatenate([u.reshape(3, -1) for u in u0], axis=1)).cuda()
    bs = L.BatchSolver(geoms, 0.8, 3 / 16, g, u0=u0_t, flags=flags)
    lats = [O.Lattice(c.nx, c.ny, c.nz, True, gm.spheres(), 0.8, 3 / 16, g).init(
        None if u0 is None else u0[i].astype(np.float64)) for i, (c, gm) in enumerate(zip(cubes, geoms))]
    return bs, lats, geoms


def test_batch_lists_per_part_bit_exact(torch_cuda):
    cubes = small_cubes()
    bs, _, geoms = _batch(cubes)
    got = bs.export_lists()
    assert bs.n_parts == len(cubes)
    li = 0
    for b, (c, gm) in enumerate(zip(cubes, geoms)):
        inf = bs.part_info(b)
        fo, co, nf, nl = inf["fluid_offset"], inf["cell_offset"], inf["n_fluid"], inf["n_links"]
        want = O.build_lists(c.nx, c.ny, c.nz, True, gm.spheres(), use_bins=True)
        assert np.array_equal(got["fluid_cell"][fo:fo + nf] - co, want["fluid_cell"])
        nb = got["nbr"][:, fo:fo + nf]
        assert np.array_equal(np.where(nb >= 0, nb - fo, -1), want["nbr"])
        sl = slice(li, li + nl)
        assert np.array_equal(got["link_cell"][sl] - fo, want["link_cell"])
        assert np.array_equal(got["link_k"][sl], want["link_k"])
        assert np.array_equal(got["link_q"][sl], want["link_q"])
        assert np.array_equal(got["link_fallback"][sl], want["link_fallback"])
        li += nl
    assert li == len(got["link_k"])


@pytest.mark.parametrize("nsteps", [0, 1, 2, 7])
def test_batch_populations_per_part(torch_cuda, nsteps):
    cubes = small_cubes()
    u0 = [W.velocity_field((c.nz, c.ny, c.nx), seed=50 + i, amplitude=2e-2) for i, c in enumerate(cubes)]
    bs, lats, _ = _batch(cubes, g=(3e-5, 1e-5, -2e-5), u0=u0)
    bs.step(nsteps)
    h = bs.populations().cpu().numpy().astype(np.float64)
    _, w = O.velocity_set()
    for b, lat in enumerate(lats):
        lat.step(nsteps)
        inf = bs.part_info(b)
        fo, nf = inf["fluid_offset"], inf["n_fluid"]
        fluid = np.flatnonzero(lat.solid().reshape(-1) == 0)
        want = lat.get_f().reshape(19, -1)[:, fluid] - w[:, None]
        assert np.max(np.abs(h[:, fo:fo + nf] - want)) <= TOL_U * np.max(np.abs(want))


def test_batch_permeability_and_plane_average(torch_cuda):
    cubes = small_cubes()
    bs, lats, _ = _batch(cubes)
    rc, n, res = bs.run_until(1e-7, 100, 100000, criterion="profile")
    assert rc == L.LBM_OK, (rc, n, res)
    assert np.all(bs.profile_residuals() < 1e-6)
    k = bs.permeabilities()
    pa = bs.plane_average()
    for b, lat in enumerate(lats):
        lat.step(n)
        assert abs(k[b] / lat.permeability() - 1) <= TOL_K
        po = bs.part_info(b)["plane_offset"]
        pa_o = lat.plane_average()
        seg = pa[po:po + cubes[b].nz]
        assert np.array_equal(seg[:, 2], pa_o[:, 2])
        assert np.max(np.abs(seg[:, 0] - pa_o[:, 0])) <= TOL_U * np.max(np.abs(pa_o[:, 0]))
    with pytest.raises(L.LBMError):
        bs.permeability()


def test_batch_recenter_per_part(torch_cuda):
    """Each cube drifts at its own rate; re-centring removes each cube's own
    mean and leaves the velocities on the oracle's."""
    cubes = small_cubes()
    bs, lats, _ = _batch(cubes)
    bs.step(2000)
    bs.recenter()
    bs.step(1)
    rho, u = bs.moments()
    for b, lat in enumerate(lats):
        lat.step(2001)
        inf = bs.part_info(b)
        co, nc = inf["cell_offset"], inf["n_cells"]
        fl = lat.solid().reshape(-1) == 0
        rho_o, u_o = lat.moments()
        drift = rho_o.reshape(-1)[fl].mean() - 1.0
        assert abs(drift) > 1e-7
        assert abs(rho.cpu().numpy()[co:co + nc][fl].mean() - 1.0) < 1e-2 * abs(drift)
        assert np.max(np.abs(u.cpu().numpy()[:, co:co + nc] - u_o.reshape(3, -1))) <= TOL_U * np.max(np.abs(u_o))


def test_schedule_does_not_change_results(torch_cuda):
    """Autotuned persistent grids and graph replay compute each cell exactly as
    one block per tile launched one by one: the states agree bit for bit."""
    cubes = [W.W4_cube(i) for i in range(3)]
    plain_flags = L.LBM_FLAG_NO_GRAPH | L.LBM_FLAG_NO_AUTOTUNE
    geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cubes]
    a = L.BatchSolver(geoms, g=(1e-5, 0, 0))
    b = L.BatchSolver(geoms, g=(1e-5, 0, 0), flags=plain_flags)
    for n in (7, 64, 101):
        a.step(n)
        b.step(n)
    sch = a.schedule()
    assert sch["tuned"] and sch["graph_steps"] > 0
    assert b.schedule()["graph_steps"] == 0
    assert a.steps == b.steps == 172
    import torch

    assert torch.equal(a.populations(), b.populations())


@pytest.mark.parametrize("flags", [L.LBM_FLAG_STAGED_NEIGHBOURS, L.LBM_FLAG_DERIVED_NEIGHBOURS],
                         ids=["staged-neighbours", "derived-neighbours"])
def test_batch_staged_neighbours_bit_exact(torch_cuda, flags):
    """Row words staged per tile (each part's words from its own offset; tiles
    across two cubes use the table) and neighbours derived along the x-rows
    give the table's bits in a batch of uneven periodic cubes."""
    import torch

    cubes = [W.W4_cube(i) for i in (59, 62, 3)]
    geoms = [L.lbm_geometry_from_spheres(*c.sphere_args()) for c in cubes]
    cells = sum(int(np.prod(g.shape)) for g in geoms)
    gen = torch.Generator(device="cuda").manual_seed(3)
    u0 = 1e-2 * torch.rand(3 * cells, device="cuda", generator=gen)
    a = L.BatchSolver(geoms, g=(1e-5, 0, 0), u0=u0, flags=flags)
    b = L.BatchSolver(geoms, g=(1e-5, 0, 0), u0=u0, flags=L.LBM_FLAG_NEIGHBOUR_TABLE)
    for n in (7, 64, 33):
        a.step(n)
        b.step(n)
    assert torch.equal(a.populations(), b.populations())


def test_single_solver_graph_replay_bit_exact(torch_cuda):
    case = W.W1
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    a = L.Solver(geom, g=(1e-5, 0, 0))
    b = L.Solver(geom, g=(1e-5, 0, 0), flags=L.LBM_FLAG_NO_GRAPH)
    a.step(3)
    b.step(3)
    a.step(130)
    b.step(130)
    import torch

    assert torch.equal(a.populations(), b.populations())
