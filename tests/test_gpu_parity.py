"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer and index results (fluid list, neighbour table, link list, link
fractions q) must be bit-exact.  Floating-point fields in FP32 storage must
agree to 1e-5 of the largest velocity (or population) of the oracle, the
tolerance of the FP32 path; permeability to 1e-4 relative.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu

TOL_U = 1e-5      # |u - u_oracle|_inf <= TOL_U * max|u_oracle|
TOL_K = 1e-4      # relative permeability


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    L.load_library()
    return torch


# The wall rule: Eq. (CLI) wherever the second fluid node exists (the paper's
# scheme), or with the corner safeguards (q < 0.1 and two-cell gaps take
# simple bounce-back) on both sides.
MODES = [False, True]
MODE_IDS = ["paper-cli", "safeguards"]


def _pair(torch, case, storage="f32", u0=None, g=None, flags=0, safeguards=False):
    g = case.g if g is None else g
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    sp = geom.spheres()
    u0_t = None if u0 is None else torch.from_numpy(u0).cuda()
    if safeguards:
        flags |= L.LBM_FLAG_CLI_SAFEGUARDS
    solver = L.Solver(geom, case.tau, case.lam, g, storage, u0=u0_t, flags=flags)
    lat = O.Lattice(case.nx, case.ny, case.nz, case.periodic_z, sp, case.tau, case.lam, g, case.q_lo,
                    case.q_hi, cli_safeguards=safeguards).init(None if u0 is None else u0.astype(np.float64))
    return solver, lat, geom


def _oracle_shifted(lat, fluid_cell):
    _, w = O.velocity_set()
    f = lat.get_f().reshape(19, -1)[:, fluid_cell]
    return f - w[:, None]


CASES = W.small_cases()


@pytest.mark.parametrize("safeguards", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("case", CASES + [W.W4_cube(0)], ids=lambda c: c.name)
def test_lists_bit_exact(torch_cuda, case, safeguards):
    solver, _, geom = _pair(torch_cuda, case, safeguards=safeguards)
    got = solver.export_lists()
    want = O.build_lists(case.nx, case.ny, case.nz, case.periodic_z, geom.spheres(), case.q_lo, case.q_hi,
                         use_bins=True, safeguards=safeguards)
    for key in want:
        assert got[key].dtype == want[key].dtype, key
        assert np.array_equal(got[key], want[key]), key


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3, 10])
@pytest.mark.parametrize("flags", [0, L.LBM_FLAG_STAGED_EVEN], ids=["plain", "staged-even"])
@pytest.mark.parametrize("safeguards", MODES, ids=MODE_IDS)
def test_populations_step_by_step(torch_cuda, case, nsteps, flags, safeguards):
    """Both AA parities: the shifted populations after n steps from a warm
    start, at every fluid cell and direction; with the even step on either
    kernel (registers, or TMA-staged through shared memory), under either
    wall rule."""
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=100 + nsteps, amplitude=2e-2)
    solver, lat, _ = _pair(torch_cuda, case, u0=u0, g=(3e-5, -1e-5, 2e-5), flags=flags, safeguards=safeguards)
    solver.step(nsteps)
    lat.step(nsteps)
    fluid = solver.export_lists()["fluid_cell"]
    got = solver.populations().cpu().numpy().astype(np.float64)
    want = _oracle_shifted(lat, fluid)
    assert np.max(np.abs(got - want)) <= TOL_U * np.max(np.abs(want))


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("nsteps", [40, 41])
def test_moments_and_plane_average(torch_cuda, case, nsteps):
    """Dense moments and plane averages at both parities after a warm start.
    The force is large enough that its per-step increment is resolved by FP32
    storage next to the warm-start populations (see the FP32 regime note)."""
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=7, amplitude=1e-2)
    solver, lat, geom = _pair(torch_cuda, case, u0=u0, g=(3e-5, -1e-5, 2e-5))
    solver.step(nsteps)
    lat.step(nsteps)
    rho, u = solver.moments()
    rho_o, u_o = lat.moments()
    solid = geom.mask().astype(bool)
    assert np.all(rho.cpu().numpy()[solid] == 0) and np.all(u.cpu().numpy()[:, solid] == 0)
    umax = np.max(np.abs(u_o))
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= TOL_U * umax
    assert np.max(np.abs(rho.cpu().numpy() - rho_o)[~solid]) <= 1e-6
    pa, pa_o = solver.plane_average(), lat.plane_average()
    assert np.array_equal(pa[:, 2], pa_o[:, 2])
    assert np.max(np.abs(pa[:, :2] - pa_o[:, :2])) <= TOL_U * umax


@pytest.mark.parametrize("safeguards", MODES, ids=MODE_IDS)
def test_w1_2000_steps_velocity(torch_cuda, safeguards):
    """32x32x64 channel with RSA spheres, cold start, 2000 steps (FP32)."""
    case = W.W1
    solver, lat, _ = _pair(torch_cuda, case, safeguards=safeguards)
    solver.step(case.steps)
    lat.step(case.steps)
    _, u = solver.moments()
    _, u_o = lat.moments()
    umax = np.max(np.abs(u_o[0]))
    assert umax > 0
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= TOL_U * umax
    pa, pa_o = solver.plane_average(), lat.plane_average()
    assert np.max(np.abs(pa[:, 0] - pa_o[:, 0])) <= TOL_U * np.max(np.abs(pa_o[:, 0]))


def _fp32_channel_bias(H, nu):
    """Relative velocity error that FP32 storage can leave in a steady channel:
    every cell of a plane rounds the same values the same way, so the rounding
    (2^-24 of the populations ~ u per step) acts like a body force that is not
    averaged away, against the real force g: 2^-24 u_max / g = 2^-24 H^2 / (8 nu)."""
    return 2.0 ** -24 * H * H / (8.0 * nu)


def _steady_channel(nx, nz, tau, lam, q_lo, q_hi, g, flags=0, storage="f32"):
    geom = L.lbm_geometry_from_list(nx, nx, nz, False, [], q_lo=q_lo, q_hi=q_hi)
    solver = L.Solver(geom, tau, lam, (g, 0.0, 0.0), storage, flags=flags)
    nu = (tau - 0.5) / 3
    H = nz - 2
    nsteps = int(40 * H * H / (math.pi ** 2 * nu)) + 201
    while nsteps > 0:   # re-centre the density: CLI walls leak mass
        solver.step(min(500, nsteps))
        nsteps -= 500
        solver.recenter()
    solver.step(1)
    _, u = solver.moments()
    ux = u[0, 1:nz - 1, 0, 0].cpu().numpy().astype(np.float64)
    z = np.arange(1, nz - 1, dtype=np.float64)
    za, zb = 1 - q_lo, nz - 2 + q_hi
    ua = -(g / nu) * (q_lo ** 2 / 2 - 2 * lam / 3)
    ub = -(g / nu) * (q_hi ** 2 / 2 - 2 * lam / 3)
    exact = g / (2 * nu) * (z - za) * (zb - z) + ua + (ub - ua) * (z - za) / (zb - za)
    return ux, exact


@pytest.mark.parametrize("tau,lam,q_lo,q_hi", [(0.8, 3 / 16, 0.5, 0.5), (1.4, 3 / 16, 0.3, 0.8),
                                               (0.8, 0.25, 0.15, 1.0)])
def test_channel_closed_form_on_gpu(torch_cuda, tau, lam, q_lo, q_hi):
    """Steady channel against the closed form of the CLI wall slip,
    u(z_w) = -(g/nu)(q^2/2 - 2 Lambda/3), in FP32 storage, to 1e-5 of u_max
    or twice the FP32 bias of a translation-invariant channel, whichever is
    larger (the bias is 1.9e-5 at H = 16, nu = 0.1)."""
    nz, g = 18, 1e-6
    nu = (tau - 0.5) / 3
    ux, exact = _steady_channel(4, nz, tau, lam, q_lo, q_hi, g)
    tol = max(TOL_U, 2 * _fp32_channel_bias(nz - 2, nu))
    assert np.max(np.abs(ux - exact)) <= tol * np.max(exact)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_plane_references_cut_the_reduced_precision_bias(torch_cuda, storage):
    """In FP16/BF16 storage the rounding of the stored populations dominates
    the error of a steady channel (the collision rounds in FP32); with the
    plane reference equilibria the stored values are the small
    non-equilibrium parts, and the error against the closed form falls by at
    least half.  (In FP32 storage the collision's own roundings at the full
    magnitude dominate, so the references do not help there: measured 1.8e-5
    plain, 2.2e-5 with references.)"""
    nz, g, tau, lam = 34, 1e-6, 0.8, 3 / 16
    ux, exact = _steady_channel(16, nz, tau, lam, 0.5, 0.5, g, storage=storage, flags=L.LBM_FLAG_NO_PLANE_REFERENCES)
    ux_r, _ = _steady_channel(16, nz, tau, lam, 0.5, 0.5, g, storage=storage)   # references: the 16-bit default
    e, e_r = (np.max(np.abs(v - exact)) / np.max(exact) for v in (ux, ux_r))
    print(f"\n{storage} channel error: plain {e:.2e}, with plane references {e_r:.2e}")
    assert e_r < 0.5 * e


def test_permeability_converged(torch_cuda):
    """Periodic sphere cube run to a plane-profile residual of 1e-9 on the GPU;
    the oracle takes the same number of steps (step-exact parity) and the
    permeabilities must agree to 1e-4.  g = 1e-4 keeps the pore velocities
    (~1e-3) in the range FP32 storage resolves; K does not depend on g in the
    Stokes regime."""
    case = CASES[2]
    g = (1e-4, 0.0, 0.0)
    solver, lat, _ = _pair(torch_cuda, case, g=g)
    # 16 planes of ~360 cells average little FP32 noise away; 1e-7 is
    # reachable here (large boxes reach 1e-8)
    rc, n, res = solver.run_until(1e-7, 100, 200000, criterion="profile")
    assert rc == L.LBM_OK, (rc, n, res)
    lat.step(n)
    k, k_o = solver.permeability(), lat.permeability()
    assert abs(k / k_o - 1) <= TOL_K
    # converged: the oracle's profile moves by less than 1e-7 over 100 more steps
    p0 = lat.plane_average()[:, 0]
    lat.step(100)
    p1 = lat.plane_average()[:, 0]
    assert np.linalg.norm(p1 - p0) / np.linalg.norm(p1) < 1e-7


def test_recenter_keeps_velocity(torch_cuda):
    """A uniform density shift commutes with the whole update: after
    re-centring, the velocities stay on the oracle's (which never re-centres)
    and the mean density deviation drops to round-off."""
    case = CASES[2]
    g = (1e-4, 0.0, 0.0)
    solver, lat, _ = _pair(torch_cuda, case, g=g)
    solver.step(3000)
    lat.step(3000)
    drift = solver.mass()
    rho_o, _ = lat.moments()
    fl = lat.solid() == 0
    # CLI mass drift, reported.  Every step the FP32 storage rounds each of a
    # cell's 19 populations once (error <= 2^-25 |h|), so after n steps the
    # mean density can be off by n * 19 * 2^-25 * max|h| at most (3000 steps
    # of 1e-3-sized populations: ~1.7e-6, 1e-3 of this drift); measured
    # 6.3e-8 (3e-5 of the drift of 2.1e-3)
    h_max = float(np.max(np.abs(_oracle_shifted(lat, solver.export_lists()["fluid_cell"]))))
    bound = 3000 * 19 * 2.0 ** -25 * h_max
    assert abs(drift - (rho_o[fl].mean() - 1.0)) <= bound
    assert abs(drift) > 1e-6
    solver.recenter()
    solver.step(1)
    lat.step(1)
    assert abs(solver.mass()) < 1e-2 * abs(drift)   # one step of new drift is left
    solver.step(100)
    lat.step(100)
    _, u = solver.moments()
    _, u_o = lat.moments()
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= TOL_U * np.max(np.abs(u_o))


# storage precision bits: FP32 keeps the FP32 tolerance; FP16/BF16 use the
# random-walk bound of their rounding, 10 (2^-p / 4) sqrt(n) 2 over n steps
@pytest.mark.parametrize("storage,p_bits", [("f32", None), ("f16", 12), ("bf16", 9)])
@pytest.mark.parametrize("flags", [0, L.LBM_FLAG_STAGED_EVEN, L.LBM_FLAG_ROW_NEIGHBOURS, L.LBM_FLAG_STAGED_NEIGHBOURS],
                         ids=["plain", "staged-even", "row-neighbours", "staged-neighbours"])
def test_reference_populations_switch(torch_cuda, storage, p_bits, flags):
    """The free layer of the W1 channel stores its populations relative to
    the plane's reference equilibrium after a re-centring: the switch (one
    step that reads with the old and writes with the new references, at
    either parity) and the steps after it leave the populations on the
    oracle's, which never re-centres."""
    tol = TOL_U if p_bits is None else 10 * 2.0 ** -p_bits / 4 * math.sqrt(184) * 2
    case = W.W1
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=3, amplitude=2e-2)
    solver, lat, _ = _pair(torch_cuda, case, storage=storage, u0=u0, g=(3e-5, 0.0, 0.0),
                           flags=flags | L.LBM_FLAG_PLANE_REFERENCES)
    assert solver.reference_planes() > 20   # the free layer z = 32..62, less its edges
    fluid = solver.export_lists()["fluid_cell"]
    shift = 0.0
    for n in (40, 41, 33):   # switches at even, odd and even parity
        solver.step(n)
        lat.step(n)
        shift += solver.recenter()
    solver.step(70)
    lat.step(70)
    # the re-centring removed the mean density drift from every population
    # (h_k - w_k c), which the oracle keeps: add it back before comparing
    _, w = O.velocity_set()
    got = solver.populations().cpu().numpy().astype(np.float64) + w[:, None] * shift
    want = _oracle_shifted(lat, fluid)
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    _, u = solver.moments()
    _, u_o = lat.moments()
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= tol * np.max(np.abs(u_o))


def test_profile_residual_matches_oracle(torch_cuda):
    case = W.W1
    solver, lat, _ = _pair(torch_cuda, case)
    assert math.isinf(solver.profile_residual())
    p0 = lat.plane_average()[:, 0]
    solver.step(300)
    lat.step(300)
    p1 = lat.plane_average()[:, 0]
    want = np.linalg.norm(p1 - p0) / np.linalg.norm(p1)
    assert abs(solver.profile_residual() / want - 1) < 1e-4


def test_permeability_window(torch_cuda):
    case = W.W1
    solver, lat, _ = _pair(torch_cuda, case)
    solver.step(500)
    lat.step(500)
    for zl, zh in [(-1, -1), (3, 20), (40, 40)]:
        assert abs(solver.permeability(zl, zh) / lat.permeability(zl, zh) - 1) <= TOL_K
    with pytest.raises(L.LBMError):
        solver.permeability(10, 64)


def test_residual_semantics(torch_cuda):
    case = CASES[1]
    solver, lat, _ = _pair(torch_cuda, case)
    assert math.isinf(solver.residual())
    lat.residual()
    solver.step(50)
    lat.step(50)
    r, r_o = solver.residual(), lat.residual()
    assert abs(r / r_o - 1) < 1e-3


def test_nan_is_reported(torch_cuda):
    """A non-finite warm start (host-made input) surfaces as LBM_ENAN."""
    case = CASES[1]
    u0 = np.zeros((3, case.nz, case.ny, case.nx), np.float32)
    u0[0, 10] = np.nan   # a plane of the free channel above the packing
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    import torch

    solver = L.Solver(geom, u0=torch.from_numpy(u0).cuda())
    solver.step(3)
    with pytest.raises(L.LBMError) as e:
        solver.residual()
    assert e.value.status == L.LBM_ENAN


def test_bounded_wait_reports_timeout(torch_cuda):
    """Failure detection without a fault: a bounded mbarrier wait on a phase
    that nothing completes gives up, the status word turns into LBM_ETIMEOUT
    at the next synchronisation, the solver refuses to step on from a state a
    timed-out block would have left half-updated, and lbm_reset makes it
    usable again (the word is cleared; the next steps and reductions
    succeed)."""
    case = CASES[0]
    solver, lat, _ = _pair(torch_cuda, case)
    lib = L.load_library()
    assert lib.lbm_wait_selftest(solver.handle, 0) == L.LBM_EINVAL
    assert lib.lbm_wait_selftest(solver.handle, 4096) == L.LBM_ETIMEOUT
    assert lib.lbm_step(solver.handle, 1) == L.LBM_ETIMEOUT
    assert solver.run_until(1e-8, 10, 100)[0] == L.LBM_ETIMEOUT
    assert solver.plane_average() is not None   # read-only calls still work
    solver.reset()
    solver.step(6)
    lat.step(6)
    assert solver.residual() is not None   # synchronises: no stale timeout
    _, u = solver.moments()
    _, u_o = lat.moments()
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= TOL_U * np.max(np.abs(u_o))


def test_workspace_too_small(torch_cuda):
    torch = torch_cuda
    geom = L.lbm_geometry_from_spheres(*CASES[1].sphere_args())
    p = L.make_params()
    n = L.lbm_workspace_size(geom, p)
    ws = torch.empty(n - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LBMError) as e:
        L.lbm_init(geom, p, ws)
    assert e.value.status == L.LBM_ESIZE


def test_step_zero_and_reset(torch_cuda):
    case = CASES[1]
    solver, lat, _ = _pair(torch_cuda, case)
    solver.step(0)
    h0 = solver.populations().cpu().numpy()
    solver.step(7)
    solver.reset()
    assert solver.steps == 0
    assert np.array_equal(solver.populations().cpu().numpy(), h0)


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 1.6e-2)])
@pytest.mark.parametrize("flags", [0, 1, 2, 64])
def test_reduced_precision_storage(torch_cuda, storage, tol, flags):
    """FP16/BF16 storage of the shifted populations (FP32 collision): the
    velocity after a few steps stays within the storage's relative precision
    (FP16 2^-11, BF16 2^-8, times a few roundings) of the FP64 oracle, for
    every odd-step variant."""
    case = CASES[0]
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=3, amplitude=2e-2)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    import torch

    solver = L.Solver(geom, case.tau, case.lam, (3e-5, 0.0, 0.0), storage, u0=torch.from_numpy(u0).cuda(), flags=flags)
    lat = O.Lattice(case.nx, case.ny, case.nz, False, geom.spheres(), case.tau, case.lam, (3e-5, 0.0, 0.0))
    lat.init(u0.astype(np.float64))
    solver.step(11)
    lat.step(11)
    _, u = solver.moments()
    _, u_o = lat.moments()
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= tol * np.max(np.abs(u_o))


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_staged_even_step_bit_exact(torch_cuda, storage, case):
    """The TMA-staged even kernel performs the register kernel's arithmetic
    (every rounding of the collision is explicit) on the same values: the
    states agree bit for bit after both parities, at every storage type (a
    tile count that is not a multiple of the grid leaves the last blocks with
    fewer tiles)."""
    import torch

    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=11, amplitude=2e-2)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    u0t = torch.from_numpy(u0).cuda()
    a = L.Solver(geom, case.tau, case.lam, (3e-5, -1e-5, 2e-5), storage, u0=u0t, flags=L.LBM_FLAG_STAGED_EVEN)
    b = L.Solver(geom, case.tau, case.lam, (3e-5, -1e-5, 2e-5), storage, u0=u0t, flags=L.LBM_FLAG_NO_AUTOTUNE)
    for n in (1, 1, 9, 40):
        a.step(n)
        b.step(n)
        assert torch.equal(a.populations(), b.populations()), n
    assert a.schedule()["grid_even"] == -1 and b.schedule()["grid_even"] > 0
    a.residual()   # synchronises and reads the kernels' timeout word (LBMError if set)


def test_geometry_without_fluid(torch_cuda):
    """Degenerate input: a walled 8 x 8 x 4 box whose two fluid planes four
    overlapping spheres fill has no fluid cell.  The solver builds, steps
    (both parities) and reports empty fields without launching empty grids."""
    spheres = [[x, y, 1.5, 3.0] for x in (1.5, 5.5) for y in (1.5, 5.5)]
    geom = L.lbm_geometry_from_list(8, 8, 4, False, spheres)
    assert geom.info()["n_fluid"] == 0
    solver = L.Solver(geom, g=(1e-5, 0, 0))
    solver.step(3)
    assert solver.steps == 3
    rho, u = solver.moments()
    assert float(rho.abs().max()) == 0.0 and float(u.abs().max()) == 0.0
    pa = solver.plane_average()
    assert np.array_equal(pa, np.zeros_like(pa))
    assert solver.populations().numel() == 0


@pytest.mark.parametrize("q", [(0.5, 0.5), (0.3, 0.8)])
def test_one_cell_wide_column(torch_cuda, q):
    """Degenerate box: 1 x 1 x 18 with walls, so every x and y neighbour of a
    cell is the cell itself (periodic wrap onto itself) and the 16 fluid
    cells fill one ragged tile.  Every population after both parities and
    after 300 steps against the oracle, on half-way and off-grid walls."""
    import torch

    g = (2e-5, 1e-5, 0.0)
    geom = L.lbm_geometry_from_list(1, 1, 18, False, [], q_lo=q[0], q_hi=q[1])
    assert geom.info()["n_fluid"] == 16
    u0 = W.velocity_field((18, 1, 1), seed=4, amplitude=1e-2)
    solver = L.Solver(geom, 0.8, 3 / 16, g, u0=torch.from_numpy(u0).cuda())
    lat = O.Lattice(1, 1, 18, False, [], 0.8, 3 / 16, g, q[0], q[1]).init(u0.astype(np.float64))
    fluid = solver.export_lists()["fluid_cell"]
    for n in (1, 1, 298):
        solver.step(n)
        lat.step(n)
        got = solver.populations().cpu().numpy().astype(np.float64)
        want = _oracle_shifted(lat, fluid)
        assert np.max(np.abs(got - want)) <= TOL_U * np.max(np.abs(want)), n


@pytest.mark.parametrize("flags", [L.LBM_FLAG_ROW_NEIGHBOURS, L.LBM_FLAG_STAGED_NEIGHBOURS, L.LBM_FLAG_DERIVED_NEIGHBOURS],
                         ids=["row-neighbours", "staged-neighbours", "derived-neighbours"])
@pytest.mark.parametrize("case", [CASES[2], W.W1, CASES[1]], ids=lambda c: c.name)
def test_odd_step_variants_agree(torch_cuda, flags, case):
    """Neighbour table, row-bitmask neighbours and row words staged per tile
    address the same slots, and every rounding of the collision is explicit:
    the kernels give the same bits (periodic cube with wrap-around rows, the
    W1 channel with dense tiles, a box whose planes hold fewer than a tile)."""
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=5, amplitude=1e-2)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    import torch

    u0t = torch.from_numpy(u0).cuda()
    a = L.Solver(geom, u0=u0t, g=(1e-5, 0, 0), flags=flags)
    b = L.Solver(geom, u0=u0t, g=(1e-5, 0, 0), flags=L.LBM_FLAG_NEIGHBOUR_TABLE)
    a.step(9)
    b.step(9)
    assert torch.equal(a.populations(), b.populations())


@pytest.mark.parametrize("variant", ["simple bounce-back", "SRT", "Lambda 1/4"])
def test_boundary_and_collision_variants(torch_cuda, variant):
    """Forced simple bounce-back (Eq. (noslip) on every link), SRT (TRT with
    Lambda = (tau - 1/2)^2) and Lambda = 1/4 on a sphere packing with off-grid
    walls: every population after 10 steps against the oracle."""
    torch = torch_cuda
    case = CASES[3]
    tau, lam, flags, sbb = case.tau, case.lam, 0, False
    if variant == "simple bounce-back":
        flags, sbb = L.LBM_FLAG_SIMPLE_BOUNCE_BACK, True
    elif variant == "SRT":
        tau = 1.1
        lam = (tau - 0.5) ** 2
    else:
        lam = 0.25
    g = (3e-5, -1e-5, 2e-5)
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=21, amplitude=2e-2)
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    solver = L.Solver(geom, tau, lam, g, u0=torch.from_numpy(u0).cuda(), flags=flags)
    lat = O.Lattice(case.nx, case.ny, case.nz, case.periodic_z, geom.spheres(), tau, lam, g, case.q_lo, case.q_hi,
                    simple_bounce_back=sbb).init(u0.astype(np.float64))
    solver.step(10)
    lat.step(10)
    lists = solver.export_lists()
    got = solver.populations().cpu().numpy().astype(np.float64)
    want = _oracle_shifted(lat, lists["fluid_cell"])
    assert np.max(np.abs(got - want)) <= TOL_U * np.max(np.abs(want))
    if sbb:
        assert lists["link_fallback"].all()
