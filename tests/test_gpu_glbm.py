"""The homogenised porous-medium LBM (Sec. 4, Guo & Zhao's generalised LBM)
on the GPU against its FP64 oracle: every population after 0..7 steps with a
porous layer, Darcy and Forchheimer drag, a body force, a moving lid and a
per-plane relaxation time (nu_eff = nu / eps in the porous layer, the paper's
proposed model); moments and plane averages; the exact uniform porous state;
the converged two-layer Brinkman-Couette profile."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.glbm_oracle import GLBM as OGLBM
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available()
    build()
    L.load_library()
    return torch


def _layered(nx=6, ny=5, nz=12, nu=0.1, eps_p=0.5, K=0.05, c_f=0.3):
    z = np.arange(nz)
    porous = (z >= 1) & (z <= nz // 2 - 1)
    eps = np.where(porous, eps_p, 1.0)
    inv_k = np.where(porous, 1.0 / K, 0.0)
    tau = 3 * nu / eps + 0.5
    return dict(nx=nx, ny=ny, nz=nz, eps=eps, inv_k=inv_k, tau=tau, nu=nu, c_f=c_f)


@pytest.mark.parametrize("nsteps", [0, 1, 2, 7])
def test_populations_match_oracle(torch_cuda, nsteps):
    torch = torch_cuda
    p = _layered()
    g, lid = (2e-5, 0.0, 1e-5), (3e-3, 1e-3, 0.0)
    u0 = W.velocity_field((p["nz"], p["ny"], p["nx"]), seed=40 + nsteps, amplitude=1e-2)
    gpu = L.GLBM(p["nx"], p["ny"], p["nz"], p["eps"], p["inv_k"], p["tau"], p["nu"], p["c_f"], g, u_top=lid,
                 u0=torch.from_numpy(u0).cuda())
    ora = OGLBM(p["nx"], p["ny"], p["nz"], p["eps"], p["inv_k"], p["tau"], p["nu"], p["c_f"], g,
                u_top=lid).init(u0.astype(np.float64))
    gpu.step(nsteps)
    ora.step(nsteps)
    _, w = O.velocity_set()
    want = ora.get_f()[:, 1:-1].reshape(19, -1) - w[:, None]
    got = gpu.populations().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))
    rho, u = gpu.moments()
    rho_o, u_o = ora.moments()
    umax = np.max(np.abs(u_o))
    assert np.max(np.abs(u.cpu().numpy() - u_o)) <= TOL * umax
    assert np.max(np.abs(rho.cpu().numpy() - rho_o)) <= 1e-6
    pa = gpu.plane_average()
    assert np.max(np.abs(pa - ora.plane_average())) <= TOL * umax


def test_uniform_porous_state(torch_cuda):
    """Periodic box: (nu/K) u + (c_F/sqrt K) u^2 = G."""
    tau, eps, K, c_f, G = 0.9, 0.45, 0.02, 0.4, 2e-4
    nu = (tau - 0.5) / 3
    gpu = L.GLBM(8, 8, 8, eps, 1 / K, tau, nu, c_f, (G, 0.0, 0.0), periodic_z=True)
    gpu.step(3000)
    _, u = gpu.moments()
    a, b = c_f / math.sqrt(K), nu / K
    want = (-b + math.sqrt(b * b + 4 * a * G)) / (2 * a)
    ux = u[0].cpu().numpy()
    assert np.max(np.abs(ux / want - 1)) < 1e-5
    assert float(u[1:].abs().max()) < 1e-9


def test_brinkman_couette_converged(torch_cuda):
    """Steady two-layer Couette (porous lower half, lid on top) against the
    oracle's converged profile on the same grid."""
    L_, tau, eps, da, U = 16, 1.5, 0.5, 0.01, 1e-3
    nz, h = L_ + 2, L_ / 2
    K, nu = da * h * h, (tau - 0.5) / 3
    z = np.arange(nz)
    porous = (z >= 1) & (z <= L_ // 2)
    eps_z, inv_k = np.where(porous, eps, 1.0), np.where(porous, 1.0 / K, 0.0)
    gpu = L.GLBM(4, 4, nz, eps_z, inv_k, tau, nu, u_top=(U, 0.0, 0.0))
    ora = OGLBM(1, 1, nz, eps_z, inv_k, tau, nu, u_top=(U, 0.0, 0.0)).init()
    gpu.step(40 * L_ * L_)
    ora.step(40 * L_ * L_)
    want = ora.plane_average()[1:-1]
    got = gpu.plane_average()[1:-1]
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(want)
