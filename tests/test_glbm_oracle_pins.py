"""Pins of the FP64 oracle of the homogenised porous-medium LBM (Sec. 4,
Eqs. (GeneralizedPor1)-(PorousForce), the generalised LBM of Guo & Zhao):
an exact uniform steady state balancing Darcy and Forchheimer drag against
the body force, the exact linear Couette profile of free fluid, the exact
two-layer Brinkman-Couette profile (Sec. 4's Couette test, solved without
the paper's low-Da approximation) approached at second order under grid
refinement, and mass conservation with a moving wall."""
import math

import numpy as np
import pytest

from oracle.glbm_oracle import GLBM


def test_equilibrium_and_source_moments():
    """The moments that define Guo & Zhao's scheme: sum f^eq = rho,
    sum e f^eq = rho u, sum e e f^eq = rho I / 3 + rho u u / eps; sum F_k = 0,
    sum e F_k = (1 - 1/(2 tau)) rho F, sum e e F_k = (1 - 1/(2 tau)) rho
    (u F + F u) / eps."""
    rng = np.random.default_rng(0)
    eps, tau = rng.uniform(0.3, 1.0, 4), rng.uniform(0.6, 1.5, 4)
    lat = GLBM(2, 3, 4, eps, 0.0, tau, 0.1)
    rho = 1 + 0.1 * rng.standard_normal((4, 3, 2))
    u = 0.05 * rng.standard_normal((3, 4, 3, 2))
    F = 1e-3 * rng.standard_normal((3, 4, 3, 2))
    e = lat.e
    ep, tp = eps[:, None, None], tau[:, None, None]
    feq, src = lat.equilibrium(rho, u), lat.source(rho, u, F)
    assert np.allclose(feq.sum(0), rho, atol=1e-14)
    assert np.allclose(np.einsum("kd,kzyx->dzyx", e, feq), rho * u, atol=1e-15)
    pi = np.einsum("ka,kb,kzyx->abzyx", e, e, feq)
    want = rho * np.eye(3)[:, :, None, None, None] / 3 + rho * np.einsum("azyx,bzyx->abzyx", u, u) / ep
    assert np.allclose(pi, want, atol=1e-14)
    c = 1 - 0.5 / tp
    assert np.allclose(src.sum(0), 0, atol=1e-17)
    assert np.allclose(np.einsum("kd,kzyx->dzyx", e, src), c * rho * F, atol=1e-17)
    uf = np.einsum("azyx,bzyx->abzyx", u, F)
    assert np.allclose(np.einsum("ka,kb,kzyx->abzyx", e, e, src), c * rho * (uf + uf.transpose(1, 0, 2, 3, 4)) / ep,
                       atol=1e-17)


def test_uniform_porous_steady_state_exact():
    """Periodic box, uniform medium: the steady velocity u solves
    (nu / K) u + (c_F / sqrt(K)) u^2 = G (Eq. (PorousForce) with F = 0); the
    uniform equilibrium at that u is an exact fixed point of the scheme."""
    tau, eps, K, c_f, G = 0.9, 0.45, 0.02, 0.4, 2e-4
    nu = (tau - 0.5) / 3
    lat = GLBM(3, 3, 3, eps, 1 / K, tau, nu, c_f, (G, 0.0, 0.0), periodic_z=True).init()
    lat.step(3000)
    _, u = lat.moments()
    a, b = c_f / math.sqrt(K), nu / K
    want = (-b + math.sqrt(b * b + 4 * a * G)) / (2 * a)
    assert np.allclose(u[0], want, rtol=1e-12, atol=0)
    assert np.max(np.abs(u[1:])) < 1e-15
    # Darcy only: u = G K / nu
    lat = GLBM(3, 3, 3, eps, 1 / K, tau, nu, 0.0, (G, 0.0, 0.0), periodic_z=True).init()
    lat.step(3000)
    _, u = lat.moments()
    assert np.allclose(u[0], G * K / nu, rtol=1e-12, atol=0)


def test_free_couette_linear_profile_exact():
    """eps = 1, no porous drag: bounce-back walls half-way, lid moving at U:
    u(z) = U (z - 1/2) / (nz - 2) exactly."""
    nz, tau, U = 12, 1.2, 1e-3
    lat = GLBM(1, 1, nz, 1.0, 0.0, tau, (tau - 0.5) / 3, u_top=(U, 0.0, 0.0)).init()
    lat.step(6000)
    _, u = lat.moments()
    z = np.arange(1, nz - 1)
    assert np.max(np.abs(u[0, 1:-1, 0, 0] - U * (z - 0.5) / (nz - 2))) < 1e-12 * U


def _brinkman_couette(L, tau=1.5, eps=0.5, da=0.01, U=1e-3, steps=None):
    """Lower half (cells z = 1..L/2) porous, upper half free, lid at the top;
    nu_eff = nu everywhere.  Exact: porous u = A sinh(r y), free u = B + C (y -
    h), y = z - 1/2, h = L/2, r = sqrt(eps / K), u and u' continuous."""
    nz = L + 2
    h = L / 2
    K = da * h * h
    nu = (tau - 0.5) / 3
    z = np.arange(nz)
    eps_z = np.where((z >= 1) & (z <= L // 2), eps, 1.0)
    inv_k = np.where((z >= 1) & (z <= L // 2), 1.0 / K, 0.0)
    lat = GLBM(1, 1, nz, eps_z, inv_k, tau, nu, u_top=(U, 0.0, 0.0))
    r = math.sqrt(eps / K)
    A = U / (math.sinh(r * h) + r * math.cosh(r * h) * (L - h))
    y = z[1:-1] - 0.5
    exact = np.where(y < h, A * np.sinh(r * y), A * math.sinh(r * h) + A * r * math.cosh(r * h) * (y - h))
    u0 = np.zeros((3, nz, 1, 1))
    u0[0, 1:-1, 0, 0] = exact
    lat.init(u0)
    lat.step(steps or 40 * L * L)
    _, u = lat.moments()
    return u[0, 1:-1, 0, 0], exact, lat


def test_brinkman_couette_second_order():
    """The largest error sits in the first free cell above the interface; it
    falls by 3.0, 3.6, 3.9 per halving from L = 8 to 64 (measured): second
    order, approached from below."""
    errs = []
    for L in (8, 16, 32):
        got, exact, _ = _brinkman_couette(L)
        errs.append(np.max(np.abs(got - exact)) / np.max(exact))
    assert errs[2] < 8e-3, errs
    assert 2.8 < errs[0] / errs[1] < 4.5 and 3.3 < errs[1] / errs[2] < 4.5, errs


def test_mass_conserved_with_moving_wall():
    _, _, lat = _brinkman_couette(8, steps=1)
    m0 = lat.get_f().sum()
    lat.step(200)
    assert abs(lat.get_f().sum() - m0) < 1e-12 * m0
