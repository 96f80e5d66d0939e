"""Two-domain interface evaluation (Sec. 3.2): interface parameters from a
plane-averaged velocity profile of free flow over a porous layer, and the
analytic two-domain profiles they define.

Host-side post-processing of a converged profile (the plane averages of
lbm_plane_average); no GPU work.

Setting: a channel driven by a body force g (per unit mass), viscosity nu,
porous layer below the interface z_i, free flow above it up to a no-slip wall
at z_top.  With U_s the velocity at the interface, dU/dz|+ and dU/dz|- the
gradients on the free and porous sides, U_m the seepage velocity far inside
the porous layer and K its permeability:

  Eq. (BJ):   dU/dz|+ = alpha / sqrt(K) (U_s - U_m)
  Eq. (BJS):  dU/dz|+ = alpha / sqrt(K) U_s          (Saffman: U_m dropped)
  Eq. (OTW):  nu_eff dU/dz|- - nu dU/dz|+ = beta nu / sqrt(K) U_s

(the conditions of Sec. 1).  As in Sec. 3.2, the free-side gradient comes
from a quadratic fitted to the profile above the interface and the
porous-side one from an exponential, here U_m + A exp(r (z - z_i)), fitted
below it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class InterfaceFit:
    z_int: float
    u_s: float           # U at the interface
    du_free: float       # dU/dz at z_int+ (quadratic fit)
    du_porous: float     # dU/dz at z_int- (exponential fit)
    u_m: float           # seepage velocity far inside the porous layer
    alpha_bj: float
    alpha_bjs: float
    beta_otw: float


def interface_position(z, eps, tol=1e-3) -> float:
    """The first plane, going up from the porous layer, whose porosity is 1
    (within tol) -- the paper's first choice of the interface position."""
    z = np.asarray(z, float)
    eps = np.asarray(eps, float)
    solid_seen = np.flatnonzero(eps < 1.0 - tol)
    if solid_seen.size == 0:
        raise ValueError("no porous plane")
    return float(z[solid_seen.max() + 1])


def fit_interface(z, u, z_int, K, nu, nu_eff=None, u_m=None, free_cells=12, porous_cells=8) -> InterfaceFit:
    """Interface parameters from a profile u(z) (superficial velocity).
    free_cells / porous_cells: planes fitted on each side; u_m (seepage
    velocity) defaults to the mean of u over the lower half of the porous
    planes below z_int; nu_eff defaults to nu."""
    z = np.asarray(z, float)
    u = np.asarray(u, float)
    nu_eff = nu if nu_eff is None else nu_eff
    above = (z >= z_int) & (z < z_int + free_cells)
    p = np.polyfit(z[above] - z_int, u[above], 2)
    u_s = float(p[2])
    du_free = float(p[1])
    if u_m is None:
        deep = (z < z_int) & (z >= z[0] + 1)
        zd = z[deep]
        u_m = float(np.mean(u[deep][zd < np.median(zd)]))
    below = (z < z_int) & (z >= z_int - porous_cells)
    d = u[below] - u_m
    zb = z[below] - z_int
    pos = d > 0
    if np.max(np.abs(d)) <= 1e-12 * abs(u_s):
        du_porous = 0.0   # a flat (Darcy) porous side
    elif pos.sum() >= 3:
        # log-linear fit of the decaying part, ln(u - u_m) = ln A + r (z - z_i),
        # over the planes above the seepage velocity (a pore-scale profile
        # fluctuates with the plane porosity)
        r, ln_a = np.polyfit(zb[pos], np.log(d[pos]), 1)
        du_porous = float(np.exp(ln_a) * r)
    else:
        du_porous = float("nan")
    sk = np.sqrt(K)
    return InterfaceFit(z_int, u_s, du_free, du_porous, u_m,
                        alpha_bj=float(sk * du_free / (u_s - u_m)),
                        alpha_bjs=float(sk * du_free / u_s),
                        beta_otw=float(sk * (nu_eff * du_porous - nu * du_free) / (nu * u_s)))


# ---------------------------------------------------------------------------
# analytic two-domain profiles (Stokes above, Darcy or Brinkman below)
# ---------------------------------------------------------------------------
def _free(z, z_int, u_s, du, g, nu):
    s = z - z_int
    return u_s + du * s - 0.5 * g / nu * s * s


def profile_bj(z, z_int, z_top, K, nu, g, alpha, saffman=False):
    """Stokes flow above the interface, Darcy below (U = U_m = g K / nu), the
    BJ (or, with saffman, BJS) condition at z_int, no slip at z_top."""
    z = np.asarray(z, float)
    L = z_top - z_int
    u_m = g * K / nu
    c = alpha / np.sqrt(K)
    # u_s + du L = g L^2 / (2 nu);  du = c (u_s - u_m)  (BJS: du = c u_s)
    rhs = 0.5 * g / nu * L * L
    u_s = (rhs + (0.0 if saffman else c * u_m * L)) / (1.0 + c * L)
    du = c * (u_s - (0.0 if saffman else u_m))
    return np.where(z >= z_int, _free(z, z_int, u_s, du, g, nu), u_m)


def profile_otw(z, z_int, z_top, K, nu, nu_eff, g, beta):
    """Stokes flow above, Brinkman below (U = U_m + A exp(r (z - z_i)),
    r = sqrt(nu / (nu_eff K)), a deep porous layer), continuous velocity and
    the OTW stress jump at z_int, no slip at z_top.  beta = 0 is the
    Brinkman model with continuous stress (Eq. (Br))."""
    z = np.asarray(z, float)
    L = z_top - z_int
    u_m = g * K / nu
    r = np.sqrt(nu / (nu_eff * K))
    # unknowns A, du:  (u_m + A) + du L = g L^2/(2 nu)
    #                  nu_eff A r - nu du = beta nu / sqrt(K) (u_m + A)
    M = np.array([[1.0, L], [nu_eff * r - beta * nu / np.sqrt(K), -nu]])
    b = np.array([0.5 * g / nu * L * L - u_m, beta * nu / np.sqrt(K) * u_m])
    A, du = np.linalg.solve(M, b)
    return np.where(z >= z_int, _free(z, z_int, u_m + A, du, g, nu), u_m + A * np.exp(r * (z - z_int)))


def profile_brinkman_layer(z, z_bot, z_int, z_top, K, eps, nu, g, nu_eff=None):
    """Single-domain Brinkman profile of a channel with a porous layer
    (Eq. (Br) with the drag of Eq. (PorousForce), Stokes regime): in the
    porous layer z_bot < z < z_int

        nu_eff u'' - (eps nu / K) u + eps g = 0,

    in the free layer z_int < z < z_top  nu u'' + g = 0; no slip at the walls
    z_bot and z_top; u and the shear stress (nu_eff u' below, nu u' above)
    continuous at z_int.  u is the superficial velocity; nu_eff defaults to
    nu / eps (Sec. 4's choice).  The porous solution is the Darcy velocity
    g K / nu plus exponentials of rate r = sqrt(eps nu / (K nu_eff)), written
    as e^{r (z - z_int)} and e^{-r (z - z_bot)} so that both stay <= 1 in the
    layer and the 4 x 4 system for their amplitudes and the free parabola's
    two coefficients stays well conditioned."""
    z = np.asarray(z, float)
    nu_e = nu / eps if nu_eff is None else nu_eff
    r = np.sqrt(eps * nu / (K * nu_e))
    u_d = g * K / nu
    H = z_int - z_bot
    Lf = z_top - z_int
    e_h = np.exp(-r * H)
    # unknowns A, B (porous), C, D (free: u = -g/(2 nu) s^2 + C s + D, s = z - z_int)
    M = np.array([[e_h, 1.0, 0.0, 0.0],                    # u(z_bot) = 0
                  [0.0, 0.0, Lf, 1.0],                     # u(z_top) = 0
                  [1.0, e_h, 0.0, -1.0],                   # u continuous at z_int
                  [nu_e * r, -nu_e * r * e_h, -nu, 0.0]])  # stress continuous at z_int
    b = np.array([-u_d, 0.5 * g / nu * Lf * Lf, -u_d, 0.0])
    A, B, C, D = np.linalg.solve(M, b)
    s = z - z_int
    porous = u_d + A * np.exp(r * np.minimum(s, 0.0)) + B * np.exp(-r * np.maximum(z - z_bot, 0.0))
    free = -0.5 * g / nu * s * s + C * s + D
    return np.where(z >= z_int, free, porous)
