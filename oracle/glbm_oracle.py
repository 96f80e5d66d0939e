"""FP64 oracle of the homogenised porous-medium LBM (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module;
the library never does.

Sec. 4 of the paper compares the pore-scale solution with the generalised
lattice Boltzmann model (GLBM) of Guo & Zhao (2002), whose macroscopic form is
Eqs. (GeneralizedPor1), (GeneralizedPor2) with the porous-medium force of
Eq. (PorousForce):  F = -(eps nu / K) u - (eps c_F / sqrt(K)) |u| u + eps G.
The paper prints no discrete scheme; this oracle takes Guo & Zhao's, written
out here in plain numpy on a dense box, two arrays, collide then stream:

  rho = sum_k f_k,  v = sum_k e_k f_k / rho + eps G / 2,
  u   = v / (c0 + sqrt(c0^2 + c1 |v|)),
        c0 = (1 + eps nu / (2 K)) / 2,  c1 = eps c_F / (2 sqrt(K))
        (the solution of u = sum e f / rho + F(u) / 2 for this F),
  F   = -(eps nu / K) u - (eps c_F / sqrt(K)) |u| u + eps G,
  f_k^eq = w_k rho (1 + 3 e.u + 9/2 (e.u)^2 / eps - 3/2 u.u / eps),
  F_k = w_k rho (1 - 1/(2 tau)) (3 e.F + 9 (e.u)(e.F) / eps - 3 u.F / eps),
  f_k(x + e_k, t + 1) = f_k - (f_k - f_k^eq) / tau + F_k,
  nu_eff = (tau - 1/2) / 3.

eps, 1/K, tau (hence nu_eff) vary with z; 1/K = 0 is free fluid.  The box is
periodic in x and y; the layers z = 0 and nz - 1 are walls at which every link
bounces back half-way, a moving wall adding -6 w_k rho (e_k . u_wall) to the
returning population (rho of the fluid node).  When periodic_z is set there
are no walls.  Fields are [.., nz, ny, nx].
"""
from __future__ import annotations

import numpy as np

from . import opposite, velocity_set


class GLBM:
    def __init__(self, nx, ny, nz, eps, inv_k, tau, nu, c_f=0.0, g=(0.0, 0.0, 0.0), u_bottom=(0.0, 0.0, 0.0),
                 u_top=(0.0, 0.0, 0.0), periodic_z=False):
        e, w = velocity_set()
        self.e = e.astype(np.float64)
        self.w = w
        self.opp = np.array([opposite(k) for k in range(19)])
        self.shape = (nz, ny, nx)
        self.periodic_z = periodic_z
        col = lambda a: np.broadcast_to(np.asarray(a, np.float64).reshape(-1), (nz,)).reshape(nz, 1, 1).copy()
        self.eps, self.inv_k, self.tau = col(eps), col(inv_k), col(tau)
        self.nu, self.c_f = float(nu), float(c_f)
        self.g = np.asarray(g, np.float64)
        self.u_wall = (np.asarray(u_bottom, np.float64), np.asarray(u_top, np.float64))
        self.f = np.zeros((19,) + self.shape)
        self.fluid = np.ones(self.shape, bool)
        if not periodic_z:
            self.fluid[0] = False
            self.fluid[-1] = False

    # -- macroscopic quantities (Guo & Zhao's implicit velocity) --
    def moments(self, f=None):
        f = self.f if f is None else f
        rho = f.sum(axis=0)
        j = np.einsum("kd,kzyx->dzyx", self.e, f)
        v = j / np.where(rho > 0, rho, 1.0) + 0.5 * self.eps[None] * self.g[:, None, None, None]
        c0 = 0.5 * (1.0 + 0.5 * self.eps * self.nu * self.inv_k)
        c1 = 0.5 * self.eps * self.c_f * np.sqrt(self.inv_k)
        vn = np.sqrt((v ** 2).sum(axis=0))
        u = v / (c0 + np.sqrt(c0 ** 2 + c1 * vn))[None]
        u[:, ~self.fluid] = 0.0
        rho = np.where(self.fluid, rho, 0.0)
        return rho, u

    def force(self, u):
        un = np.sqrt((u ** 2).sum(axis=0))
        return (-(self.eps * self.nu * self.inv_k)[None] * u
                - (self.eps * self.c_f * np.sqrt(self.inv_k))[None] * un[None] * u
                + self.eps[None] * self.g[:, None, None, None])

    def equilibrium(self, rho, u):
        eu = np.einsum("kd,dzyx->kzyx", self.e, u)
        uu = (u ** 2).sum(axis=0)
        return self.w[:, None, None, None] * rho[None] * (1.0 + 3.0 * eu + 4.5 * eu ** 2 / self.eps[None]
                                                          - 1.5 * uu[None] / self.eps[None])

    def source(self, rho, u, F):
        """F_k = w_k rho (1 - 1/(2 tau)) (3 e.F + 9 (e.u)(e.F) / eps - 3 u.F / eps)."""
        eu = np.einsum("kd,dzyx->kzyx", self.e, u)
        eF = np.einsum("kd,dzyx->kzyx", self.e, F)
        uF = (u * F).sum(axis=0)
        return self.w[:, None, None, None] * rho[None] * (1.0 - 0.5 / self.tau[None]) * (
            3.0 * eF + 9.0 * eu * eF / self.eps[None] - 3.0 * uF[None] / self.eps[None])

    def init(self, u0=None, rho0=1.0):
        """f = f^eq(rho0, u0) in the fluid (u0 [3, nz, ny, nx] or None)."""
        u = np.zeros((3,) + self.shape) if u0 is None else np.asarray(u0, np.float64).reshape((3,) + self.shape)
        rho = np.full(self.shape, rho0)
        self.f = self.equilibrium(rho, u) * self.fluid[None]
        return self

    def step(self, n=1):
        e, w, opp = self.e, self.w, self.opp
        for _ in range(n):
            rho, u = self.moments()
            F = self.force(u)
            feq = self.equilibrium(rho, u)
            src = self.source(rho, u, F)
            post = (self.f - (self.f - feq) / self.tau[None] + src) * self.fluid[None]
            new = np.zeros_like(self.f)
            for k in range(19):
                ex, ey, ez = (int(c) for c in e[k])
                new[k] = np.roll(post[k], shift=(ez, ey, ex), axis=(0, 1, 2))
            if not self.periodic_z:
                # links into the wall layers return to their node, with the
                # moving-wall term
                for k in range(1, 19):
                    ez = int(e[k, 2])
                    if ez == 0:
                        continue
                    zf = self.shape[0] - 2 if ez > 0 else 1     # fluid layer next to that wall
                    uw = self.u_wall[1] if ez > 0 else self.u_wall[0]
                    corr = 6.0 * w[k] * rho[zf] * float(e[k] @ uw)
                    new[opp[k], zf] = post[k, zf] - corr
            new *= self.fluid[None]
            self.f = new

    def get_f(self):
        return self.f.copy()

    def plane_average(self):
        """[nz]: mean stream-wise velocity of each plane (fluid planes)."""
        _, u = self.moments()
        return u[0].mean(axis=(1, 2))
