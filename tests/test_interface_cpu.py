"""Two-domain interface evaluation (Sec. 3.2): the analytic profiles satisfy
their interface conditions (Eqs. (BJ), (BJS), (OTW), (Br)) and limits, and
fitting them recovers the parameters they were built with."""
import numpy as np
import pytest

from paper_1507_06565_gb300 import interface as I

Z = np.arange(0.0, 256.0) + 0.5     # plane centres
ZI, ZT, NU, G = 128.0, 254.5, 0.1, 1e-6


@pytest.mark.parametrize("alpha", [0.1, 0.3163, 2.0])
def test_bj_profile_and_fit(alpha):
    K = 3.0
    u = I.profile_bj(Z, ZI, ZT, K, NU, G, alpha)
    u_m = G * K / NU
    # the condition itself, from the profile by differences
    h = 1e-4
    du = (I.profile_bj(ZI + h, ZI, ZT, K, NU, G, alpha) - I.profile_bj(ZI, ZI, ZT, K, NU, G, alpha)) / h
    us = float(I.profile_bj(ZI, ZI, ZT, K, NU, G, alpha))
    assert du == pytest.approx(alpha / np.sqrt(K) * (us - u_m), rel=1e-3)
    assert float(I.profile_bj(ZT, ZI, ZT, K, NU, G, alpha)) == pytest.approx(0.0, abs=1e-15)
    f = I.fit_interface(Z, u, ZI, K, NU)
    assert f.alpha_bj == pytest.approx(alpha, rel=1e-8)
    assert f.u_m == pytest.approx(u_m, rel=1e-12)


def test_bjs_profile_and_fit():
    K, alpha = 1.5, 0.5
    u = I.profile_bj(Z, ZI, ZT, K, NU, G, alpha, saffman=True)
    f = I.fit_interface(Z, u, ZI, K, NU)
    assert f.alpha_bjs == pytest.approx(alpha, rel=1e-8)


def test_bj_limits():
    """alpha -> infinity: no slip relative to the seepage velocity; alpha -> 0:
    no shear at the interface, the free layer's Poiseuille maximum."""
    K = 2.0
    L = ZT - ZI
    big = I.profile_bj(np.array([ZI]), ZI, ZT, K, NU, G, 1e9)[0]
    assert big == pytest.approx(G * K / NU, rel=1e-6)
    small = I.profile_bj(np.array([ZI]), ZI, ZT, K, NU, G, 1e-12)[0]
    assert small == pytest.approx(0.5 * G / NU * L * L, rel=1e-9)


@pytest.mark.parametrize("beta,j", [(-0.8, 1 / 0.6), (0.0, 1.0), (0.4, 2.0)])
def test_otw_profile_and_fit(beta, j):
    K = 2.0
    nu_eff = j * NU
    u = I.profile_otw(Z, ZI, ZT, K, NU, nu_eff, G, beta)
    f = I.fit_interface(Z, u, ZI, K, NU, nu_eff=nu_eff, u_m=G * K / NU)
    assert f.beta_otw == pytest.approx(beta, abs=1e-7)
    # velocity continuous, porous side decays to the Darcy velocity
    assert f.u_s == pytest.approx(float(I.profile_otw(ZI - 1e-9, ZI, ZT, K, NU, nu_eff, G, beta)), rel=1e-6)
    assert float(u[0]) == pytest.approx(G * K / NU, rel=1e-6)


def test_interface_position():
    eps = np.concatenate([np.full(100, 0.6), [0.8, 0.95], np.ones(50)])
    z = np.arange(eps.size, dtype=float)
    assert I.interface_position(z, eps) == 102.0


@pytest.mark.parametrize("K,eps", [(3.0, 0.6), (0.4, 0.35), (25.0, 0.9)])
def test_brinkman_layer_profile_satisfies_its_problem(K, eps):
    """The two-layer Brinkman profile solves its ODEs (second differences on
    a fine grid), meets both walls, and is continuous in u and in stress
    (nu_eff u' = nu u') at the interface."""
    nu, g = 0.1, 1e-6
    zb, zi, zt = 0.5, 40.0, 80.0
    nu_e = nu / eps
    u = lambda z: I.profile_brinkman_layer(z, zb, zi, zt, K, eps, nu, g)
    h = 1e-3
    for z in np.linspace(zb + 0.5, zi - 0.5, 7):
        d2 = (u(z + h) - 2 * u(z) + u(z - h)) / h ** 2
        assert abs(nu_e * d2 - eps * nu / K * u(z) + eps * g) < 1e-6 * eps * g
    for z in np.linspace(zi + 0.5, zt - 0.5, 7):
        d2 = (u(z + h) - 2 * u(z) + u(z - h)) / h ** 2
        assert abs(nu * d2 + g) < 1e-6 * g
    umax = float(np.max(u(np.linspace(zb, zt, 801))))
    assert abs(float(u(zb))) < 1e-12 * umax and abs(float(u(zt))) < 1e-12 * umax
    d = 1e-7
    assert abs(float(u(zi - d)) - float(u(zi + d))) < 1e-6 * umax
    # second-order one-sided differences on each side of the interface
    a, b = zi - d, zi + d
    s_below = nu_e * (3 * float(u(a)) - 4 * float(u(a - h)) + float(u(a - 2 * h))) / (2 * h)
    s_above = nu * (-3 * float(u(b)) + 4 * float(u(b + h)) - float(u(b + 2 * h))) / (2 * h)
    assert abs(s_below - s_above) < 1e-5 * abs(s_above)


def test_brinkman_layer_limits():
    """No drag (K -> infinity, eps = 1, nu_eff = nu): plane Poiseuille flow
    between the walls.  Vanishing permeability: the porous layer is at rest
    and the free layer is Poiseuille flow between the interface and the top
    wall."""
    nu, g = 0.1, 1e-6
    zb, zi, zt = 0.5, 30.0, 70.0
    z = np.linspace(zb, zt, 281)
    u = I.profile_brinkman_layer(z, zb, zi, zt, 1e12, 1.0, nu, g, nu_eff=nu)
    want = 0.5 * g / nu * (z - zb) * (zt - z)
    assert np.max(np.abs(u - want)) < 1e-6 * np.max(want)
    u0 = I.profile_brinkman_layer(z, zb, zi, zt, 1e-10, 0.5, nu, g)
    want0 = np.where(z >= zi, 0.5 * g / nu * (z - zi) * (zt - z), 0.0)
    assert np.max(np.abs(u0 - want0)) < 1e-4 * np.max(want0)
