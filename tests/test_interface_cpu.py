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
