"""Pins of the FP64 numpy oracle of the learned warm start: finite differences
for every gradient, adjointness of the resampling operators, a brute-force
convolution written with scalar loops, closed forms for Adam's first step and
for the signed distance, and bf16 rounding of known values."""
import math

import numpy as np
import pytest

from oracle import unet_oracle as U


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 1.0 + 2 ** -7, 3.0e-39, 65504.0])
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1;
    # 1 + 3 2^-9 rounds up to 1 + 2^-7
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, -2.5, 1.0 + 2 ** -7, U.bf16(3.0e-39)[()], 65536.0])
    assert np.array_equal(U.bf16(vals)[:5], want[:5])
    assert U.bf16(65504.0) == 65536.0          # 8-bit significand
    assert abs(U.bf16(math.pi) - math.pi) <= 2 ** -8 * math.pi


def test_shift_and_resampling_adjoints():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 6, 4, 8))
    y = rng.standard_normal((3, 6, 4, 8))
    for off in U.TAPS:
        assert abs(np.sum(U.shift(x, *off) * y) - np.sum(x * U.unshift(y, *off))) < 1e-12
    yp = rng.standard_normal((3, 3, 2, 4))
    assert abs(np.sum(U.pool(x) * yp) - np.sum(x * U.upsample(yp) / 8.0)) < 1e-12


def _conv_brute(x, w, b):
    c, nz, ny, nx = x.shape
    co = w.shape[1]
    out = np.zeros((co, nz, ny, nx))
    for o in range(co):
        for z in range(nz):
            for y in range(ny):
                for xx in range(nx):
                    s = b[o]
                    for t, (dz, dy, dx) in enumerate(U.TAPS):
                        zz = z + dz
                        if zz < 0 or zz >= nz:
                            continue
                        s += np.dot(w[t, o], x[:, zz, (y + dy) % ny, (xx + dx) % nx])
                    out[o, z, y, xx] = s
    return out


def test_conv_matches_scalar_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 3, 5))
    w = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(3)
    assert np.allclose(U.conv3(x, w, b), _conv_brute(x, w, b), atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 3, 4))
    w = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(3)
    gout = rng.standard_normal((3, 4, 3, 4))
    f = lambda x_, w_, b_: np.sum(U.conv3(x_, w_, b_) * gout)
    dx, dw, db = U.conv3_backward(x, w, gout)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (1, 3, 2, 1), (0, 2, 1, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        assert abs((f(xp, w, b) - f(xm, w, b)) / (2 * eps) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0), (13, 2, 1), (26, 1, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        assert abs((f(x, wp, b) - f(x, wm, b)) / (2 * eps) - dw[idx]) < 1e-6
    assert np.allclose(db, gout.sum(axis=(1, 2, 3)))


def test_unet_gradients_finite_differences():
    """Every parameter group of a narrow U-Net against central differences of
    the loss (fp64, no rounding)."""
    widths = (2, 3, 3, 4)
    rng = np.random.default_rng(3)
    p = U.init_params(7, widths=widths, c_in=2)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((2, 8, 8, 8))
    target = rng.standard_normal((3, 8, 8, 8))
    net = U.UNet(p, widths=widths)
    net.loss(net.forward(x), target)
    g = net.backward(target)

    def loss_at(params):
        n2 = U.UNet(params, widths=widths)
        return n2.loss(n2.forward(x), target)

    eps = 1e-6
    checked = 0
    for k in sorted(p):
        flat = p[k].reshape(-1)
        for j in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            pp = {kk: v.copy() for kk, v in p.items()}
            pm = {kk: v.copy() for kk, v in p.items()}
            pp[k].reshape(-1)[j] += eps
            pm[k].reshape(-1)[j] -= eps
            fd = (loss_at(pp) - loss_at(pm)) / (2 * eps)
            an = g[k].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, j, fd, an)
            checked += 1
    assert checked > 40


def test_adam_first_step_closed_form():
    """After one step the bias-corrected moments are g and g^2, so every
    parameter moves by lr * g / (|g| + eps)."""
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -1e-3, 4.0])}
    st = {}
    U.adam(p, g, st, lr=1e-2)
    assert np.allclose(p["a"], np.array([1.0, -2.0, 0.5]) - 1e-2 * g["a"] / (np.abs(g["a"]) + 1e-8), atol=1e-15)


def test_sdf_closed_forms():
    nx = ny = 16
    nz = 20
    sp = [[8.0, 8.0, 10.0, 3.0]]
    d = U.sdf(nx, ny, nz, False, sp, trunc=8.0)
    # centre of the sphere: -r, clipped distance -3/8
    assert abs(d[10, 8, 8] - (-3.0 / 8.0)) < 1e-15
    # a cell 5 along x from the centre: 5 - 3 = 2
    assert abs(d[10, 8, 13] - 2.0 / 8.0) < 1e-15
    # next to the bottom wall (plane z = 0.5): z = 1 is 0.5 away
    assert abs(d[1, 0, 0] - 0.5 / 8.0) < 1e-15
    # wall layer itself is inside the solid
    assert d[0, 3, 3] < 0
    # periodic image: sphere near x = 0 is seen from x = 15
    d2 = U.sdf(nx, ny, nz, True, [[0.5, 8.0, 10.0, 2.0]], trunc=8.0)
    assert abs(d2[10, 8, 15] - (1.5 - 2.0) / 8.0) < 1e-15
    assert np.all(np.abs(d2) <= 1.0)
