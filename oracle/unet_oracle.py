"""FP64 numpy oracle of the learned warm start (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may use this module; it shares no code with the CUDA library.

The paper has no learned component: the warm start is an addition that feeds
the LBM of Sec. 2 a better initial velocity (Eq. (equilibrium) evaluated at a
predicted u0), and the converged LBM stays the arbiter of its error.  This file
states, plainly and slowly, what the GPU kernels compute:

* ``sdf``: truncated signed distance to the solid (spheres of the packing and
  the channel walls), negative inside solids, divided by the truncation T and
  clipped to [-1, 1].
* ``UNet``: a 3-D convolutional U-Net (Ronneberger et al. 2015, in 3-D) on
  fields laid out [C, nz, ny, nx]:
    enc1  conv(16->16) relu conv(16->16) relu          (full resolution)
    pool  2x2x2 average
    enc2  conv(16->32) relu conv(32->32) relu
    pool
    enc3  conv(32->64) relu conv(64->64) relu
    pool
    bott  conv(64->128) relu conv(128->128) relu
    up    nearest x2, concat [up, skip]
    dec3  conv(192->64) relu conv(64->64) relu
    up, concat
    dec2  conv(96->32) relu conv(32->32) relu
    up, concat
    dec1  conv(48->16) relu conv(16->16) relu
    head  1x1x1 conv(16->3) + bias
  Every 3x3x3 convolution has a bias and pads circularly in x and y (the
  periodic directions of the channel) and with zeros in z (the walls).  The
  input has 16 channels: [sdf, z feature, 14 zero channels].
* ``backward``: gradients of the mean squared error by the chain rule, layer
  by layer in reverse (no automatic differentiation).
* ``adam``: Kingma & Ba (2015) with bias correction.
* ``bf16``: round-to-nearest-even to bfloat16 (the GPU stores activations,
  activation gradients and weight copies in bf16 and accumulates in fp32);
  when enabled, the forward and backward passes round weights and every
  stored activation and activation gradient the same way.

Weights are [27][C_out][C_in] per 3x3x3 layer (tap t = 9 (dz+1) + 3 (dy+1) +
(dx+1)), [C_out][C_in] for the head.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (16, 32, 64, 128)
C_IN = 16
C_OUT = 3
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16(a):
    """Round float64 values to bfloat16 (via float32, round to nearest even)."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Signed distance field
# ---------------------------------------------------------------------------
def sdf(nx, ny, nz, periodic_z, spheres, trunc, q_lo=0.5, q_hi=0.5):
    """Truncated signed distance / trunc in [-1, 1], shape [nz, ny, nx].
    Spheres: every periodic image; walls (when z is not periodic): the planes
    z = 1 - q_lo and z = nz - 2 + q_hi bounding the fluid."""
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    d = np.full((nz, ny, nx), np.inf)
    if not periodic_z:
        d = np.minimum(z - (1.0 - q_lo), (nz - 2 + q_hi) - z)
    mzs = (-1, 0, 1) if periodic_z else (0,)
    for cx, cy, cz, r in np.asarray(spheres, np.float64).reshape(-1, 4):
        for mx in (-1, 0, 1):
            for my in (-1, 0, 1):
                for mz in mzs:
                    dist = np.sqrt((x - cx - mx * nx) ** 2 + (y - cy - my * ny) ** 2 + (z - cz - mz * nz) ** 2) - r
                    d = np.minimum(d, dist)
    return np.clip(d / trunc, -1.0, 1.0)


def input_channels(sdf_field):
    """[16, nz, ny, nx]: sdf, z feature in [-1, 1], zeros."""
    nz = sdf_field.shape[0]
    x = np.zeros((C_IN,) + sdf_field.shape)
    x[0] = sdf_field
    zc = np.linspace(-1.0, 1.0, nz) if nz > 1 else np.zeros(1)
    x[1] = zc[:, None, None]
    return x


# ---------------------------------------------------------------------------
# Building blocks
# ---------------------------------------------------------------------------
def shift(x, dz, dy, dx):
    """xs[c, z, y, x] = x[c, z+dz, y+dy, x+dx]: circular in y, x; zero outside z."""
    s = np.roll(x, shift=(-dy, -dx), axis=(2, 3))
    out = np.zeros_like(s)
    nz = x.shape[1]
    if dz == 0:
        out[:] = s
    elif dz > 0:
        out[:, :nz - dz] = s[:, dz:]
    else:
        out[:, -dz:] = s[:, :nz + dz]
    return out


def unshift(y, dz, dy, dx):
    """Adjoint of shift: out[c, p] = y[c, p - off]."""
    nz = y.shape[1]
    out = np.zeros_like(y)
    if dz == 0:
        out[:] = y
    elif dz > 0:
        out[:, dz:] = y[:, :nz - dz]
    else:
        out[:, :nz + dz] = y[:, -dz:]
    return np.roll(out, shift=(dy, dx), axis=(2, 3))


def conv3(x, w, b):
    """3x3x3 convolution: out[o] = b[o] + sum_t sum_c w[t][o][c] x[c](p + off_t)."""
    out = np.zeros((w.shape[1],) + x.shape[1:])
    for t, off in enumerate(TAPS):
        out += np.einsum("oc,czyx->ozyx", w[t], shift(x, *off))
    return out + b[:, None, None, None]


def conv3_backward(x, w, dout):
    """Gradients of conv3 w.r.t. its input, weights and bias."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, off in enumerate(TAPS):
        dw[t] = np.einsum("ozyx,czyx->oc", dout, shift(x, *off))
        dx += unshift(np.einsum("oc,ozyx->czyx", w[t], dout), *off)
    return dx, dw, dout.sum(axis=(1, 2, 3))


def pool(x):
    c, d, h, w = x.shape
    return x.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).mean(axis=(2, 4, 6))


def upsample(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


# ---------------------------------------------------------------------------
# The network
# ---------------------------------------------------------------------------
def layer_shapes(widths=WIDTHS, c_in=C_IN):
    """(name, C_out, C_in) of the 3x3x3 layers in order, then the head."""
    c1, c2, c3, c4 = widths
    return [("enc1a", c1, c_in), ("enc1b", c1, c1), ("enc2a", c2, c1), ("enc2b", c2, c2),
            ("enc3a", c3, c2), ("enc3b", c3, c3), ("botta", c4, c3), ("bottb", c4, c4),
            ("dec3a", c3, c4 + c3), ("dec3b", c3, c3), ("dec2a", c2, c3 + c2), ("dec2b", c2, c2),
            ("dec1a", c1, c2 + c1), ("dec1b", c1, c1)]


def init_params(seed, widths=WIDTHS, c_in=C_IN, c_out=C_OUT):
    """He-uniform weights, zero biases, from numpy's seeded generator (these
    are inputs to both implementations)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, co, ci in layer_shapes(widths, c_in):
        bound = np.sqrt(6.0 / (27 * ci))
        p[name + ".w"] = rng.uniform(-bound, bound, (27, co, ci))
        p[name + ".b"] = np.zeros(co)
    bound = np.sqrt(6.0 / widths[0])
    p["head.w"] = rng.uniform(-bound, bound, (c_out, widths[0]))
    p["head.b"] = np.zeros(c_out)
    return p


class UNet:
    def __init__(self, params, widths=WIDTHS, bf16_emulation=False):
        self.p = params
        self.widths = widths
        self.q = bf16 if bf16_emulation else (lambda a: a)

    def _conv(self, name, x):
        return np.maximum(self.q(conv3(x, self.q(self.p[name + ".w"]), self.p[name + ".b"])), 0.0)

    def forward(self, x):
        """x [16, nz, ny, nx] -> [3, nz, ny, nx]; keeps the activations."""
        q = self.q
        a = {"in": q(x)}
        a["enc1a"] = self._conv("enc1a", a["in"])
        a["enc1b"] = self._conv("enc1b", a["enc1a"])
        a["p1"] = q(pool(a["enc1b"]))
        a["enc2a"] = self._conv("enc2a", a["p1"])
        a["enc2b"] = self._conv("enc2b", a["enc2a"])
        a["p2"] = q(pool(a["enc2b"]))
        a["enc3a"] = self._conv("enc3a", a["p2"])
        a["enc3b"] = self._conv("enc3b", a["enc3a"])
        a["p3"] = q(pool(a["enc3b"]))
        a["botta"] = self._conv("botta", a["p3"])
        a["bottb"] = self._conv("bottb", a["botta"])
        a["c3"] = np.concatenate([upsample(a["bottb"]), a["enc3b"]])
        a["dec3a"] = self._conv("dec3a", a["c3"])
        a["dec3b"] = self._conv("dec3b", a["dec3a"])
        a["c2"] = np.concatenate([upsample(a["dec3b"]), a["enc2b"]])
        a["dec2a"] = self._conv("dec2a", a["c2"])
        a["dec2b"] = self._conv("dec2b", a["dec2a"])
        a["c1"] = np.concatenate([upsample(a["dec2b"]), a["enc1b"]])
        a["dec1a"] = self._conv("dec1a", a["c1"])
        a["dec1b"] = self._conv("dec1b", a["dec1a"])
        a["out"] = np.einsum("oc,czyx->ozyx", q(self.p["head.w"]), a["dec1b"]) + self.p["head.b"][:, None, None, None]
        self.acts = a
        return a["out"]

    def loss(self, out, target):
        """Mean squared error over all voxels and components."""
        return float(np.mean((out - target) ** 2))

    def backward(self, target):
        """Gradients of the loss of the last forward pass: the fp64 chain rule
        through the stored activations.  With bf16 emulation the weights enter
        in bf16 and every stored activation gradient is rounded to bf16, as the
        kernels store them; weight gradients stay unrounded sums."""
        a, p, q = self.acts, self.p, self.q
        g = {}
        dout = 2.0 * (a["out"] - target) / a["out"].size
        g["head.w"] = np.einsum("ozyx,czyx->oc", dout, a["dec1b"])
        g["head.b"] = dout.sum(axis=(1, 2, 3))
        d = q(np.einsum("oc,ozyx->czyx", q(p["head.w"]), dout))

        def conv_back(name, x_in, d_out):
            d_out = d_out * (a[name] > 0)
            dx, dw, db = conv3_backward(x_in, q(p[name + ".w"]), d_out)
            g[name + ".w"], g[name + ".b"] = dw, db
            return q(dx)

        d = conv_back("dec1b", a["dec1a"], d)
        d = conv_back("dec1a", a["c1"], d)
        c = self.widths[1]
        d_up, d_skip1 = d[:c], d[c:]
        d = q(8.0 * pool(d_up))
        d = conv_back("dec2b", a["dec2a"], d)
        d = conv_back("dec2a", a["c2"], d)
        c = self.widths[2]
        d_up, d_skip2 = d[:c], d[c:]
        d = q(8.0 * pool(d_up))
        d = conv_back("dec3b", a["dec3a"], d)
        d = conv_back("dec3a", a["c3"], d)
        c = self.widths[3]
        d_up, d_skip3 = d[:c], d[c:]
        d = q(8.0 * pool(d_up))
        d = conv_back("bottb", a["botta"], d)
        d = conv_back("botta", a["p3"], d)
        d = q(upsample(d) / 8.0 + d_skip3)
        d = conv_back("enc3b", a["enc3a"], d)
        d = conv_back("enc3a", a["p2"], d)
        d = q(upsample(d) / 8.0 + d_skip2)
        d = conv_back("enc2b", a["enc2a"], d)
        d = conv_back("enc2a", a["p1"], d)
        d = q(upsample(d) / 8.0 + d_skip1)
        d = conv_back("enc1b", a["enc1a"], d)
        conv_back("enc1a", a["in"], d)
        return g


def adam(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m." + k, np.zeros_like(params[k]))
        v = state.setdefault("v." + k, np.zeros_like(params[k]))
        m[:] = beta1 * m + (1 - beta1) * grads[k]
        v[:] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params
