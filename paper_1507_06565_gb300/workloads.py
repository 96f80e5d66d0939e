"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

The paper's reference geometry (1274 settled spheres of diameter 16-48 in a
walled channel driven by a pressure drop of 1e-6, Sec. 3.1) and its
weak-scaling block (151^3 cells with one sphere of diameter 90 per core,
Sec. 3) are not available as data; these presets stand in for them with the
same structure: a channel with no-slip walls at top and bottom, periodic
stream- and span-wise, a porous lower layer of spheres, body-force driving
g = 1e-6, tau = 0.8, Lambda = 3/16.  Both the CUDA path and the CPU oracle are
driven from these presets.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Channel:
    name: str
    nx: int
    ny: int
    nz: int
    layer_z0: float
    layer_z1: float
    r_min: float
    r_max: float
    porosity: float
    allow_overlap: bool
    seed: int
    periodic_z: bool = False
    q_lo: float = 0.5
    q_hi: float = 0.5
    tau: float = 0.8
    lam: float = 3.0 / 16.0
    g: tuple = (1e-6, 0.0, 0.0)
    steps: int = 0
    perm_window: tuple = field(default=(-1, -1))

    def sphere_args(self):
        """Positional arguments of the sphere-placement calls (both sides)."""
        return (self.nx, self.ny, self.nz, self.periodic_z, self.layer_z0, self.layer_z1, self.r_min,
                self.r_max, self.porosity, self.allow_overlap, self.seed)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


# 32x32x64 channel, walls z = 0 and 63, lower half z in [1, 32) filled with
# non-overlapping spheres of radius 4 to porosity 0.7; 2000 steps.
W1 = Channel("W1 32x32x64 RSA r=4 phi=0.7", 32, 32, 64, 1.0, 32.0, 4.0, 4.0, 0.7, False, 1, steps=2000)

# 256x256x512 channel, porous layer z in [1, 256) of overlapping r = 8 spheres.
W2_POROSITIES = (0.4, 0.6, 0.8, 0.9)


def W2(phi: float) -> Channel:
    seed = {0.4: 2040, 0.6: 2060, 0.8: 2080, 0.9: 2090}[phi]
    return Channel(f"W2 256x256x512 r=8 phi={phi}", 256, 256, 512, 1.0, 256.0, 8.0, 8.0, phi, True, seed,
                   perm_window=(33, 224))


# 512x512x1024 channel (throughput of the reduced-precision storage).
W3_LARGE = Channel("W3 512x512x1024 r=8 phi=0.6", 512, 512, 1024, 1.0, 512.0, 8.0, 8.0, 0.6, True, 3060,
                   perm_window=(65, 448))


def W4_cube(i: int) -> Channel:
    """REV cube i of the batched permeability sweep: periodic cube, edge in
    [48,160], radii in [3,10], porosity in [0.35,0.95], overlapping."""
    rng = np.random.default_rng(4000 + i)
    edge = int(rng.integers(48, 161))
    phi = float(rng.uniform(0.35, 0.95))
    return Channel(f"W4 cube {i} edge={edge}", edge, edge, edge, 0.0, float(edge), 3.0, 10.0, round(phi, 6), True,
                   4000 + i, periodic_z=True)


def W2_half(phi: float) -> Channel:
    """The W2 channel at half the size (128x128x256, porous layer z < 128,
    same radius and seeds), for profiler captures and converged profiles;
    permeability window z in [17, 112)."""
    return Channel(f"half-size channel phi={phi}", 128, 128, 256, 1.0, 128.0, 8.0, 8.0, phi, True, W2(phi).seed,
                   perm_window=(17, 112))


# The paper's weak-scaling block: 151^3 periodic cube, one centred sphere of
# diameter 90 (explicit list).
W0_BOX = (151, 151, 151)
W0_SPHERES = np.array([[75.0, 75.0, 75.0, 45.0]])
# its flow parameters (the sphere comes from W0_SPHERES, not from placement)
W0 = Channel("W0 151^3 periodic, one sphere D=90", 151, 151, 151, 0.0, 151.0, 45.0, 45.0, 0.0, False, 0,
             periodic_z=True)


def small_cases():
    """Small boxes that the oracle finishes in seconds but that still span
    several thread blocks and leave a ragged last block."""
    return [
        W1,
        Channel("tiny walls r=2.5 rsa", 12, 10, 14, 1.0, 8.0, 2.0, 3.0, 0.75, False, 11, steps=40),
        Channel("periodic cube overlap", 20, 18, 16, 0.0, 16.0, 2.0, 3.5, 0.6, True, 12, periodic_z=True, steps=40),
        Channel("off-grid walls", 16, 16, 20, 1.0, 10.0, 1.5, 3.0, 0.7, True, 13, q_lo=0.3, q_hi=0.8, steps=40),
    ]


def velocity_field(shape, seed: int, amplitude: float = 1e-3) -> np.ndarray:
    """Smooth seeded velocity field [3, nz, ny, nx] (float32) for warm starts:
    a few random Fourier modes."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    for d in range(3):
        for _ in range(4):
            kx, ky, kz = rng.integers(0, 3, 3)
            ph = rng.uniform(0, 2 * np.pi)
            u[d] += rng.standard_normal() * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    return (amplitude * u / max(1e-30, np.abs(u).max())).astype(np.float32)


# The warm-start network's 3x3x3 layers (name, c_out, c_in) in parameter
# order, as documented in include/unet.h; then the head [3][16] and bias [3].
UNET_LAYERS = [("enc1a", 16, 16), ("enc1b", 16, 16), ("enc2a", 32, 16), ("enc2b", 32, 32),
               ("enc3a", 64, 32), ("enc3b", 64, 64), ("botta", 128, 64), ("bottb", 128, 128),
               ("dec3a", 64, 192), ("dec3b", 64, 64), ("dec2a", 32, 96), ("dec2b", 32, 32),
               ("dec1a", 16, 48), ("dec1b", 16, 16)]


def unet_init(seed: int) -> np.ndarray:
    """Seeded He-uniform weights and zero biases as the flat fp32 parameter
    vector of the warm-start network."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, co, ci in UNET_LAYERS:
        bound = np.sqrt(6.0 / (27 * ci))
        parts += [rng.uniform(-bound, bound, 27 * co * ci), np.zeros(co)]
    bound = np.sqrt(6.0 / 16)
    parts += [rng.uniform(-bound, bound, 3 * 16), np.zeros(3)]
    return np.concatenate(parts).astype(np.float32)
