"""FP64 CPU oracle for the D3Q19 TRT lattice Boltzmann method with CLI walls.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle is plain C
(``lbm_oracle.c``) loaded through ctypes; it shares no code with the CUDA
library and imports nothing from it.

Every function restates a passage of Fattahi, Waluga, Wohlmuth & Ruede,
"Large scale lattice Boltzmann simulation for the coupling of free and porous
media flow": Sec. 2.1 (Eqs. (LBM), (TRT), (TRT2), (equilibrium), (Macro),
(collision), (streaming)), Sec. 2.2 (Eqs. (noslip), (CLI)), Sec. 3.1 (plane
averages) and Eq. (Darcy) (permeability).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")

_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available, no FP contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "orc_velocity_set": (None, [_p, _p]),
        "orc_opposite": (_i, [_i]),
        "orc_splitmix64_next": (_u64, [_p]),
        "orc_uniform": (_d, [_p]),
        "orc_voxelize": (None, [_i, _i, _i, _i, _p, _i64, _p]),
        "orc_place_spheres": (_i, [_i, _i, _i, _i, _d, _d, _d, _d, _d, _i, _u64, _i64, _i64, _p, _p, _p]),
        "orc_link_q": (_d, [_i, _i, _i, _i, _d, _d, _p, _i64, _i, _i, _i, _i]),
        "orc_build_lists": (_i, [_i, _i, _i, _i, _d, _d, _p, _i64, _p, _p, _p, _p, _p, _p, _p, _p, _i, _i]),
        "orc_rates": (None, [_d, _d, _p, _p, _p]),
        "orc_equilibrium": (None, [_d, _p, _p]),
        "orc_lbm_create": (_p, [_i, _i, _i, _i, _d, _d, _p, _i64, _d, _d, _d, _d, _d, _i]),
        "orc_lbm_set_simple_bounce_back": (None, [_p]),
        "orc_lbm_destroy": (None, [_p]),
        "orc_lbm_init": (None, [_p, _p]),
        "orc_lbm_step": (None, [_p, _i64]),
        "orc_lbm_steps": (_i64, [_p]),
        "orc_lbm_moments": (None, [_p, _p, _p]),
        "orc_lbm_plane_average": (None, [_p, _p]),
        "orc_lbm_permeability": (_d, [_p, _i, _i]),
        "orc_lbm_residual": (_d, [_p]),
        "orc_lbm_get_f": (None, [_p, _p]),
        "orc_lbm_set_f": (None, [_p, _p]),
        "orc_lbm_solid": (None, [_p, _p]),
        "orc_lbm_nu": (_d, [_p]),
        "orc_lbm_omega_minus": (_d, [_p]),
        "orc_threads": (_i, []),
        "orc_set_threads": (None, [_i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# D3Q19 and the random stream
# --------------------------------------------------------------------------
def velocity_set():
    """(e[19,3] int32, w[19] float64) of the D3Q19 lattice (Sec. 2.1)."""
    e = np.zeros((19, 3), np.int32)
    w = np.zeros(19, np.float64)
    _load().orc_velocity_set(_ptr(e), _ptr(w))
    return e, w


def opposite(k: int) -> int:
    return int(_load().orc_opposite(k))


def splitmix64(seed: int, n: int) -> list[int]:
    """First n outputs of SplitMix64 seeded with ``seed``."""
    st = ctypes.c_uint64(seed)
    return [int(_load().orc_splitmix64_next(ctypes.byref(st))) for _ in range(n)]


def rates(tau: float, lam: float):
    """(omega+, omega-, nu) from tau = 1/omega+ and the magic parameter Lambda."""
    op, om, nu = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_rates(tau, lam, ctypes.byref(op), ctypes.byref(om), ctypes.byref(nu))
    return op.value, om.value, nu.value


def equilibrium(rho: float, u) -> np.ndarray:
    """Incompressible equilibrium f^eq_k(rho, u) for full populations (Eq. (equilibrium))."""
    uu = np.ascontiguousarray(u, np.float64)
    out = np.zeros(19, np.float64)
    _load().orc_equilibrium(rho, _ptr(uu), _ptr(out))
    return out


# --------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------
def place_spheres(nx, ny, nz, periodic_z, z0, z1, r_min, r_max, porosity, allow_overlap, seed,
                  max_spheres=1 << 20, max_rejects=100000):
    """Seeded sphere placement; returns (xyzr[n,4], achieved layer porosity, status)."""
    buf = np.zeros((max_spheres, 4), np.float64)
    n = ctypes.c_int64()
    phi = ctypes.c_double()
    rc = _load().orc_place_spheres(nx, ny, nz, int(periodic_z), z0, z1, r_min, r_max, porosity,
                                   int(allow_overlap), seed, max_spheres, max_rejects, _ptr(buf),
                                   ctypes.byref(n), ctypes.byref(phi))
    return buf[: n.value].copy(), phi.value, rc


def voxelize(nx, ny, nz, periodic_z, xyzr) -> np.ndarray:
    """Solid mask [nz, ny, nx] uint8 (1 = solid)."""
    sp = np.ascontiguousarray(np.asarray(xyzr, np.float64).reshape(-1, 4))
    out = np.zeros((nz, ny, nx), np.uint8)
    _load().orc_voxelize(nx, ny, nz, int(periodic_z), _ptr(sp), sp.shape[0], _ptr(out))
    return out


def link_q(nx, ny, nz, periodic_z, xyzr, x, y, z, k, q_lo=0.5, q_hi=0.5) -> float:
    sp = np.ascontiguousarray(np.asarray(xyzr, np.float64).reshape(-1, 4))
    return float(_load().orc_link_q(nx, ny, nz, int(periodic_z), q_lo, q_hi, _ptr(sp), sp.shape[0],
                                    x, y, z, k))


def build_lists(nx, ny, nz, periodic_z, xyzr, q_lo=0.5, q_hi=0.5, use_bins=False, safeguards=False) -> dict:
    """Fluid list, neighbour table and wall-link list (see lbm_oracle.c).
    ``use_bins`` prunes the sphere search for large boxes (same result).
    ``safeguards`` adds the two corner fallbacks (q < 0.1, two-cell gap) to the
    paper's one (x_f2 solid)."""
    lib = _load()
    sp = np.ascontiguousarray(np.asarray(xyzr, np.float64).reshape(-1, 4))
    nf, nl = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.orc_build_lists(nx, ny, nz, int(periodic_z), q_lo, q_hi, _ptr(sp), sp.shape[0],
                             ctypes.byref(nf), ctypes.byref(nl), None, None, None, None, None, None, 0, 0)
    assert rc == 0
    fluid = np.zeros(nf.value, np.int32)
    nbr = np.zeros((18, nf.value), np.int32)
    lc = np.zeros(nl.value, np.int32)
    lk = np.zeros(nl.value, np.int8)
    lq = np.zeros(nl.value, np.float64)
    lf = np.zeros(nl.value, np.uint8)
    rc = lib.orc_build_lists(nx, ny, nz, int(periodic_z), q_lo, q_hi, _ptr(sp), sp.shape[0],
                             ctypes.byref(nf), ctypes.byref(nl), _ptr(fluid), _ptr(nbr), _ptr(lc),
                             _ptr(lk), _ptr(lq), _ptr(lf), int(use_bins), int(safeguards))
    assert rc == 0
    return {"fluid_cell": fluid, "nbr": nbr, "link_cell": lc, "link_k": lk, "link_q": lq,
            "link_fallback": lf}


def threads() -> int:
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# The LBM
# --------------------------------------------------------------------------
class Lattice:
    """Dense two-array FP64 TRT/CLI lattice; fields are [.., nz, ny, nx].

    Eq. (CLI) on every wall link with a second fluid node (the paper's scheme);
    ``cli_safeguards`` also turns links with q < 0.1 or across a two-cell gap
    into simple bounce-back, ``simple_bounce_back`` every link."""

    def __init__(self, nx, ny, nz, periodic_z, xyzr=(), tau=0.8, lam=3.0 / 16.0, g=(1e-6, 0.0, 0.0),
                 q_lo=0.5, q_hi=0.5, simple_bounce_back=False, cli_safeguards=False):
        self._lib = _load()
        sp = np.ascontiguousarray(np.asarray(xyzr, np.float64).reshape(-1, 4))
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz
        self.g = tuple(float(v) for v in g)
        self._h = self._lib.orc_lbm_create(nx, ny, nz, int(periodic_z), q_lo, q_hi, _ptr(sp),
                                           sp.shape[0], tau, lam, *self.g, int(cli_safeguards))
        if not self._h:
            raise MemoryError("oracle lattice allocation failed")
        if simple_bounce_back:
            self._lib.orc_lbm_set_simple_bounce_back(self._h)
        self.nu = float(self._lib.orc_lbm_nu(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_lbm_destroy(h)
            self._h = None

    def init(self, u0=None):
        if u0 is None:
            self._lib.orc_lbm_init(self._h, None)
        else:
            a = np.ascontiguousarray(np.asarray(u0, np.float64).reshape(3, *self.shape))
            self._lib.orc_lbm_init(self._h, _ptr(a))
        return self

    def step(self, n: int = 1):
        self._lib.orc_lbm_step(self._h, int(n))
        return self

    @property
    def steps(self) -> int:
        return int(self._lib.orc_lbm_steps(self._h))

    def moments(self):
        rho = np.zeros(self.shape, np.float64)
        u = np.zeros((3, *self.shape), np.float64)
        self._lib.orc_lbm_moments(self._h, _ptr(rho), _ptr(u))
        return rho, u

    def plane_average(self) -> np.ndarray:
        out = np.zeros((self.shape[0], 3), np.float64)
        self._lib.orc_lbm_plane_average(self._h, _ptr(out))
        return out

    def permeability(self, z_lo: int = -1, z_hi: int = -1) -> float:
        return float(self._lib.orc_lbm_permeability(self._h, z_lo, z_hi))

    def residual(self) -> float:
        return float(self._lib.orc_lbm_residual(self._h))

    def solid(self) -> np.ndarray:
        out = np.zeros(self.shape, np.uint8)
        self._lib.orc_lbm_solid(self._h, _ptr(out))
        return out

    def get_f(self) -> np.ndarray:
        out = np.zeros((19, *self.shape), np.float64)
        self._lib.orc_lbm_get_f(self._h, _ptr(out))
        return out

    def set_f(self, f) -> None:
        a = np.ascontiguousarray(np.asarray(f, np.float64).reshape(19, *self.shape))
        self._lib.orc_lbm_set_f(self._h, _ptr(a))
