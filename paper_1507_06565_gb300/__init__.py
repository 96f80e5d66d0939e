"""Python binding of liblbm (GB300 pore-scale lattice Boltzmann, sm_103a).

Thin ctypes marshalling over the C ABI in ``include/lbm.h``; every step of the
method runs in the library's CUDA kernels.  PyTorch supplies device memory
(the caller-owned workspace and field tensors) and streams.  The binding
refuses to load when the compiled library is missing: there is no fallback.

Names follow the C ABI: lbm_geometry_from_spheres, lbm_geometry_from_list,
lbm_workspace_size, lbm_init, lbm_step, lbm_moments, lbm_plane_average,
lbm_permeability, lbm_residual, lbm_profile_residual, lbm_run_until, lbm_export_lists,
lbm_populations.  ``Solver`` bundles a handle with its workspace tensor.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_EPACKING = -4
LBM_ENAN = -5
LBM_ENOTCONVERGED = -6
LBM_ETIMEOUT = -7
LBM_ESIZE = -8

LBM_FLAG_NEIGHBOUR_TABLE = 1
LBM_FLAG_ROW_NEIGHBOURS = 2
LBM_FLAG_NO_GRAPH = 4
LBM_FLAG_NO_AUTOTUNE = 8
LBM_FLAG_SIMPLE_BOUNCE_BACK = 32
LBM_FLAG_STAGED_EVEN = 64
LBM_FLAG_CLI_SAFEGUARDS = 128
LBM_FLAG_STAGED_NEIGHBOURS = 256
LBM_FLAG_PLANE_REFERENCES = 512
LBM_FLAG_NO_PLANE_REFERENCES = 1024
LBM_FLAG_DERIVED_NEIGHBOURS = 2048

LBM_CONVERGE_FIELD = 0
LBM_CONVERGE_PROFILE = 1

LBM_F32 = 0
LBM_F16 = 1
LBM_BF16 = 2
STORAGE = {"f32": LBM_F32, "f16": LBM_F16, "bf16": LBM_BF16}


class LBMError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class lbm_box(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic_z", ctypes.c_int32), ("q_lo", ctypes.c_double), ("q_hi", ctypes.c_double)]


class lbm_sphere_params(ctypes.Structure):
    _fields_ = [("box", lbm_box), ("layer_z0", ctypes.c_double), ("layer_z1", ctypes.c_double),
                ("r_min", ctypes.c_double), ("r_max", ctypes.c_double), ("porosity", ctypes.c_double),
                ("allow_overlap", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("max_spheres", ctypes.c_int64), ("max_rejects", ctypes.c_int64)]


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("lambda_", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("storage", ctypes.c_int32), ("flags", ctypes.c_int32)]


class glbm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic_z", ctypes.c_int32), ("nu", ctypes.c_double), ("c_f", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("u_bottom", ctypes.c_double * 3), ("u_top", ctypes.c_double * 3)]


class lbm_geometry_info(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_fluid", ctypes.c_int64), ("n_links", ctypes.c_int64),
                ("n_spheres", ctypes.c_int64), ("porosity", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SZ = ctypes.c_size_t

# symbol -> (restype, argtypes); every symbol declared in include/lbm.h and include/unet.h
SIGNATURES = {
    "lbm_geometry_from_spheres": (_I, [ctypes.POINTER(lbm_sphere_params), ctypes.POINTER(_P)]),
    "lbm_geometry_from_list": (_I, [ctypes.POINTER(lbm_box), _P, _I64, ctypes.POINTER(_P)]),
    "lbm_geometry_info_get": (_I, [_P, ctypes.POINTER(lbm_geometry_info)]),
    "lbm_geometry_spheres": (_I, [_P, _P, _I64, ctypes.POINTER(_I64)]),
    "lbm_geometry_mask": (_I, [_P, _P]),
    "lbm_geometry_destroy": (None, [_P]),
    "lbm_workspace_size": (_I, [_P, ctypes.POINTER(lbm_params), ctypes.POINTER(_SZ)]),
    "lbm_init": (_I, [_P, ctypes.POINTER(lbm_params), _P, _SZ, _P, _P, ctypes.POINTER(_P)]),
    "lbm_reset": (_I, [_P, _P]),
    "lbm_step": (_I, [_P, _I64]),
    "lbm_moments": (_I, [_P, _P, _P]),
    "lbm_plane_average": (_I, [_P, _P]),
    "lbm_permeability": (_I, [_P, _I32, _I32, ctypes.POINTER(_D)]),
    "lbm_residual": (_I, [_P, ctypes.POINTER(_D)]),
    "lbm_profile_residual": (_I, [_P, ctypes.POINTER(_D)]),
    "lbm_mass": (_I, [_P, ctypes.POINTER(_D)]),
    "lbm_recenter": (_I, [_P, ctypes.POINTER(_D)]),
    "lbm_run_until": (_I, [_P, _D, _I64, _I64, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_D)]),
    "lbm_steps_done": (_I, [_P, ctypes.POINTER(_I64)]),
    "lbm_reference_planes": (_I, [_P, ctypes.POINTER(_I32)]),
    "lbm_checkpoint_size": (_I, [_P, ctypes.POINTER(_SZ)]),
    "lbm_save": (_I, [_P, _P, _SZ]),
    "lbm_load": (_I, [_P, _P, _SZ]),
    "lbm_solver_info": (_I, [_P, ctypes.POINTER(lbm_geometry_info)]),
    "lbm_export_lists": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "lbm_populations": (_I, [_P, _P]),
    "lbm_wait_selftest": (_I, [_P, _I32]),
    "lbm_plane_average_static": (_I, [_P, _P, _I32, _I32, _I32, _P, _P]),
    "lbm_batch_workspace_size": (_I, [_P, _I32, ctypes.POINTER(lbm_params), ctypes.POINTER(_SZ)]),
    "lbm_batch_init": (_I, [_P, _I32, ctypes.POINTER(lbm_params), _P, _SZ, _P, _P, ctypes.POINTER(_P)]),
    "lbm_batch_parts": (_I, [_P, ctypes.POINTER(_I32)]),
    "lbm_batch_part_info": (_I, [_P, _I32, ctypes.POINTER(lbm_geometry_info), ctypes.POINTER(_I64),
                                 ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "lbm_batch_permeability": (_I, [_P, _P]),
    "lbm_batch_profile_residual": (_I, [_P, _P]),
    "lbm_schedule": (_I, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                          ctypes.POINTER(_I32)]),
    # include/glbm.h
    "glbm_workspace_size": (_I, [ctypes.POINTER(glbm_params), ctypes.POINTER(_SZ)]),
    "glbm_init": (_I, [ctypes.POINTER(glbm_params), _P, _P, _P, _P, _SZ, _P, _P, ctypes.POINTER(_P)]),
    "glbm_step": (_I, [_P, _I64]),
    "glbm_moments": (_I, [_P, _P, _P]),
    "glbm_plane_average": (_I, [_P, _P]),
    "glbm_populations": (_I, [_P, _P]),
    "glbm_steps_done": (_I, [_P, ctypes.POINTER(_I64)]),
    "glbm_destroy": (None, [_P]),
    # include/unet.h
    "lbm_sdf_workspace_size": (_I, [_P, ctypes.c_float, ctypes.POINTER(_SZ)]),
    "lbm_sdf": (_I, [_P, ctypes.c_float, _P, _SZ, _P, _P]),
    "unet_create": (_I, [_I32, _I32, _I32, _I32, ctypes.POINTER(_P)]),
    "unet_destroy": (None, [_P]),
    "unet_param_count": (_I, [_P, ctypes.POINTER(_I64)]),
    "unet_workspace_size": (_I, [_P, ctypes.POINTER(_SZ)]),
    "unet_bind": (_I, [_P, _P, _SZ, _P]),
    "unet_set_params": (_I, [_P, _P]),
    "unet_get_params": (_I, [_P, _P]),
    "unet_get_grads": (_I, [_P, _P]),
    "unet_forward": (_I, [_P, _P, _P, ctypes.c_float]),
    "unet_backward": (_I, [_P, _P, ctypes.c_float, ctypes.POINTER(_D)]),
    "unet_adam_step": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "unet_conv3d": (_I, [_P, _I32, _P, _P, _P, _I32, _I32, _I32, _I32, _I32, _I32, _P, _P]),
    "unet_conv3d_wgrad": (_I, [_P, _I32, _P, _I32, _P, _I32, _I32, _I32, _I32, _P, _P]),
    "lbm_solver_destroy": (None, [_P]),
    "lbm_status_string": (ctypes.c_char_p, [_I]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so (built by ``paper_1507_06565_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbm.so not built ({path}); run paper_1507_06565_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load_library().lbm_status_string(int(status)).decode()


def _check(rc: int, what: str) -> None:
    if rc != LBM_OK:
        raise LBMError(rc, what)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------
class Geometry:
    """Owning wrapper of an lbm_geometry handle."""

    def __init__(self, handle, box: lbm_box):
        self._h = handle
        self.box = box

    def __del__(self):
        if getattr(self, "_h", None):
            load_library().lbm_geometry_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.box.nz, self.box.ny, self.box.nx)

    def info(self) -> dict:
        inf = lbm_geometry_info()
        _check(load_library().lbm_geometry_info_get(self._h, ctypes.byref(inf)), "lbm_geometry_info_get")
        return {k: getattr(inf, k) for k, _ in lbm_geometry_info._fields_}

    def spheres(self) -> np.ndarray:
        n = _I64()
        load_library().lbm_geometry_spheres(self._h, None, 0, ctypes.byref(n))
        out = np.zeros((n.value, 4), np.float64)
        _check(load_library().lbm_geometry_spheres(self._h, _np_ptr(out), n.value, ctypes.byref(n)),
               "lbm_geometry_spheres")
        return out

    def mask(self) -> np.ndarray:
        out = np.zeros(self.shape, np.uint8)
        _check(load_library().lbm_geometry_mask(self._h, _np_ptr(out)), "lbm_geometry_mask")
        return out


def make_box(nx, ny, nz, periodic_z=False, q_lo=0.5, q_hi=0.5) -> lbm_box:
    return lbm_box(int(nx), int(ny), int(nz), int(bool(periodic_z)), float(q_lo), float(q_hi))


def lbm_geometry_from_spheres(nx, ny, nz, periodic_z, layer_z0, layer_z1, r_min, r_max, porosity,
                              allow_overlap, seed, q_lo=0.5, q_hi=0.5, max_spheres=1 << 22,
                              max_rejects=100000) -> Geometry:
    box = make_box(nx, ny, nz, periodic_z, q_lo, q_hi)
    p = lbm_sphere_params(box, float(layer_z0), float(layer_z1), float(r_min), float(r_max), float(porosity),
                          int(bool(allow_overlap)), int(seed), int(max_spheres), int(max_rejects))
    h = _P()
    _check(load_library().lbm_geometry_from_spheres(ctypes.byref(p), ctypes.byref(h)),
           "lbm_geometry_from_spheres")
    return Geometry(h, box)


def lbm_geometry_from_list(nx, ny, nz, periodic_z, xyzr, q_lo=0.5, q_hi=0.5) -> Geometry:
    box = make_box(nx, ny, nz, periodic_z, q_lo, q_hi)
    sp = np.ascontiguousarray(np.asarray(xyzr, np.float64).reshape(-1, 4))
    h = _P()
    _check(load_library().lbm_geometry_from_list(ctypes.byref(box), _np_ptr(sp), sp.shape[0], ctypes.byref(h)),
           "lbm_geometry_from_list")
    return Geometry(h, box)


# ---------------------------------------------------------------------------
# Solver
# ---------------------------------------------------------------------------
def make_params(tau=0.8, lam=3.0 / 16.0, g=(1e-6, 0.0, 0.0), storage="f32", flags=0) -> lbm_params:
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    return lbm_params(float(tau), float(lam), (ctypes.c_double * 3)(*[float(v) for v in g]), st, int(flags))


def lbm_workspace_size(geom: Geometry, params: lbm_params) -> int:
    n = _SZ()
    _check(load_library().lbm_workspace_size(geom.handle, ctypes.byref(params), ctypes.byref(n)),
           "lbm_workspace_size")
    return int(n.value)


def lbm_init(geom: Geometry, params: lbm_params, workspace, u0=None, stream=None):
    """Returns the raw solver handle; ``workspace`` is a CUDA uint8 tensor."""
    h = _P()
    s = ctypes.c_void_p(stream) if stream is not None else None
    _check(load_library().lbm_init(geom.handle, ctypes.byref(params), _dev_ptr(workspace), workspace.numel(),
                                   _dev_ptr(u0), s, ctypes.byref(h)), "lbm_init")
    return h


class Solver:
    """A solver handle with its caller-owned workspace (a torch uint8 tensor)."""

    def __init__(self, geom: Geometry, tau=0.8, lam=3.0 / 16.0, g=(1e-6, 0.0, 0.0), storage="f32", u0=None,
                 device="cuda", stream=None, flags=0):
        import torch

        self.params = make_params(tau, lam, g, storage, flags)
        self.box = geom.box
        self.shape = geom.shape
        nbytes = lbm_workspace_size(geom, self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        if stream is None:
            stream = torch.cuda.current_stream(self.workspace.device).cuda_stream
        self.stream = stream
        self._h = lbm_init(geom, self.params, self.workspace, u0, stream)
        self.nu = (tau - 0.5) / 3.0
        self.g = tuple(float(v) for v in g)

    def __del__(self):
        if getattr(self, "_h", None):
            load_library().lbm_solver_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = lbm_geometry_info()
        _check(load_library().lbm_solver_info(self._h, ctypes.byref(inf)), "lbm_solver_info")
        return {k: getattr(inf, k) for k, _ in lbm_geometry_info._fields_}

    def reset(self, u0=None):
        _check(load_library().lbm_reset(self._h, _dev_ptr(u0)), "lbm_reset")

    def step(self, n: int = 1):
        _check(load_library().lbm_step(self._h, int(n)), "lbm_step")

    @property
    def steps(self) -> int:
        n = _I64()
        _check(load_library().lbm_steps_done(self._h, ctypes.byref(n)), "lbm_steps_done")
        return n.value

    def moments(self, rho=None, u=None):
        import torch

        dev = self.workspace.device
        if rho is None:
            rho = torch.empty(self.shape, dtype=torch.float32, device=dev)
        if u is None:
            u = torch.empty((3, *self.shape), dtype=torch.float32, device=dev)
        _check(load_library().lbm_moments(self._h, _dev_ptr(rho), _dev_ptr(u)), "lbm_moments")
        return rho, u

    def plane_average(self) -> np.ndarray:
        out = np.zeros((self.shape[0], 3), np.float64)
        _check(load_library().lbm_plane_average(self._h, _np_ptr(out)), "lbm_plane_average")
        return out

    def permeability(self, z_lo: int = -1, z_hi: int = -1) -> float:
        k = _D()
        _check(load_library().lbm_permeability(self._h, int(z_lo), int(z_hi), ctypes.byref(k)), "lbm_permeability")
        return k.value

    def residual(self) -> float:
        r = _D()
        _check(load_library().lbm_residual(self._h, ctypes.byref(r)), "lbm_residual")
        return r.value

    def profile_residual(self) -> float:
        r = _D()
        _check(load_library().lbm_profile_residual(self._h, ctypes.byref(r)), "lbm_profile_residual")
        return r.value

    def mass(self) -> float:
        """Mean density deviation <rho - 1> over the fluid cells."""
        m = _D()
        _check(load_library().lbm_mass(self._h, ctypes.byref(m)), "lbm_mass")
        return m.value

    def recenter(self) -> float:
        c = _D()
        _check(load_library().lbm_recenter(self._h, ctypes.byref(c)), "lbm_recenter")
        return c.value

    def run_until(self, tol=1e-8, interval=100, max_steps=10 ** 7, criterion="profile"):
        """Returns (status, steps, residual); criterion "profile" or "field"."""
        crit = LBM_CONVERGE_PROFILE if criterion == "profile" else LBM_CONVERGE_FIELD
        n, r = _I64(), _D()
        rc = load_library().lbm_run_until(self._h, float(tol), int(interval), int(max_steps), crit,
                                          ctypes.byref(n), ctypes.byref(r))
        return rc, n.value, r.value

    def export_lists(self) -> dict:
        inf = self.info()
        nf, nl = inf["n_fluid"], inf["n_links"]
        out = {"fluid_cell": np.zeros(nf, np.int32), "nbr": np.zeros((18, nf), np.int32),
               "link_cell": np.zeros(nl, np.int32), "link_k": np.zeros(nl, np.int8),
               "link_q": np.zeros(nl, np.float64), "link_fallback": np.zeros(nl, np.uint8)}
        _check(load_library().lbm_export_lists(self._h, *[_np_ptr(out[k]) for k in
                                                           ("fluid_cell", "nbr", "link_cell", "link_k", "link_q",
                                                            "link_fallback")]), "lbm_export_lists")
        return out

    def save(self) -> bytes:
        """Checkpoint of the solver's state (lbm_save) as bytes."""
        n = _SZ()
        lib = load_library()
        _check(lib.lbm_checkpoint_size(self._h, ctypes.byref(n)), "lbm_checkpoint_size")
        buf = np.zeros(int(n.value), np.uint8)
        _check(lib.lbm_save(self._h, _np_ptr(buf), buf.size), "lbm_save")
        return buf.tobytes()

    def load(self, data: bytes) -> None:
        """Resume from a checkpoint of the same problem (lbm_load)."""
        buf = np.frombuffer(data, np.uint8).copy()
        _check(load_library().lbm_load(self._h, _np_ptr(buf), buf.size), "lbm_load")

    def reference_planes(self) -> int:
        """Planes whose slots store populations relative to the plane's
        reference equilibrium (refreshed by recenter())."""
        n = _I32()
        _check(load_library().lbm_reference_planes(self._h, ctypes.byref(n)), "lbm_reference_planes")
        return n.value

    def link_fallback(self) -> np.ndarray:
        """Per wall link (in (cell, k) order): 1 where it takes simple
        bounce-back instead of Eq. (CLI)."""
        out = np.zeros(self.info()["n_links"], np.uint8)
        _check(load_library().lbm_export_lists(self._h, None, None, None, None, None, _np_ptr(out)),
               "lbm_export_lists")
        return out

    def populations(self):
        """Shifted populations h_k = f_k - w_k, [19, n_fluid] float32 on the device."""
        import torch

        nf = self.info()["n_fluid"]
        out = torch.empty((19, nf), dtype=torch.float32, device=self.workspace.device)
        _check(load_library().lbm_populations(self._h, _dev_ptr(out)), "lbm_populations")
        return out


def _schedule(handle) -> dict:
    ge, go, tu, gs = _I32(), _I32(), _I32(), _I32()
    _check(load_library().lbm_schedule(handle, ctypes.byref(ge), ctypes.byref(go), ctypes.byref(tu),
                                       ctypes.byref(gs)), "lbm_schedule")
    return {"grid_even": ge.value, "grid_odd": go.value, "tuned": bool(tu.value), "graph_steps": gs.value}


Solver.schedule = lambda self: _schedule(self._h)


class BatchSolver(Solver):
    """Several independent boxes advanced together (one launch per step)."""

    def __init__(self, geoms, tau=0.8, lam=3.0 / 16.0, g=(1e-6, 0.0, 0.0), storage="f32", u0=None,
                 device="cuda", stream=None, flags=0):
        import torch

        self.params = make_params(tau, lam, g, storage, flags)
        self.geoms = list(geoms)
        arr = (_P * len(self.geoms))(*[gm.handle for gm in self.geoms])
        self._arr = arr
        n = _SZ()
        _check(load_library().lbm_batch_workspace_size(arr, len(self.geoms), ctypes.byref(self.params),
                                                       ctypes.byref(n)), "lbm_batch_workspace_size")
        self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=device)
        if stream is None:
            stream = torch.cuda.current_stream(self.workspace.device).cuda_stream
        self.stream = stream
        h = _P()
        _check(load_library().lbm_batch_init(arr, len(self.geoms), ctypes.byref(self.params),
                                             _dev_ptr(self.workspace), self.workspace.numel(), _dev_ptr(u0),
                                             ctypes.c_void_p(stream), ctypes.byref(h)), "lbm_batch_init")
        self._h = h
        self.box = self.geoms[0].box
        self.nu = (tau - 0.5) / 3.0
        self.g = tuple(float(v) for v in g)
        self.n_cells_total = sum(int(np.prod(gm.shape)) for gm in self.geoms)

    @property
    def n_parts(self) -> int:
        n = _I32()
        _check(load_library().lbm_batch_parts(self._h, ctypes.byref(n)), "lbm_batch_parts")
        return n.value

    def part_info(self, b: int) -> dict:
        inf = lbm_geometry_info()
        fo, co, po = _I64(), _I64(), _I64()
        _check(load_library().lbm_batch_part_info(self._h, int(b), ctypes.byref(inf), ctypes.byref(fo),
                                                  ctypes.byref(co), ctypes.byref(po)), "lbm_batch_part_info")
        d = {k: getattr(inf, k) for k, _ in lbm_geometry_info._fields_}
        d.update(fluid_offset=fo.value, cell_offset=co.value, plane_offset=po.value)
        return d

    def moments(self, rho=None, u=None):
        import torch

        dev = self.workspace.device
        if rho is None:
            rho = torch.empty(self.n_cells_total, dtype=torch.float32, device=dev)
        if u is None:
            u = torch.empty((3, self.n_cells_total), dtype=torch.float32, device=dev)
        _check(load_library().lbm_moments(self._h, _dev_ptr(rho), _dev_ptr(u)), "lbm_moments")
        return rho, u

    def plane_average(self) -> np.ndarray:
        nplanes = sum(gm.box.nz for gm in self.geoms)
        out = np.zeros((nplanes, 3), np.float64)
        _check(load_library().lbm_plane_average(self._h, _np_ptr(out)), "lbm_plane_average")
        return out

    def permeabilities(self) -> np.ndarray:
        out = np.zeros(len(self.geoms), np.float64)
        _check(load_library().lbm_batch_permeability(self._h, _np_ptr(out)), "lbm_batch_permeability")
        return out

    def profile_residuals(self) -> np.ndarray:
        out = np.zeros(len(self.geoms), np.float64)
        _check(load_library().lbm_batch_profile_residual(self._h, _np_ptr(out)), "lbm_batch_profile_residual")
        return out


def lbm_sdf(geom: Geometry, trunc: float = 8.0, out=None, stream=None):
    """Truncated signed distance / trunc of a geometry, [nz, ny, nx] float32 on the device."""
    import torch

    n = _SZ()
    _check(load_library().lbm_sdf_workspace_size(geom.handle, float(trunc), ctypes.byref(n)),
           "lbm_sdf_workspace_size")
    ws = torch.empty(int(n.value), dtype=torch.uint8, device="cuda")
    if out is None:
        out = torch.empty(geom.shape, dtype=torch.float32, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load_library().lbm_sdf(geom.handle, float(trunc), _dev_ptr(ws), ws.numel(), _dev_ptr(out),
                                  ctypes.c_void_p(stream)), "lbm_sdf")
    return out


class GLBM:
    """The homogenised porous-medium LBM (include/glbm.h) with its device
    workspace.  eps, inv_k (1/K) and tau are per z-plane (length nz or
    scalars)."""

    def __init__(self, nx, ny, nz, eps, inv_k, tau, nu, c_f=0.0, g=(0.0, 0.0, 0.0), u_bottom=(0.0, 0.0, 0.0),
                 u_top=(0.0, 0.0, 0.0), periodic_z=False, u0=None, stream=None):
        import torch

        lib = load_library()
        p = glbm_params(int(nx), int(ny), int(nz), int(bool(periodic_z)), float(nu), float(c_f),
                        (ctypes.c_double * 3)(*g), (ctypes.c_double * 3)(*u_bottom), (ctypes.c_double * 3)(*u_top))
        self.shape = (int(nz), int(ny), int(nx))
        col = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64).reshape(-1), (nz,)))
        e, ik, t = col(eps), col(inv_k), col(tau)
        ws = _SZ()
        _check(lib.glbm_workspace_size(ctypes.byref(p), ctypes.byref(ws)), "glbm_workspace_size")
        self.workspace = torch.empty(int(ws.value), dtype=torch.uint8, device="cuda")
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = _P()
        _check(lib.glbm_init(ctypes.byref(p), _np_ptr(e), _np_ptr(ik), _np_ptr(t), _dev_ptr(self.workspace),
                             self.workspace.numel(), _dev_ptr(u0) if u0 is not None else None,
                             ctypes.c_void_p(stream), ctypes.byref(h)), "glbm_init")
        self._h = h
        self.n_fluid = int(nx) * int(ny) * (int(nz) if periodic_z else int(nz) - 2)

    def __del__(self):
        if getattr(self, "_h", None):
            load_library().glbm_destroy(self._h)
            self._h = None

    def step(self, n: int = 1):
        _check(load_library().glbm_step(self._h, int(n)), "glbm_step")
        return self

    @property
    def steps(self) -> int:
        v = _I64()
        _check(load_library().glbm_steps_done(self._h, ctypes.byref(v)), "glbm_steps_done")
        return v.value

    def moments(self):
        import torch

        rho = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        u = torch.empty((3,) + self.shape, dtype=torch.float32, device="cuda")
        _check(load_library().glbm_moments(self._h, _dev_ptr(rho), _dev_ptr(u)), "glbm_moments")
        return rho, u

    def plane_average(self) -> np.ndarray:
        out = np.zeros(self.shape[0], np.float64)
        _check(load_library().glbm_plane_average(self._h, _np_ptr(out)), "glbm_plane_average")
        return out

    def populations(self):
        """f_k - w_k of the current time, [19, n_fluid] float32 on the device."""
        import torch

        out = torch.empty((19, self.n_fluid), dtype=torch.float32, device="cuda")
        _check(load_library().glbm_populations(self._h, _dev_ptr(out)), "glbm_populations")
        return out


class UNet:
    """The warm-start network (include/unet.h) with its device workspace."""

    def __init__(self, n, nz, ny, nx, params=None, stream=None):
        import torch

        lib = load_library()
        h = _P()
        _check(lib.unet_create(int(n), int(nz), int(ny), int(nx), ctypes.byref(h)), "unet_create")
        self._h = h
        self.shape = (int(n), int(nz), int(ny), int(nx))
        cnt, ws = _I64(), _SZ()
        _check(lib.unet_param_count(h, ctypes.byref(cnt)), "unet_param_count")
        _check(lib.unet_workspace_size(h, ctypes.byref(ws)), "unet_workspace_size")
        self.n_params = cnt.value
        self.workspace = torch.empty(int(ws.value), dtype=torch.uint8, device="cuda")
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        _check(lib.unet_bind(h, _dev_ptr(self.workspace), self.workspace.numel(), ctypes.c_void_p(stream)),
               "unet_bind")
        if params is not None:
            self.set_params(params)

    def __del__(self):
        if getattr(self, "_h", None):
            load_library().unet_destroy(self._h)
            self._h = None

    def set_params(self, params):
        import torch

        t = torch.as_tensor(params, dtype=torch.float32).contiguous().cuda()
        assert t.numel() == self.n_params
        _check(load_library().unet_set_params(self._h, _dev_ptr(t)), "unet_set_params")

    def params(self):
        import torch

        t = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(load_library().unet_get_params(self._h, _dev_ptr(t)), "unet_get_params")
        return t

    def grads(self):
        import torch

        t = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(load_library().unet_get_grads(self._h, _dev_ptr(t)), "unet_get_grads")
        return t

    def forward(self, sdf, out=None, out_scale=1.0):
        import torch

        n, nz, ny, nx = self.shape
        if out is None:
            out = torch.empty((n, 3, nz, ny, nx), dtype=torch.float32, device="cuda")
        _check(load_library().unet_forward(self._h, _dev_ptr(sdf), _dev_ptr(out), float(out_scale)), "unet_forward")
        return out

    def backward(self, target, target_scale=1.0) -> float:
        loss = _D()
        _check(load_library().unet_backward(self._h, _dev_ptr(target), float(target_scale), ctypes.byref(loss)),
               "unet_backward")
        return loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(load_library().unet_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps)),
               "unet_adam_step")


def unet_conv3d(x, w, bias, co: int, dims, relu: bool = True, out=None, status=None, stream=None):
    """One 3x3x3 convolution layer (include/unet.h): x bf16 [n, nz, ny, nx, ci]
    CUDA tensor, w bf16 [27, co, ci], bias fp32 [co] or None; returns the bf16
    output [n, nz, ny, nx, co].  ``status`` (int32 [1], zero) records a wait
    that gave up."""
    import torch

    n, nz, ny, nx = dims
    ci = int(x.shape[-1])
    if out is None:
        out = torch.empty((n, nz, ny, nx, co), dtype=torch.bfloat16, device=x.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream(x.device).cuda_stream
    _check(load_library().unet_conv3d(_dev_ptr(x), ci, _dev_ptr(w), _dev_ptr(bias), _dev_ptr(out), co, n, nz, ny, nx,
                                      int(relu), _dev_ptr(status), ctypes.c_void_p(st)), "unet_conv3d")
    return out


def unet_conv3d_wgrad(dy, x, dims, dw=None, status=None, stream=None):
    """Weight gradient of a 3x3x3 layer: dw fp32 [27, co, ci] += sum_v dy[v, o]
    x[v + off_t, c] (dy bf16 [.., co], x bf16 [.., ci])."""
    import torch

    n, nz, ny, nx = dims
    co, ci = int(dy.shape[-1]), int(x.shape[-1])
    if dw is None:
        dw = torch.zeros((27, co, ci), dtype=torch.float32, device=x.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream(x.device).cuda_stream
    _check(load_library().unet_conv3d_wgrad(_dev_ptr(dy), co, _dev_ptr(x), ci, _dev_ptr(dw), n, nz, ny, nx,
                                            _dev_ptr(status), ctypes.c_void_p(st)), "unet_conv3d_wgrad")
    return dw


def lbm_batch_init(geoms, **kw) -> BatchSolver:
    return BatchSolver(geoms, **kw)


def lbm_step(solver: Solver, n: int = 1):
    solver.step(n)


def lbm_moments(solver: Solver, rho=None, u=None):
    return solver.moments(rho, u)


def lbm_plane_average(solver: Solver) -> np.ndarray:
    return solver.plane_average()


def lbm_permeability(solver: Solver, z_lo: int = -1, z_hi: int = -1) -> float:
    return solver.permeability(z_lo, z_hi)


def lbm_residual(solver: Solver) -> float:
    return solver.residual()


def lbm_profile_residual(solver: Solver) -> float:
    return solver.profile_residual()


def lbm_run_until(solver: Solver, tol=1e-8, interval=100, max_steps=10 ** 7, criterion="profile"):
    return solver.run_until(tol, interval, max_steps, criterion)


def lbm_export_lists(solver: Solver) -> dict:
    return solver.export_lists()


def lbm_populations(solver: Solver):
    return solver.populations()
