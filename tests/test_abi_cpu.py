"""CPU-side checks of the C-ABI library: it builds, loads and exports every
symbol of include/*.h, and its host geometry (sphere placement, voxel mask)
equals the oracle's bit for bit.  No GPU kernel is launched here."""
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return L.load_library()


def _declared_symbols():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b((?:lbm|unet|glbm)_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_symbols_exported(lib):
    declared = _declared_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(L.SIGNATURES) == declared


def test_status_strings(lib):
    for code in range(-8, 1):
        assert L.status_string(code) != "unknown status"


@pytest.mark.parametrize("case", W.small_cases() + [W.W4_cube(0), W.W4_cube(1)], ids=lambda c: c.name)
def test_sphere_placement_and_mask_bit_exact(lib, case):
    sp_o, phi_o, rc = O.place_spheres(*case.sphere_args())
    assert rc == 0
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    sp = geom.spheres()
    assert sp.shape == sp_o.shape and np.array_equal(sp, sp_o)
    assert geom.info()["porosity"] == phi_o
    mask_o = O.voxelize(case.nx, case.ny, case.nz, case.periodic_z, sp_o)
    assert np.array_equal(geom.mask(), mask_o)
    lists = O.build_lists(case.nx, case.ny, case.nz, case.periodic_z, sp_o, case.q_lo, case.q_hi, use_bins=True)
    inf = geom.info()
    assert inf["n_fluid"] == len(lists["fluid_cell"]) and inf["n_links"] == len(lists["link_k"])


@pytest.mark.parametrize("phi", W.W2_POROSITIES)
def test_full_size_channel_spheres_bit_exact(lib, phi):
    """The 256x256x512 channel packings: same sphere list and voxel count."""
    case = W.W2(phi)
    sp_o, phi_o, rc = O.place_spheres(*case.sphere_args())
    assert rc == 0
    geom = L.lbm_geometry_from_spheres(*case.sphere_args())
    assert np.array_equal(geom.spheres(), sp_o)
    assert geom.info()["porosity"] == phi_o
    assert phi_o <= phi


def test_explicit_list_geometry(lib):
    sp = np.array([[5.25, 4.5, 3.0, 2.5], [-0.5, 0.25, 6.0, 1.75]])
    geom = L.lbm_geometry_from_list(10, 9, 12, False, sp)
    assert np.array_equal(geom.mask(), O.voxelize(10, 9, 12, False, sp))
    assert np.array_equal(geom.spheres(), sp)


# hand-made sphere lists: a centre on grid points (cells at exactly distance r
# are solid: the test is |x - c|^2 <= r^2), spheres across the periodic x and
# y faces, two overlapping spheres, a sphere cut by the bottom wall layer and
# one reaching into the top wall layer
HAND_CASES = {
    "on grid points": (9, 9, 12, [[4.0, 4.0, 6.0, 3.0]]),
    "across periodic faces": (10, 9, 12, [[-0.25, 8.75, 5.5, 2.25], [9.9, 0.1, 6.0, 1.5]]),
    "two overlapping": (12, 10, 12, [[4.5, 5.0, 6.0, 3.0], [7.0, 5.0, 6.5, 2.5]]),
    "cut by the walls": (8, 8, 10, [[4.0, 4.0, 0.5, 2.75], [3.5, 3.5, 9.25, 1.5]]),
}


@pytest.mark.parametrize("name", sorted(HAND_CASES))
def test_hand_made_geometries_bit_exact(lib, name):
    nx, ny, nz, sp = HAND_CASES[name]
    sp = np.array(sp)
    geom = L.lbm_geometry_from_list(nx, ny, nz, False, sp)
    mask = geom.mask()
    assert np.array_equal(mask, O.voxelize(nx, ny, nz, False, sp))
    assert np.array_equal(geom.spheres(), sp)
    # brute force from the definition: solid where some periodic image (in x
    # and y) of a sphere holds the cell centre, or in the wall layers z = 0, nz - 1
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    solid = (z == 0) | (z == nz - 1)
    for cx, cy, cz, r in sp:
        for sx in (-nx, 0, nx):
            for sy in (-ny, 0, ny):
                solid |= (x - cx - sx) ** 2 + (y - cy - sy) ** 2 + (z - cz) ** 2 <= r * r
    assert np.array_equal(mask.astype(bool), solid)


def test_error_codes(lib):
    with pytest.raises(L.LBMError) as e:
        L.lbm_geometry_from_spheres(24, 24, 24, True, 0.0, 24.0, 4.0, 4.0, 0.1, False, 3, max_rejects=2000)
    assert e.value.status == L.LBM_EPACKING
    with pytest.raises(L.LBMError) as e:   # 2r >= nx
        L.lbm_geometry_from_spheres(8, 8, 8, True, 0.0, 8.0, 4.0, 4.0, 0.5, True, 3)
    assert e.value.status == L.LBM_EINVAL
    with pytest.raises(L.LBMError) as e:
        L.lbm_geometry_from_list(8, 8, 8, False, [[1.0, 1.0, 1.0, -1.0]])
    assert e.value.status == L.LBM_EINVAL
    geom = L.lbm_geometry_from_list(8, 8, 8, False, [])
    with pytest.raises(L.LBMError) as e:
        L.lbm_workspace_size(geom, L.make_params(tau=0.5))
    assert e.value.status == L.LBM_EINVAL
    assert L.lbm_workspace_size(geom, L.make_params()) > 0


def test_flags_validated_on_host(lib):
    """Every documented LBM_FLAG_* value (and the allowed combinations) is
    accepted by the host-side size query; undefined bits and the two
    neighbour variants together are refused."""
    geom = L.lbm_geometry_from_list(8, 8, 8, False, [[4.0, 4.0, 4.0, 2.0]])
    base = L.lbm_workspace_size(geom, L.make_params())
    for f in (L.LBM_FLAG_NEIGHBOUR_TABLE, L.LBM_FLAG_ROW_NEIGHBOURS, L.LBM_FLAG_NO_GRAPH, L.LBM_FLAG_NO_AUTOTUNE,
              L.LBM_FLAG_SIMPLE_BOUNCE_BACK, L.LBM_FLAG_STAGED_EVEN, L.LBM_FLAG_CLI_SAFEGUARDS,
              L.LBM_FLAG_STAGED_NEIGHBOURS, L.LBM_FLAG_PLANE_REFERENCES, L.LBM_FLAG_NO_PLANE_REFERENCES, L.LBM_FLAG_DERIVED_NEIGHBOURS,
              L.LBM_FLAG_STAGED_EVEN | L.LBM_FLAG_NO_AUTOTUNE | L.LBM_FLAG_NEIGHBOUR_TABLE):
        assert L.lbm_workspace_size(geom, L.make_params(flags=f)) == base
    for f in (16, 4096, 1 << 20, L.LBM_FLAG_PLANE_REFERENCES | L.LBM_FLAG_NO_PLANE_REFERENCES, L.LBM_FLAG_NEIGHBOUR_TABLE | L.LBM_FLAG_ROW_NEIGHBOURS,
              L.LBM_FLAG_ROW_NEIGHBOURS | L.LBM_FLAG_STAGED_NEIGHBOURS):
        with pytest.raises(L.LBMError) as e:
            L.lbm_workspace_size(geom, L.make_params(flags=f))
        assert e.value.status == L.LBM_EINVAL


def test_geometry_keeps_its_sphere_bins(lib):
    """The link bins are part of the geometry: repeated size queries agree,
    and two geometries from the same spheres give the same sizes."""
    sp = [[5.25, 4.5, 3.0, 2.5], [-0.5, 0.25, 6.0, 1.75]]
    a = L.lbm_geometry_from_list(10, 9, 12, False, sp)
    b = L.lbm_geometry_from_list(10, 9, 12, False, sp)
    p = L.make_params()
    assert L.lbm_workspace_size(a, p) == L.lbm_workspace_size(a, p) == L.lbm_workspace_size(b, p)


def test_size_limit_of_32bit_slot_offsets(lib):
    """The step kernels address population slots with 32-bit offsets, so a
    solver takes at most 2^32 / 19 padded fluid cells (~226 M): a 624^3
    channel (242 M fluid cells) is refused, a 600^3 one (215 M) accepted."""
    big = L.lbm_geometry_from_list(624, 624, 624, False, [])
    assert big.info()["n_fluid"] * 19 > 2 ** 32
    with pytest.raises(L.LBMError) as e:
        L.lbm_workspace_size(big, L.make_params())
    assert e.value.status == L.LBM_EINVAL
    del big
    ok = L.lbm_workspace_size(L.lbm_geometry_from_list(600, 600, 600, False, []), L.make_params())
    assert ok > 600 * 600 * 598 * 19 * 4
