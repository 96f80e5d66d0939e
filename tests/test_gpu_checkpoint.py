"""Checkpoint and resume: a solver rebuilt from the same geometry that loads a
checkpoint continues bit for bit like the uninterrupted run, at either
parity, with a density shift and a switch of reference populations pending,
and through a file."""
import numpy as np
import pytest

import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300 import workloads as W
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    L.load_library()
    return torch


def _solver(torch, case, storage, u0, flags=0):
    geom = L.lbm_geometry_from_spheres(*case.sphere_args(), q_lo=case.q_lo, q_hi=case.q_hi)
    return L.Solver(geom, case.tau, case.lam, (3e-5, 1e-5, 0.0), storage, u0=torch.from_numpy(u0).cuda(),
                    flags=flags)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("first", [57, 58], ids=["save-at-odd", "save-at-even"])
@pytest.mark.parametrize("case", [W.W1, W.small_cases()[2]], ids=lambda c: c.name)
def test_resume_is_bit_identical(torch_cuda, tmp_path, case, first, storage):
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=8, amplitude=1e-2)
    flags = L.LBM_FLAG_PLANE_REFERENCES   # W1's free layer: a reference switch pending at the save
    a = _solver(torch_cuda, case, storage, u0, flags)
    a.step(first)
    a.recenter()   # a density shift and (W1) a reference switch are pending
    a.residual()
    a.profile_residual()
    ck = a.save()
    path = tmp_path / "state.ckpt"
    path.write_bytes(ck)
    a.step(45)
    res_a = a.profile_residual()
    want = a.populations().cpu().numpy()
    b = _solver(torch_cuda, case, storage, np.zeros_like(u0), flags)
    b.load(path.read_bytes())
    assert b.steps == first
    b.step(45)
    assert b.steps == a.steps
    got = b.populations().cpu().numpy()
    assert np.array_equal(got, want)
    assert b.profile_residual() == res_a


def test_load_refuses_another_problem(torch_cuda):
    case = W.small_cases()[1]
    u0 = W.velocity_field((case.nz, case.ny, case.nx), seed=8, amplitude=1e-2)
    a = _solver(torch_cuda, case, "f32", u0)
    ck = a.save()
    other = _solver(torch_cuda, case, "f16", u0)
    with pytest.raises(L.LBMError) as e:
        other.load(ck)
    assert e.value.status == L.LBM_EINVAL
    guarded = _solver(torch_cuda, case, "f32", u0, flags=L.LBM_FLAG_CLI_SAFEGUARDS)
    with pytest.raises(L.LBMError) as e:
        guarded.load(ck)
    assert e.value.status == L.LBM_EINVAL
    with pytest.raises(L.LBMError) as e:
        a.load(ck[:-8])
    assert e.value.status == L.LBM_ESIZE
