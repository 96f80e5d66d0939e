"""The U-Net's tensor-core contractions one layer at a time, element by
element, against the FP64 oracle evaluated on the same bf16 inputs.

With bf16 inputs every product is exact in fp32, so the kernels differ from
the exact result only by the fp32 accumulation (at most n u sum|terms| over n
additions, u = 2^-24) and, for the forward output, one rounding to bf16
(u = 2^-8 relative).  Those are the element-wise bounds here."""
import numpy as np
import pytest

from oracle import unet_oracle as U
import paper_1507_06565_gb300 as L
from paper_1507_06565_gb300.build import build

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24   # fp32 unit roundoff
U16 = 2.0 ** -8    # bf16 unit roundoff


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build()
    L.load_library()
    return torch


DIMS = (2, 6, 10, 12)   # n, nz, ny, nx: 1440 voxels, a ragged last tile of 128
# boxes with the x-rows of the network's two finest levels (32 / 64 voxels):
# a tile of 128 voxels is 4 / 2 whole rows, with wrap-around in y and zeros
# beyond z
HALO_DIMS = [(2, 3, 4, 32), (1, 4, 2, 64), (1, 2, 8, 64)]


def _bf16_tensor(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)


def _per_sample(a):
    """[n, nz, ny, nx, c] -> list of oracle-layout [c, nz, ny, nx]."""
    return [np.moveaxis(a[s], -1, 0) for s in range(a.shape[0])]


@pytest.mark.parametrize("dims", [DIMS] + HALO_DIMS, ids=lambda d: "x".join(map(str, d)))
@pytest.mark.parametrize("ci,co", [(16, 16), (48, 16), (32, 64), (64, 128), (192, 64), (96, 32), (32, 96)])
def test_conv3d_forward_elementwise(torch_cuda, ci, co, dims):
    torch = torch_cuda
    rng = np.random.default_rng(ci * 1000 + co)
    x = U.bf16(rng.standard_normal(dims + (ci,)))
    w = U.bf16(rng.standard_normal((27, co, ci)) / np.sqrt(27 * ci))
    b = rng.standard_normal(co).astype(np.float32).astype(np.float64)
    y = L.unet_conv3d(_bf16_tensor(torch, x), _bf16_tensor(torch, w), torch.from_numpy(b.astype(np.float32)).cuda(),
                      co, dims, relu=True).float().cpu().numpy().astype(np.float64)
    for s, xs in enumerate(_per_sample(x)):
        exact = np.maximum(U.conv3(xs, w, b), 0.0)
        absum = U.conv3(np.abs(xs), np.abs(w), np.abs(b))
        bound = U16 * np.abs(exact) + (1 + U16) * (27 * ci + 1) * U32 * absum
        err = np.abs(np.moveaxis(y[s], -1, 0) - exact)
        assert np.all(err <= bound), (s, float(np.max(err / np.maximum(bound, 1e-300))))


@pytest.mark.parametrize("ci,co", [(16, 16), (48, 16), (16, 32), (64, 64), (192, 64), (64, 128)])
def test_conv3d_wgrad_elementwise(torch_cuda, ci, co):
    torch = torch_cuda
    rng = np.random.default_rng(ci * 7 + co)
    x = U.bf16(rng.standard_normal(DIMS + (ci,)))
    dy = U.bf16(rng.standard_normal(DIMS + (co,)))
    dw = L.unet_conv3d_wgrad(_bf16_tensor(torch, dy), _bf16_tensor(torch, x), DIMS).cpu().numpy().astype(np.float64)
    exact = np.zeros((27, co, ci))
    absum = np.zeros((27, co, ci))
    wz = np.zeros((27, co, ci))
    for xs, ds in zip(_per_sample(x), _per_sample(dy)):
        exact += U.conv3_backward(xs, wz, ds)[1]
        absum += U.conv3_backward(np.abs(xs), wz, np.abs(ds))[1]
    n_add = int(np.prod(DIMS))   # additions per element: one per voxel
    bound = n_add * U32 * absum
    err = np.abs(dw - exact)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
