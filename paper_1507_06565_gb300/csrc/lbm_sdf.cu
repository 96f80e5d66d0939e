// lbm_sdf.cu -- truncated signed distance field of a geometry (input of the
// learned warm start).
//
// sdf(p) = min over the solid surfaces of the signed distance (negative inside
// a solid): |p - c| - r for every periodic image of every sphere, and, when z
// is not periodic, the distances to the wall planes z = 1 - q_lo and
// z = nz - 2 + q_hi that bound the fluid.  The result is divided by the
// truncation T and clipped to [-1, 1]; only spheres within T of a cell can
// matter, so each cell scans the sphere images binned near it.
#include <algorithm>
#include <new>

#include "lbm_internal.h"

namespace lbm {
namespace {

__global__ void k_sdf(int nx, int ny, int nz, int periodic_z, double q_lo, double q_hi, float trunc,
                      const int32_t *__restrict__ bin_start, const SphereImage *__restrict__ images, int nbx, int nby,
                      float *__restrict__ out)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ncell = (int64_t)nx * ny * nz;
    if (c >= ncell) return;
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
    float d = trunc;
    if (!periodic_z) d = fminf(d, fminf((float)z - (float)(1.0 - q_lo), (float)(nz - 2 + q_hi) - (float)z));
    const int bin = x / kBinEdge + nbx * (y / kBinEdge + nby * (z / kBinEdge));
    for (int b = bin_start[bin]; b < bin_start[bin + 1]; ++b) {
        const SphereImage im = images[b];
        const float dx = (float)x - (float)im.x, dy = (float)y - (float)im.y, dz = (float)z - (float)im.z;
        d = fminf(d, sqrtf(dx * dx + dy * dy + dz * dz) - (float)im.r);
    }
    out[c] = fminf(1.0f, fmaxf(-1.0f, d / trunc));
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_sdf_workspace_size(const lbm_geometry *g, float trunc, size_t *bytes)
{
    if (!g || !bytes || !(trunc > 0.0f)) return LBM_EINVAL;
    Bins bins;
    try {
        build_bins(g->box, g->spheres, bins, std::ceil((double)trunc) + 1.0);
    } catch (const std::bad_alloc &) {
        return LBM_ENOMEM;
    }
    *bytes = align_up(bins.start.size() * 4, 256) + bins.images.size() * sizeof(SphereImage) + 256;
    return LBM_OK;
}

extern "C" int lbm_sdf(const lbm_geometry *g, float trunc, void *dev_ws, size_t bytes, float *dev_out, void *stream)
{
    if (!g || !dev_ws || !dev_out || !(trunc > 0.0f) || ((uintptr_t)dev_ws & 255u)) return LBM_EINVAL;
    Bins bins;
    try {
        build_bins(g->box, g->spheres, bins, std::ceil((double)trunc) + 1.0);
    } catch (const std::bad_alloc &) {
        return LBM_ENOMEM;
    }
    const size_t off = align_up(bins.start.size() * 4, 256);
    if (bytes < off + bins.images.size() * sizeof(SphereImage)) return LBM_ESIZE;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *d_start = (int32_t *)dev_ws;
    SphereImage *d_img = (SphereImage *)((char *)dev_ws + off);
    if (cudaMemcpyAsync(d_start, bins.start.data(), bins.start.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LBM_ECUDA;
    if (!bins.images.empty() && cudaMemcpyAsync(d_img, bins.images.data(), bins.images.size() * sizeof(SphereImage),
                                                cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LBM_ECUDA;
    const lbm_box &b = g->box;
    const int64_t ncell = g->ncell();
    k_sdf<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(b.nx, b.ny, b.nz, b.periodic_z, b.q_lo, b.q_hi, trunc,
                                                          d_start, d_img, bins.nbx, bins.nby, dev_out);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    // the host bins must outlive the staged copies
    return cudaStreamSynchronize(st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
