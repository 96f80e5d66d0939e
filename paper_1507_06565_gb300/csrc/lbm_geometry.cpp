// lbm_geometry.cpp -- host side of the geometry: seeded sphere placement,
// voxelisation, fluid/link counts and the sphere-image bins used by the device
// link-fraction kernel.
//
// Sphere placement replaces the rigid-body settling of Sec. 3.1 (the paper's
// particle code is not available): a SplitMix64 stream (Steele, Lea & Flood,
// OOPSLA 2014) draws centre and radius, each rounded down to the 2^-10 grid so
// that every voxel test below is exact in FP64 whatever the evaluation order.
// This file is compiled with -ffp-contract=off: the few inexact operations
// (scaling a uniform draw) must round the same way on every host.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lbm_internal.h"

namespace lbm {
namespace {

struct SplitMix64 {
    uint64_t state;
    uint64_t next()
    {
        state += 0x9e3779b97f4a7c15ULL;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        return z ^ (z >> 31);
    }
    // 53 random bits as a double in [0,1)
    double unit() { return (double)(next() >> 11) * 0x1.0p-53; }
};

inline double snap(double v) { return std::floor(v * 1024.0) / 1024.0; }

struct BoxView {
    int nx, ny, nz;
    bool pz;
    bool wall_layer(int z) const { return !pz && (z == 0 || z == nz - 1); }
    int64_t cell(int x, int y, int z) const { return x + (int64_t)nx * (y + (int64_t)ny * z); }
};

// Marks the cells of one sphere (every periodic image) solid; returns how many
// cells with zlo <= z < zhi (outside wall layers) were fluid before.
int64_t stamp(const BoxView &b, uint8_t *mask, double cx, double cy, double cz, double r, int zlo,
              int zhi)
{
    const double r2 = r * r;
    int64_t turned = 0;
    const int mzr = b.pz ? 1 : 0;
    for (int mz = -mzr; mz <= mzr; ++mz) {
        const double iz = cz + (double)mz * b.nz;
        const int za = std::max(0, (int)std::ceil(iz - r)), zb = std::min(b.nz - 1, (int)std::floor(iz + r));
        for (int my = -1; my <= 1; ++my) {
            const double iy = cy + (double)my * b.ny;
            const int ya = std::max(0, (int)std::ceil(iy - r)), yb = std::min(b.ny - 1, (int)std::floor(iy + r));
            for (int mx = -1; mx <= 1; ++mx) {
                const double ix = cx + (double)mx * b.nx;
                const int xa = std::max(0, (int)std::ceil(ix - r)), xb = std::min(b.nx - 1, (int)std::floor(ix + r));
                if (xa > xb || ya > yb || za > zb) continue;
                for (int z = za; z <= zb; ++z) {
                    const double dz = (double)z - iz;
                    const bool counted = z >= zlo && z < zhi && !b.wall_layer(z);
                    for (int y = ya; y <= yb; ++y) {
                        const double dy = (double)y - iy;
                        const double ryz = r2 - dz * dz - dy * dy;   // exact
                        if (ryz < 0.0) continue;
                        uint8_t *row = mask + b.cell(0, y, z);
                        for (int x = xa; x <= xb; ++x) {
                            const double dx = (double)x - ix;
                            if (dx * dx <= ryz && !row[x]) {
                                row[x] = 1;
                                turned += counted;
                            }
                        }
                    }
                }
            }
        }
    }
    return turned;
}

void init_walls(const BoxView &b, uint8_t *mask)
{
    if (b.pz) return;
    const size_t plane = (size_t)b.nx * b.ny;
    std::memset(mask, 1, plane);
    std::memset(mask + (size_t)(b.nz - 1) * plane, 1, plane);
}

bool box_ok(const lbm_box &box)
{
    if (box.nx < 1 || box.ny < 1 || box.nz < 1) return false;
    if ((int64_t)box.nx * box.ny * box.nz >= (int64_t)1 << 31) return false;
    if (!box.periodic_z) {
        if (box.nz < 3) return false;
        if (!(box.q_lo > 0.0 && box.q_lo <= 1.0 && box.q_hi > 0.0 && box.q_hi <= 1.0)) return false;
    }
    return true;
}

}  // namespace

int place_and_voxelise(const lbm_sphere_params &p, Geometry &g)
{
    const lbm_box &box = p.box;
    if (!box_ok(box)) return LBM_EINVAL;
    if (!(p.layer_z1 > p.layer_z0) || !(p.r_min > 0.0) || !(p.r_max >= p.r_min)) return LBM_EINVAL;
    if (2.0 * p.r_max >= box.nx || 2.0 * p.r_max >= box.ny || (box.periodic_z && 2.0 * p.r_max >= box.nz))
        return LBM_EINVAL;
    if (p.max_spheres < 0 || p.max_rejects < 1) return LBM_EINVAL;
    const BoxView b{box.nx, box.ny, box.nz, box.periodic_z != 0};
    g.box = box;
    g.mask.assign((size_t)g.ncell(), 0);
    init_walls(b, g.mask.data());
    g.spheres.clear();

    const int zlo = (int)std::ceil(p.layer_z0), zhi = (int)std::ceil(p.layer_z1);
    int64_t layer_cells = 0;
    for (int z = std::max(zlo, 0); z < std::min(zhi, box.nz); ++z)
        if (!b.wall_layer(z)) layer_cells += (int64_t)box.nx * box.ny;
    int64_t layer_fluid = layer_cells;
    double phi = layer_cells > 0 ? 1.0 : 0.0;

    SplitMix64 rng{p.seed};
    int64_t misses = 0;
    while (layer_cells > 0 && phi > p.porosity) {
        const double cx = snap(rng.unit() * box.nx);
        const double cy = snap(rng.unit() * box.ny);
        const double cz = snap(p.layer_z0 + rng.unit() * (p.layer_z1 - p.layer_z0));
        const double r = snap(p.r_min + rng.unit() * (p.r_max - p.r_min));
        if (!p.allow_overlap) {
            bool hit = false;
            const size_t n = g.spheres.size() / 4;
            for (size_t j = 0; j < n && !hit; ++j) {
                const double *o = &g.spheres[4 * j];
                double d[3] = {cx - o[0], cy - o[1], cz - o[2]};
                const double ext[3] = {(double)box.nx, (double)box.ny, (double)box.nz};
                const int per = box.periodic_z ? 3 : 2;
                for (int a = 0; a < per; ++a) {
                    if (d[a] > 0.5 * ext[a]) d[a] -= ext[a];
                    else if (d[a] < -0.5 * ext[a]) d[a] += ext[a];
                }
                const double reach = r + o[3];
                hit = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < reach * reach;
            }
            if (hit) {
                if (++misses >= p.max_rejects) return LBM_EPACKING;
                continue;
            }
        }
        misses = 0;
        if ((int64_t)(g.spheres.size() / 4) >= p.max_spheres) return LBM_EINVAL;
        g.spheres.insert(g.spheres.end(), {cx, cy, cz, r});
        layer_fluid -= stamp(b, g.mask.data(), cx, cy, cz, r, zlo, zhi);
        phi = (double)layer_fluid / (double)layer_cells;
    }
    g.porosity = phi;
    count_fluid_and_links(g);
    return LBM_OK;
}

int voxelise_list(const lbm_box &box, const double *xyzr, int64_t n, Geometry &g)
{
    if (!box_ok(box) || n < 0 || (n > 0 && !xyzr)) return LBM_EINVAL;
    for (int64_t s = 0; s < n; ++s) {
        const double r = xyzr[4 * s + 3];
        if (!(r > 0.0) || 2.0 * r >= box.nx || 2.0 * r >= box.ny || (box.periodic_z && 2.0 * r >= box.nz))
            return LBM_EINVAL;
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(xyzr[4 * s + a])) return LBM_EINVAL;
    }
    const BoxView b{box.nx, box.ny, box.nz, box.periodic_z != 0};
    g.box = box;
    g.mask.assign((size_t)g.ncell(), 0);
    init_walls(b, g.mask.data());
    g.spheres.assign(xyzr, xyzr + 4 * n);
    for (int64_t s = 0; s < n; ++s)
        stamp(b, g.mask.data(), xyzr[4 * s], xyzr[4 * s + 1], xyzr[4 * s + 2], xyzr[4 * s + 3], 0, 0);
    count_fluid_and_links(g);
    int64_t fl = g.n_fluid;
    g.porosity = (double)fl / (double)g.ncell();
    return LBM_OK;
}

// Fluid cells and wall links (fluid cell, k) whose neighbour x + e_k is solid
// or beyond a non-periodic face.
void count_fluid_and_links(Geometry &g)
{
    const lbm_box &box = g.box;
    const int nx = box.nx, ny = box.ny, nz = box.nz;
    const bool pz = box.periodic_z != 0;
    const uint8_t *m = g.mask.data();
    int64_t nf = 0, nl = 0;
#pragma omp parallel for reduction(+ : nf, nl) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (m[x + (int64_t)nx * (y + (int64_t)ny * z)]) continue;
                ++nf;
                for (int k = 1; k < kQ; ++k) {
                    int xn = x + ex(k), yn = y + ey(k), zn = z + ez(k);
                    xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
                    yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
                    if (pz) zn = zn < 0 ? zn + nz : (zn >= nz ? zn - nz : zn);
                    else if (zn < 0 || zn >= nz) { ++nl; continue; }
                    nl += m[xn + (int64_t)nx * (yn + (int64_t)ny * zn)];
                }
            }
    g.n_fluid = nf;
    g.n_links = nl;
}

// Every sphere image is listed in each bin of kBinEdge^3 cells that its
// bounding box grown by `grow` cells overlaps.  With grow = 2 a link starting
// in a bin (at most sqrt(2) long) can only enter images listed for that bin;
// with grow = T every image within distance T of a cell of the bin is listed.
void build_bins(const lbm_box &box, const std::vector<double> &spheres, Bins &bins, double grow)
{
    bins.nbx = (box.nx + kBinEdge - 1) / kBinEdge;
    bins.nby = (box.ny + kBinEdge - 1) / kBinEdge;
    bins.nbz = (box.nz + kBinEdge - 1) / kBinEdge;
    const size_t nb = (size_t)bins.nbx * bins.nby * bins.nbz;
    std::vector<std::vector<SphereImage>> per_bin(nb);
    const int mzr = box.periodic_z ? 1 : 0;
    const int ext[3] = {box.nx, box.ny, box.nz};
    for (size_t s = 0; s < spheres.size() / 4; ++s) {
        const double *sp = &spheres[4 * s];
        for (int mz = -mzr; mz <= mzr; ++mz)
            for (int my = -1; my <= 1; ++my)
                for (int mx = -1; mx <= 1; ++mx) {
                    const SphereImage im{sp[0] + (double)mx * box.nx, sp[1] + (double)my * box.ny,
                                         sp[2] + (double)mz * box.nz, sp[3]};
                    const double c[3] = {im.x, im.y, im.z};
                    int lo[3], hi[3];
                    bool empty = false;
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = std::max(0, (int)std::floor(c[a] - im.r - grow));
                        hi[a] = std::min(ext[a] - 1, (int)std::ceil(c[a] + im.r + grow));
                        empty |= lo[a] > hi[a];
                    }
                    if (empty) continue;
                    for (int bz = lo[2] / kBinEdge; bz <= hi[2] / kBinEdge; ++bz)
                        for (int by = lo[1] / kBinEdge; by <= hi[1] / kBinEdge; ++by)
                            for (int bx = lo[0] / kBinEdge; bx <= hi[0] / kBinEdge; ++bx)
                                per_bin[bx + (size_t)bins.nbx * (by + (size_t)bins.nby * bz)].push_back(im);
                }
    }
    bins.start.assign(nb + 1, 0);
    size_t total = 0;
    for (size_t i = 0; i < nb; ++i) {
        bins.start[i] = (int32_t)total;
        total += per_bin[i].size();
    }
    bins.start[nb] = (int32_t)total;
    bins.images.clear();
    bins.images.reserve(total);
    for (auto &v : per_bin) bins.images.insert(bins.images.end(), v.begin(), v.end());
}

}  // namespace lbm
