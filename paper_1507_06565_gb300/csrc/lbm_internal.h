// lbm_internal.h -- internal declarations of liblbm (not part of the ABI).
//
// Data layout in device memory (all arrays in the caller's workspace):
//   pdf        [19][n_pad]  shifted populations h_k = f_k - w_k, storage type T,
//                           in-place AA pattern (see lbm_step.cu)
//   nbr        [18][n_pad]  int32 fluid index of x + e_k (k = 1..18), -1 if solid
//   lmask      [n_pad]      uint32, bit k set when x + e_k is solid (wall link k)
//   warp_off   [n_pad/32]   uint32, index of the first link of each aligned group
//                           of 32 fluid cells in the link arrays
//   link_a     [n_links]    float, CLI coefficient (1-2q)/(1+2q), 0 for bounce-back
//   link_q     [n_links]    double, link fraction q (kept for export)
//   fluid_cell [n_pad]      int32 cell index c = x + nx (y + ny z)
//   plane_off  [nz+1]       int32 first fluid index of each z plane
//   row_words  [ny*nz][nw]  uint2 per 32-cell word of each x-row (y, z):
//                           {fluid bitmask, fluid index of its first fluid cell};
//                           a neighbour's index is base + popc(bits below x)
//   cell_xr    [n_pad]      uint32 x | (row << x_bits), row = y + ny z
//   u_cur/u_prev [3][n_pad] float velocity snapshots (fluid order), rho_cur [n_pad]
//                           holds rho - 1
// Links of a cell are stored in increasing k; cells in fluid order, so the
// first link of cell i is warp_off[i/32] + (links of cells i&~31 .. i-1).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "lbm.h"

namespace lbm {

constexpr int kQ = 19;
constexpr int kBlock = 256;   // threads per block of the per-cell kernels
constexpr int kBinEdge = 8;   // edge (cells) of the sphere-image bins

// ---------------------------------------------------------------------------
// D3Q19 velocity set (ordering documented in lbm.h).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex(int k)
{
    return (k == 1 || k == 7 || k == 9 || k == 11 || k == 13) ? 1
         : (k == 2 || k == 8 || k == 10 || k == 12 || k == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int k)
{
    return (k == 3 || k == 7 || k == 10 || k == 15 || k == 17) ? 1
         : (k == 4 || k == 8 || k == 9 || k == 16 || k == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez(int k)
{
    return (k == 5 || k == 11 || k == 14 || k == 15 || k == 18) ? 1
         : (k == 6 || k == 12 || k == 13 || k == 16 || k == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
__host__ __device__ constexpr double weight(int k)
{
    return k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// One sphere image with its periodic shift applied (x, y, z, r).
struct SphereImage {
    double x, y, z, r;
};

// Host geometry behind the lbm_geometry handle.
struct Geometry {
    lbm_box box{};
    std::vector<double> spheres;   // [n][4]
    std::vector<uint8_t> mask;     // [ncell], 1 = solid
    int64_t n_fluid = 0;
    int64_t n_links = 0;
    double porosity = 1.0;
    int64_t ncell() const { return (int64_t)box.nx * box.ny * box.nz; }
};

// Sphere images binned on a grid of kBinEdge^3 cells (host build, device use).
struct Bins {
    int nbx = 0, nby = 0, nbz = 0;
    std::vector<int32_t> start;          // [nbins+1]
    std::vector<SphereImage> images;
};

// Workspace carve-up.
struct Layout {
    size_t pdf, nbr, lmask, warp_off, warp_cnt, link_a, link_q, fluid_cell, plane_off, row_words, cell_xr;
    size_t u_cur, u_prev, rho_cur, prof_prev, bins_start, bins_img, scan_tmp, partials, result, total;
    // build-time aliases inside the pdf region
    size_t idx_map, mask;
    int32_t n_pad;
    int64_t n_scan_blocks, n_partials;
};

struct Solver {
    lbm_box box{};
    lbm_params params{};
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    Layout lay{};
    int64_t n_cells = 0;
    int32_t n_fluid = 0;
    int32_t n_pad = 0;
    int64_t n_links = 0;
    int64_t n_spheres = 0;
    int64_t steps = 0;
    bool has_prev = false;
    bool has_prev_profile = false;
    double omega_p = 0, omega_m = 0, nu = 0;
    double drho_shift = 0;   // uniform density shift applied by the next step
    int nbins_x = 0, nbins_y = 0, nbins_z = 0;
    int n_words = 0;          // 32-cell words per row
    int x_bits = 0;           // bits of x in cell_xr
    bool odd_rows = true;     // odd step computes neighbours from row bitmasks
    // device pointers
    void *pdf = nullptr;
    int32_t *nbr = nullptr;
    uint32_t *lmask = nullptr;
    uint32_t *warp_off = nullptr;
    float *link_a = nullptr;
    double *link_q = nullptr;
    int32_t *fluid_cell = nullptr;
    int32_t *plane_off = nullptr;
    uint2 *row_words = nullptr;
    uint32_t *cell_xr = nullptr;
    float *u_cur = nullptr;
    float *u_prev = nullptr;
    float *rho_cur = nullptr;
    double *prof_prev = nullptr;
    double *partials = nullptr;
    double *result = nullptr;
};

// ---- host geometry (lbm_geometry.cpp) ----
int place_and_voxelise(const lbm_sphere_params &p, Geometry &g);
int voxelise_list(const lbm_box &box, const double *xyzr, int64_t n, Geometry &g);
void count_fluid_and_links(Geometry &g);
void build_bins(const lbm_box &box, const std::vector<double> &spheres, Bins &bins);

// ---- workspace (lbm_api.cpp) ----
Layout make_layout(const lbm_box &box, int64_t n_fluid, int64_t n_links, int storage,
                   size_t n_bins, size_t n_images);
// bits needed for x in cell_xr; rows must fit in the remaining bits
int x_bits_for(int nx);
bool rows_packable(const lbm_box &box);

// ---- device build (lbm_build.cu) ----
int device_build(Solver &s, const Geometry &g, const Bins &bins);

// ---- step kernels (lbm_step.cu) ----
int launch_init(Solver &s, const float *dev_u0);
int launch_steps(Solver &s, int64_t n);

// ---- post-processing (lbm_post.cu) ----
int launch_fluid_moments(Solver &s);                       // -> u_cur, rho_cur
int launch_scatter_moments(Solver &s, float *rho, float *u);
int launch_plane_average(Solver &s);                       // -> result[0 .. 3 nz)
int launch_permeability(Solver &s, int z_lo, int z_hi);    // -> result[0]
int launch_residual(Solver &s);                            // -> result[0..2]
int launch_mass(Solver &s);                                // -> result[3nz+4]
int launch_profile_residual(Solver &s);                    // -> result[3nz+1 .. 3nz+3]
int launch_populations(Solver &s, float *out);

// ---- shared host helpers ----
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int storage_bytes(int storage) { return storage == LBM_F32 ? 4 : 2; }

}  // namespace lbm

// The handle types of the ABI are the internal classes.
struct lbm_geometry : public lbm::Geometry {};
struct lbm_solver : public lbm::Solver {};
