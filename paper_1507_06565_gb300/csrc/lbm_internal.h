// lbm_internal.h -- internal declarations of liblbm (not part of the ABI).
//
// Data layout in device memory (all arrays in the caller's workspace):
//   pdf        [19][n_pad]  shifted populations h_k = f_k - w_k, storage type T,
//                           in-place AA pattern (see lbm_step.cu)
//   nbr        [18][n_pad]  int32 fluid index of x + e_k (k = 1..18), -1 if solid
//   lmask      [n_pad]      uint32, bit k set when x + e_k is solid (wall link k,
//                           kLinkBits); bit 19 when x = nx - 1, bit 20 when x = 0
//   warp_off   [n_pad/32]   uint32, index of the first link of each aligned group
//                           of 32 fluid cells in the link arrays
//   link_a     [n_links]    float, CLI coefficient (1-2q)/(1+2q), 0 for bounce-back
//   link_q     [n_links]    double, link fraction q (kept for export)
//   fluid_cell [n_pad]      int32 cell index c = x + nx (y + ny z)
//   plane_off  [nz+1]       int32 first fluid index of each z plane
//   row_words  [ny*nz][nw]  uint2 per 32-cell word of each x-row (y, z) of
//                           every part (part b from words_base):
//                           {fluid bitmask, fluid index of its first fluid cell};
//                           a neighbour's index is base + popc(bits below x)
//   cell_xr    [n_pad]      uint32 x | y << 11 | z << 22 (kXyz* bits)
//   tile_rows  [n_pad/256]  int4 descriptor of a tile whose odd-step
//                           neighbours come from row words staged in shared
//                           memory (see k_stage_tiles), {-1, ..} otherwise
//   u_cur/u_prev [3][n_pad] float velocity snapshots (fluid order), rho_cur [n_pad]
//                           holds rho - 1
//   ref, ref_next [n_planes][kRefStride] float reference populations of the
//                           referenced planes (see below), zero elsewhere
//   tile_ref   [n_pad/256]  int2 {global plane of the tile's first cell, fluid
//                           index where the next plane starts} for tiles that
//                           use reference populations, {-1, 0} otherwise
//
// Reference populations.  In a fully fluid plane far from the porous layer
// the flow is the same at every cell, so FP32 rounding of the stored
// populations is the same at every cell of the plane and does not average
// out: it acts like a spurious body force of up to ~2^-24 |f| per step.  In
// such planes the slot A[.][y] of a population of direction k (owner cell y
// in plane z) stores f_k - w_k - R_k(z), where R_k(z) = f_k^eq(1, u_z) - w_k
// is the equilibrium of the plane's mean velocity u_z (refreshed by
// lbm_recenter), which leaves only the small non-equilibrium part to round.
// A plane is referenced when it and both neighbour planes lie entirely in
// dense tiles (every cell that reads or writes its slots then knows its
// plane); everywhere else R = 0 and the storage is the plain shifted one.
// Links of a cell are stored in increasing k; cells in fluid order, so the
// first link of cell i is warp_off[i/32] + (links of cells i&~31 .. i-1).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "lbm.h"

namespace lbm {

constexpr int kQ = 19;
constexpr int kBlock = 256;   // threads per block of the per-cell kernels
constexpr int kBinEdge = 8;   // edge (cells) of the sphere-image bins
// With LBM_FLAG_CLI_SAFEGUARDS, links whose wall lies closer than this
// fraction of the link to the node use simple bounce-back instead of
// Eq. (CLI) (stability in sharp corners, with the two-cell-gap rule of
// k_links).
constexpr double kCliQmin = 0.1;
constexpr int kRefStride = 20;   // floats per plane of reference populations (19 used)
// lmask: the link bits 1..18, and two bits for the cells at the ends of an
// x-row (their x -+ 1 neighbour wraps around the periodic x span)
constexpr uint32_t kLinkBits = 0x7FFFEu;
constexpr uint32_t kXLast = 1u << 19;    // x = nx - 1
constexpr uint32_t kXFirst = 1u << 20;   // x = 0
// packed cell position x | y << 11 | z << 22 (row bitmask variants)
constexpr int kXyzBitsX = 11, kXyzBitsY = 11, kXyzBitsZ = 10;
// row words one tile of the odd step stages in shared memory (3 bands of
// rows: the planes z - 1, z, z + 1 of the tile's rows and one more row on
// either side)
constexpr int kMaxStagedWords = 512;

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
// Sphere images binned on a grid of kBinEdge^3 cells (host build, device use).
struct Bins {
    int nbx = 0, nby = 0, nbz = 0;
    std::vector<int32_t> start;          // [nbins+1]
    std::vector<SphereImage> images;
};

struct Geometry {
    lbm_box box{};
    std::vector<double> spheres;   // [n][4]
    std::vector<uint8_t> mask;     // [ncell], 1 = solid
    int64_t n_fluid = 0;
    int64_t n_links = 0;
    double porosity = 1.0;
    Bins link_bins;                // the bins of the link fractions, built with the geometry
    int64_t ncell() const { return (int64_t)box.nx * box.ny * box.nz; }
};

// One independent box of a solver.  A solver advances the union of its parts
// in one launch per step: fluid cells of part b occupy the fluid indices
// [fluid_off, fluid_off + n_fluid) and the concatenated cell indices
// [cell_base, cell_base + n_cells); neighbour indices are global, so the step
// kernels never need to know which part a cell belongs to.
struct Part {
    lbm_box box{};
    int64_t cell_base = 0;
    int64_t n_cells = 0;
    int32_t fluid_off = 0;
    int32_t n_fluid = 0;
    int64_t n_links = 0;
    int64_t n_spheres = 0;
    int32_t plane_base = 0;   // first plane of this part in the concatenated plane arrays
    int32_t poff_base = 0;    // first entry of this part in plane_off (nz + 1 per part)
    int64_t words_base = 0;   // first row word of this part
    bool has_prev_profile = false;
};

// Workspace carve-up.
struct Layout {
    size_t pdf, nbr, lmask, warp_off, warp_cnt, link_a, link_q, fluid_cell, plane_off, row_words, cell_xr, tile_desc,
        tile_rows;
    size_t u_cur, u_prev, rho_cur, prof_prev, bins_start, bins_img, scan_tmp, partials, result, total;
    size_t part_shift, part_foff, status, ref, ref_next, tile_ref, plane_flag;
    // build-time aliases inside the pdf region
    size_t idx_map, mask;
    int32_t n_pad;
    int64_t n_scan_blocks, n_partials;
    int32_t n_planes;           // sum of nz over parts
    int32_t n_parts;
};

// Offsets (in doubles) inside the result region.
inline size_t res_field(const Layout &L) { return 3 * (size_t)L.n_planes; }        // 3 field-residual sums
inline size_t res_mass(const Layout &L) { return res_field(L) + 4; }               // 2 global mass sums
inline size_t res_part(const Layout &L, int b) { return res_mass(L) + 4 + 8 * (size_t)b; }
// per part: [0] K, [1..3] profile residual sums, [4..5] mass sums

struct Solver {
    lbm_box box{};                 // box of part 0 (the whole solver when unbatched)
    lbm_params params{};
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    Layout lay{};
    std::vector<Part> parts;
    int64_t n_cells = 0;
    int32_t n_fluid = 0;
    int32_t n_pad = 0;
    int64_t n_links = 0;
    int64_t n_spheres = 0;
    int64_t steps = 0;
    bool has_prev = false;
    double omega_p = 0, omega_m = 0, nu = 0;
    bool shift_pending = false;    // the next step applies part_shift
    std::vector<float> shift_host; // per-part shifts (host copy)
    int n_words = 0;               // 32-cell words per row (part 0)
    bool rows_ok = false;          // every part fits the packed positions: row words and cell_xr exist
    bool odd_rows = true;          // odd step computes neighbours from row bitmasks
    bool staged_rows = false;      // odd step stages row words per tile (LBM_FLAG_STAGED_NEIGHBOURS)
    bool derived_nbrs = false;     // odd step derives x-shifted neighbours (LBM_FLAG_DERIVED_NEIGHBOURS)
    // launch schedule: grid sizes of the even/odd step (0 = one block per
    // tile, -1 = the staged even kernel on one wave of resident blocks)
    int grid_even = 0, grid_odd = 0;
    int tune_state = 0;            // 0 untuned, 1 tuning, 2 done
    int tune_idx = 0;
    std::vector<int> tune_grids_even, tune_grids_odd;   // candidates (-1: staged even kernel)
    std::vector<float> tune_ms_even, tune_ms_odd;
    int tune_count_even = 0, tune_count_odd = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // CUDA graph of kGraphSteps steps starting at even parity
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    bool use_graph = true;
    bool autotune = true;
    bool staged_even = false;      // LBM_FLAG_STAGED_EVEN
    // device pointers
    void *pdf = nullptr;
    int32_t *nbr = nullptr;
    uint32_t *lmask = nullptr;
    uint32_t *warp_off = nullptr;
    float *link_a = nullptr;
    double *link_q = nullptr;
    int32_t *fluid_cell = nullptr;
    int32_t *plane_off = nullptr;
    // per tile of kBlock cells: {fluid index of cell (0, 0, z) of the tile's
    // first plane, nx | ny << 16} when every cell of the tile lies in a fully
    // fluid plane whose neighbour planes are fully fluid too (its neighbour
    // indices are then arithmetic and it has no wall link), else {-1, 0}
    int2 *tile_desc = nullptr;
    int32_t dense_lo = 0, dense_hi = 0;   // tiles [dense_lo, dense_hi) hold every dense tile
    // reference populations (see the layout notes): per plane of all parts,
    // the current ones and those the next step switches to
    float *ref = nullptr;
    float *ref_next = nullptr;
    int2 *tile_ref = nullptr;
    int32_t ref_lo = 0, ref_hi = 0;       // tiles [ref_lo, ref_hi) hold every tile with tile_ref.x >= 0
    std::vector<uint8_t> plane_referenced;   // per global plane (host copy)
    uint8_t *plane_flag = nullptr;        // the same on the device
    bool has_ref = false;                 // some plane is referenced
    bool ref_pending = false;             // the next step reads with ref and writes with ref_next
    uint2 *row_words = nullptr;
    uint32_t *cell_xr = nullptr;
    int4 *tile_rows = nullptr;
    int32_t rows_lo = 0, rows_hi = 0;    // tiles [rows_lo, rows_hi) hold every staged tile
    float *u_cur = nullptr;
    float *u_prev = nullptr;
    float *rho_cur = nullptr;
    double *prof_prev = nullptr;
    double *partials = nullptr;
    double *result = nullptr;
    float *part_shift = nullptr;
    int32_t *part_foff = nullptr;
    int *status = nullptr;   // set by a step kernel whose bounded wait gave up
    // a step kernel gave up a wait (reported once as LBM_ETIMEOUT): its block
    // left the tile's populations half-updated, so steps are refused until
    // lbm_reset re-initialises the state
    bool stale = false;
    ~Solver();
};

// ---- host geometry (lbm_geometry.cpp) ----
int place_and_voxelise(const lbm_sphere_params &p, Geometry &g);
int voxelise_list(const lbm_box &box, const double *xyzr, int64_t n, Geometry &g);
void count_fluid_and_links(Geometry &g);
void build_bins(const lbm_box &box, const std::vector<double> &spheres, Bins &bins, double grow = 2.0);

// ---- workspace (lbm_api.cpp) ----
Layout make_layout(const std::vector<const Geometry *> &geoms, int storage, size_t n_bins, size_t n_images);
// positions of the box fit the packing of cell_xr
bool rows_packable(const lbm_box &box);

// ---- device build (lbm_build.cu) ----
int device_build(Solver &s, const std::vector<const Geometry *> &geoms);

// ---- step kernels (lbm_step.cu) ----
int launch_init(Solver &s, const float *dev_u0);
int launch_steps(Solver &s, int64_t n);
int launch_wait_selftest(Solver &s, int max_polls);

// ---- post-processing (lbm_post.cu) ----
int launch_fluid_moments(Solver &s);                       // -> u_cur, rho_cur
int launch_scatter_moments(Solver &s, float *rho, float *u);
int launch_plane_average(Solver &s);                       // -> result[0 .. 3 n_planes)
int launch_permeability(Solver &s, int part, int z_lo, int z_hi);  // -> part slot [0]
int launch_residual(Solver &s);                            // -> res_field
int launch_profile_residual(Solver &s);                    // -> part slots [1..3]
int launch_mass(Solver &s);                                // -> res_mass, part slots [4..5]
int launch_populations(Solver &s, float *out);
int launch_reference_update(Solver &s);                    // u_cur -> ref_next

// ---- shared host helpers ----
// plane reference equilibria in use: FP16/BF16 storage unless turned off,
// FP32 storage when asked for
inline bool plane_references_on(const lbm_params &p)
{
    if (p.flags & LBM_FLAG_PLANE_REFERENCES) return true;
    return p.storage != LBM_F32 && !(p.flags & LBM_FLAG_NO_PLANE_REFERENCES);
}
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int storage_bytes(int storage) { return storage == LBM_F32 ? 4 : 2; }

}  // namespace lbm

// The handle types of the ABI are the internal classes.
struct lbm_geometry : public lbm::Geometry {};
struct lbm_solver : public lbm::Solver {};
