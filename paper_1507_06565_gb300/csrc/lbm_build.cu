// lbm_build.cu -- device construction of the sparse fluid list, the neighbour
// table and the wall-link list with the link fractions q of Eq. (CLI).
//
// Steps (all on the solver's stream), for each part (independent box) in turn:
//   1. per block of cells: count fluid cells of the uploaded solid mask;
//      exclusive scan of the block counts;
//   2. dense index map cell -> global fluid index (-1 solid) and fluid_cell[]
//      (concatenated cell index);
//   3. neighbour table nbr[k][i] and link mask lmask[i] (bit k: x + e_k solid),
//      packed positions and row bitmask words (boxes of up to 2048 x 2048 x
//      1024 cells), and the tiles whose odd step stages row words;
//   4. first fluid index of each z plane of the part;
// then over the whole solver: link counts per aligned group of 32 fluid cells
// and their exclusive scan; and again per part:
//   5. link fraction q and CLI coefficient a = (1-2q)/(1+2q) per link
//      (a = 0, bounce-back, when the second node x - e_k is solid; with the
//      corner safeguards also when x - 2 e_k is solid or when q < 0.1).
// The index map and the mask live in the population region, which is written
// only afterwards by the initialisation.
#include <algorithm>
#include <cstdio>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// 1. fluid count per block of kBlock cells
__global__ void k_count_fluid(const uint8_t *__restrict__ mask, int64_t ncell, uint32_t *__restrict__ counts)
{
    const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int fluid = c < ncell && !mask[c];
    const int n = __syncthreads_count(fluid);
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)n;
}

// Exclusive scan of n uint32 values in place by one block; the total goes to
// *total.  Sequential over chunks of kScanThreads with a running carry.
__global__ void k_scan_exclusive(uint32_t *__restrict__ v, int64_t n, uint32_t *__restrict__ total)
{
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    __shared__ uint32_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < n; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const uint32_t x = i < n ? v[i] : 0u;
        uint32_t s = x;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane == 31) warp_sums[warp] = s;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_sums[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            warp_sums[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const uint32_t carry = carry_s;
        const uint32_t before = (warp ? warp_sums[warp - 1] : 0u) + s - x;
        if (i < n) v[i] = carry + before;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry_s = carry + warp_sums[kScanThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

// 2. index map and fluid list (fluid cells keep increasing cell order)
__global__ void k_fill_index(const uint8_t *__restrict__ mask, int64_t ncell,
                             const uint32_t *__restrict__ block_off, int32_t fluid_off, int64_t cell_base,
                             int32_t *__restrict__ idx_map, int32_t *__restrict__ fluid_cell)
{
    __shared__ uint32_t warp_cnt[kBlock / 32];
    const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const bool fluid = c < ncell && !mask[c];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ballot = __ballot_sync(0xffffffffu, fluid);
    if (lane == 0) warp_cnt[warp] = __popc(ballot);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_cnt[w];
    before += __popc(ballot & ((1u << lane) - 1u));
    if (c < ncell) {
        const int32_t idx = fluid ? fluid_off + (int32_t)(block_off[blockIdx.x] + before) : -1;
        idx_map[c] = idx;
        if (fluid) fluid_cell[idx] = (int32_t)(cell_base + c);
    }
}

// Row bitmask words of one part (idx_map holds global fluid indices): one
// thread per (row, word) of 32 cells along x.
__global__ void k_row_words(const int32_t *__restrict__ idx_map, int nx, int64_t nrows, int nw,
                            uint2 *__restrict__ words)
{
    const int64_t t = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (t >= nrows * nw) return;
    const int64_t row = t / nw;
    const int w = (int)(t % nw);
    uint32_t bits = 0, base = 0;
    bool seen = false;
    for (int b = 0; b < 32; ++b) {
        const int x = 32 * w + b;
        if (x >= nx) break;
        const int32_t j = idx_map[row * nx + x];
        if (j >= 0) {
            bits |= 1u << b;
            if (!seen) base = (uint32_t)j;
            seen = true;
        }
    }
    words[t] = make_uint2(bits, base);
}

// 3. neighbour table, link mask and packed (x, row) of the fluid cells of one
//    part; idx_map holds global fluid indices.
__global__ void k_neighbours(const int32_t *__restrict__ idx_map, const int32_t *__restrict__ fluid_cell,
                             int32_t begin, int32_t end, int64_t cell_base, int32_t n_pad, int nx, int ny, int nz,
                             int periodic_z, int32_t *__restrict__ nbr, uint32_t *__restrict__ lmask,
                             uint32_t *__restrict__ cell_xr)
{
    const int32_t i = begin + (int32_t)(blockIdx.x * kBlock + threadIdx.x);
    if (i >= end) return;
    const int32_t c = (int32_t)(fluid_cell[i] - cell_base);
    const int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
    if (cell_xr) cell_xr[i] = (uint32_t)x | ((uint32_t)y << kXyzBitsX) | ((uint32_t)z << (kXyzBitsX + kXyzBitsY));
    uint32_t m = 0;
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        const int xn = wrap(x + ex(k), nx), yn = wrap(y + ey(k), ny);
        int zn = z + ez(k);
        int32_t j = -1;
        if (periodic_z) zn = wrap(zn, nz);
        if (zn >= 0 && zn < nz) j = idx_map[xn + nx * (yn + ny * zn)];
        nbr[(size_t)(k - 1) * n_pad + i] = j;
        m |= (uint32_t)(j < 0) << k;
    }
    if (x == nx - 1) m |= kXLast;
    if (x == 0) m |= kXFirst;
    lmask[i] = m;
}

// Padding cells beyond the last fluid cell: no links, neighbours -1.
__global__ void k_pad_cells(int32_t n_fluid, int32_t n_pad, int32_t *__restrict__ nbr, uint32_t *__restrict__ lmask,
                            int32_t *__restrict__ fluid_cell, uint32_t *__restrict__ cell_xr)
{
    const int32_t i = n_fluid + (int32_t)(blockIdx.x * kBlock + threadIdx.x);
    if (i >= n_pad) return;
    for (int k = 1; k < kQ; ++k) nbr[(size_t)(k - 1) * n_pad + i] = -1;
    lmask[i] = 0;
    fluid_cell[i] = 0;
    if (cell_xr) cell_xr[i] = 0;
}

// Link counts per aligned group of 32 fluid cells.
__global__ void k_warp_counts(const uint32_t *__restrict__ lmask, uint32_t *__restrict__ warp_cnt)
{
    const int32_t i = blockIdx.x * kBlock + threadIdx.x;
    uint32_t cnt = __popc(lmask[i] & kLinkBits);
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0) warp_cnt[i >> 5] = cnt;
}

// Entry parameter s in (0,1] of the ray p + s e into the sphere |x - c| <= r,
// d = p - c, p outside.  2.0 when the ray does not enter within the link.
// Every product and sum here is exact for coordinates on the 2^-10 grid; the
// explicit round-to-nearest intrinsics keep the compiler from contracting.
__device__ double sphere_entry(double dx, double dy, double dz, int kx, int ky, int kz, double r)
{
    const double A = (double)(kx * kx + ky * ky + kz * kz);
    const double B = __dadd_rn(__dadd_rn(__dmul_rn(dx, (double)kx), __dmul_rn(dy, (double)ky)),
                               __dmul_rn(dz, (double)kz));
    const double C = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)),
                               __dmul_rn(r, r));
    const double disc = __dsub_rn(__dmul_rn(B, B), __dmul_rn(A, C));
    if (!(B < 0.0) || disc < 0.0) return 2.0;
    // A = e.e is 1 or 2, so the division is exact as a multiplication by 1
    // or 1/2 (same bits, no FP64 division)
    const double s = __dmul_rn(__dsub_rn(-B, __dsqrt_rn(disc)), A == 1.0 ? 1.0 : 0.5);
    return s <= 1.0 ? s : 2.0;
}

struct LinkArgs {
    const int32_t *fluid_cell;
    const int32_t *nbr;
    const uint32_t *lmask;
    const uint32_t *warp_off;
    const int32_t *bin_start;
    const SphereImage *images;
    float *link_a;
    double *link_q;
    int32_t begin, end, n_fluid, n_pad;
    int64_t cell_base;
    int nx, ny, nz, periodic_z;
    int nbx, nby;
    double q_lo, q_hi;
    int simple_bounce_back;   // every link a = 0 (LBM_FLAG_SIMPLE_BOUNCE_BACK)
    int safeguards;           // LBM_FLAG_CLI_SAFEGUARDS
};

// 5. link fractions and CLI coefficients of the cells of one part.  The grid
// covers the aligned groups of 32 that contain the part; a warp owns the
// links of its 32 cells (stored contiguously from warp_off, cell by cell, in
// increasing k) and processes them 32 at a time, one link per lane: the lane
// finds the link's cell by a binary search over the warp's inclusive prefix
// sum of link counts and its direction as the r-th set bit of that cell's
// link mask.  (One cell per lane would run the candidate loop for every
// direction in which any lane of the warp has a link.)
__global__ void k_links(LinkArgs a)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t i = (a.begin & ~31) + (int32_t)(blockIdx.x * kBlock + threadIdx.x);
    const int32_t i0 = i - lane;   // first cell of the warp's group
    const uint32_t m = i < a.n_fluid ? a.lmask[i] & kLinkBits : 0u;
    const uint32_t cnt = __popc(m);
    uint32_t incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kAll, incl, d);
        if (lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(kAll, incl, 31);
    if (total == 0) return;   // warp-uniform
    const uint32_t wbase = a.warp_off[i0 >> 5];
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t l = base + (uint32_t)lane;   // this lane's link, relative to wbase
        // owner: the first lane whose inclusive count exceeds l
        int lo = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t v = __shfl_sync(kAll, incl, lo + step - 1);
            if (v <= l) lo += step;
        }
        const int j = lo < 31 ? lo : 31;
        const uint32_t mj = __shfl_sync(kAll, m, j);
        const uint32_t excl = __shfl_sync(kAll, incl, j) - __popc(mj);
        const int32_t c_i = i0 + j;
        if (l >= total || c_i < a.begin || c_i >= a.end) continue;
        // direction: the (l - excl)-th set bit of mj (0 <= l - excl < popc(mj),
        // since incl[j-1] <= l < incl[j])
        uint32_t mm = mj;
        for (uint32_t r = l - excl; r > 0; --r) mm &= mm - 1u;
        const int k = __ffs(mm) - 1;
        const int32_t c = (int32_t)(a.fluid_cell[c_i] - a.cell_base);
        const int x = c % a.nx, y = (c / a.nx) % a.ny, z = c / (a.nx * a.ny);
        const int bin = x / kBinEdge + a.nbx * (y / kBinEdge + a.nby * (z / kBinEdge));
        const int b0 = a.bin_start[bin], b1 = a.bin_start[bin + 1];
        const int kx = ex(k), ky = ey(k), kz = ez(k);
        double q = 2.0;
        if (!a.periodic_z) {
            const int bz = z + kz;
            if (bz <= 0) q = a.q_lo;
            if (bz >= a.nz - 1 && a.q_hi < q) q = a.q_hi;
        }
        for (int b = b0; b < b1; ++b) {
            const SphereImage im = a.images[b];
            // A link of length <= sqrt(2) can only enter a sphere whose centre is
            // within r + sqrt(2) of its start; the FP32 test keeps a margin of
            // ~0.17 r over that bound, so it never drops a candidate.
            const float fx = (float)x - (float)im.x, fy = (float)y - (float)im.y, fz = (float)z - (float)im.z;
            const float reach = (float)im.r + 1.5f;
            if (fx * fx + fy * fy + fz * fz > reach * reach) continue;
            const double s = sphere_entry((double)x - im.x, (double)y - im.y, (double)z - im.z, kx, ky, kz, im.r);
            if (s < q) q = s;
        }
        // bounce-back when the second node x_f2 = x - e_k is solid (Eq. (CLI)
        // has no second node); with the safeguards also when x_f2 is itself a
        // wall node on the link's line (x - 2 e_k solid) or when the wall is
        // within kCliQmin of the node: Eq. (CLI) can grow without bound in such
        // sharp corners of overlapping packings
        bool fallback = a.simple_bounce_back || ((mj >> opp(k)) & 1u) || (a.safeguards && q < kCliQmin);
        if (!fallback && a.safeguards) {
            const int32_t x2 = a.nbr[(size_t)(opp(k) - 1) * a.n_pad + c_i];
            fallback = (a.lmask[x2] >> opp(k)) & 1u;
        }
        const double coef = fallback ? 0.0 : __ddiv_rn(__dsub_rn(1.0, __dmul_rn(2.0, q)), __dadd_rn(1.0, __dmul_rn(2.0, q)));
        a.link_q[wbase + l] = q;
        a.link_a[wbase + l] = (float)coef;
    }
}

// 4. first fluid index of each z plane of one part (plane_off[nz] = end)
__global__ void k_plane_offsets(const int32_t *__restrict__ fluid_cell, int32_t begin, int32_t end,
                                int64_t cell_base, int plane, int nz, int32_t *__restrict__ plane_off)
{
    const int32_t i = begin + (int32_t)(blockIdx.x * kBlock + threadIdx.x);
    if (i >= end) return;
    const int z = (int)((fluid_cell[i] - cell_base) / plane);
    const int zp = i == begin ? -1 : (int)((fluid_cell[i - 1] - cell_base) / plane);
    for (int zz = zp + 1; zz <= z; ++zz) plane_off[zz] = i;
    if (i == end - 1)
        for (int zz = z + 1; zz <= nz; ++zz) plane_off[zz] = end;
}

// Staged tiles of one part (Solver::tile_rows): a tile of kBlock fluid cells
// that lies in the part and is not dense gets the descriptor of the three
// bands of rows its odd step stages: the rows r_first - 1 .. r_last + 1
// (r = y + ny z) of its first and last cell, and the same rows one plane
// below and above.  {first row word of the part, r_first - 1,
// band_rows | nw << 8 | periodic_z << 15 | nz << 16, nx | ny << 16}; tiles
// whose bands exceed kMaxStagedWords keep the table.
__global__ void k_stage_tiles(const int32_t *__restrict__ fluid_cell, const int2 *__restrict__ dense,
                              int32_t begin, int32_t end, int64_t cell_base, int nx, int ny, int nz, int periodic_z,
                              int64_t words_base, int4 *__restrict__ out)
{
    const int32_t t = begin / kBlock + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    const int32_t first = t * kBlock, last = first + kBlock - 1;
    if (first >= end) return;
    if (first < begin || last >= end) return;   // straddles a part boundary or the end: table
    if (dense[t].x >= 0) return;                 // computed indices
    const int32_t r_first = (int32_t)((fluid_cell[first] - cell_base) / nx);
    const int32_t r_last = (int32_t)((fluid_cell[last] - cell_base) / nx);
    const int band_rows = r_last - r_first + 3, nw = (nx + 31) / 32;
    if (band_rows > 255 || 3 * band_rows * nw > kMaxStagedWords) return;
    out[t] = make_int4((int32_t)words_base, r_first - 1, band_rows | (nw << 8) | (periodic_z << 15) | (nz << 16),
                       nx | (ny << 16));
}

// Dense tiles of one part (see Solver::tile_desc): tile t holds fluid cells
// t*kBlock .. t*kBlock+kBlock-1; it is dense when they all belong to this part
// and lie in planes z with 1 <= z <= nz - 2 such that planes z - 1, z, z + 1
// are fully fluid.  One thread per tile of the part.
__global__ void k_dense_tiles(const int32_t *__restrict__ fluid_cell, const int32_t *__restrict__ plane_off,
                              int32_t begin, int32_t end, int64_t cell_base, int nx, int ny, int nz,
                              int2 *__restrict__ desc)
{
    const int32_t t = begin / kBlock + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    const int32_t first = t * kBlock, last = first + kBlock - 1;
    if (first >= end) return;
    if (first < begin || last >= end) return;   // straddles a part boundary or the end: not dense
    const int64_t plane = (int64_t)nx * ny;
    const int z0 = (int)((fluid_cell[first] - cell_base) / plane);
    const int z1 = (int)((fluid_cell[last] - cell_base) / plane);
    if (z0 < 1 || z1 > nz - 2) return;
    for (int z = z0 - 1; z <= z1 + 1; ++z)
        if ((int64_t)(plane_off[z + 1] - plane_off[z]) != plane) return;
    desc[t] = make_int2(plane_off[z0], nx | (ny << 16));
}

}  // namespace

// Referenced planes (lbm_internal.h): plane z of a part is referenced when
// planes z-1, z and z+1 are fully fluid and every tile that holds one of
// their cells is dense, so that every cell reading or writing a slot of the
// plane knows the plane.  A dense tile uses reference populations when one of
// the planes of its cells or their neighbour planes is referenced; it then
// gets {global plane of its first cell, first fluid index of the next plane}.
// Only parts whose planes hold at least a tile of cells qualify (a tile then
// spans at most two planes).
static void mark_reference_planes(Solver &s, const std::vector<int2> &desc, const std::vector<int32_t> &poff,
                                  std::vector<int2> &tref)
{
    for (const Part &P : s.parts) {
        const int nz = P.box.nz;
        const int64_t plane = (int64_t)P.box.nx * P.box.ny;
        if (plane < kBlock || P.n_fluid == 0) continue;
        const int32_t *po = poff.data() + P.poff_base;
        std::vector<uint8_t> cov((size_t)nz, 0), refd((size_t)nz, 0);
        for (int z = 0; z < nz; ++z) {
            const int32_t b = po[z], e = po[z + 1];
            if ((int64_t)(e - b) != plane) continue;
            bool all = true;
            for (int32_t t = b / kBlock; t <= (e - 1) / kBlock && all; ++t) all = desc[(size_t)t].x >= 0;
            cov[(size_t)z] = all;
        }
        for (int z = 1; z + 1 < nz; ++z) {
            refd[(size_t)z] = cov[(size_t)z - 1] && cov[(size_t)z] && cov[(size_t)z + 1];
            s.plane_referenced[(size_t)(P.plane_base + z)] = refd[(size_t)z];
        }
        const int32_t t0 = P.fluid_off / kBlock, t1 = (P.fluid_off + P.n_fluid - 1) / kBlock;
        for (int32_t t = t0; t <= t1; ++t) {
            const int2 d = desc[(size_t)t];
            if (d.x < 0) continue;
            // planes of the tile's first and last cell
            const int32_t first = t * kBlock, last = first + kBlock - 1;
            const int z0 = (int)(std::upper_bound(po, po + nz + 1, first) - po) - 1;
            const int z1 = (int)(std::upper_bound(po, po + nz + 1, last) - po) - 1;
            bool touch = false;
            for (int z = std::max(z0 - 1, 0); z <= std::min(z1 + 1, nz - 1); ++z) touch |= refd[(size_t)z] != 0;
            if (touch) tref[(size_t)t] = make_int2(P.plane_base + z0, po[z0 + 1]);
        }
    }
}

#define LBM_CUDA_TRY(x)                                     \
    do {                                                    \
        if ((x) != cudaSuccess) return LBM_ECUDA;           \
    } while (0)

static unsigned blocks_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

int device_build(Solver &s, const std::vector<const Geometry *> &geoms)
{
    const Layout &L = s.lay;
    cudaStream_t st = s.stream;
    uint8_t *d_mask = (uint8_t *)(s.ws + L.mask);
    int32_t *d_idx = (int32_t *)(s.ws + L.idx_map);
    uint32_t *d_scan = (uint32_t *)(s.ws + L.scan_tmp);
    uint32_t *d_wcnt = (uint32_t *)(s.ws + L.warp_cnt);
    uint32_t *d_total = (uint32_t *)(s.ws + L.result);
    int32_t *d_bstart = (int32_t *)(s.ws + L.bins_start);
    SphereImage *d_img = (SphereImage *)(s.ws + L.bins_img);
    uint32_t *cell_xr = s.rows_ok ? s.cell_xr : nullptr;
    std::vector<uint32_t> counts(s.parts.size() + 1, 0);

    LBM_CUDA_TRY(cudaMemsetAsync(s.tile_desc, 0xFF, sizeof(int2) * (s.n_pad / kBlock), st));
    LBM_CUDA_TRY(cudaMemsetAsync(s.tile_rows, 0xFF, sizeof(int4) * (s.n_pad / kBlock), st));
    LBM_CUDA_TRY(cudaMemsetAsync(s.status, 0, sizeof(int), st));
    for (size_t b = 0; b < s.parts.size(); ++b) {
        const Part &P = s.parts[b];
        const Geometry &g = *geoms[b];
        const int nx = P.box.nx, ny = P.box.ny, nz = P.box.nz;
        const int64_t ncell = P.n_cells;
        LBM_CUDA_TRY(cudaMemcpyAsync(d_mask, g.mask.data(), (size_t)ncell, cudaMemcpyHostToDevice, st));
        const int64_t nblk = (ncell + kBlock - 1) / kBlock;
        k_count_fluid<<<(unsigned)nblk, kBlock, 0, st>>>(d_mask, ncell, d_scan);
        k_scan_exclusive<<<1, kScanThreads, 0, st>>>(d_scan, nblk, d_total + b);
        k_fill_index<<<(unsigned)nblk, kBlock, 0, st>>>(d_mask, ncell, d_scan, P.fluid_off, P.cell_base, d_idx,
                                                         s.fluid_cell);
        LBM_CUDA_TRY(cudaGetLastError());
        if (P.n_fluid > 0) {
            const int32_t begin = P.fluid_off, end = P.fluid_off + P.n_fluid;
            k_neighbours<<<blocks_for(P.n_fluid), kBlock, 0, st>>>(d_idx, s.fluid_cell, begin, end, P.cell_base,
                                                                    s.n_pad, nx, ny, nz, P.box.periodic_z, s.nbr,
                                                                    s.lmask, cell_xr);
            k_plane_offsets<<<blocks_for(P.n_fluid), kBlock, 0, st>>>(s.fluid_cell, begin, end, P.cell_base, nx * ny,
                                                                       nz, s.plane_off + P.poff_base);
            if (nx < 65536 && ny < 32768) {
                const int32_t tiles = end / kBlock - begin / kBlock + 1;
                k_dense_tiles<<<blocks_for(tiles), kBlock, 0, st>>>(s.fluid_cell, s.plane_off + P.poff_base, begin,
                                                                     end, P.cell_base, nx, ny, nz, s.tile_desc);
            }
            if (s.staged_rows) {
                const int32_t tiles = end / kBlock - begin / kBlock + 1;
                k_stage_tiles<<<blocks_for(tiles), kBlock, 0, st>>>(s.fluid_cell, s.tile_desc, begin, end, P.cell_base,
                                                                     nx, ny, nz, P.box.periodic_z, P.words_base,
                                                                     s.tile_rows);
            }
        } else {
            LBM_CUDA_TRY(cudaMemsetAsync(s.plane_off + P.poff_base, 0, sizeof(int32_t) * (nz + 1), st));
        }
        if (s.rows_ok) {
            const int nw = (nx + 31) / 32;
            const int64_t nrows = (int64_t)ny * nz, nwords = nrows * nw;
            k_row_words<<<blocks_for(nwords), kBlock, 0, st>>>(d_idx, nx, nrows, nw, s.row_words + P.words_base);
        }
        LBM_CUDA_TRY(cudaGetLastError());
        // the next part reuses the mask and index map: keep the order
    }
    if (s.n_pad > s.n_fluid)
        k_pad_cells<<<blocks_for(s.n_pad - s.n_fluid), kBlock, 0, st>>>(s.n_fluid, s.n_pad, s.nbr, s.lmask,
                                                                          s.fluid_cell, cell_xr);
    k_warp_counts<<<(unsigned)(s.n_pad / kBlock), kBlock, 0, st>>>(s.lmask, d_wcnt);
    LBM_CUDA_TRY(cudaMemcpyAsync(s.warp_off, d_wcnt, sizeof(uint32_t) * (s.n_pad / 32), cudaMemcpyDeviceToDevice, st));
    k_scan_exclusive<<<1, kScanThreads, 0, st>>>(s.warp_off, s.n_pad / 32, d_total + s.parts.size());
    LBM_CUDA_TRY(cudaGetLastError());

    for (size_t b = 0; b < s.parts.size(); ++b) {
        const Part &P = s.parts[b];
        if (P.n_links == 0) continue;
        const Bins &bins = geoms[b]->link_bins;
        LBM_CUDA_TRY(cudaMemcpyAsync(d_bstart, bins.start.data(), bins.start.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, st));
        if (!bins.images.empty())
            LBM_CUDA_TRY(cudaMemcpyAsync(d_img, bins.images.data(), bins.images.size() * sizeof(SphereImage),
                                         cudaMemcpyHostToDevice, st));
        const int32_t begin = P.fluid_off, end = P.fluid_off + P.n_fluid;
        LinkArgs la{s.fluid_cell, s.nbr, s.lmask, s.warp_off, d_bstart, d_img, s.link_a, s.link_q, begin, end,
                    s.n_fluid, s.n_pad, P.cell_base, P.box.nx, P.box.ny, P.box.nz, P.box.periodic_z, bins.nbx,
                    bins.nby, P.box.q_lo, P.box.q_hi, (s.params.flags & LBM_FLAG_SIMPLE_BOUNCE_BACK) ? 1 : 0,
                    (s.params.flags & LBM_FLAG_CLI_SAFEGUARDS) ? 1 : 0};
        k_links<<<blocks_for(end - (begin & ~31)), kBlock, 0, st>>>(la);
        LBM_CUDA_TRY(cudaGetLastError());
        // the host bins must outlive their (pageable, staged) copies: synchronise
        LBM_CUDA_TRY(cudaStreamSynchronize(st));
    }

    LBM_CUDA_TRY(cudaMemcpyAsync(counts.data(), d_total, sizeof(uint32_t) * counts.size(), cudaMemcpyDeviceToHost, st));
    {
        // the span of dense tiles, for the odd step's dense kernel
        std::vector<int2> desc((size_t)(s.n_pad / kBlock));
        std::vector<int4> trows(desc.size());
        std::vector<int32_t> poff((size_t)(s.lay.n_planes + s.parts.size()));
        LBM_CUDA_TRY(cudaMemcpyAsync(desc.data(), s.tile_desc, sizeof(int2) * desc.size(), cudaMemcpyDeviceToHost, st));
        LBM_CUDA_TRY(cudaMemcpyAsync(trows.data(), s.tile_rows, sizeof(int4) * trows.size(), cudaMemcpyDeviceToHost, st));
        LBM_CUDA_TRY(cudaMemcpyAsync(poff.data(), s.plane_off, sizeof(int32_t) * poff.size(), cudaMemcpyDeviceToHost, st));
        LBM_CUDA_TRY(cudaStreamSynchronize(st));
        s.dense_lo = s.dense_hi = 0;
        for (size_t t = 0; t < desc.size(); ++t)
            if (desc[t].x >= 0) {
                if (s.dense_hi == 0) s.dense_lo = (int32_t)t;
                s.dense_hi = (int32_t)t + 1;
            }
        s.rows_lo = s.rows_hi = 0;
        for (size_t t = 0; t < trows.size(); ++t)
            if (trows[t].x >= 0) {
                if (s.rows_hi == 0) s.rows_lo = (int32_t)t;
                s.rows_hi = (int32_t)t + 1;
            }
        // reference planes and the tiles that use them (see lbm_internal.h)
        std::vector<int2> tref(desc.size(), make_int2(-1, 0));
        s.plane_referenced.assign((size_t)s.lay.n_planes, 0);
        if (plane_references_on(s.params)) mark_reference_planes(s, desc, poff, tref);
        s.ref_lo = s.ref_hi = 0;
        for (size_t t = 0; t < tref.size(); ++t)
            if (tref[t].x >= 0) {
                if (s.ref_hi == 0) s.ref_lo = (int32_t)t;
                s.ref_hi = (int32_t)t + 1;
            }
        s.has_ref = s.ref_hi > s.ref_lo;
        LBM_CUDA_TRY(cudaMemcpyAsync(s.tile_ref, tref.data(), sizeof(int2) * tref.size(), cudaMemcpyHostToDevice, st));
        LBM_CUDA_TRY(cudaMemcpyAsync(s.plane_flag, s.plane_referenced.data(), s.plane_referenced.size(),
                                     cudaMemcpyHostToDevice, st));
        LBM_CUDA_TRY(cudaMemsetAsync(s.ref, 0, sizeof(float) * kRefStride * (size_t)s.lay.n_planes, st));
        LBM_CUDA_TRY(cudaMemsetAsync(s.ref_next, 0, sizeof(float) * kRefStride * (size_t)s.lay.n_planes, st));
        // the host vectors must outlive their (pageable) copies
        LBM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    LBM_CUDA_TRY(cudaStreamSynchronize(st));
    for (size_t b = 0; b < s.parts.size(); ++b)
        if ((int64_t)counts[b] != s.parts[b].n_fluid) {
            std::fprintf(stderr, "liblbm: device list build disagrees with host count of part %zu (%u/%d fluid)\n", b,
                         counts[b], s.parts[b].n_fluid);
            return LBM_ECUDA;
        }
    if ((int64_t)counts[s.parts.size()] != s.n_links) {
        std::fprintf(stderr, "liblbm: device link count %u differs from host count %lld\n", counts[s.parts.size()],
                     (long long)s.n_links);
        return LBM_ECUDA;
    }
    return LBM_OK;
}

}  // namespace lbm
