// lbm_step.cu -- the fused stream-collide + CLI update over the sparse fluid
// list (in-place AA pattern, see lbm_kernels.cuh), the initialisation, and the
// launch schedule (tile-loop grid chosen by timing, CUDA-graph replay).
//
// One thread per fluid cell; a block handles tiles of 256 consecutive fluid
// cells (8 aligned warps) and loops over tiles with the grid stride, so a grid
// smaller than the tile count makes the kernel persistent.  The even step
// touches only the cell's own 19 slots (contiguous structure-of-arrays rows);
// the odd step gathers through the neighbour indices and scatters back to the
// same slots.  Wall links cost one coefficient load each.  The kernels never
// need to know which independent box (part) a cell belongs to, because the
// neighbour indices are global; only the optional density re-centring looks
// up the part of a cell.
#include <algorithm>

#include "lbm_kernels.cuh"

namespace lbm {
namespace {

// Resident blocks per SM requested from the register allocator (256 threads
// each).  Measured on GB300 over the 256x256x512 channel sweep: both steps at
// 6 blocks (40 registers, no spills; 7 blocks spill).  The odd step stages
// only its neighbour slots in shared memory (18 KB per block) and reads the
// CLI coefficients where it uses them, as the even step does: 10% faster
// than also staging the coefficients at 5 blocks (48 registers, 36 KB per
// block), which left too little L1 for the gathers.
constexpr int kEvenBlocksPerSM = 6;
constexpr int kOddBlocksPerSM = 6;

// Where the odd step takes a cell's neighbour indices from: the table, the
// row bitmasks, or the table except in dense tiles (Solver::tile_desc), whose
// indices are computed.  Without dense tiles the table-only kernel is used:
// it carries no descriptor load or branch (the periodic REV cubes, 2.7% faster
// in the odd step).
// kNbStaged: the table's role outside the dense tiles is taken by row words
// staged per tile in shared memory (LBM_FLAG_STAGED_NEIGHBOURS).
// kNbDerived: outside the dense tiles the table's x-shifted entries are
// derived from its other entries (LBM_FLAG_DERIVED_NEIGHBOURS).
enum NbSource { kNbTable = 0, kNbRows = 1, kNbDense = 2, kNbStaged = 3, kNbDerived = 4 };
constexpr int kGridBulk = -1;       // schedule entry: the staged even step
constexpr int kGraphSteps = 32;     // steps per CUDA-graph replay (even)
constexpr int kTuneReps = 3;        // timed launches per candidate grid

template <typename T>
struct StepArgs {
    T *pdf;
    const int32_t *nbr;
    const uint32_t *lmask;
    const uint32_t *warp_off;
    const int2 *tile_desc;
    int32_t dense_lo, dense_hi;   // every dense tile lies in [dense_lo, dense_hi)
    const int4 *tile_rows;
    int32_t rows_lo, rows_hi;     // every staged tile lies in [rows_lo, rows_hi)
    const float *link_a;
    int *status;   // set to 1 when a bounded wait gives up
    int32_t n_fluid;
    int32_t n_pad;
    int32_t n_tiles;
    RowGeo rows;
    const float *part_shift;   // per-part density shift
    const int32_t *part_foff;  // [n_parts + 1] first fluid index of each part
    int32_t n_parts;
    int32_t shift_on;          // apply part_shift in this launch
    // reference populations (lbm_internal.h): tiles [ref_lo, ref_hi) may use
    // them; slots are read relative to ref_rd and written relative to ref_wr
    // (the same array except in the step that switches to new references)
    const int2 *tile_ref;
    int32_t ref_lo, ref_hi;
    const float *ref_rd;
    const float *ref_wr;
    Coef c;
};

// Density shift of the part that holds fluid cell i (binary search).
template <typename T>
__device__ __forceinline__ float part_shift_of(const StepArgs<T> &p, int32_t i)
{
    int lo = 0, hi = p.n_parts - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(p.part_foff + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return __ldg(p.part_shift + lo);
}

// Even step: the cell's own 19 slots.  The CLI coefficients of its links are
// read where they are used, before and after the collision; the second read
// hits L1.  Holding no staging buffer keeps shared memory free for L1 and the
// register count at 40, so six blocks fit on an SM.
// With reference populations (REF, a tile in or next to referenced planes),
// the population of direction k is read as slot + R_k(z) and written as
// f~_k - R_k(z), z the plane of the slot's owner (the cell itself in the even
// step).  Dense tiles have no wall links, so in FP32 storage, where the step
// is bound by its bytes, their cells skip the link-mask load (4 B per cell;
// the tile's descriptor is one broadcast load per warp).
template <typename T, bool REF>
__device__ __forceinline__ void even_cell(const StepArgs<T> &p, int32_t i)
{
    const bool live = i < p.n_fluid;
    const int32_t tile = i / kBlock;
    const bool dense = sizeof(T) == 4 && tile >= p.dense_lo && tile < p.dense_hi && __ldg(p.tile_desc + tile).x >= 0;
    const uint32_t m = live && !dense ? p.lmask[i] & kLinkBits : 0u;
    const uint32_t off = first_link(p.warp_off, i, m);
    if (!live) return;
    const int32_t rr = ref_row<REF>(p, i);
    const size_t n_pad = (size_t)p.n_pad;
    float h[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) h[k] = ld_raw(p.pdf + k * n_pad + i);
    if (REF && rr >= 0) ref_rows<true, 0, sizeof(T) == 2>(h, p.ref_rd + rr);
    if (m) cli_links<true>(h, p.link_a, off, m);
    if (p.shift_on) apply_shift(h, part_shift_of(p, i) * StoreScale<T>::v);
    collide(h, p.c);
    if (m) cli_links<false>(h, p.link_a, off, m);
    if (REF && rr >= 0) ref_rows<false, 0, sizeof(T) == 2>(h, p.ref_wr + rr);
#pragma unroll
    for (int k = 0; k < kQ; ++k) st_raw(p.pdf + opp(k) * n_pad + i, h[k]);
}

// Odd step: per-thread staging of the neighbour slots in shared memory (each
// thread writes and reads its own column, so no barrier is needed).  Keeping
// them out of registers across the collision lowers register pressure and
// raises the number of resident warps, which is what hides the memory latency
// of the two dependent loads (indices, then populations).  The CLI
// coefficients are read where they are used, before and after the collision
// (the second read hits L1).
// NB: where the neighbour indices come from (NbSource).
template <typename T, int NB, bool REF>
__device__ __forceinline__ void odd_cell(const StepArgs<T> &p, int32_t i, int32_t (*nb_s)[kBlock], uint2 *ws)
{
    const int t = threadIdx.x;
    const bool live = i < p.n_fluid;
    // 32-bit element offsets (19 n_pad < 2^32 is checked on the host)
    const uint32_t n_pad = (uint32_t)p.n_pad, ui = (uint32_t)i;
    uint32_t m = 0;
    // a dense tile (same for the whole block) computes its indices and has no links
    const int32_t tile = i / kBlock;
    const int2 d = (NB == kNbDense || NB == kNbStaged || NB == kNbDerived) && tile >= p.dense_lo && tile < p.dense_hi
                       ? __ldg(p.tile_desc + tile)
                       : make_int2(-1, 0);
    // a staged tile (same for the whole block): its bands of row words go to
    // shared memory once, after every thread is done with the previous tile's
    const int4 sd = NB == kNbStaged && d.x < 0 && tile >= p.rows_lo && tile < p.rows_hi ? __ldg(p.tile_rows + tile)
                                                                                       : make_int4(-1, 0, 0, 0);
    if (NB == kNbStaged && sd.x >= 0) {
        __syncthreads();
        stage_rows(ws, p.rows.words, staged_tile(sd));
        __syncthreads();
    }
    if (live) {
        int32_t nb[kQ];
        if (d.x >= 0) dense_neighbours(nb, d, i);
        else if (NB == kNbStaged && sd.x >= 0 && staged_neighbours(nb, m, ws, sd, __ldg(p.rows.cell_xr + i), i)) {
        }
        else if (NB == kNbDerived) m = derived_nbr(nb, p.nbr, (size_t)n_pad, i, __ldg(p.lmask + i));
        else m = NB == kNbRows ? row_neighbours(nb, p.rows, i) : load_nbr(nb, p.nbr, (size_t)n_pad, i);
        // stage the slot of direction k, A[k][x + e_k] or the dead slot
        // A[opp k][x] of a wall link: the gather of h_opp(k) reads it and the
        // scatter of the new h_k writes it (the AA pattern), so it is
        // resolved once
#pragma unroll
        for (int k = 1; k < kQ; ++k)
            nb_s[k - 1][t] = (int32_t)(nb[k] >= 0 ? k * n_pad + (uint32_t)nb[k] : opp(k) * n_pad + ui);
    }
    // skip the link-offset scan in link-free warps only where such warps
    // exist (solvers with dense tiles): measured faster on the channel and
    // 0.8% slower on the periodic REV cubes, where nearly every warp has links
    const uint32_t off = first_link<NB == kNbDense>(p.warp_off, i, m);
    if (!live) return;
    auto slot = [&](int k) -> uint32_t { return (uint32_t)nb_s[k - 1][t]; };   // slot of direction k
    float h[kQ];
    h[0] = ld_raw(p.pdf + ui);
#pragma unroll
    for (int k = 1; k < kQ; ++k) h[k] = ld_raw(p.pdf + slot(opp(k)));   // A[opp k][x - e_k]
    // reference rows: the slot read for h_k belongs to x - e_k (plane z - ez_k),
    // the slot written with h_k to x + e_k (plane z + ez_k)
    const int32_t rr = ref_row<REF>(p, i);
    if (REF && rr >= 0) ref_rows<true, -1, sizeof(T) == 2>(h, p.ref_rd + rr);
    if (m) cli_links<true>(h, p.link_a, off, m);
    if (p.shift_on) apply_shift(h, part_shift_of(p, i) * StoreScale<T>::v);
    collide(h, p.c);
    if (m) cli_links<false>(h, p.link_a, off, m);
    if (REF && rr >= 0) ref_rows<false, 1, sizeof(T) == 2>(h, p.ref_wr + rr);
    st_raw(p.pdf + ui, h[0]);
#pragma unroll
    for (int k = 1; k < kQ; ++k) st_raw(p.pdf + slot(k), h[k]);
}

template <typename T, int MINB, bool REF>
__global__ void __launch_bounds__(kBlock, MINB) k_step_even(StepArgs<T> p)
{
    for (int32_t tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x)
        even_cell<T, REF>(p, tile * kBlock + threadIdx.x);
}

// Even step with the populations staged through shared memory.  A persistent
// block takes the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; warp 0
// fetches each tile's 19 rows (kBlock contiguous slots per direction, 16-byte
// aligned since n_pad and the tiles are multiples of 256 cells) with TMA bulk
// copies into one of S stages, S tiles ahead of the collision, so the bytes
// in flight are set by the stages rather than by the registers of the
// resident threads.  Results are stored directly (stores need no latency
// hiding).  A stage is refilled after the block barrier that follows its last
// read.  On GB300 the register kernel measured faster at every storage type:
// in FP32 it already moves its bytes at 95% of the copy bandwidth, and in
// 16-bit storage both are bound by instruction issue, not by bytes in flight.
// The tuner keeps this kernel as a candidate.
template <typename T, int S>
constexpr size_t even_bulk_smem()
{
    return (size_t)S * kQ * kBlock * sizeof(T) + (size_t)S * sizeof(uint64_t);
}

template <typename T, int S, int MINB, bool REF>
__global__ void __launch_bounds__(kBlock, MINB) k_step_even_bulk(StepArgs<T> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *buf = (T *)smem_raw;   // [S][kQ][kBlock]
    uint64_t *full = (uint64_t *)(smem_raw + (size_t)S * kQ * kBlock * sizeof(T));
    constexpr uint32_t kRow = kBlock * sizeof(T);
    const int t = threadIdx.x;
    const int32_t first = blockIdx.x, stride = gridDim.x;
    const int32_t count = first < p.n_tiles ? (p.n_tiles - 1 - first) / stride + 1 : 0;
    const size_t n_pad = (size_t)p.n_pad;
    auto issue = [&](int32_t j) {   // warp 0
        const int st_ = j % S;
        const size_t base = (size_t)(first + j * stride) * kBlock;
        const int lane = t & 31;
        if (lane == 0) bulk::expect_tx(&full[st_], kQ * kRow);
        __syncwarp();
        if (lane < kQ) bulk::copy(buf + ((size_t)st_ * kQ + lane) * kBlock, p.pdf + lane * n_pad + base, kRow, &full[st_]);
    };
    if (t == 0) {
        for (int q = 0; q < S; ++q) bulk::init(&full[q], 1);
        bulk::fence_init();
    }
    __syncthreads();
    if (t < 32)
        for (int32_t j = 0; j < S && j < count; ++j) issue(j);
    int32_t j = 0;
    bool ok = true;
    for (; j < count; ++j) {
        const int32_t i = (first + j * stride) * kBlock + t;
        const bool live = i < p.n_fluid;
        const uint32_t m = live ? p.lmask[i] & kLinkBits : 0u;
        const uint32_t off = first_link(p.warp_off, i, m);
        const T *row = buf + (size_t)(j % S) * kQ * kBlock + t;
        ok = bulk::wait(&full[j % S], (uint32_t)((j / S) & 1));
        float h[kQ];
#pragma unroll
        for (int k = 0; k < kQ; ++k) h[k] = ok ? ld_raw(row + k * kBlock) : 0.0f;
        if (__syncthreads_or(!ok)) break;   // the stage is free again
        if (t < 32 && j + S < count) issue(j + S);
        if (!live) continue;
        const int32_t rr = ref_row<REF>(p, i);
        if (REF && rr >= 0) ref_rows<true, 0, sizeof(T) == 2>(h, p.ref_rd + rr);
        if (m) cli_links<true>(h, p.link_a, off, m);
        if (p.shift_on) apply_shift(h, part_shift_of(p, i) * StoreScale<T>::v);
        collide(h, p.c);
        if (m) cli_links<false>(h, p.link_a, off, m);
        if (REF && rr >= 0) ref_rows<false, 0, sizeof(T) == 2>(h, p.ref_wr + rr);
#pragma unroll
        for (int k = 0; k < kQ; ++k) st_raw(p.pdf + opp(k) * n_pad + i, h[k]);
    }
    if (j < count && t == 0) {
        // a wait gave up: report it, and let the copies still in flight land
        // before the block's shared memory is released
        atomicExch(p.status, 1);
        for (int32_t q = j; q < count && q < j + S; ++q) bulk::wait(&full[q % S], (uint32_t)((q / S) & 1));
    }
}

// Self-test of the bounded waits: one warp waits on an mbarrier phase that
// nothing completes (no arrival, no copy), gives up after max_polls polls and
// reports it in the status word, as a step kernel whose copies never landed
// would.  Touches only its shared barrier and the status word.
__global__ void k_wait_selftest(int *status, int max_polls)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        bulk::init(&bar, 1);
        bulk::fence_init();
    }
    __syncthreads();
    const bool ok = bulk::wait(&bar, 0u, max_polls);
    if (!ok && threadIdx.x == 0) atomicExch(status, 1);
}

template <typename T, int NB, int MINB, bool REF>
__global__ void __launch_bounds__(kBlock, MINB) k_step_odd(StepArgs<T> p)
{
    __shared__ int32_t nb_s[kQ - 1][kBlock];
    __shared__ uint2 ws[NB == kNbStaged ? kMaxStagedWords : 1];
    for (int32_t tile = blockIdx.x; tile < p.n_tiles; tile += gridDim.x)
        odd_cell<T, NB, REF>(p, tile * kBlock + threadIdx.x, nb_s, ws);
}

// Initial state f_k = f_k^eq(rho = 1, u0) (Eq. (equilibrium)) stored shifted
// at even parity; the dead slot of each link receives the partial
// P = h_kbar - a_k h_k so that the first step completes it to h_kbar.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_init(StepArgs<T> p, const int32_t *__restrict__ fluid_cell,
                                                 const float *__restrict__ u0, int64_t ncell)
{
    const int32_t i = blockIdx.x * kBlock + threadIdx.x;
    const bool live = i < p.n_fluid;
    const uint32_t m = live ? p.lmask[i] & kLinkBits : 0u;
    const uint32_t off = first_link(p.warp_off, i, m);
    if (!live) return;
    float ux = 0.0f, uy = 0.0f, uz = 0.0f;
    if (u0) {
        const int64_t c = fluid_cell[i];
        ux = u0[c];
        uy = u0[ncell + c];
        uz = u0[2 * ncell + c];
    }
    const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
    float h[kQ], a[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
        const float eu = (float)ex(k) * ux + (float)ey(k) * uy + (float)ez(k) * uz;
        h[k] = (float)weight(k) * (3.0f * eu + 4.5f * eu * eu - usq);
    }
    load_links(a, m, p.link_a, off);
    float out[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) out[k] = h[k];
#pragma unroll
    for (int k = 1; k < kQ; ++k) out[opp(k)] = fmaf(-a[k], h[k], out[opp(k)]);
    const size_t n_pad = (size_t)p.n_pad;
#pragma unroll
    for (int k = 0; k < kQ; ++k) st(p.pdf + k * n_pad + i, out[k]);
}

template <typename T>
StepArgs<T> make_args(const Solver &s)
{
    StepArgs<T> p;
    p.pdf = (T *)s.pdf;
    p.nbr = s.nbr;
    p.lmask = s.lmask;
    p.warp_off = s.warp_off;
    p.tile_desc = s.tile_desc;
    p.dense_lo = s.dense_lo;
    p.dense_hi = s.dense_hi;
    p.link_a = s.link_a;
    p.status = s.status;
    p.n_fluid = s.n_fluid;
    p.n_pad = s.n_pad;
    p.n_tiles = s.n_pad / kBlock;
    p.rows = RowGeo{s.row_words, s.cell_xr, s.box.nx, s.box.ny, s.box.nz, s.n_words, s.box.periodic_z};
    p.tile_rows = s.tile_rows;
    p.rows_lo = s.rows_lo;
    p.rows_hi = s.rows_hi;
    p.part_shift = s.part_shift;
    p.part_foff = s.part_foff;
    p.n_parts = (int32_t)s.parts.size();
    p.shift_on = 0;
    p.tile_ref = s.tile_ref;
    p.ref_lo = s.ref_lo;
    p.ref_hi = s.ref_hi;
    p.ref_rd = s.ref;
    p.ref_wr = s.ref;
    p.c.omega_p = (float)s.omega_p;
    p.c.omega_m = (float)s.omega_m;
    // storage units: the scale (a power of two) multiplies F_k and divides
    // the quadratic terms' constants, so the results are exactly scaled
    const float scale = StoreScale<T>::v;
    p.c.usq_c = 1.5f / scale;
    p.c.eu_c = 4.5f / scale;
    p.c.half_omega_m = (float)(0.5 * s.omega_m);
    for (int cls = 0; cls < 2; ++cls) {
        const double w = cls == 0 ? weight(1) : weight(7);
        p.c.ep_c[cls] = (float)(w * 4.5 / scale);
        p.c.em_c[cls] = (float)(3.0 * w * s.omega_m);
    }
    for (int k = 0; k < kQ; ++k) {
        const double eg = ex(k) * s.params.g[0] + ey(k) * s.params.g[1] + ez(k) * s.params.g[2];
        p.c.force[k] = (float)(3.0 * weight(k) * eg) * scale;
    }
    for (int d = 0; d < 3; ++d) p.c.half_g[d] = (float)(0.5 * s.params.g[d]);
    return p;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// Stages and resident blocks of the staged even step per storage type.
template <typename T>
struct EvenBulk {
    static constexpr int S = 2, MINB = 5;   // FP32: 39 KB of stages per block
};
template <>
struct EvenBulk<__half> {
    static constexpr int S = 4, MINB = 5;
};
template <>
struct EvenBulk<__nv_bfloat16> {
    static constexpr int S = 4, MINB = 5;
};

// The staged even step on one wave of resident blocks.
template <typename T, int S, int MINB, bool REF>
void launch_even_bulk(const StepArgs<T> &p, cudaStream_t st)
{
    constexpr size_t smem = even_bulk_smem<T, S>();
    static const int wave = [] {
        cudaFuncSetAttribute(k_step_even_bulk<T, S, MINB, REF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_even_bulk<T, S, MINB, REF>, kBlock, smem) !=
            cudaSuccess)
            nb = 1;
        return sm_count() * std::max(nb, 1);
    }();
    k_step_even_bulk<T, S, MINB, REF><<<(unsigned)std::min(wave, p.n_tiles), kBlock, smem, st>>>(p);
}

// One step launch at the current parity with the chosen grid (0: a block per
// tile; kGridBulk: the staged even step).  Solvers with referenced planes run
// the kernels compiled with reference populations.
template <typename T, bool REF>
void launch_step_ref(const Solver &s, const StepArgs<T> &p, bool odd, int grid, cudaStream_t st)
{
    const unsigned g = (unsigned)(grid > 0 ? std::min(grid, p.n_tiles) : p.n_tiles);
    if (!odd && grid == kGridBulk) launch_even_bulk<T, EvenBulk<T>::S, EvenBulk<T>::MINB, REF>(p, st);
    else if (!odd) k_step_even<T, kEvenBlocksPerSM, REF><<<g, kBlock, 0, st>>>(p);
    else if (s.odd_rows) k_step_odd<T, kNbRows, kOddBlocksPerSM, REF><<<g, kBlock, 0, st>>>(p);
    else if (s.staged_rows && p.rows_hi > p.rows_lo)
        k_step_odd<T, kNbStaged, kOddBlocksPerSM, REF><<<g, kBlock, 0, st>>>(p);
    else if (s.derived_nbrs) k_step_odd<T, kNbDerived, kOddBlocksPerSM, REF><<<g, kBlock, 0, st>>>(p);
    else if (p.dense_hi > p.dense_lo) k_step_odd<T, kNbDense, kOddBlocksPerSM, REF><<<g, kBlock, 0, st>>>(p);
    else k_step_odd<T, kNbTable, kOddBlocksPerSM, false><<<g, kBlock, 0, st>>>(p);
}

template <typename T>
void launch_step(const Solver &s, const StepArgs<T> &p, bool odd, int grid, cudaStream_t st)
{
    if (s.has_ref) launch_step_ref<T, true>(s, p, odd, grid, st);
    else launch_step_ref<T, false>(s, p, odd, grid, st);
}

// Candidate schedules: a block per tile, or 1, 2, 4 waves of resident blocks
// looping over the tiles; the even step also tries its staged kernel.  Only
// solvers of more than four waves are tuned.
void start_tuning(Solver &s, int n_tiles)
{
    const int wave = sm_count() * kOddBlocksPerSM;
    s.tune_grids_odd = {0};
    if (s.autotune && n_tiles > 4 * sm_count() * kEvenBlocksPerSM)
        for (int w : {1, 2, 4}) s.tune_grids_odd.push_back(w * wave);
    s.tune_grids_even = s.tune_grids_odd;
    if (s.staged_even) s.tune_grids_even = {kGridBulk};
    else if (s.tune_grids_even.size() > 1) s.tune_grids_even.push_back(kGridBulk);
    s.tune_ms_even.assign(s.tune_grids_even.size(), 0.0f);
    s.tune_ms_odd.assign(s.tune_grids_odd.size(), 0.0f);
    s.tune_count_even = s.tune_count_odd = 0;
    s.tune_state = s.tune_grids_odd.size() > 1 ? 1 : 2;
    s.grid_even = s.staged_even ? kGridBulk : 0;
    s.grid_odd = 0;
    if (s.tune_state == 1 && (!s.ev0 || !s.ev1)) {
        if (cudaEventCreate(&s.ev0) != cudaSuccess || cudaEventCreate(&s.ev1) != cudaSuccess) s.tune_state = 2;
    }
}

template <typename T>
int run_steps(Solver &s, int64_t n)
{
    if (s.n_fluid == 0) {
        s.steps += n;
        return LBM_OK;
    }
    StepArgs<T> p = make_args<T>(s);
    if (s.tune_state == 0) start_tuning(s, p.n_tiles);
    const int Ce = (int)s.tune_grids_even.size(), Co = (int)s.tune_grids_odd.size();
    int64_t t = 0;
    const size_t ref_bytes = sizeof(float) * kRefStride * (size_t)s.lay.n_planes;
    while (t < n) {
        const bool odd = (s.steps & 1) != 0;
        p.shift_on = s.shift_pending ? 1 : 0;
        s.shift_pending = false;
        // a step that switches to new reference populations reads with the
        // old ones and writes with the new ones, which then become current
        const bool ref_switch = s.ref_pending;
        s.ref_pending = false;
        p.ref_wr = ref_switch ? s.ref_next : s.ref;
        auto after_switch = [&]() -> int {
            if (!ref_switch) return LBM_OK;
            p.ref_wr = s.ref;
            return cudaMemcpyAsync(s.ref, s.ref_next, ref_bytes, cudaMemcpyDeviceToDevice, s.stream) == cudaSuccess
                       ? LBM_OK
                       : LBM_ECUDA;
        };
        if (s.tune_state == 1) {
            int &cnt = odd ? s.tune_count_odd : s.tune_count_even;
            const std::vector<int> &grids = odd ? s.tune_grids_odd : s.tune_grids_even;
            if (cnt < (int)grids.size() * kTuneReps) {
                const int c = cnt / kTuneReps;
                if (cudaEventRecord(s.ev0, s.stream) != cudaSuccess) return LBM_ECUDA;
                launch_step(s, p, odd, grids[c], s.stream);
                if (cudaEventRecord(s.ev1, s.stream) != cudaSuccess || cudaEventSynchronize(s.ev1) != cudaSuccess)
                    return LBM_ECUDA;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, s.ev0, s.ev1);
                (odd ? s.tune_ms_odd : s.tune_ms_even)[c] += ms;
                ++cnt;
            } else {
                launch_step(s, p, odd, odd ? s.grid_odd : s.grid_even, s.stream);
            }
            if (after_switch() != LBM_OK) return LBM_ECUDA;
            if (s.tune_count_even >= Ce * kTuneReps && s.tune_count_odd >= Co * kTuneReps) {
                s.grid_even = s.tune_grids_even[std::min_element(s.tune_ms_even.begin(), s.tune_ms_even.end()) -
                                                s.tune_ms_even.begin()];
                s.grid_odd = s.tune_grids_odd[std::min_element(s.tune_ms_odd.begin(), s.tune_ms_odd.end()) -
                                              s.tune_ms_odd.begin()];
                s.tune_state = 2;
            }
            ++s.steps;
            ++t;
            continue;
        }
        // replay whole graph chunks from an even step, once the schedule is fixed
        if (s.use_graph && !odd && !p.shift_on && !ref_switch && n - t >= kGraphSteps) {
            if (!s.graph_exec) {
                if (!s.cap_stream && cudaStreamCreateWithFlags(&s.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                    return LBM_ECUDA;
                if (cudaStreamBeginCapture(s.cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return LBM_ECUDA;
                for (int k = 0; k < kGraphSteps; ++k) launch_step(s, p, (k & 1) != 0, (k & 1) ? s.grid_odd : s.grid_even, s.cap_stream);
                if (cudaStreamEndCapture(s.cap_stream, &s.graph) != cudaSuccess) return LBM_ECUDA;
                if (cudaGraphInstantiate(&s.graph_exec, s.graph, 0) != cudaSuccess) return LBM_ECUDA;
            }
            while (n - t >= kGraphSteps) {
                if (cudaGraphLaunch(s.graph_exec, s.stream) != cudaSuccess) return LBM_ECUDA;
                s.steps += kGraphSteps;
                t += kGraphSteps;
            }
            continue;
        }
        launch_step(s, p, odd, odd ? s.grid_odd : s.grid_even, s.stream);
        if (after_switch() != LBM_OK) return LBM_ECUDA;
        ++s.steps;
        ++t;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

template <typename T>
int run_init(Solver &s, const float *u0)
{
    s.steps = 0;
    s.shift_pending = false;
    s.ref_pending = false;
    if (s.n_fluid == 0) return LBM_OK;
    // the initial state is stored without reference populations
    if (cudaMemsetAsync(s.ref, 0, sizeof(float) * kRefStride * (size_t)s.lay.n_planes, s.stream) != cudaSuccess)
        return LBM_ECUDA;
    const StepArgs<T> p = make_args<T>(s);
    k_init<T><<<(unsigned)(s.n_pad / kBlock), kBlock, 0, s.stream>>>(p, s.fluid_cell, u0, s.n_cells);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // namespace

Solver::~Solver()
{
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
}

Coef make_coef(const Solver &s) { return make_args<float>(s).c; }

int launch_init(Solver &s, const float *dev_u0)
{
    switch (s.params.storage) {
    case LBM_F32: return run_init<float>(s, dev_u0);
    case LBM_F16: return run_init<__half>(s, dev_u0);
    case LBM_BF16: return run_init<__nv_bfloat16>(s, dev_u0);
    }
    return LBM_EINVAL;
}

int launch_wait_selftest(Solver &s, int max_polls)
{
    k_wait_selftest<<<1, 32, 0, s.stream>>>(s.status, max_polls);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_steps(Solver &s, int64_t n)
{
    switch (s.params.storage) {
    case LBM_F32: return run_steps<float>(s, n);
    case LBM_F16: return run_steps<__half>(s, n);
    case LBM_BF16: return run_steps<__nv_bfloat16>(s, n);
    }
    return LBM_EINVAL;
}

int graph_steps() { return kGraphSteps; }

}  // namespace lbm

extern "C" int lbm_schedule(const lbm_solver *s, int32_t *grid_even, int32_t *grid_odd, int32_t *tuned,
                            int32_t *graph_steps_out)
{
    if (!s) return LBM_EINVAL;
    const int32_t tiles = s->n_pad / lbm::kBlock;
    if (grid_even) *grid_even = s->grid_even > 0 ? std::min(s->grid_even, tiles) : (s->grid_even < 0 ? -1 : tiles);
    if (grid_odd) *grid_odd = s->grid_odd > 0 ? std::min(s->grid_odd, tiles) : tiles;
    if (tuned) *tuned = s->tune_state == 2 ? 1 : 0;
    if (graph_steps_out) *graph_steps_out = s->use_graph ? lbm::graph_steps() : 0;
    return LBM_OK;
}
