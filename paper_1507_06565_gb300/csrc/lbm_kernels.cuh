// lbm_kernels.cuh -- device building blocks of the fused stream-collide + CLI
// update (shared by the step, moment and export kernels).
//
// In-place AA streaming over the fluid list.  Storage A[k][i] (pdf[k*n_pad+i])
// holds shifted populations h_k = f_k - w_k.
//   even time t: A[k][x] = f_k(x,t) for every direction whose upstream node
//                x - e_k is fluid;
//   even step:   read A[k][x], collide, write f~_k to A[opp k][x];
//   odd time:    f_k(x,t) = A[opp k][x - e_k];
//   odd step:    read A[opp k][x - e_k], collide, write f~_k to A[k][x + e_k].
// Both steps read and write the same set of slots per cell, so one array
// suffices and no two cells touch the same slot.
//
// Wall link (x, k): x + e_k solid.  Its "dead" slot S = A[opp k][x] is the one
// the solid node would have received; only x reads and writes it:
//   even step writes f~_k(x) to S; odd step redirects its write of f~_k(x) to
//   S; both steps read S for direction opp k.
// Eq. (CLI) needs f~_k(x_f1), f~_kbar(x_f1) (both local to the collision of
// x_f1) and f~_k(x_f2), x_f2 = x - e_k, which is exactly what x receives next
// step in direction k.  So the collision of x stores the partial
//   P = f~_k(x) - a f~_kbar(x)           (a = (1-2q)/(1+2q))
// in S, and the next step completes
//   f_kbar(x) = P + a f_k(x)             (f_k(x) = f~_k(x_f2), streamed).
// No extra population traffic; a = 0 gives simple bounce-back (Eq. (noslip)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

// ---- storage conversions ----
// Shifted populations are small (|h| << 1).  FP16 stores them scaled by 2^14
// (exact) so that values down to ~4e-9 stay normal numbers with the full
// 11-bit significand; |h| < 4 keeps them below the FP16 maximum.  BF16 shares
// the FP32 exponent range and is stored unscaled.
constexpr float kHalfScale = 16384.0f;
constexpr float kHalfUnscale = 1.0f / 16384.0f;
__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(*p) * kHalfUnscale; }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v * kHalfScale); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// The step kernels work in storage units: FP16 values stay scaled by 2^14
// through the collision (its constants carry the scale, see Coef), which
// saves the two multiplications per population and changes no bit, since
// every scaling is by a power of two.
template <typename T>
struct StoreScale {
    static constexpr float v = 1.0f;
};
template <>
struct StoreScale<__half> {
    static constexpr float v = kHalfScale;
};
__device__ __forceinline__ float ld_raw(const float *p) { return *p; }
__device__ __forceinline__ float ld_raw(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float ld_raw(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st_raw(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_raw(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st_raw(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// ---- TMA bulk copies global -> shared memory, completed on an mbarrier ----
// A copy moves a contiguous run of bytes (16-byte aligned at both ends, a
// multiple of 16 bytes long); the barrier's phase completes once the bytes
// announced with expect_tx have landed.  Waits are bounded: a wait that gives
// up returns false and the caller reports LBM_ETIMEOUT instead of hanging.
namespace bulk {
constexpr int kMaxPolls = 1 << 22;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
}

// makes barrier initialisation visible to the async proxy (the TMA unit)
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ bool test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(saddr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity, int max_polls = kMaxPolls)
{
    for (int it = 0; it < max_polls; ++it)
        if (test(bar, parity)) return true;
    return false;
}
}  // namespace bulk

// Relaxation constants and source term of one solver (kernel parameter).
// Index 0 of ep_c/em_c is the axis class (w = 1/18), 1 the diagonal class
// (w = 1/36).
struct Coef {
    float omega_p, omega_m;
    float half_omega_m;  // omega- / 2
    float usq_c, eu_c;   // 3/2 and 9/2 over the storage scale (quadratic terms)
    float ep_c[2];       // w eu_c: the quadratic term of the symmetric equilibrium
    float em_c[2];       // 3 w omega-: the antisymmetric equilibrium, relaxed
    float force[kQ];     // F_k = 3 w_k e_k.g, times the storage scale
    float half_g[3];   // g/2, added to j for the reported velocity
};

// Uniform density shift of the logical populations: h_k -= w_k c.
__device__ __forceinline__ void apply_shift(float h[kQ], float c)
{
    if (c != 0.0f) {
#pragma unroll
        for (int k = 0; k < kQ; ++k) h[k] = fmaf(-(float)weight(k), c, h[k]);
    }
}

// Constants of a solver (defined in lbm_step.cu).
Coef make_coef(const Solver &s);

// Offset of the reference row of cell i's plane (lbm_internal.h), or -1 when
// its tile stores no reference populations (REF: the solver has referenced
// planes at all).  A holds tile_ref, ref_lo and ref_hi.
template <bool REF, typename A>
__device__ __forceinline__ int32_t ref_row(const A &p, int32_t i)
{
    if (!REF) return -1;
    const int32_t tile = i / kBlock;
    if (tile < p.ref_lo || tile >= p.ref_hi) return -1;
    const int2 tr = __ldg(p.tile_ref + tile);
    return tr.x < 0 ? -1 : (tr.x + (i >= tr.y ? 1 : 0)) * kRefStride;
}

// Adds (ADD) or subtracts the reference populations R_k to or from h.  The
// row of direction k lies SIGN * ez(k) rows from `row` (SIGN 0: every
// direction from `row` itself; -1: the plane z - ez_k, where the odd step's
// population h_k comes from; +1: z + ez_k, where it goes).  Rows are
// kRefStride = 20 floats and 16-byte aligned.  VEC reads them in float4
// chunks, one load per chunk that holds a direction taking that row (5 loads
// for SIGN 0, 10 otherwise, instead of 19): measured 0.6-0.8% faster for the
// issue-bound 16-bit steps, 1% slower in FP32 (the even step then spills), so
// the FP32 steps take the scalar form.  Either way each element gets the same
// single rounding.
template <bool ADD, int SIGN, bool VEC>
__device__ __forceinline__ void ref_rows(float h[kQ], const float *row)
{
    if (!VEC) {
#pragma unroll
        for (int k = 0; k < kQ; ++k) {
            const float r = __ldg(row + SIGN * ez(k) * kRefStride + k);
            h[k] = ADD ? __fadd_rn(h[k], r) : __fsub_rn(h[k], r);
        }
        return;
    }
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
#pragma unroll
        for (int j = 0; j < kRefStride / 4; ++j) {
            bool any = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) any = any || (4 * j + q < kQ && SIGN * ez(4 * j + q) == d);
            if (!any) continue;
            const float4 v = __ldg(reinterpret_cast<const float4 *>(row + d * kRefStride) + j);
            const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * j + q;
                if (k < kQ && SIGN * ez(k) == d) h[k] = ADD ? __fadd_rn(h[k], c[q]) : __fsub_rn(h[k], c[q]);
            }
        }
    }
}

// First link index of cell i and its link mask.  Must be called by all 32
// lanes of a warp with lanes mapped to the aligned cells 32w .. 32w+31; m is
// this lane's mask (0 for padding lanes).
template <bool SKIP = true>
__device__ __forceinline__ uint32_t first_link(const uint32_t *__restrict__ warp_off, int32_t i, uint32_t m)
{
    // SKIP: no link in the warp, no scan (the offset is then never used)
    if (SKIP && !__any_sync(0xffffffffu, m != 0u)) return 0u;
    const uint32_t cnt = __popc(m);
    uint32_t incl = cnt;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    return warp_off[i >> 5] + incl - cnt;
}

// Eq. (CLI) on the links of mask m, whose coefficients are stored from off in
// increasing k: before the collision (INCOMING) the incoming populations are
// completed, h_opp(k) += a_k h_k; after it the partials are formed,
// h_k -= a_k h_opp(k).  A running index over the set bits replaces a
// popcount per direction; directions without a link are left untouched.
template <bool INCOMING>
__device__ __forceinline__ void cli_links(float h[kQ], const float *__restrict__ link_a, uint32_t off, uint32_t m)
{
    uint32_t r = off;
#pragma unroll
    for (int k = 1; k < kQ; ++k)
        if ((m >> k) & 1u) {
            const float a = link_a[r++];
            if (INCOMING) h[opp(k)] = fmaf(a, h[k], h[opp(k)]);
            else h[k] = fmaf(-a, h[opp(k)], h[k]);
        }
}

// CLI coefficients a[k] of the links in m (0 elsewhere).
__device__ __forceinline__ void load_links(float a[kQ], uint32_t m, const float *__restrict__ link_a, uint32_t off)
{
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
        a[k] = 0.0f;
        if ((m >> k) & 1u) a[k] = link_a[off++];
    }
}

// Completes the incoming populations of link-reverse directions:
// f_kbar = P + a_k f_k.  If a_k != 0 then opp(k) is no link, so the order of
// the updates does not matter.
__device__ __forceinline__ void cli_incoming(float h[kQ], const float a[kQ])
{
#pragma unroll
    for (int k = 1; k < kQ; ++k) h[opp(k)] = fmaf(a[k], h[k], h[opp(k)]);
}

// Replaces f~_k of link directions by the partial P = f~_k - a_k f~_kbar.
__device__ __forceinline__ void cli_outgoing(float h[kQ], const float a[kQ])
{
#pragma unroll
    for (int k = 1; k < kQ; ++k) h[k] = fmaf(-a[k], h[opp(k)], h[k]);
}

// Density deviation and momentum of shifted populations (Eq. (Macro); the
// shift w_k carries rho0 = 1 and no momentum).
__device__ __forceinline__ void moments(const float h[kQ], float &drho, float &jx, float &jy, float &jz)
{
    drho = 0.0f;
    jx = jy = jz = 0.0f;
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
        drho += h[k];
        if (ex(k) > 0) jx += h[k];
        if (ex(k) < 0) jx -= h[k];
        if (ey(k) > 0) jy += h[k];
        if (ey(k) < 0) jy -= h[k];
        if (ez(k) > 0) jz += h[k];
        if (ez(k) < 0) jz -= h[k];
    }
}

// e_k . j from the non-zero components only (exact: e_k has entries 0, +-1).
__device__ __forceinline__ float e_dot(int k, float jx, float jy, float jz)
{
    float s = 0.0f;
    bool any = false;
    if (ex(k)) {
        s = ex(k) > 0 ? jx : -jx;
        any = true;
    }
    if (ey(k)) {
        s = any ? __fadd_rn(s, ey(k) > 0 ? jy : -jy) : (ey(k) > 0 ? jy : -jy);
        any = true;
    }
    if (ez(k)) s = any ? __fadd_rn(s, ez(k) > 0 ? jz : -jz) : (ez(k) > 0 ? jz : -jz);
    return s;
}

// TRT collision with source (Eqs. (TRT), (TRT2), (equilibrium), (collision)),
// on shifted populations: h~_k = h_k - w+ (h_k^+ - e_k^+) - w- (h_k^- - e_k^-) + F_k,
// e_k^+ = w_k (drho + 9/2 (e.j)^2 - 3/2 j.j), e_k^- = 3 w_k e.j, with the
// pre-collision momentum j.  h is in storage units (Coef carries the scale of
// the quadratic terms and of F_k).  Pair by pair (k, kbar = k + 1 for odd k),
// with s = h_k + h_kbar and a = h_k - h_kbar:
//   dp = w+ (s/2 - e_k^+),   dm' = w-/2 a - (w- e_k^- + F_k),
//   h~_k = h_k - dp - dm',   h~_kbar = h_kbar - dp + dm'.
// Every rounding is spelled out (fmaf, __fmul_rn, __fadd_rn: the compiler may
// not contract or reorder them), so all step kernels produce the same bits for
// the same inputs whatever code surrounds the collision.
__device__ __forceinline__ void collide(float h[kQ], const Coef &c)
{
    float drho, jx, jy, jz;
    moments(h, drho, jx, jy, jz);
    const float usq = __fmul_rn(c.usq_c, fmaf(jz, jz, fmaf(jy, jy, __fmul_rn(jx, jx))));
    const float q = __fsub_rn(drho, usq);   // drho - 3/2 j.j: the isotropic part of e^+
    const float e0 = __fmul_rn((float)weight(0), q);
    h[0] = fmaf(-c.omega_p, __fsub_rn(h[0], e0), h[0]);
    const float qw[2] = {__fmul_rn((float)weight(1), q), __fmul_rn((float)weight(7), q)};
#pragma unroll
    for (int k = 1; k < kQ; k += 2) {
        const int kb = k + 1, cls = k <= 6 ? 0 : 1;
        const float eu = e_dot(k, jx, jy, jz);
        const float ep = fmaf(__fmul_rn(c.ep_c[cls], eu), eu, qw[cls]);
        const float dp = __fmul_rn(c.omega_p, fmaf(0.5f, __fadd_rn(h[k], h[kb]), -ep));
        const float dm = fmaf(c.half_omega_m, __fsub_rn(h[k], h[kb]), -fmaf(c.em_c[cls], eu, c.force[k]));
        const float hk = __fsub_rn(__fsub_rn(h[k], dp), dm);
        h[kb] = __fadd_rn(__fsub_rn(h[kb], dp), dm);
        h[k] = hk;
    }
}

// Gather of the streamed populations of cell i at time parity `odd`
// (before the CLI completion).  nb[k] = nbr[k-1][i] is needed for odd.
template <typename T>
__device__ __forceinline__ void gather_even(float h[kQ], const T *__restrict__ pdf, size_t n_pad, int32_t i)
{
#pragma unroll
    for (int k = 0; k < kQ; ++k) h[k] = ld(pdf + k * n_pad + i);
}

template <typename T>
__device__ __forceinline__ void gather_odd(float h[kQ], const T *__restrict__ pdf, size_t n_pad, int32_t i,
                                           const int32_t nb[kQ])
{
    h[0] = ld(pdf + i);
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        const int32_t up = nb[opp(k)];   // x - e_k = x + e_opp(k)
        const T *src = up >= 0 ? pdf + opp(k) * n_pad + up : pdf + k * n_pad + i;
        h[k] = ld(src);
    }
}

// Geometry of the row bitmasks of a single box (see lbm_internal.h).
struct RowGeo {
    const uint2 *words;
    const uint32_t *cell_xr;
    int nx, ny, nz, nw, periodic_z;
};

__device__ __forceinline__ void unpack_xyz(uint32_t v, int &x, int &y, int &z)
{
    x = (int)(v & ((1u << kXyzBitsX) - 1u));
    y = (int)((v >> kXyzBitsX) & ((1u << kXyzBitsY) - 1u));
    z = (int)(v >> (kXyzBitsX + kXyzBitsY));
}

// Fluid index of bit b of a row word, -1 when the cell is solid.
__device__ __forceinline__ int32_t word_pick(uint2 w, int b)
{
    const uint32_t bit = 1u << b;
    return (w.x & bit) ? (int32_t)(w.y + __popc(w.x & (bit - 1u))) : -1;
}

// Fluid indices of x-1, x, x+1 (periodic in x) in the row whose words start at
// `row` (global or shared memory): one word load, plus the neighbouring word
// at a word edge.
template <bool SHARED>
__device__ __forceinline__ void row_triple(int nx, const uint2 *row, int x, int xm, int xp, int32_t &im, int32_t &i0,
                                           int32_t &ip)
{
    auto load = [&](int w) { return SHARED ? row[w] : __ldg(row + w); };
    const int b = x & 31;
    const uint2 c = load(x >> 5);
    i0 = word_pick(c, b);
    im = b > 0 ? word_pick(c, b - 1) : word_pick(load(xm >> 5), xm & 31);
    ip = (b < 31 && x + 1 < nx) ? word_pick(c, b + 1) : word_pick(load(xp >> 5), xp & 31);
}

// The 18 neighbours of a cell from the row words of its row (y, z) and the
// rows (y +- 1, z +- 1); R(dy, dz) gives the words of row (y + dy, z + dz).
// Writes nb[k] (-1: solid) and returns the link mask (bit k: x + e_k solid).
template <bool SHARED, typename Rows>
__device__ __forceinline__ uint32_t neighbours_from_rows(int32_t nb[kQ], Rows R, int nx, int x, int32_t i)
{
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    int32_t self;
    nb[0] = i;
    row_triple<SHARED>(nx, R(0, 0), x, xm, xp, nb[2], self, nb[1]);      // -x, +x
    row_triple<SHARED>(nx, R(1, 0), x, xm, xp, nb[10], nb[3], nb[7]);    // (-1,1,0) (0,1,0) (1,1,0)
    row_triple<SHARED>(nx, R(-1, 0), x, xm, xp, nb[8], nb[4], nb[9]);    // (-1,-1,0) (0,-1,0) (1,-1,0)
    row_triple<SHARED>(nx, R(0, 1), x, xm, xp, nb[14], nb[5], nb[11]);   // (-1,0,1) (0,0,1) (1,0,1)
    row_triple<SHARED>(nx, R(0, -1), x, xm, xp, nb[12], nb[6], nb[13]);  // (-1,0,-1) (0,0,-1) (1,0,-1)
    const int b = x & 31, w = x >> 5;
    auto pick = [&](const uint2 *row) { return word_pick(SHARED ? row[w] : __ldg(row + w), b); };
    nb[15] = pick(R(1, 1));     // (0,1,1)
    nb[16] = pick(R(-1, -1));   // (0,-1,-1)
    nb[17] = pick(R(1, -1));    // (0,1,-1)
    nb[18] = pick(R(-1, 1));    // (0,-1,1)
    uint32_t m = 0;
#pragma unroll
    for (int k = 1; k < kQ; ++k) m |= (uint32_t)(nb[k] < 0) << k;
    return m;
}

// Neighbour indices of a fluid cell from the row bitmasks: the neighbour
// (x', y', z') is fluid when bit x' of row (y', z') is set, and its fluid index
// is the word's base plus the fluid cells below x' in the word.  Writes nb[k]
// (-1: solid) and returns the link mask (bit k: x + e_k solid).  Fluid cells
// never lie in a wall layer, so z +- 1 stays in the box when z is not periodic.
__device__ __forceinline__ uint32_t row_neighbours(int32_t nb[kQ], const RowGeo &g, int32_t i)
{
    int x, y, z;
    unpack_xyz(g.cell_xr[i], x, y, z);
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    int zm = z - 1, zp = z + 1;
    if (g.periodic_z) {
        zm = zm < 0 ? zm + g.nz : zm;
        zp = zp >= g.nz ? zp - g.nz : zp;
    }
    const uint32_t nw = (uint32_t)g.nw, ny = (uint32_t)g.ny;
    auto R = [&](int dy, int dz) {
        const int yy = dy < 0 ? ym : (dy > 0 ? yp : y), zz = dz < 0 ? zm : (dz > 0 ? zp : z);
        return g.words + ((uint32_t)yy + ny * (uint32_t)zz) * nw;
    };
    return neighbours_from_rows<false>(nb, R, g.nx, x, i);
}

// A tile whose odd step stages row words in shared memory (Solver::tile_rows,
// see k_stage_tiles): three bands (planes z - 1, z, z + 1) of band_rows rows
// each, starting at row r0 (r = y + ny z) of the part whose words start at
// words_base.
struct StagedTile {
    int32_t words_base, r0;
    int band_rows, nw, periodic_z, nz, nx, ny;
};

__device__ __forceinline__ StagedTile staged_tile(int4 d)
{
    StagedTile t;
    t.words_base = d.x;
    t.r0 = d.y;
    t.band_rows = d.z & 0xFF;
    t.nw = (d.z >> 8) & 0x7F;
    t.periodic_z = (d.z >> 15) & 1;
    t.nz = d.z >> 16;
    t.nx = d.w & 0xFFFF;
    t.ny = d.w >> 16;
    return t;
}

// Cooperative copy of the tile's bands into ws[3][band_rows][nw] (all
// threads of the block); rows outside the part read as empty.
__device__ __forceinline__ void stage_rows(uint2 *ws, const uint2 *__restrict__ words, const StagedTile &t)
{
    const int per_band = t.band_rows * t.nw, total = 3 * per_band, rows = t.ny * t.nz;
    for (int e = threadIdx.x; e < total; e += kBlock) {
        const int b = e / per_band, rem = e - b * per_band;
        const int j = rem / t.nw, w = rem - j * t.nw;
        const int row = t.r0 + (b - 1) * t.ny + j;
        ws[e] = row >= 0 && row < rows ? __ldg(words + t.words_base + (int64_t)row * t.nw + w) : make_uint2(0u, 0u);
    }
}

// Neighbour indices from the staged bands; false (nb untouched) when the cell
// needs a row outside them: a neighbour row across the periodic wrap in y, or
// in z for a periodic box.
__device__ __forceinline__ bool staged_neighbours(int32_t nb[kQ], uint32_t &m, const uint2 *ws, int4 sd, uint32_t xyz,
                                                  int32_t i)
{
    const StagedTile t = staged_tile(sd);
    int x, y, z;
    unpack_xyz(xyz, x, y, z);
    if (y == 0 || y == t.ny - 1 || (t.periodic_z && (z == 0 || z == t.nz - 1))) return false;
    const int lr = y + t.ny * z - t.r0;   // the cell's row within a band
    auto R = [&](int dy, int dz) { return ws + ((dz + 1) * t.band_rows + lr + dy) * t.nw; };
    m = neighbours_from_rows<true>(nb, R, t.nx, x, i);
    return true;
}

// Neighbour indices of a cell of a dense tile (Solver::tile_desc d): the
// tile's planes and their neighbours are fully fluid, so the fluid index of
// (x, y, z) is d.x + x + nx (y + ny (z - z_first)) and a neighbour is a fixed
// offset, with the periodic wrap in x and y.
__device__ __forceinline__ void dense_neighbours(int32_t nb[kQ], int2 d, int32_t i)
{
    const int nx = d.y & 0xFFFF, ny = d.y >> 16;
    const int32_t r = i - d.x, plane = nx * ny;
    const int x = r % nx, y = (r / nx) % ny;
    const int32_t ox[3] = {x == 0 ? nx - 1 : -1, 0, x == nx - 1 ? -(nx - 1) : 1};
    const int32_t oy[3] = {y == 0 ? (ny - 1) * nx : -nx, 0, y == ny - 1 ? -(ny - 1) * nx : nx};
    nb[0] = i;
#pragma unroll
    for (int k = 1; k < kQ; ++k) nb[k] = i + ox[ex(k) + 1] + oy[ey(k) + 1] + ez(k) * plane;
}

// Neighbour indices from the table for the eight directions without an x
// component and from arithmetic for the ten with one: fluid cells are
// numbered along x-rows, so the neighbour at x +- 1 of a fluid cell j in the
// same row is j +- 1 whenever it is fluid.  (x +- 1, y', z') is therefore the
// index of (x, y', z') +- 1 -- the table's entry of an axis direction, or i
// itself for +-x -- when both cells are fluid and x +- 1 does not wrap around
// the row (lm: the cell's link bits and row-end bits); otherwise, if the
// neighbour is fluid, its table entry is read.  Returns the link mask.
__device__ __forceinline__ uint32_t derived_nbr(int32_t nb[kQ], const int32_t *__restrict__ nbr, size_t n_pad, int32_t i,
                                                uint32_t lm)
{
    nb[0] = i;
#pragma unroll
    for (int k = 1; k < kQ; ++k)
        if (ex(k) == 0) nb[k] = nbr[(k - 1) * n_pad + i];
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        if (ex(k) == 0) continue;
        // the x-free direction with the same (ey, ez): 0 (the cell) or 3..6
        const int b = ey(k) > 0 ? 3 : ey(k) < 0 ? 4 : ez(k) > 0 ? 5 : ez(k) < 0 ? 6 : 0;
        const bool wraps = (lm & (ex(k) > 0 ? kXLast : kXFirst)) != 0u;
        const bool base_fluid = b == 0 || ((lm >> b) & 1u) == 0u;
        const int32_t base = b == 0 ? i : nb[b];
        if ((lm >> k) & 1u) nb[k] = -1;
        else if (base_fluid && !wraps) nb[k] = base + ex(k);
        else nb[k] = nbr[(k - 1) * n_pad + i];
    }
    return lm & kLinkBits;
}

__device__ __forceinline__ uint32_t load_nbr(int32_t nb[kQ], const int32_t *__restrict__ nbr, size_t n_pad, int32_t i)
{
    uint32_t m = 0;
    nb[0] = i;
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        nb[k] = nbr[(k - 1) * n_pad + i];
        m |= (uint32_t)(nb[k] < 0) << k;
    }
    return m;
}

}  // namespace lbm
