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
__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Relaxation constants and source term of one solver (kernel parameter).
struct Coef {
    float omega_p, omega_m;
    float force[kQ];   // F_k = 3 w_k e_k.g
    float half_g[3];   // g/2, added to j for the reported velocity
    float shift;       // uniform density shift removed before the collision (0: none)
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

// First link index of cell i and its link mask.  Must be called by all 32
// lanes of a warp with lanes mapped to the aligned cells 32w .. 32w+31; m is
// this lane's mask (0 for padding lanes).
__device__ __forceinline__ uint32_t first_link(const uint32_t *__restrict__ warp_off, int32_t i, uint32_t m)
{
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

// TRT collision with source (Eqs. (TRT), (TRT2), (equilibrium), (collision)),
// on shifted populations: h~_k = h_k - w+ (h_k^+ - e_k^+) - w- (h_k^- - e_k^-) + F_k,
// e_k^+ = w_k (drho + 9/2 (e.j)^2 - 3/2 j.j), e_k^- = 3 w_k e.j, with the
// pre-collision momentum j.
__device__ __forceinline__ void collide(float h[kQ], const Coef &c)
{
    float drho, jx, jy, jz;
    moments(h, drho, jx, jy, jz);
    const float usq = 1.5f * (jx * jx + jy * jy + jz * jz);
    h[0] -= c.omega_p * (h[0] - (float)weight(0) * (drho - usq));
#pragma unroll
    for (int k = 1; k < kQ; k += 2) {
        const int kb = k + 1;
        const float eu = (float)ex(k) * jx + (float)ey(k) * jy + (float)ez(k) * jz;
        const float w = (float)weight(k);
        const float ep = w * (drho + 4.5f * eu * eu - usq);
        const float em = 3.0f * w * eu;
        const float dp = c.omega_p * (0.5f * (h[k] + h[kb]) - ep);
        const float dm = c.omega_m * (0.5f * (h[k] - h[kb]) - em);
        const float hk = h[k] - dp - dm + c.force[k];
        const float hb = h[kb] - dp + dm - c.force[k];
        h[k] = hk;
        h[kb] = hb;
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
