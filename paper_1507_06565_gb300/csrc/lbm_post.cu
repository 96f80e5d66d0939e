// lbm_post.cu -- moments, plane averages, permeability, residual and the
// population export.  All reductions accumulate in FP64 with a fixed
// reduction tree (deterministic for a given geometry).
#include <cmath>

#include "lbm_kernels.cuh"

namespace lbm {
namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxPartials = 1024;

// Block sum of a double (all threads of the block must call it); valid in
// thread 0.
__device__ double block_sum(double v)
{
    __shared__ double warp_part[kRedThreads / 32];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_part[warp] = v;
    __syncthreads();
    v = threadIdx.x < kRedThreads / 32 ? warp_part[threadIdx.x] : 0.0;
    if (warp == 0)
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

struct PostArgs {
    const int32_t *nbr;
    const uint32_t *lmask;
    const uint32_t *warp_off;
    const float *link_a;
    int32_t n_fluid, n_pad;
    const int2 *tile_ref;
    int32_t ref_lo, ref_hi;
    const float *ref;
    float unscale;   // storage units -> populations (FP16 stores x 2^14)
    Coef c;
};

// Streamed populations of cell i at the current time (CLI-completed).
template <typename T, bool ODD>
__device__ __forceinline__ bool current_populations(const T *pdf, const PostArgs &p, int32_t i, float h[kQ])
{
    const bool live = i < p.n_fluid;
    const size_t n_pad = (size_t)p.n_pad;
    int32_t nb[kQ];
    uint32_t m = 0;
    if (live) m = ODD ? load_nbr(nb, p.nbr, n_pad, i) : p.lmask[i] & kLinkBits;
    const uint32_t off = first_link(p.warp_off, i, m);
    if (!live) return false;
    float a[kQ];
    load_links(a, m, p.link_a, off);
    if (ODD) gather_odd(h, pdf, n_pad, i, nb);
    else gather_even(h, pdf, n_pad, i);
    // reference populations of the slots' owners: the cell itself (even
    // time) or x - e_k (odd time, plane z - ez_k); dense tiles have no links
    const int32_t rr = ref_row<true>(p, i);
    if (rr >= 0) {
#pragma unroll
        for (int k = 0; k < kQ; ++k)
            h[k] = __fadd_rn(h[k], __ldg(p.ref + rr - (ODD ? ez(k) : 0) * kRefStride + k) * p.unscale);
    }
    cli_incoming(h, a);
    return true;
}

// rho - 1 = sum h and u = j + g/2 per fluid cell (fluid order).
template <typename T, bool ODD>
__global__ void __launch_bounds__(kBlock) k_fluid_moments(const T *__restrict__ pdf, PostArgs p,
                                                          float *__restrict__ rho, float *__restrict__ u)
{
    const int32_t i = blockIdx.x * kBlock + threadIdx.x;
    float h[kQ];
    if (!current_populations<T, ODD>(pdf, p, i, h)) return;
    float drho, jx, jy, jz;
    moments(h, drho, jx, jy, jz);
    const size_t n_pad = (size_t)p.n_pad;
    rho[i] = drho;
    u[i] = jx + p.c.half_g[0];
    u[n_pad + i] = jy + p.c.half_g[1];
    u[2 * n_pad + i] = jz + p.c.half_g[2];
}

template <typename T, bool ODD>
__global__ void __launch_bounds__(kBlock) k_populations(const T *__restrict__ pdf, PostArgs p, float *__restrict__ out)
{
    const int32_t i = blockIdx.x * kBlock + threadIdx.x;
    float h[kQ];
    if (!current_populations<T, ODD>(pdf, p, i, h)) return;
#pragma unroll
    for (int k = 0; k < kQ; ++k) out[(size_t)k * p.n_fluid + i] = h[k];
}

__global__ void k_scatter(const int32_t *__restrict__ fluid_cell, const float *__restrict__ rho_f,
                          const float *__restrict__ u_f, int32_t n_fluid, int32_t n_pad, int64_t ncell,
                          float *__restrict__ rho, float *__restrict__ u)
{
    const int32_t i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n_fluid) return;
    const int64_t c = fluid_cell[i];
    if (rho) rho[c] = 1.0f + rho_f[i];
    if (u) {
        u[c] = u_f[i];
        u[ncell + c] = u_f[(size_t)n_pad + i];
        u[2 * ncell + c] = u_f[2 * (size_t)n_pad + i];
    }
}

// One block per z plane: superficial and intrinsic mean of u_x, porosity.
__global__ void __launch_bounds__(kRedThreads) k_plane_average(const float *__restrict__ ux,
                                                               const int32_t *__restrict__ plane_off,
                                                               double area, double *__restrict__ out)
{
    const int z = blockIdx.x;
    const int32_t b = plane_off[z], e = plane_off[z + 1];
    double s = 0.0;
    for (int32_t i = b + threadIdx.x; i < e; i += kRedThreads) s += (double)ux[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        const int32_t n = e - b;
        out[3 * z + 0] = s / area;
        out[3 * z + 1] = n > 0 ? s / (double)n : 0.0;
        out[3 * z + 2] = (double)n / area;
    }
}

// K = nu <u_x>_sup / g_x over planes z_lo..z_hi of the plane averages.
__global__ void __launch_bounds__(kRedThreads) k_permeability(const double *__restrict__ planes, int z_lo, int z_hi,
                                                              double nu, double gx, double *__restrict__ k_out)
{
    double s = 0.0;
    for (int z = z_lo + threadIdx.x; z <= z_hi; z += kRedThreads) s += planes[3 * z];
    s = block_sum(s);
    if (threadIdx.x == 0) *k_out = nu * (s / (double)(z_hi - z_lo + 1)) / gx;
}

// Partial sums of |u - u_prev|^2, |u|^2 and the count of non-finite values.
__global__ void __launch_bounds__(kRedThreads) k_residual_partials(const float *__restrict__ u,
                                                                   const float *__restrict__ up, int32_t n_fluid,
                                                                   int32_t n_pad, int has_prev,
                                                                   double *__restrict__ partials)
{
    double num = 0.0, den = 0.0, bad = 0.0;
    for (int32_t i = blockIdx.x * kRedThreads + threadIdx.x; i < n_fluid; i += gridDim.x * kRedThreads) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float v = u[(size_t)d * n_pad + i];
            const double dv = has_prev ? (double)v - (double)up[(size_t)d * n_pad + i] : 0.0;
            num += dv * dv;
            den += (double)v * (double)v;
            bad += isfinite(v) ? 0.0 : 1.0;
        }
    }
    num = block_sum(num);
    den = block_sum(den);
    bad = block_sum(bad);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = num;
        partials[3 * blockIdx.x + 1] = den;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

// Partial sums of rho - 1 (mass drift).
__global__ void __launch_bounds__(kRedThreads) k_mass_partials(const float *__restrict__ drho, int32_t n_fluid,
                                                               double *__restrict__ partials)
{
    double m = 0.0, bad = 0.0;
    for (int32_t i = blockIdx.x * kRedThreads + threadIdx.x; i < n_fluid; i += gridDim.x * kRedThreads) {
        m += (double)drho[i];
        bad += isfinite(drho[i]) ? 0.0 : 1.0;
    }
    m = block_sum(m);
    bad = block_sum(bad);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = m;
        partials[3 * blockIdx.x + 1] = bad;
        partials[3 * blockIdx.x + 2] = 0.0;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_partials(const double *__restrict__ partials, int n,
                                                                 double *__restrict__ out)
{
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int b = threadIdx.x; b < n; b += kRedThreads) s += partials[3 * b + c];
        s = block_sum(s);
        if (threadIdx.x == 0) out[c] = s;
        __syncthreads();
    }
}

// Profile residual sums over the nz superficial plane averages; the current
// profile becomes the previous one.
__global__ void __launch_bounds__(kRedThreads) k_profile_residual(const double *__restrict__ planes,
                                                                  double *__restrict__ prev, int nz, int has_prev,
                                                                  double *__restrict__ out)
{
    double num = 0.0, den = 0.0, bad = 0.0;
    for (int z = threadIdx.x; z < nz; z += kRedThreads) {
        const double p = planes[3 * z];
        const double d = has_prev ? p - prev[z] : 0.0;
        num += d * d;
        den += p * p;
        bad += isfinite(p) ? 0.0 : 1.0;
    }
    num = block_sum(num);
    den = block_sum(den);
    bad = block_sum(bad);
    __syncthreads();
    for (int z = threadIdx.x; z < nz; z += kRedThreads) prev[z] = planes[3 * z];
    if (threadIdx.x == 0) {
        out[0] = num;
        out[1] = den;
        out[2] = bad;
    }
}

// Reference populations of the planes of one part from the current mean
// velocity of each referenced plane (u in fluid order, fresh from the
// moments kernel): R_k = f_k^eq(1, u_z) - w_k in storage units, zero rows for
// the other planes.  One block per plane.
__global__ void __launch_bounds__(kRedThreads) k_reference_update(const float *__restrict__ u, int32_t n_pad,
                                                                  const int32_t *__restrict__ plane_off,
                                                                  int32_t plane_base,
                                                                  const uint8_t *__restrict__ plane_flag, float scale,
                                                                  float *__restrict__ ref_next)
{
    __shared__ double mean[3];
    const int z = blockIdx.x;
    const int32_t gp = plane_base + z;
    float *out = ref_next + (size_t)gp * kRefStride;
    if (!plane_flag[gp]) {   // uniform over the block
        if (threadIdx.x < kRefStride) out[threadIdx.x] = 0.0f;
        return;
    }
    const int32_t b = plane_off[z], e = plane_off[z + 1];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int32_t i = b + threadIdx.x; i < e; i += kRedThreads) {
        sx += (double)u[i];
        sy += (double)u[(size_t)n_pad + i];
        sz += (double)u[2 * (size_t)n_pad + i];
    }
    sx = block_sum(sx);
    sy = block_sum(sy);
    sz = block_sum(sz);
    if (threadIdx.x == 0) {
        const double n = (double)(e - b);
        mean[0] = sx / n;
        mean[1] = sy / n;
        mean[2] = sz / n;
    }
    __syncthreads();
    const int k = threadIdx.x;
    if (k < kRefStride) {
        double r = 0.0;
        if (k < kQ) {
            const double eu = ex(k) * mean[0] + ey(k) * mean[1] + ez(k) * mean[2];
            const double uu = mean[0] * mean[0] + mean[1] * mean[1] + mean[2] * mean[2];
            r = weight(k) * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu) * (double)scale;
        }
        out[k] = (float)r;
    }
}

float storage_scale(const Solver &s) { return s.params.storage == LBM_F16 ? 16384.0f : 1.0f; }

PostArgs make_post(const Solver &s)
{
    PostArgs p;
    p.nbr = s.nbr;
    p.lmask = s.lmask;
    p.warp_off = s.warp_off;
    p.link_a = s.link_a;
    p.n_fluid = s.n_fluid;
    p.n_pad = s.n_pad;
    p.tile_ref = s.tile_ref;
    p.ref_lo = s.ref_lo;
    p.ref_hi = s.ref_hi;
    p.ref = s.ref;
    p.unscale = 1.0f / storage_scale(s);
    p.c = make_coef(s);
    return p;
}

template <typename T>
void fluid_moments_t(Solver &s)
{
    const PostArgs p = make_post(s);
    const unsigned grid = (unsigned)(s.n_pad / kBlock);
    if (s.steps & 1) k_fluid_moments<T, true><<<grid, kBlock, 0, s.stream>>>((const T *)s.pdf, p, s.rho_cur, s.u_cur);
    else k_fluid_moments<T, false><<<grid, kBlock, 0, s.stream>>>((const T *)s.pdf, p, s.rho_cur, s.u_cur);
}

template <typename T>
void populations_t(Solver &s, float *out)
{
    const PostArgs p = make_post(s);
    const unsigned grid = (unsigned)(s.n_pad / kBlock);
    if (s.steps & 1) k_populations<T, true><<<grid, kBlock, 0, s.stream>>>((const T *)s.pdf, p, out);
    else k_populations<T, false><<<grid, kBlock, 0, s.stream>>>((const T *)s.pdf, p, out);
}

}  // namespace

int launch_fluid_moments(Solver &s)
{
    if (s.n_fluid == 0) return LBM_OK;
    switch (s.params.storage) {
    case LBM_F32: fluid_moments_t<float>(s); break;
    case LBM_F16: fluid_moments_t<__half>(s); break;
    case LBM_BF16: fluid_moments_t<__nv_bfloat16>(s); break;
    default: return LBM_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_populations(Solver &s, float *out)
{
    if (s.n_fluid == 0) return LBM_OK;
    switch (s.params.storage) {
    case LBM_F32: populations_t<float>(s, out); break;
    case LBM_F16: populations_t<__half>(s, out); break;
    case LBM_BF16: populations_t<__nv_bfloat16>(s, out); break;
    default: return LBM_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_scatter_moments(Solver &s, float *rho, float *u)
{
    const size_t n = (size_t)s.n_cells;
    if (rho && cudaMemsetAsync(rho, 0, n * sizeof(float), s.stream) != cudaSuccess) return LBM_ECUDA;
    if (u && cudaMemsetAsync(u, 0, 3 * n * sizeof(float), s.stream) != cudaSuccess) return LBM_ECUDA;
    if (s.n_fluid == 0) return LBM_OK;
    int rc = launch_fluid_moments(s);
    if (rc != LBM_OK) return rc;
    k_scatter<<<(unsigned)(s.n_pad / kBlock), kBlock, 0, s.stream>>>(s.fluid_cell, s.rho_cur, s.u_cur, s.n_fluid,
                                                                      s.n_pad, s.n_cells, rho, u);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_plane_average(Solver &s)
{
    int rc = launch_fluid_moments(s);
    if (rc != LBM_OK) return rc;
    for (const Part &P : s.parts)
        k_plane_average<<<(unsigned)P.box.nz, kRedThreads, 0, s.stream>>>(
            s.u_cur, s.plane_off + P.poff_base, (double)P.box.nx * (double)P.box.ny, s.result + 3 * (size_t)P.plane_base);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_permeability(Solver &s, int part, int z_lo, int z_hi)
{
    if (part == 0 || s.parts.size() == 1) {
        const int rc = launch_plane_average(s);
        if (rc != LBM_OK) return rc;
    }
    const Part &P = s.parts[part];
    k_permeability<<<1, kRedThreads, 0, s.stream>>>(s.result + 3 * (size_t)P.plane_base, z_lo, z_hi, s.nu,
                                                    s.params.g[0], s.result + res_part(s.lay, part));
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_residual(Solver &s)
{
    int rc = launch_fluid_moments(s);
    if (rc != LBM_OK) return rc;
    const int np = (int)s.lay.n_partials;
    k_residual_partials<<<np, kRedThreads, 0, s.stream>>>(s.u_cur, s.u_prev, s.n_fluid, s.n_pad, s.has_prev ? 1 : 0,
                                                          s.partials);
    k_reduce_partials<<<1, kRedThreads, 0, s.stream>>>(s.partials, np, s.result + res_field(s.lay));
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_profile_residual(Solver &s)
{
    int rc = launch_plane_average(s);
    if (rc != LBM_OK) return rc;
    for (size_t b = 0; b < s.parts.size(); ++b) {
        const Part &P = s.parts[b];
        k_profile_residual<<<1, kRedThreads, 0, s.stream>>>(s.result + 3 * (size_t)P.plane_base,
                                                            s.prof_prev + P.plane_base, P.box.nz,
                                                            P.has_prev_profile ? 1 : 0, s.result + res_part(s.lay, (int)b) + 1);
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_mass(Solver &s)
{
    int rc = launch_fluid_moments(s);
    if (rc != LBM_OK) return rc;
    const int np = (int)s.lay.n_partials;
    k_mass_partials<<<np, kRedThreads, 0, s.stream>>>(s.rho_cur, s.n_fluid, s.partials);
    k_reduce_partials<<<1, kRedThreads, 0, s.stream>>>(s.partials, np, s.result + res_mass(s.lay));
    for (size_t b = 0; b < s.parts.size(); ++b) {
        const Part &P = s.parts[b];
        k_mass_partials<<<np, kRedThreads, 0, s.stream>>>(s.rho_cur + P.fluid_off, P.n_fluid, s.partials);
        k_reduce_partials<<<1, kRedThreads, 0, s.stream>>>(s.partials, np, s.result + res_part(s.lay, (int)b) + 4);
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int launch_reference_update(Solver &s)
{
    if (!s.has_ref) return LBM_OK;
    for (const Part &P : s.parts)
        k_reference_update<<<(unsigned)P.box.nz, kRedThreads, 0, s.stream>>>(
            s.u_cur, s.n_pad, s.plane_off + P.poff_base, P.plane_base, s.plane_flag, storage_scale(s), s.ref_next);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    s.ref_pending = true;
    return LBM_OK;
}

int residual_partial_count(int64_t n_fluid)
{
    int64_t b = (n_fluid + kRedThreads - 1) / kRedThreads;
    if (b < 1) b = 1;
    return (int)(b < kMaxPartials ? b : kMaxPartials);
}

}  // namespace lbm
