// glbm.cu -- the homogenised porous-medium LBM of Sec. 4 (Guo & Zhao's
// generalised LBM, see include/glbm.h) on a dense box.
//
// Layout: one slot per fluid cell and direction, pdf[k * n_pad + c] with c =
// x + nx (y + ny (z - z0)) over the fluid planes z0..z1 (x fastest), FP32,
// holding f_k - w_k.  Neighbours are arithmetic (periodic in x, y; in z
// periodic or bounded by the wall planes), so no index table is read.
//
// In-place AA pattern as in the pore-scale step (lbm_kernels.cuh): the even
// step reads A[k][c] and writes f~_k to A[opp k][c]; the odd step reads
// A[opp k][c - e_k] and writes f~_k to A[k][c + e_k].  A link into a wall
// plane has a dead slot A[opp k][c] that only its cell uses: the collision
// writes the bounced population f~_k - 6 w_k rho (e_k . u_wall) there, and
// the cell reads it back as f_{opp k} on the next step (half-way bounce-back
// with a moving wall).
//
// Per-plane constants (eps, 1/eps, omega = 1/tau, the source factor
// 1 - 1/(2 tau), c0, c1, the linear and quadratic drag coefficients) sit in a
// small table read through the read-only cache.
#include <climits>
#include <cmath>
#include <new>
#include <vector>

#include "glbm.h"
#include "lbm_internal.h"

namespace glbm {

using lbm::ex;
using lbm::ey;
using lbm::ez;
using lbm::kQ;
using lbm::opp;
using lbm::weight;

constexpr int kBlock = 256;

struct Plane {
    float eps, inv_eps, omega, src, c0, c1, drag1, drag2;
};

struct Args {
    float *pdf;
    const Plane *planes;   // [nz]
    int nx, ny, nz, z0, nzf;
    int32_t n_cells, n_pad;
    float g[3];
    float u_wall[2][3];    // [0] bottom, [1] top
    int periodic_z;
};

// Index offsets of the neighbours of a cell along each axis, for steps -1,
// 0, +1 (periodic wrap in x, y and, if set, z); a step into a wall plane is
// marked by kWall.  neighbour = c + ox[dx+1] + oy[dy+1] + oz[dz+1].
constexpr int32_t kWall = INT32_MIN / 2;

struct Offsets {
    int32_t ox[3], oy[3], oz[3];
};

__device__ __forceinline__ Offsets offsets(const Args &a, int32_t c, int &z)
{
    const int x = c % a.nx, y = (c / a.nx) % a.ny, zf = c / (a.nx * a.ny);
    z = a.z0 + zf;
    const int32_t sx = 1, sy = a.nx, sz = a.nx * a.ny;
    Offsets o;
    o.ox[0] = x == 0 ? (a.nx - 1) * sx : -sx;
    o.ox[1] = 0;
    o.ox[2] = x == a.nx - 1 ? -(a.nx - 1) * sx : sx;
    o.oy[0] = y == 0 ? (a.ny - 1) * sy : -sy;
    o.oy[1] = 0;
    o.oy[2] = y == a.ny - 1 ? -(a.ny - 1) * sy : sy;
    if (a.periodic_z) {
        o.oz[0] = zf == 0 ? (a.nzf - 1) * sz : -sz;
        o.oz[2] = zf == a.nzf - 1 ? -(a.nzf - 1) * sz : sz;
    } else {
        o.oz[0] = zf == 0 ? kWall : -sz;
        o.oz[2] = zf == a.nzf - 1 ? kWall : sz;
    }
    o.oz[1] = 0;
    return o;
}

// neighbour of c along direction k (sign +1) or -k (sign -1); negative: wall
__device__ __forceinline__ int32_t nb(const Offsets &o, int32_t c, int k, int sign)
{
    return c + o.ox[sign * ex(k) + 1] + o.oy[sign * ey(k) + 1] + o.oz[sign * ez(k) + 1];
}

// Density deviation drho = sum h (summed from zero so that FP32 keeps the
// small shifted values), Guo & Zhao's velocity and the force of
// Eq. (PorousForce) from the shifted populations h (rho = 1 + drho; the shift
// carries no momentum).
// FAST: the hardware reciprocal and reciprocal square root (a few ulp)
// instead of the IEEE division and square root, whose slow paths cost
// registers; used where that lets more blocks fit (the even step).
template <bool FAST = false>
__device__ __forceinline__ void macro(const float h[kQ], const Plane &P, const Args &a, float &drho, float u[3],
                                      float F[3])
{
    drho = 0.0f;
    float j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
        drho += h[k];
        if (ex(k)) j[0] += ex(k) * h[k];
        if (ey(k)) j[1] += ey(k) * h[k];
        if (ez(k)) j[2] += ez(k) * h[k];
    }
    const float rho = 1.0f + drho;
    auto root = [](float x) { return FAST ? (x > 0.0f ? x * rsqrtf(x) : 0.0f) : sqrtf(x); };
    const float inv_rho = FAST ? __fdividef(1.0f, rho) : 0.0f;
    float v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = (FAST ? j[d] * inv_rho : j[d] / rho) + 0.5f * P.eps * a.g[d];
    const float vn = root(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float den = P.c0 + root(P.c0 * P.c0 + P.c1 * vn);
    const float s = FAST ? __fdividef(1.0f, den) : 1.0f / den;
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = v[d] * s;
    const float un = root(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) F[d] = -(P.drag1 + P.drag2 * un) * u[d] + P.eps * a.g[d];
}

// BGK collision with Guo & Zhao's equilibrium and source, in place on h,
// over opposite pairs (k, k+1): e_{k+1} = -e_k, so the pair shares w, e.u and
// e.F up to sign, which keeps few values live.
template <bool FAST>
__device__ __forceinline__ float collide(float h[kQ], const Plane &P, const Args &a)
{
    float drho, u[3], F[3];
    macro<FAST>(h, P, a, drho, u, F);
    const float rho = 1.0f + drho;
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const float rs = rho * P.src;
    // rest population: e = 0
    {
        const float w = (float)weight(0);
        const float heq = w * (drho - rho * 1.5f * uu * P.inv_eps);
        h[0] = h[0] - P.omega * (h[0] - heq) - w * rs * 3.0f * uF * P.inv_eps;
    }
#pragma unroll
    for (int k = 1; k < kQ; k += 2) {
        const float w = (float)weight(k);
        const float eu = ex(k) * u[0] + ey(k) * u[1] + ez(k) * u[2];
        const float eF = ex(k) * F[0] + ey(k) * F[1] + ez(k) * F[2];
        // symmetric and antisymmetric parts of the pair's equilibrium and source
        const float eq_s = w * (drho + rho * (4.5f * eu * eu - 1.5f * uu) * P.inv_eps);
        const float eq_a = w * rho * 3.0f * eu;
        const float src_s = w * rs * (9.0f * eu * eF - 3.0f * uF) * P.inv_eps;
        const float src_a = w * rs * 3.0f * eF;
        const float hk = h[k], hb = h[k + 1];
        h[k] = hk - P.omega * (hk - (eq_s + eq_a)) + src_s + src_a;
        h[k + 1] = hb - P.omega * (hb - (eq_s - eq_a)) + src_s - src_a;
    }
    return rho;
}

// value written to the dead slot of wall link k: f~_k - 6 w_k rho (e_k . u_wall)
__device__ __forceinline__ float bounced(const Args &a, int k, float hk, float rho)
{
    const float *uw = a.u_wall[ez(k) > 0 ? 1 : 0];
    const float eu = ex(k) * uw[0] + ey(k) * uw[1] + ez(k) * uw[2];
    return hk - 6.0f * (float)weight(k) * rho * eu;
}

// Resident blocks per SM: measured on the 256x256x512 channel, the even step
// with the FAST velocity forms at 4 blocks (64 registers) and the odd step
// with the IEEE forms at 5 (48 registers); the other pairings were slower.
__global__ void __launch_bounds__(kBlock, 4) k_glbm_even(Args a)
{
    const int32_t c = blockIdx.x * kBlock + threadIdx.x;
    if (c >= a.n_cells) return;
    const uint32_t n_pad = (uint32_t)a.n_pad;
    float h[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) h[k] = a.pdf[k * n_pad + (uint32_t)c];
    const int zf = c / (a.nx * a.ny);
    const float rho = collide<true>(h, a.planes[a.z0 + zf], a);
    // f~_k goes to slot opp(k) of this cell
#pragma unroll
    for (int k = 0; k < kQ; ++k) a.pdf[opp(k) * n_pad + (uint32_t)c] = h[k];
    // next to a wall plane that slot is the dead slot of the link: it holds
    // the bounced population instead (a second store, on two planes only)
    const int side = a.periodic_z ? 0 : (zf == 0 ? -1 : (zf == a.nzf - 1 ? 1 : 0));
    if (side) {
#pragma unroll
        for (int k = 1; k < kQ; ++k)
            if (ez(k) == side) a.pdf[opp(k) * n_pad + (uint32_t)c] = bounced(a, k, h[k], rho);
    }
}

__global__ void __launch_bounds__(kBlock, 5) k_glbm_odd(Args a)
{
    const int32_t c = blockIdx.x * kBlock + threadIdx.x;
    if (c >= a.n_cells) return;
    int z;
    const uint32_t n_pad = (uint32_t)a.n_pad;
    float h[kQ];
    {
        const Offsets o = offsets(a, c, z);
        h[0] = a.pdf[(uint32_t)c];
#pragma unroll
        for (int k = 1; k < kQ; ++k) {
            const int32_t up = nb(o, c, k, -1);
            h[k] = up >= 0 ? a.pdf[opp(k) * n_pad + (uint32_t)up] : a.pdf[k * n_pad + (uint32_t)c];
        }
    }
    const float rho = collide<false>(h, a.planes[z], a);
    // the offsets again (cheaper than keeping them live across the collision)
    const Offsets o = offsets(a, c, z);
    a.pdf[(uint32_t)c] = h[0];
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        const int32_t down = nb(o, c, k, 1);
        if (down >= 0) a.pdf[k * n_pad + (uint32_t)down] = h[k];
        else a.pdf[opp(k) * n_pad + (uint32_t)c] = bounced(a, k, h[k], rho);
    }
}

// f_k - w_k of the current time (parity-aware read)
__device__ __forceinline__ void gather(const Args &a, bool odd, int32_t c, float h[kQ])
{
    int z;
    const Offsets o = offsets(a, c, z);
    const uint32_t n_pad = (uint32_t)a.n_pad;
    h[0] = a.pdf[(uint32_t)c];
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        const int32_t up = odd ? nb(o, c, k, -1) : -1;
        h[k] = up >= 0 ? a.pdf[opp(k) * n_pad + (uint32_t)up] : a.pdf[k * n_pad + (uint32_t)c];
    }
}

__global__ void k_glbm_populations(Args a, int odd, float *__restrict__ out)
{
    const int32_t c = blockIdx.x * kBlock + threadIdx.x;
    if (c >= a.n_cells) return;
    float h[kQ];
    gather(a, odd != 0, c, h);
#pragma unroll
    for (int k = 0; k < kQ; ++k) out[(size_t)k * a.n_cells + c] = h[k];
}

// dense moments over the whole box (wall planes zero)
__global__ void k_glbm_moments(Args a, int odd, float *__restrict__ rho_out, float *__restrict__ u_out)
{
    const int64_t cell = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int64_t ncell = (int64_t)a.nx * a.ny * a.nz;
    if (cell >= ncell) return;
    const int z = (int)(cell / ((int64_t)a.nx * a.ny));
    float rho = 0.0f, u[3] = {0.0f, 0.0f, 0.0f};
    if (z >= a.z0 && z < a.z0 + a.nzf) {
        const int32_t c = (int32_t)(cell - (int64_t)a.z0 * a.nx * a.ny);
        float h[kQ], F[3], drho;
        gather(a, odd != 0, c, h);
        macro(h, a.planes[z], a, drho, u, F);
        rho = 1.0f + drho;
    }
    if (rho_out) rho_out[cell] = rho;
    if (u_out)
        for (int d = 0; d < 3; ++d) u_out[d * ncell + cell] = u[d];
}

// plane sums of u_x: one block per plane, FP64 accumulation
__global__ void __launch_bounds__(kBlock) k_glbm_plane_sum(Args a, int odd, double *__restrict__ out)
{
    const int zf = blockIdx.x;
    const int32_t per = a.nx * a.ny;
    double s = 0.0;
    for (int32_t i = threadIdx.x; i < per; i += kBlock) {
        float h[kQ], drho, u[3], F[3];
        gather(a, odd != 0, zf * per + i, h);
        macro(h, a.planes[a.z0 + zf], a, drho, u, F);
        s += (double)u[0];
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    __shared__ double part[kBlock / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) t += part[w];
        out[a.z0 + zf] = t / (double)per;
    }
}

// f = f^eq(rho = 1, u0) (Guo & Zhao's equilibrium at the plane's eps)
__global__ void k_glbm_init(Args a, const float *__restrict__ u0)
{
    const int32_t c = blockIdx.x * kBlock + threadIdx.x;
    if (c >= a.n_cells) return;
    const int z = a.z0 + c / (a.nx * a.ny);
    const Plane P = a.planes[z];
    const int64_t ncell = (int64_t)a.nx * a.ny * a.nz;
    const int64_t cell = (int64_t)a.z0 * a.nx * a.ny + c;
    float u[3] = {0.0f, 0.0f, 0.0f};
    if (u0)
        for (int d = 0; d < 3; ++d) u[d] = u0[d * ncell + cell];
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
        const float eu = ex(k) * u[0] + ey(k) * u[1] + ez(k) * u[2];
        a.pdf[k * (uint32_t)a.n_pad + (uint32_t)c] =
            (float)weight(k) * (3.0f * eu + (4.5f * eu * eu - 1.5f * uu) * P.inv_eps);
    }
}

}  // namespace glbm

using namespace glbm;

struct glbm_solver {
    Args a{};
    cudaStream_t st = nullptr;
    int64_t steps = 0;
    double *plane_out = nullptr;   // device [nz]
};

namespace {

bool box_ok(const glbm_params *p, int64_t &n_cells)
{
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < (p->periodic_z ? 1 : 3)) return false;
    const int64_t nzf = p->periodic_z ? p->nz : p->nz - 2;
    n_cells = (int64_t)p->nx * p->ny * nzf;
    return n_cells < ((int64_t)1 << 31) / kQ;
}

struct Lay {
    size_t pdf, planes, plane_out, total;
    int32_t n_pad;
};

Lay layout(const glbm_params *p, int64_t n_cells)
{
    Lay L{};
    const int64_t n_pad = (n_cells + kBlock - 1) / kBlock * kBlock;
    L.n_pad = (int32_t)n_pad;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t at = off;
        off = lbm::align_up(off + (b ? b : 1), 256);
        return at;
    };
    L.pdf = take((size_t)kQ * n_pad * 4);
    L.planes = take((size_t)p->nz * sizeof(Plane));
    L.plane_out = take((size_t)p->nz * 8);
    L.total = off;
    return L;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace

extern "C" {

int glbm_workspace_size(const glbm_params *params, size_t *bytes)
{
    int64_t n = 0;
    if (!bytes || !box_ok(params, n)) return LBM_EINVAL;
    *bytes = layout(params, n).total;
    return LBM_OK;
}

int glbm_init(const glbm_params *p, const double *eps, const double *inv_k, const double *tau, void *dev_ws,
              size_t bytes, const float *dev_u0, void *stream, glbm_solver **out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    int64_t n_cells = 0;
    if (!box_ok(p, n_cells) || !eps || !inv_k || !tau || !(p->nu >= 0.0) || !(p->c_f >= 0.0)) return LBM_EINVAL;
    if (!dev_ws || ((uintptr_t)dev_ws & 255u)) return LBM_ESIZE;
    const Lay L = layout(p, n_cells);
    if (bytes < L.total) return LBM_ESIZE;
    const int z0 = p->periodic_z ? 0 : 1, nzf = p->periodic_z ? p->nz : p->nz - 2;
    std::vector<Plane> planes(p->nz);
    for (int z = 0; z < p->nz; ++z) {
        const bool fluid = z >= z0 && z < z0 + nzf;
        const double e = fluid ? eps[z] : 1.0, ik = fluid ? inv_k[z] : 0.0, t = fluid ? tau[z] : 1.0;
        if (!(e > 0.0 && e <= 1.0) || !(ik >= 0.0) || !(t > 0.5) || !std::isfinite(ik)) return LBM_EINVAL;
        Plane &P = planes[z];
        P.eps = (float)e;
        P.inv_eps = (float)(1.0 / e);
        P.omega = (float)(1.0 / t);
        P.src = (float)(1.0 - 0.5 / t);
        P.c0 = (float)(0.5 * (1.0 + 0.5 * e * p->nu * ik));
        P.c1 = (float)(0.5 * e * p->c_f * std::sqrt(ik));
        P.drag1 = (float)(e * p->nu * ik);
        P.drag2 = (float)(e * p->c_f * std::sqrt(ik));
    }
    glbm_solver *s = new (std::nothrow) glbm_solver();
    if (!s) return LBM_ENOMEM;
    char *ws = (char *)dev_ws;
    s->st = (cudaStream_t)stream;
    Args &a = s->a;
    a.pdf = (float *)(ws + L.pdf);
    a.planes = (const Plane *)(ws + L.planes);
    a.nx = p->nx;
    a.ny = p->ny;
    a.nz = p->nz;
    a.z0 = z0;
    a.nzf = nzf;
    a.n_cells = (int32_t)n_cells;
    a.n_pad = L.n_pad;
    for (int d = 0; d < 3; ++d) {
        a.g[d] = (float)p->g[d];
        a.u_wall[0][d] = (float)p->u_bottom[d];
        a.u_wall[1][d] = (float)p->u_top[d];
    }
    a.periodic_z = p->periodic_z;
    s->plane_out = (double *)(ws + L.plane_out);
    int rc = LBM_OK;
    if (cudaMemcpyAsync((void *)a.planes, planes.data(), planes.size() * sizeof(Plane), cudaMemcpyHostToDevice,
                        s->st) != cudaSuccess ||
        cudaMemsetAsync(a.pdf, 0, (size_t)kQ * a.n_pad * 4, s->st) != cudaSuccess)
        rc = LBM_ECUDA;
    if (rc == LBM_OK) {
        k_glbm_init<<<blocks_for(n_cells), kBlock, 0, s->st>>>(a, dev_u0);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s->st) != cudaSuccess) rc = LBM_ECUDA;
    }
    if (rc != LBM_OK) {
        delete s;
        return rc;
    }
    *out = s;
    return LBM_OK;
}

int glbm_step(glbm_solver *s, int64_t n)
{
    if (!s || n < 0) return LBM_EINVAL;
    const unsigned g = blocks_for(s->a.n_cells);
    for (int64_t t = 0; t < n; ++t, ++s->steps) {
        if ((s->steps & 1) == 0) k_glbm_even<<<g, kBlock, 0, s->st>>>(s->a);
        else k_glbm_odd<<<g, kBlock, 0, s->st>>>(s->a);
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int glbm_moments(glbm_solver *s, float *dev_rho, float *dev_u)
{
    if (!s) return LBM_EINVAL;
    const int64_t ncell = (int64_t)s->a.nx * s->a.ny * s->a.nz;
    k_glbm_moments<<<blocks_for(ncell), kBlock, 0, s->st>>>(s->a, (int)(s->steps & 1), dev_rho, dev_u);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int glbm_plane_average(glbm_solver *s, double *host_out)
{
    if (!s || !host_out) return LBM_EINVAL;
    if (cudaMemsetAsync(s->plane_out, 0, (size_t)s->a.nz * 8, s->st) != cudaSuccess) return LBM_ECUDA;
    k_glbm_plane_sum<<<(unsigned)s->a.nzf, kBlock, 0, s->st>>>(s->a, (int)(s->steps & 1), s->plane_out);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(host_out, s->plane_out, (size_t)s->a.nz * 8, cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
        cudaStreamSynchronize(s->st) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

int glbm_populations(glbm_solver *s, float *dev_out)
{
    if (!s || !dev_out) return LBM_EINVAL;
    k_glbm_populations<<<blocks_for(s->a.n_cells), kBlock, 0, s->st>>>(s->a, (int)(s->steps & 1), dev_out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int glbm_steps_done(const glbm_solver *s, int64_t *steps)
{
    if (!s || !steps) return LBM_EINVAL;
    *steps = s->steps;
    return LBM_OK;
}

void glbm_destroy(glbm_solver *s) { delete s; }

}  // extern "C"
