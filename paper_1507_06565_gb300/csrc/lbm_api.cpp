// lbm_api.cpp -- the extern "C" entry points declared in include/lbm.h.
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <utility>

#include "lbm_internal.h"

namespace lbm {

int residual_partial_count(int64_t n_fluid);   // lbm_post.cu

Layout make_layout(const lbm_box &box, int64_t n_fluid, int64_t n_links, int storage, size_t n_bins,
                   size_t n_images)
{
    Layout L{};
    const size_t A = 256;
    const int64_t ncell = (int64_t)box.nx * box.ny * box.nz;
    const int64_t n_pad = ((n_fluid > 0 ? n_fluid : 1) + kBlock - 1) / kBlock * kBlock;
    L.n_pad = (int32_t)n_pad;
    L.n_scan_blocks = (ncell + kBlock - 1) / kBlock;
    L.n_partials = residual_partial_count(n_fluid);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + (bytes ? bytes : 1), A);
        return at;
    };
    const size_t pdf_bytes = (size_t)kQ * n_pad * storage_bytes(storage);
    const size_t build_bytes = align_up((size_t)ncell * 4, A) + align_up((size_t)ncell, A);
    L.pdf = take(pdf_bytes > build_bytes ? pdf_bytes : build_bytes);
    L.idx_map = L.pdf;
    L.mask = L.pdf + align_up((size_t)ncell * 4, A);
    L.nbr = take((size_t)(kQ - 1) * n_pad * 4);
    L.lmask = take((size_t)n_pad * 4);
    L.warp_off = take((size_t)n_pad / 32 * 4);
    L.warp_cnt = take((size_t)n_pad / 32 * 4);
    L.link_a = take((size_t)(n_links > 0 ? n_links : 1) * 4);
    L.link_q = take((size_t)(n_links > 0 ? n_links : 1) * 8);
    L.fluid_cell = take((size_t)n_pad * 4);
    L.plane_off = take((size_t)(box.nz + 1) * 4);
    L.row_words = take((size_t)box.ny * box.nz * ((box.nx + 31) / 32) * 8);
    L.cell_xr = take((size_t)n_pad * 4);
    L.u_cur = take((size_t)3 * n_pad * 4);
    L.u_prev = take((size_t)3 * n_pad * 4);
    L.rho_cur = take((size_t)n_pad * 4);
    L.prof_prev = take((size_t)box.nz * 8);
    L.bins_start = take((n_bins + 1) * 4);
    L.bins_img = take(n_images * sizeof(SphereImage));
    L.scan_tmp = take((size_t)(L.n_scan_blocks + 1) * 4);
    L.partials = take((size_t)L.n_partials * 3 * 8);
    L.result = take((size_t)(3 * box.nz + 8) * 8);
    L.total = off;
    return L;
}

int x_bits_for(int nx)
{
    int b = 1;
    while ((1 << b) < nx) ++b;
    return b;
}

bool rows_packable(const lbm_box &box)
{
    const int xb = x_bits_for(box.nx);
    return (int64_t)box.ny * box.nz <= ((int64_t)1 << (32 - xb));
}

// The kernels address populations with 32-bit element offsets (19 n_pad <
// 2^32, about 226 million fluid cells) and links with 32-bit indices.
static bool size_ok(const Geometry &g)
{
    const int64_t n_pad = (g.n_fluid + kBlock - 1) / kBlock * kBlock;
    return (int64_t)kQ * n_pad < ((int64_t)1 << 32) && g.n_links <= (int64_t)std::numeric_limits<uint32_t>::max();
}

static bool params_ok(const lbm_params *p)
{
    if (!p) return false;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return false;
    if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return false;
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p->g[d])) return false;
    if (p->flags != 0 && p->flags != LBM_FLAG_NEIGHBOUR_TABLE && p->flags != LBM_FLAG_ROW_NEIGHBOURS) return false;
    return p->storage == LBM_F32 || p->storage == LBM_F16 || p->storage == LBM_BF16;
}

static int bins_for(const Geometry &g, Bins &bins)
{
    try {
        build_bins(g.box, g.spheres, bins);
    } catch (const std::bad_alloc &) {
        return LBM_ENOMEM;
    }
    return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_geometry_from_spheres(const lbm_sphere_params *params, lbm_geometry **out)
{
    if (!params || !out) return LBM_EINVAL;
    *out = nullptr;
    lbm_geometry *g = new (std::nothrow) lbm_geometry();
    if (!g) return LBM_ENOMEM;
    int rc;
    try {
        rc = place_and_voxelise(*params, *g);
    } catch (const std::bad_alloc &) {
        rc = LBM_ENOMEM;
    }
    if (rc != LBM_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return LBM_OK;
}

int lbm_geometry_from_list(const lbm_box *box, const double *xyzr, int64_t n, lbm_geometry **out)
{
    if (!box || !out) return LBM_EINVAL;
    *out = nullptr;
    lbm_geometry *g = new (std::nothrow) lbm_geometry();
    if (!g) return LBM_ENOMEM;
    int rc;
    try {
        rc = voxelise_list(*box, xyzr, n, *g);
    } catch (const std::bad_alloc &) {
        rc = LBM_ENOMEM;
    }
    if (rc != LBM_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return LBM_OK;
}

int lbm_geometry_info_get(const lbm_geometry *g, lbm_geometry_info *out)
{
    if (!g || !out) return LBM_EINVAL;
    out->n_cells = g->ncell();
    out->n_fluid = g->n_fluid;
    out->n_links = g->n_links;
    out->n_spheres = (int64_t)(g->spheres.size() / 4);
    out->porosity = g->porosity;
    return LBM_OK;
}

int lbm_geometry_spheres(const lbm_geometry *g, double *xyzr, int64_t cap, int64_t *n)
{
    if (!g || !n) return LBM_EINVAL;
    const int64_t cnt = (int64_t)(g->spheres.size() / 4);
    *n = cnt;
    if (cap < cnt) return LBM_ESIZE;
    if (cnt > 0) {
        if (!xyzr) return LBM_EINVAL;
        std::memcpy(xyzr, g->spheres.data(), sizeof(double) * 4 * (size_t)cnt);
    }
    return LBM_OK;
}

int lbm_geometry_mask(const lbm_geometry *g, uint8_t *mask)
{
    if (!g || !mask) return LBM_EINVAL;
    std::memcpy(mask, g->mask.data(), g->mask.size());
    return LBM_OK;
}

void lbm_geometry_destroy(lbm_geometry *g) { delete g; }

int lbm_workspace_size(const lbm_geometry *g, const lbm_params *params, size_t *bytes)
{
    if (!g || !bytes || !params_ok(params)) return LBM_EINVAL;
    if (!size_ok(*g)) return LBM_EINVAL;
    Bins bins;
    const int rc = bins_for(*g, bins);
    if (rc != LBM_OK) return rc;
    *bytes = make_layout(g->box, g->n_fluid, g->n_links, params->storage, bins.start.size() - 1,
                         bins.images.size()).total;
    return LBM_OK;
}

int lbm_init(const lbm_geometry *g, const lbm_params *params, void *dev_workspace, size_t bytes,
             const float *dev_u0, void *stream, lbm_solver **out)
{
    if (!g || !out || !params_ok(params)) return LBM_EINVAL;
    *out = nullptr;
    if (!size_ok(*g)) return LBM_EINVAL;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255u) != 0) return LBM_ESIZE;
    Bins bins;
    int rc = bins_for(*g, bins);
    if (rc != LBM_OK) return rc;
    const Layout L = make_layout(g->box, g->n_fluid, g->n_links, params->storage, bins.start.size() - 1,
                                 bins.images.size());
    if (bytes < L.total) return LBM_ESIZE;
    lbm_solver *s = new (std::nothrow) lbm_solver();
    if (!s) return LBM_ENOMEM;
    s->box = g->box;
    s->params = *params;
    s->stream = (cudaStream_t)stream;
    s->ws = (char *)dev_workspace;
    s->lay = L;
    s->n_cells = g->ncell();
    s->n_fluid = (int32_t)g->n_fluid;
    s->n_pad = L.n_pad;
    s->n_links = g->n_links;
    s->n_spheres = (int64_t)(g->spheres.size() / 4);
    s->nu = (params->tau - 0.5) / 3.0;
    s->omega_p = 1.0 / params->tau;
    s->omega_m = 1.0 / (params->lambda / (params->tau - 0.5) + 0.5);
    s->pdf = s->ws + L.pdf;
    s->nbr = (int32_t *)(s->ws + L.nbr);
    s->lmask = (uint32_t *)(s->ws + L.lmask);
    s->warp_off = (uint32_t *)(s->ws + L.warp_off);
    s->link_a = (float *)(s->ws + L.link_a);
    s->link_q = (double *)(s->ws + L.link_q);
    s->fluid_cell = (int32_t *)(s->ws + L.fluid_cell);
    s->plane_off = (int32_t *)(s->ws + L.plane_off);
    s->row_words = (uint2 *)(s->ws + L.row_words);
    s->cell_xr = (uint32_t *)(s->ws + L.cell_xr);
    s->n_words = (g->box.nx + 31) / 32;
    s->x_bits = x_bits_for(g->box.nx);
    {
        bool rows = params->storage != LBM_F32;   // auto: see LBM_FLAG_* in lbm.h
        if (params->flags == LBM_FLAG_NEIGHBOUR_TABLE) rows = false;
        if (params->flags == LBM_FLAG_ROW_NEIGHBOURS) rows = true;
        s->odd_rows = rows && rows_packable(g->box);
    }
    s->u_cur = (float *)(s->ws + L.u_cur);
    s->u_prev = (float *)(s->ws + L.u_prev);
    s->rho_cur = (float *)(s->ws + L.rho_cur);
    s->prof_prev = (double *)(s->ws + L.prof_prev);
    s->partials = (double *)(s->ws + L.partials);
    s->result = (double *)(s->ws + L.result);
    s->nbins_x = bins.nbx;
    s->nbins_y = bins.nby;
    s->nbins_z = bins.nbz;
    rc = device_build(*s, *g, bins);
    if (rc == LBM_OK) rc = launch_init(*s, dev_u0);
    if (rc == LBM_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = LBM_ECUDA;
    if (rc != LBM_OK) {
        delete s;
        return rc;
    }
    *out = s;
    return LBM_OK;
}

int lbm_reset(lbm_solver *s, const float *dev_u0)
{
    if (!s) return LBM_EINVAL;
    s->has_prev = false;
    s->has_prev_profile = false;
    return launch_init(*s, dev_u0);
}

int lbm_step(lbm_solver *s, int64_t n)
{
    if (!s || n < 0) return LBM_EINVAL;
    return launch_steps(*s, n);
}

int lbm_moments(lbm_solver *s, float *dev_rho, float *dev_u)
{
    if (!s) return LBM_EINVAL;
    return launch_scatter_moments(*s, dev_rho, dev_u);
}

int lbm_plane_average(lbm_solver *s, double *host_out)
{
    if (!s || !host_out) return LBM_EINVAL;
    int rc = launch_plane_average(*s);
    if (rc != LBM_OK) return rc;
    if (cudaMemcpyAsync(host_out, s->result, sizeof(double) * 3 * (size_t)s->box.nz, cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
        return LBM_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_permeability(lbm_solver *s, int32_t z_lo, int32_t z_hi, double *k_out)
{
    if (!s || !k_out) return LBM_EINVAL;
    if (z_lo == -1 && z_hi == -1) {
        z_lo = 0;
        z_hi = s->box.nz - 1;
    }
    if (z_lo < 0 || z_hi >= s->box.nz || z_lo > z_hi || s->params.g[0] == 0.0) return LBM_EINVAL;
    int rc = launch_permeability(*s, z_lo, z_hi);
    if (rc != LBM_OK) return rc;
    if (cudaMemcpyAsync(k_out, s->result + 3 * (size_t)s->box.nz, sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
        return LBM_ECUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_residual(lbm_solver *s, double *res_out)
{
    if (!s || !res_out) return LBM_EINVAL;
    int rc = launch_residual(*s);
    if (rc != LBM_OK) return rc;
    double r[3];
    if (cudaMemcpyAsync(r, s->result, sizeof(r), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) return LBM_ECUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return LBM_ECUDA;
    const bool had_prev = s->has_prev;
    std::swap(s->u_cur, s->u_prev);
    s->has_prev = true;
    if (r[2] != 0.0 || !std::isfinite(r[0]) || !std::isfinite(r[1])) {
        *res_out = std::numeric_limits<double>::quiet_NaN();
        return LBM_ENAN;
    }
    *res_out = had_prev ? std::sqrt(r[0]) / std::sqrt(r[1]) : std::numeric_limits<double>::infinity();
    return LBM_OK;
}

int lbm_profile_residual(lbm_solver *s, double *res_out)
{
    if (!s || !res_out) return LBM_EINVAL;
    int rc = launch_profile_residual(*s);
    if (rc != LBM_OK) return rc;
    double r[3];
    if (cudaMemcpyAsync(r, s->result + 3 * (size_t)s->box.nz + 1, sizeof(r), cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return LBM_ECUDA;
    const bool had_prev = s->has_prev_profile;
    s->has_prev_profile = true;
    if (r[2] != 0.0 || !std::isfinite(r[0]) || !std::isfinite(r[1])) {
        *res_out = std::numeric_limits<double>::quiet_NaN();
        return LBM_ENAN;
    }
    *res_out = had_prev ? std::sqrt(r[0]) / std::sqrt(r[1]) : std::numeric_limits<double>::infinity();
    return LBM_OK;
}

int lbm_mass(lbm_solver *s, double *mean_drho)
{
    if (!s || !mean_drho) return LBM_EINVAL;
    if (s->n_fluid == 0) {
        *mean_drho = 0.0;
        return LBM_OK;
    }
    int rc = launch_mass(*s);
    if (rc != LBM_OK) return rc;
    double r[2];
    if (cudaMemcpyAsync(r, s->result + 3 * (size_t)s->box.nz + 4, sizeof(r), cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return LBM_ECUDA;
    if (r[1] != 0.0 || !std::isfinite(r[0])) return LBM_ENAN;
    *mean_drho = r[0] / (double)s->n_fluid;
    return LBM_OK;
}

int lbm_recenter(lbm_solver *s, double *shift_out)
{
    double m = 0.0;
    int rc = lbm_mass(s, &m);
    if (rc != LBM_OK) return rc;
    s->drho_shift = m;   // the state is measured afresh: replace, do not accumulate
    if (shift_out) *shift_out = s->drho_shift;
    return LBM_OK;
}

int lbm_run_until(lbm_solver *s, double tol, int64_t interval, int64_t max_steps, int32_t criterion,
                  int64_t *steps_done, double *res_out)
{
    if (!s || interval < 1 || max_steps < 0 || !(tol > 0.0)) return LBM_EINVAL;
    if (criterion != LBM_CONVERGE_FIELD && criterion != LBM_CONVERGE_PROFILE) return LBM_EINVAL;
    auto residual = [&](double *r) {
        return criterion == LBM_CONVERGE_FIELD ? lbm_residual(s, r) : lbm_profile_residual(s, r);
    };
    int64_t done = 0;
    double res = std::numeric_limits<double>::infinity();
    int rc = residual(&res);
    while (rc == LBM_OK) {
        if (done > 0 && res < tol) break;
        if (done >= max_steps) {
            rc = LBM_ENOTCONVERGED;
            break;
        }
        const int64_t n = interval < max_steps - done ? interval : max_steps - done;
        rc = launch_steps(*s, n);
        if (rc != LBM_OK) break;
        done += n;
        rc = residual(&res);
        if (rc == LBM_OK) rc = lbm_recenter(s, nullptr);
    }
    if (steps_done) *steps_done = done;
    if (res_out) *res_out = res;
    return rc;
}

int lbm_steps_done(const lbm_solver *s, int64_t *steps)
{
    if (!s || !steps) return LBM_EINVAL;
    *steps = s->steps;
    return LBM_OK;
}

int lbm_solver_info(const lbm_solver *s, lbm_geometry_info *out)
{
    if (!s || !out) return LBM_EINVAL;
    out->n_cells = s->n_cells;
    out->n_fluid = s->n_fluid;
    out->n_links = s->n_links;
    out->n_spheres = s->n_spheres;
    out->porosity = (double)s->n_fluid / (double)s->n_cells;
    return LBM_OK;
}

int lbm_export_lists(lbm_solver *s, int32_t *fluid_cell, int32_t *nbr, int32_t *link_cell, int8_t *link_k,
                     double *link_q, uint8_t *link_fallback)
{
    if (!s) return LBM_EINVAL;
    const size_t nf = (size_t)s->n_fluid;
    cudaStream_t st = s->stream;
    if (fluid_cell && nf &&
        cudaMemcpyAsync(fluid_cell, s->fluid_cell, nf * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LBM_ECUDA;
    if (nbr && nf &&
        cudaMemcpy2DAsync(nbr, nf * 4, s->nbr, (size_t)s->n_pad * 4, nf * 4, kQ - 1, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return LBM_ECUDA;
    if (link_q && s->n_links &&
        cudaMemcpyAsync(link_q, s->link_q, (size_t)s->n_links * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return LBM_ECUDA;
    if (link_cell || link_k || link_fallback) {
        uint32_t *mask = new (std::nothrow) uint32_t[nf ? nf : 1];
        if (!mask) return LBM_ENOMEM;
        if (nf && cudaMemcpyAsync(mask, s->lmask, nf * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            delete[] mask;
            return LBM_ECUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            delete[] mask;
            return LBM_ECUDA;
        }
        size_t l = 0;
        for (size_t i = 0; i < nf; ++i)
            for (int k = 1; k < kQ; ++k)
                if ((mask[i] >> k) & 1u) {
                    if (link_cell) link_cell[l] = (int32_t)i;
                    if (link_k) link_k[l] = (int8_t)k;
                    if (link_fallback) link_fallback[l] = (uint8_t)((mask[i] >> opp(k)) & 1u);
                    ++l;
                }
        delete[] mask;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_populations(lbm_solver *s, float *dev_out)
{
    if (!s || !dev_out) return LBM_EINVAL;
    return launch_populations(*s, dev_out);
}

void lbm_solver_destroy(lbm_solver *s) { delete s; }

const char *lbm_status_string(int status)
{
    switch (status) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "host allocation failed";
    case LBM_ECUDA: return "CUDA runtime error";
    case LBM_EPACKING: return "target porosity unreachable without overlap";
    case LBM_ENAN: return "non-finite velocity field";
    case LBM_ENOTCONVERGED: return "not converged within max_steps";
    case LBM_ETIMEOUT: return "device-side wait timed out";
    case LBM_ESIZE: return "workspace too small or misaligned";
    }
    return "unknown status";
}

}  // extern "C"
