// lbm_api.cpp -- the extern "C" entry points declared in include/lbm.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <utility>

#include "lbm_internal.h"

namespace lbm {

int residual_partial_count(int64_t n_fluid);   // lbm_post.cu

Layout make_layout(const std::vector<const Geometry *> &geoms, int storage, size_t n_bins, size_t n_images)
{
    Layout L{};
    const size_t A = 256;
    int64_t n_fluid = 0, n_links = 0, ncell_max = 0;
    int32_t n_planes = 0, n_poff = 0;
    for (const Geometry *g : geoms) {
        n_fluid += g->n_fluid;
        n_links += g->n_links;
        ncell_max = std::max(ncell_max, g->ncell());
        n_planes += g->box.nz;
        n_poff += g->box.nz + 1;
    }
    bool packable = true;
    int64_t n_words = 0;
    for (const Geometry *g : geoms) {
        packable = packable && rows_packable(g->box);
        n_words += (int64_t)g->box.ny * g->box.nz * ((g->box.nx + 31) / 32);
    }
    const int64_t n_pad = ((n_fluid > 0 ? n_fluid : 1) + kBlock - 1) / kBlock * kBlock;
    L.n_pad = (int32_t)n_pad;
    L.n_parts = (int32_t)geoms.size();
    L.n_planes = n_planes;
    L.n_scan_blocks = (ncell_max + kBlock - 1) / kBlock;
    L.n_partials = residual_partial_count(n_fluid);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + (bytes ? bytes : 1), A);
        return at;
    };
    const size_t pdf_bytes = (size_t)kQ * n_pad * storage_bytes(storage);
    const size_t build_bytes = align_up((size_t)ncell_max * 4, A) + align_up((size_t)ncell_max, A);
    L.pdf = take(pdf_bytes > build_bytes ? pdf_bytes : build_bytes);
    L.idx_map = L.pdf;
    L.mask = L.pdf + align_up((size_t)ncell_max * 4, A);
    L.nbr = take((size_t)(kQ - 1) * n_pad * 4);
    L.lmask = take((size_t)n_pad * 4);
    L.warp_off = take((size_t)n_pad / 32 * 4);
    L.warp_cnt = take((size_t)n_pad / 32 * 4);
    L.link_a = take((size_t)(n_links > 0 ? n_links : 1) * 4);
    L.link_q = take((size_t)(n_links > 0 ? n_links : 1) * 8);
    L.fluid_cell = take((size_t)n_pad * 4);
    L.plane_off = take((size_t)n_poff * 4);
    L.tile_desc = take((size_t)n_pad / kBlock * 8);
    L.row_words = take(packable ? (size_t)n_words * 8 : 0);
    L.cell_xr = take(packable ? (size_t)n_pad * 4 : 0);
    L.tile_rows = take((size_t)n_pad / kBlock * 16);
    L.u_cur = take((size_t)3 * n_pad * 4);
    L.u_prev = take((size_t)3 * n_pad * 4);
    L.rho_cur = take((size_t)n_pad * 4);
    L.prof_prev = take((size_t)n_planes * 8);
    L.bins_start = take((n_bins + 1) * 4);
    L.bins_img = take(n_images * sizeof(SphereImage));
    L.scan_tmp = take((size_t)(L.n_scan_blocks + 1) * 4);
    L.partials = take((size_t)L.n_partials * 3 * 8);
    L.result = take((res_part(L, L.n_parts) + 8) * 8);
    L.part_shift = take((size_t)L.n_parts * 4);
    L.part_foff = take((size_t)(L.n_parts + 1) * 4);
    L.status = take(sizeof(int));
    L.ref = take((size_t)n_planes * kRefStride * 4);
    L.ref_next = take((size_t)n_planes * kRefStride * 4);
    L.tile_ref = take((size_t)n_pad / kBlock * 8);
    L.plane_flag = take((size_t)n_planes);
    L.total = off;
    return L;
}

bool rows_packable(const lbm_box &box)
{
    return box.nx <= (1 << kXyzBitsX) && box.ny <= (1 << kXyzBitsY) && box.nz <= (1 << kXyzBitsZ);
}

// The kernels address populations with 32-bit element offsets (19 n_pad <
// 2^32, about 226 million fluid cells) and links with 32-bit indices.
static bool size_ok(const std::vector<const Geometry *> &geoms)
{
    int64_t nf = 0, nl = 0;
    for (const Geometry *g : geoms) {
        nf += g->n_fluid;
        nl += g->n_links;
    }
    const int64_t n_pad = (nf + kBlock - 1) / kBlock * kBlock;
    return (int64_t)kQ * n_pad < ((int64_t)1 << 32) && nl <= (int64_t)std::numeric_limits<uint32_t>::max();
}

static bool params_ok(const lbm_params *p)
{
    if (!p) return false;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return false;
    if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return false;
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p->g[d])) return false;
    const int32_t known = LBM_FLAG_NEIGHBOUR_TABLE | LBM_FLAG_ROW_NEIGHBOURS | LBM_FLAG_NO_GRAPH | LBM_FLAG_NO_AUTOTUNE |
                          LBM_FLAG_SIMPLE_BOUNCE_BACK | LBM_FLAG_STAGED_EVEN | LBM_FLAG_CLI_SAFEGUARDS |
                          LBM_FLAG_STAGED_NEIGHBOURS | LBM_FLAG_PLANE_REFERENCES | LBM_FLAG_NO_PLANE_REFERENCES |
                          LBM_FLAG_DERIVED_NEIGHBOURS;
    if ((p->flags & ~known) != 0) return false;
    const int32_t variants = p->flags & (LBM_FLAG_NEIGHBOUR_TABLE | LBM_FLAG_ROW_NEIGHBOURS | LBM_FLAG_STAGED_NEIGHBOURS |
                                         LBM_FLAG_DERIVED_NEIGHBOURS);
    if (variants & (variants - 1)) return false;   // at most one neighbour variant
    if ((p->flags & LBM_FLAG_PLANE_REFERENCES) && (p->flags & LBM_FLAG_NO_PLANE_REFERENCES)) return false;
    return p->storage == LBM_F32 || p->storage == LBM_F16 || p->storage == LBM_BF16;
}

// Largest bin table over the parts (the device build uploads one part at a time).
static int bins_extent(const std::vector<const Geometry *> &geoms, size_t &n_bins, size_t &n_images)
{
    n_bins = 0;
    n_images = 0;
    for (const Geometry *g : geoms) {
        n_bins = std::max(n_bins, g->link_bins.start.size() - 1);
        n_images = std::max(n_images, g->link_bins.images.size());
    }
    return LBM_OK;
}

static int collect(const lbm_geometry *const *geoms, int32_t n, std::vector<const Geometry *> &out)
{
    if (!geoms || n < 1) return LBM_EINVAL;
    out.clear();
    for (int32_t b = 0; b < n; ++b) {
        if (!geoms[b]) return LBM_EINVAL;
        out.push_back(geoms[b]);
    }
    return LBM_OK;
}

static int workspace_size(const std::vector<const Geometry *> &geoms, const lbm_params *params, size_t *bytes)
{
    if (!bytes || !params_ok(params) || !size_ok(geoms)) return LBM_EINVAL;
    size_t nb = 0, ni = 0;
    const int rc = bins_extent(geoms, nb, ni);
    if (rc != LBM_OK) return rc;
    *bytes = make_layout(geoms, params->storage, nb, ni).total;
    return LBM_OK;
}

static int init_parts(const std::vector<const Geometry *> &geoms, const lbm_params *params, void *dev_workspace,
                      size_t bytes, const float *dev_u0, void *stream, lbm_solver **out)
{
    if (!out || !params_ok(params)) return LBM_EINVAL;
    *out = nullptr;
    if (!size_ok(geoms)) return LBM_EINVAL;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255u) != 0) return LBM_ESIZE;
    size_t nb = 0, ni = 0;
    int rc = bins_extent(geoms, nb, ni);
    if (rc != LBM_OK) return rc;
    const Layout L = make_layout(geoms, params->storage, nb, ni);
    if (bytes < L.total) return LBM_ESIZE;
    lbm_solver *s = new (std::nothrow) lbm_solver();
    if (!s) return LBM_ENOMEM;
    s->box = geoms[0]->box;
    s->params = *params;
    s->stream = (cudaStream_t)stream;
    s->ws = (char *)dev_workspace;
    s->lay = L;
    int64_t cell_base = 0, words_base = 0;
    int32_t fluid_off = 0, plane_base = 0, poff_base = 0;
    for (const Geometry *g : geoms) {
        Part P;
        P.box = g->box;
        P.cell_base = cell_base;
        P.n_cells = g->ncell();
        P.fluid_off = fluid_off;
        P.n_fluid = (int32_t)g->n_fluid;
        P.n_links = g->n_links;
        P.n_spheres = (int64_t)(g->spheres.size() / 4);
        P.plane_base = plane_base;
        P.poff_base = poff_base;
        P.words_base = words_base;
        s->parts.push_back(P);
        words_base += (int64_t)g->box.ny * g->box.nz * ((g->box.nx + 31) / 32);
        cell_base += P.n_cells;
        fluid_off += P.n_fluid;
        plane_base += g->box.nz;
        poff_base += g->box.nz + 1;
        s->n_links += g->n_links;
        s->n_spheres += P.n_spheres;
    }
    s->n_cells = cell_base;
    s->n_fluid = fluid_off;
    s->n_pad = L.n_pad;
    s->shift_host.assign(s->parts.size(), 0.0f);
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
    s->tile_desc = (int2 *)(s->ws + L.tile_desc);
    s->tile_rows = (int4 *)(s->ws + L.tile_rows);
    s->u_cur = (float *)(s->ws + L.u_cur);
    s->u_prev = (float *)(s->ws + L.u_prev);
    s->rho_cur = (float *)(s->ws + L.rho_cur);
    s->prof_prev = (double *)(s->ws + L.prof_prev);
    s->partials = (double *)(s->ws + L.partials);
    s->result = (double *)(s->ws + L.result);
    s->part_shift = (float *)(s->ws + L.part_shift);
    s->part_foff = (int32_t *)(s->ws + L.part_foff);
    s->status = (int *)(s->ws + L.status);
    s->ref = (float *)(s->ws + L.ref);
    s->ref_next = (float *)(s->ws + L.ref_next);
    s->tile_ref = (int2 *)(s->ws + L.tile_ref);
    s->plane_flag = (uint8_t *)(s->ws + L.plane_flag);
    const bool single = geoms.size() == 1;
    s->n_words = (s->box.nx + 31) / 32;
    s->rows_ok = true;   // make_layout gives every part row words and cell_xr then
    for (const Geometry *g : geoms) s->rows_ok = s->rows_ok && rows_packable(g->box);
    {
        bool rows = false;   // auto: the table (see LBM_FLAG_* in lbm.h)
        if (params->flags & LBM_FLAG_NEIGHBOUR_TABLE) rows = false;
        if (params->flags & LBM_FLAG_ROW_NEIGHBOURS) rows = true;
        s->odd_rows = rows && single && s->rows_ok;
        s->staged_rows = (params->flags & LBM_FLAG_STAGED_NEIGHBOURS) && s->rows_ok && !s->odd_rows;
        s->derived_nbrs = (params->flags & LBM_FLAG_DERIVED_NEIGHBOURS) != 0;
    }
    s->use_graph = !(params->flags & LBM_FLAG_NO_GRAPH);
    s->autotune = !(params->flags & LBM_FLAG_NO_AUTOTUNE);
    s->staged_even = (params->flags & LBM_FLAG_STAGED_EVEN) != 0;
    std::vector<int32_t> foff;
    for (const Part &P : s->parts) foff.push_back(P.fluid_off);
    foff.push_back(s->n_fluid);
    rc = device_build(*s, geoms);
    if (rc == LBM_OK && cudaMemcpyAsync(s->part_foff, foff.data(), foff.size() * 4, cudaMemcpyHostToDevice,
                                        s->stream) != cudaSuccess)
        rc = LBM_ECUDA;
    if (rc == LBM_OK) rc = launch_init(*s, dev_u0);
    if (rc == LBM_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = LBM_ECUDA;
    if (rc != LBM_OK) {
        delete s;
        return rc;
    }
    *out = s;
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
        if (rc == LBM_OK) build_bins(g->box, g->spheres, g->link_bins);
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
        if (rc == LBM_OK) build_bins(g->box, g->spheres, g->link_bins);
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
    if (!g) return LBM_EINVAL;
    return workspace_size({g}, params, bytes);
}

int lbm_init(const lbm_geometry *g, const lbm_params *params, void *dev_workspace, size_t bytes,
             const float *dev_u0, void *stream, lbm_solver **out)
{
    if (!g) return LBM_EINVAL;
    return init_parts({g}, params, dev_workspace, bytes, dev_u0, stream, out);
}

int lbm_batch_workspace_size(const lbm_geometry *const *geoms, int32_t n, const lbm_params *params, size_t *bytes)
{
    std::vector<const Geometry *> v;
    const int rc = collect(geoms, n, v);
    return rc != LBM_OK ? rc : workspace_size(v, params, bytes);
}

int lbm_batch_init(const lbm_geometry *const *geoms, int32_t n, const lbm_params *params, void *dev_workspace,
                   size_t bytes, const float *dev_u0, void *stream, lbm_solver **out)
{
    std::vector<const Geometry *> v;
    const int rc = collect(geoms, n, v);
    return rc != LBM_OK ? rc : init_parts(v, params, dev_workspace, bytes, dev_u0, stream, out);
}

int lbm_batch_parts(const lbm_solver *s, int32_t *n_parts)
{
    if (!s || !n_parts) return LBM_EINVAL;
    *n_parts = (int32_t)s->parts.size();
    return LBM_OK;
}

int lbm_batch_part_info(const lbm_solver *s, int32_t part, lbm_geometry_info *info, int64_t *fluid_offset,
                        int64_t *cell_offset, int64_t *plane_offset)
{
    if (!s || part < 0 || part >= (int32_t)s->parts.size()) return LBM_EINVAL;
    const Part &P = s->parts[part];
    if (info) {
        info->n_cells = P.n_cells;
        info->n_fluid = P.n_fluid;
        info->n_links = P.n_links;
        info->n_spheres = P.n_spheres;
        info->porosity = (double)P.n_fluid / (double)P.n_cells;
    }
    if (fluid_offset) *fluid_offset = P.fluid_off;
    if (cell_offset) *cell_offset = P.cell_base;
    if (plane_offset) *plane_offset = P.plane_base;
    return LBM_OK;
}

// Synchronise the solver's stream and read the step kernels' status word:
// LBM_ETIMEOUT (and the word cleared) if a bounded device-side wait gave up
// since the last check.  The state is then marked stale: a block that gave
// up returned without finishing its tile, so lbm_step refuses to continue
// until lbm_reset.
static int sync_checked(lbm_solver *s)
{
    int st = 0;
    if (cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (st) {
        s->stale = true;
        if (cudaMemsetAsync(s->status, 0, sizeof(int), s->stream) != cudaSuccess) return LBM_ECUDA;
        return LBM_ETIMEOUT;
    }
    return LBM_OK;
}

int lbm_batch_permeability(lbm_solver *s, double *k_out)
{
    if (!s || !k_out || s->params.g[0] == 0.0) return LBM_EINVAL;
    for (int b = 0; b < (int)s->parts.size(); ++b) {
        const int rc = launch_permeability(*s, b, 0, s->parts[b].box.nz - 1);
        if (rc != LBM_OK) return rc;
    }
    std::vector<double> r(8 * s->parts.size());
    if (cudaMemcpyAsync(r.data(), s->result + res_part(s->lay, 0), r.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (int rc = sync_checked(s)) return rc;
    for (size_t b = 0; b < s->parts.size(); ++b) k_out[b] = r[8 * b];
    return LBM_OK;
}

int lbm_reset(lbm_solver *s, const float *dev_u0)
{
    if (!s) return LBM_EINVAL;
    s->stale = false;
    s->has_prev = false;
    for (Part &P : s->parts) P.has_prev_profile = false;
    return launch_init(*s, dev_u0);
}

int lbm_step(lbm_solver *s, int64_t n)
{
    if (!s || n < 0) return LBM_EINVAL;
    if (s->stale) return LBM_ETIMEOUT;
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
    if (cudaMemcpyAsync(host_out, s->result, sizeof(double) * 3 * (size_t)s->lay.n_planes, cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
        return LBM_ECUDA;
    return sync_checked(s);
}

int lbm_permeability(lbm_solver *s, int32_t z_lo, int32_t z_hi, double *k_out)
{
    if (!s || !k_out || s->parts.size() != 1) return LBM_EINVAL;
    if (z_lo == -1 && z_hi == -1) {
        z_lo = 0;
        z_hi = s->box.nz - 1;
    }
    if (z_lo < 0 || z_hi >= s->box.nz || z_lo > z_hi || s->params.g[0] == 0.0) return LBM_EINVAL;
    int rc = launch_permeability(*s, 0, z_lo, z_hi);
    if (rc != LBM_OK) return rc;
    if (cudaMemcpyAsync(k_out, s->result + res_part(s->lay, 0), sizeof(double), cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    return sync_checked(s);
}

int lbm_residual(lbm_solver *s, double *res_out)
{
    if (!s || !res_out) return LBM_EINVAL;
    int rc = launch_residual(*s);
    if (rc != LBM_OK) return rc;
    double r[3];
    if (cudaMemcpyAsync(r, s->result + res_field(s->lay), sizeof(r), cudaMemcpyDeviceToHost, s->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    if (int rc2 = sync_checked(s)) return rc2;
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

// Per-part profile residuals (host array of n_parts); the largest is returned.
static int profile_residuals(lbm_solver *s, double *per_part, double *worst)
{
    int rc = launch_profile_residual(*s);
    if (rc != LBM_OK) return rc;
    std::vector<double> r(8 * s->parts.size());
    if (cudaMemcpyAsync(r.data(), s->result + res_part(s->lay, 0), r.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (int rc2 = sync_checked(s)) return rc2;
    double w = 0.0;
    bool bad = false;
    for (size_t b = 0; b < s->parts.size(); ++b) {
        Part &P = s->parts[b];
        const double num = r[8 * b + 1], den = r[8 * b + 2];
        bad |= r[8 * b + 3] != 0.0 || !std::isfinite(num) || !std::isfinite(den);
        double v = std::numeric_limits<double>::infinity();
        if (P.has_prev_profile) v = den > 0.0 ? std::sqrt(num) / std::sqrt(den) : (num > 0.0 ? v : 0.0);
        P.has_prev_profile = true;
        if (per_part) per_part[b] = v;
        w = std::max(w, v);
    }
    if (bad) {
        *worst = std::numeric_limits<double>::quiet_NaN();
        return LBM_ENAN;
    }
    *worst = w;
    return LBM_OK;
}

int lbm_profile_residual(lbm_solver *s, double *res_out)
{
    if (!s || !res_out) return LBM_EINVAL;
    return profile_residuals(s, nullptr, res_out);
}

int lbm_batch_profile_residual(lbm_solver *s, double *res_out)
{
    if (!s || !res_out) return LBM_EINVAL;
    double worst;
    return profile_residuals(s, res_out, &worst);
}

// Mean density deviation per part (host array) and over the whole solver.
static int part_masses(lbm_solver *s, std::vector<double> &per_part, double *mean_all)
{
    per_part.assign(s->parts.size(), 0.0);
    *mean_all = 0.0;
    if (s->n_fluid == 0) return LBM_OK;
    int rc = launch_mass(*s);
    if (rc != LBM_OK) return rc;
    std::vector<double> r(8 * s->parts.size());
    double g[2];
    if (cudaMemcpyAsync(r.data(), s->result + res_part(s->lay, 0), r.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess ||
        cudaMemcpyAsync(g, s->result + res_mass(s->lay), sizeof(g), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (int rc2 = sync_checked(s)) return rc2;
    bool bad = g[1] != 0.0 || !std::isfinite(g[0]);
    for (size_t b = 0; b < s->parts.size(); ++b) {
        bad |= r[8 * b + 5] != 0.0 || !std::isfinite(r[8 * b + 4]);
        per_part[b] = s->parts[b].n_fluid ? r[8 * b + 4] / (double)s->parts[b].n_fluid : 0.0;
    }
    if (bad) return LBM_ENAN;
    *mean_all = g[0] / (double)s->n_fluid;
    return LBM_OK;
}

int lbm_mass(lbm_solver *s, double *mean_drho)
{
    if (!s || !mean_drho) return LBM_EINVAL;
    std::vector<double> per;
    return part_masses(s, per, mean_drho);
}

int lbm_recenter(lbm_solver *s, double *shift_out)
{
    if (!s) return LBM_EINVAL;
    std::vector<double> per;
    double all = 0.0;
    int rc = part_masses(s, per, &all);
    if (rc != LBM_OK) return rc;
    // the state is measured afresh: replace any pending shift, do not accumulate
    for (size_t b = 0; b < per.size(); ++b) s->shift_host[b] = (float)per[b];
    if (cudaMemcpyAsync(s->part_shift, s->shift_host.data(), sizeof(float) * per.size(), cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return LBM_ECUDA;
    s->shift_pending = true;
    // new reference populations from the same velocity field (part_masses
    // ran the moments kernel); the next step switches to them
    rc = launch_reference_update(*s);
    if (rc != LBM_OK) return rc;
    if (shift_out) *shift_out = all;
    return LBM_OK;
}

int lbm_run_until(lbm_solver *s, double tol, int64_t interval, int64_t max_steps, int32_t criterion,
                  int64_t *steps_done, double *res_out)
{
    if (!s || interval < 1 || max_steps < 0 || !(tol > 0.0)) return LBM_EINVAL;
    if (criterion != LBM_CONVERGE_FIELD && criterion != LBM_CONVERGE_PROFILE) return LBM_EINVAL;
    if (s->stale) return LBM_ETIMEOUT;
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

int lbm_reference_planes(const lbm_solver *s, int32_t *n_planes)
{
    if (!s || !n_planes) return LBM_EINVAL;
    int32_t n = 0;
    for (uint8_t f : s->plane_referenced) n += f ? 1 : 0;
    *n_planes = n;
    return LBM_OK;
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
        // links in (cell, k) order from the link masks; a link falls back to
        // bounce-back when x - e_k is solid, and with the corner safeguards
        // also when x - 2 e_k is solid or q < kCliQmin
        std::vector<uint32_t> mask(nf ? nf : 1);
        std::vector<double> qs;
        std::vector<int32_t> nb;
        if (link_fallback) {
            qs.resize(s->n_links ? (size_t)s->n_links : 1);
            nb.resize((size_t)(kQ - 1) * (nf ? nf : 1));
        }
        if (nf && cudaMemcpyAsync(mask.data(), s->lmask, nf * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return LBM_ECUDA;
        if (link_fallback && s->n_links &&
            cudaMemcpyAsync(qs.data(), s->link_q, (size_t)s->n_links * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return LBM_ECUDA;
        if (link_fallback && nf &&
            cudaMemcpy2DAsync(nb.data(), nf * 4, s->nbr, (size_t)s->n_pad * 4, nf * 4, kQ - 1, cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
            return LBM_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ECUDA;
        size_t l = 0;
        for (size_t i = 0; i < nf; ++i)
            for (int k = 1; k < kQ; ++k)
                if ((mask[i] >> k) & 1u) {
                    if (link_cell) link_cell[l] = (int32_t)i;
                    if (link_k) link_k[l] = (int8_t)k;
                    if (link_fallback) {
                        const bool guard = (s->params.flags & LBM_FLAG_CLI_SAFEGUARDS) != 0;
                        bool fb = (s->params.flags & LBM_FLAG_SIMPLE_BOUNCE_BACK) || ((mask[i] >> opp(k)) & 1u) ||
                                  (guard && qs[l] < kCliQmin);
                        if (!fb && guard) fb = (mask[nb[(size_t)(opp(k) - 1) * nf + i]] >> opp(k)) & 1u;
                        link_fallback[l] = (uint8_t)fb;
                    }
                    ++l;
                }
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_wait_selftest(lbm_solver *s, int32_t max_polls)
{
    if (!s || max_polls < 1) return LBM_EINVAL;
    const int rc = launch_wait_selftest(*s, max_polls);
    if (rc != LBM_OK) return rc;
    return sync_checked(s);
}

int lbm_populations(lbm_solver *s, float *dev_out)
{
    if (!s) return LBM_EINVAL;
    if (s->n_fluid == 0) return LBM_OK;   // nothing to write
    if (!dev_out) return LBM_EINVAL;
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
