// lbm_checkpoint.cpp -- checkpoint and resume of a solver's state.
//
// A checkpoint holds what the next steps and the convergence checks depend
// on: the stored populations at the current parity (storage type, fluid
// cells only), the step count, the pending density shift, the reference
// populations (current, and the next ones when a switch is pending) and the
// residual histories.  The lists (fluid cells, neighbours, links) are not in
// it: they follow from the geometry, which the caller rebuilds (from the same
// seed or sphere list) to create the solver that loads the checkpoint.  The
// step kernels give the same bits for every launch schedule, so a resumed run
// is bit-identical to the uninterrupted one.
//
// Layout (host byte order): a fixed header, then the arrays in the order of
// the header's fields, each padded to 8 bytes.
#include <cstring>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;
// flags that change the wall links or the arithmetic (the others only pick
// kernels or schedules, which give the same bits)
constexpr int32_t kStateFlags = LBM_FLAG_SIMPLE_BOUNCE_BACK | LBM_FLAG_CLI_SAFEGUARDS | LBM_FLAG_PLANE_REFERENCES;

struct Header {
    char magic[8];
    uint32_t version;
    int32_t storage;
    int32_t flags;
    int32_t n_parts;
    int64_t n_cells, n_fluid, n_links, n_planes;
    double tau, lambda, g[3];
    int64_t steps;
    int32_t shift_pending, ref_pending, has_prev, pad;
};

size_t pad8(size_t v) { return (v + 7) / 8 * 8; }

struct Sizes {
    size_t pdf, shift, prof_flags, ref, prof, uprev, total;
};

Sizes sizes_of(const Solver &s)
{
    Sizes z{};
    z.pdf = pad8((size_t)kQ * (size_t)s.n_fluid * (size_t)storage_bytes(s.params.storage));
    z.shift = pad8(sizeof(float) * s.parts.size());
    z.prof_flags = pad8(s.parts.size());
    z.ref = pad8(sizeof(float) * kRefStride * (size_t)s.lay.n_planes);
    z.prof = pad8(sizeof(double) * (size_t)s.lay.n_planes);
    z.uprev = pad8(sizeof(float) * 3 * (size_t)s.n_fluid);
    // ref twice: current and next
    z.total = sizeof(Header) + z.pdf + z.shift + z.prof_flags + 2 * z.ref + z.prof + z.uprev;
    return z;
}

Header header_of(const Solver &s)
{
    Header h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.storage = s.params.storage;
    h.flags = (s.params.flags & kStateFlags & ~LBM_FLAG_PLANE_REFERENCES) |
              (plane_references_on(s.params) ? LBM_FLAG_PLANE_REFERENCES : 0);
    h.n_parts = (int32_t)s.parts.size();
    h.n_cells = s.n_cells;
    h.n_fluid = s.n_fluid;
    h.n_links = s.n_links;
    h.n_planes = s.lay.n_planes;
    h.tau = s.params.tau;
    h.lambda = s.params.lambda;
    for (int d = 0; d < 3; ++d) h.g[d] = s.params.g[d];
    h.steps = s.steps;
    h.shift_pending = s.shift_pending ? 1 : 0;
    h.ref_pending = s.ref_pending ? 1 : 0;
    h.has_prev = s.has_prev ? 1 : 0;
    return h;
}

bool same_problem(const Header &a, const Header &b)
{
    return std::memcmp(a.magic, b.magic, 8) == 0 && a.version == b.version && a.storage == b.storage &&
           a.flags == b.flags && a.n_parts == b.n_parts && a.n_cells == b.n_cells && a.n_fluid == b.n_fluid &&
           a.n_links == b.n_links && a.n_planes == b.n_planes && a.tau == b.tau && a.lambda == b.lambda &&
           a.g[0] == b.g[0] && a.g[1] == b.g[1] && a.g[2] == b.g[2];
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_checkpoint_size(const lbm_solver *s, size_t *bytes)
{
    if (!s || !bytes) return LBM_EINVAL;
    *bytes = sizes_of(*s).total;
    return LBM_OK;
}

int lbm_save(lbm_solver *s, void *host_buf, size_t bytes)
{
    if (!s || !host_buf) return LBM_EINVAL;
    if (s->stale) return LBM_ETIMEOUT;
    const Sizes z = sizes_of(*s);
    if (bytes < z.total) return LBM_ESIZE;
    char *out = (char *)host_buf;
    std::memset(out, 0, z.total);
    const Header h = header_of(*s);
    std::memcpy(out, &h, sizeof(h));
    char *p = out + sizeof(Header);
    cudaStream_t st = s->stream;
    const size_t sb = (size_t)storage_bytes(s->params.storage);
    const size_t nf = (size_t)s->n_fluid;
    // populations: 19 rows of n_fluid values out of the [19][n_pad] array
    if (nf && cudaMemcpy2DAsync(p, nf * sb, s->pdf, (size_t)s->n_pad * sb, nf * sb, kQ, cudaMemcpyDeviceToHost, st) !=
                  cudaSuccess)
        return LBM_ECUDA;
    p += z.pdf;
    std::memcpy(p, s->shift_host.data(), sizeof(float) * s->parts.size());
    p += z.shift;
    for (size_t b = 0; b < s->parts.size(); ++b) p[b] = s->parts[b].has_prev_profile ? 1 : 0;
    p += z.prof_flags;
    const size_t ref_bytes = sizeof(float) * kRefStride * (size_t)s->lay.n_planes;
    if (cudaMemcpyAsync(p, s->ref, ref_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBM_ECUDA;
    p += z.ref;
    if (cudaMemcpyAsync(p, s->ref_next, ref_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBM_ECUDA;
    p += z.ref;
    if (cudaMemcpyAsync(p, s->prof_prev, sizeof(double) * (size_t)s->lay.n_planes, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return LBM_ECUDA;
    p += z.prof;
    if (nf && cudaMemcpy2DAsync(p, nf * 4, s->u_prev, (size_t)s->n_pad * 4, nf * 4, 3, cudaMemcpyDeviceToHost, st) !=
                  cudaSuccess)
        return LBM_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

int lbm_load(lbm_solver *s, const void *host_buf, size_t bytes)
{
    if (!s || !host_buf) return LBM_EINVAL;
    const Sizes z = sizes_of(*s);
    if (bytes < sizeof(Header)) return LBM_ESIZE;
    Header h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (!same_problem(h, header_of(*s))) return LBM_EINVAL;
    if (bytes < z.total) return LBM_ESIZE;
    const char *p = (const char *)host_buf + sizeof(Header);
    cudaStream_t st = s->stream;
    const size_t sb = (size_t)storage_bytes(s->params.storage);
    const size_t nf = (size_t)s->n_fluid;
    if (nf && cudaMemcpy2DAsync(s->pdf, (size_t)s->n_pad * sb, p, nf * sb, nf * sb, kQ, cudaMemcpyHostToDevice, st) !=
                  cudaSuccess)
        return LBM_ECUDA;
    p += z.pdf;
    std::vector<float> shift(s->parts.size());
    std::memcpy(shift.data(), p, sizeof(float) * shift.size());
    p += z.shift;
    std::vector<uint8_t> pflags(p, p + s->parts.size());
    p += z.prof_flags;
    const size_t ref_bytes = sizeof(float) * kRefStride * (size_t)s->lay.n_planes;
    if (cudaMemcpyAsync(s->ref, p, ref_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return LBM_ECUDA;
    p += z.ref;
    if (cudaMemcpyAsync(s->ref_next, p, ref_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return LBM_ECUDA;
    p += z.ref;
    if (cudaMemcpyAsync(s->prof_prev, p, sizeof(double) * (size_t)s->lay.n_planes, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return LBM_ECUDA;
    p += z.prof;
    if (nf && cudaMemcpy2DAsync(s->u_prev, (size_t)s->n_pad * 4, p, nf * 4, nf * 4, 3, cudaMemcpyHostToDevice, st) !=
                  cudaSuccess)
        return LBM_ECUDA;
    if (cudaMemcpyAsync(s->part_shift, shift.data(), sizeof(float) * shift.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LBM_ECUDA;
    s->shift_host = shift;
    for (size_t b = 0; b < s->parts.size(); ++b) s->parts[b].has_prev_profile = pflags[b] != 0;
    s->steps = h.steps;
    s->shift_pending = h.shift_pending != 0;
    s->ref_pending = h.ref_pending != 0;
    s->has_prev = h.has_prev != 0;
    s->stale = false;
    return LBM_OK;
}

}  // extern "C"
