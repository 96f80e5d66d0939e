// lbm_step.cu -- the fused stream-collide + CLI update over the sparse fluid
// list (in-place AA pattern, see lbm_kernels.cuh) and the initialisation.
//
// One thread per fluid cell, 256 threads per block.  The even step touches only
// the cell's own 19 slots (contiguous structure-of-arrays rows, fully
// coalesced); the odd step gathers through the neighbour table and scatters
// back to the same slots.  Wall links cost one coefficient load each.
#include "lbm_kernels.cuh"

namespace lbm {
namespace {

// Resident blocks per SM requested from the register allocator (256 threads
// each).  Measured on GB300 over the 256x256x512 channel sweep: the even step
// reaches 91% of the copy bandwidth at 5 blocks (48 registers, no spills); the
// odd step is best at 4 (64 registers); more blocks make the odd step spill.
constexpr int kEvenBlocksPerSM = 5;
constexpr int kOddBlocksPerSM = 4;

template <typename T>
struct StepArgs {
    T *pdf;
    const int32_t *nbr;
    const uint32_t *lmask;
    const uint32_t *warp_off;
    const float *link_a;
    int32_t n_fluid;
    int32_t n_pad;
    RowGeo rows;
    Coef c;
};

// Per-thread staging in shared memory: the CLI coefficients (and, for the odd
// step, the neighbour indices) of a thread are written and read by that thread
// only, so no barrier is needed.  Keeping them out of registers across the
// collision lowers register pressure and raises the number of resident warps,
// which is what hides the memory latency of these kernels.
template <typename T, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_step_even(StepArgs<T> p)
{
    __shared__ float a_s[kQ - 1][kBlock];
    const int t = threadIdx.x;
    const int32_t i = blockIdx.x * kBlock + t;
    const bool live = i < p.n_fluid;
    const uint32_t m = live ? p.lmask[i] : 0u;
    const uint32_t off = first_link(p.warp_off, i, m);
    if (!live) return;
    const size_t n_pad = (size_t)p.n_pad;
    float h[kQ];
    gather_even(h, p.pdf, n_pad, i);
    if (m) {
        stage_links(a_s, t, m, p.link_a, off);
        cli_incoming_s(h, a_s, t);
    }
    apply_shift(h, p.c.shift);
    collide(h, p.c);
    if (m) cli_outgoing_s(h, a_s, t);
#pragma unroll
    for (int k = 0; k < kQ; ++k) st(p.pdf + opp(k) * n_pad + i, h[k]);
}

// ROWS: neighbour indices from the row bitmasks; otherwise from the table.
template <typename T, bool ROWS, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_step_odd(StepArgs<T> p)
{
    __shared__ int32_t nb_s[kQ - 1][kBlock];
    __shared__ float a_s[kQ - 1][kBlock];
    const int t = threadIdx.x;
    const int32_t i = blockIdx.x * kBlock + t;
    const bool live = i < p.n_fluid;
    // 32-bit element offsets (19 n_pad < 2^32 is checked on the host)
    const uint32_t n_pad = (uint32_t)p.n_pad, ui = (uint32_t)i;
    uint32_t m = 0;
    if (live) {
        int32_t nb[kQ];
        m = ROWS ? row_neighbours(nb, p.rows, i) : load_nbr(nb, p.nbr, (size_t)n_pad, i);
#pragma unroll
        for (int k = 1; k < kQ; ++k) nb_s[k - 1][t] = nb[k];
    }
    const uint32_t off = first_link(p.warp_off, i, m);
    if (!live) return;
    if (m) stage_links(a_s, t, m, p.link_a, off);
    float h[kQ];
    h[0] = ld(p.pdf + ui);
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        const int32_t up = nb_s[opp(k) - 1][t];   // x - e_k = x + e_opp(k)
        h[k] = ld(p.pdf + (up >= 0 ? opp(k) * n_pad + (uint32_t)up : k * n_pad + ui));
    }
    if (m) cli_incoming_s(h, a_s, t);
    apply_shift(h, p.c.shift);
    collide(h, p.c);
    if (m) cli_outgoing_s(h, a_s, t);
    st(p.pdf + ui, h[0]);
#pragma unroll
    for (int k = 1; k < kQ; ++k) {
        const int32_t down = nb_s[k - 1][t];
        st(p.pdf + (down >= 0 ? k * n_pad + (uint32_t)down : opp(k) * n_pad + ui), h[k]);
    }
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
    const uint32_t m = live ? p.lmask[i] : 0u;
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
StepArgs<T> make_args(Solver &s)
{
    StepArgs<T> p;
    p.pdf = (T *)s.pdf;
    p.nbr = s.nbr;
    p.lmask = s.lmask;
    p.warp_off = s.warp_off;
    p.link_a = s.link_a;
    p.n_fluid = s.n_fluid;
    p.n_pad = s.n_pad;
    p.rows = RowGeo{s.row_words, s.cell_xr, s.box.nx, s.box.ny, s.box.nz, s.n_words, s.x_bits, s.box.periodic_z};
    p.c.omega_p = (float)s.omega_p;
    p.c.omega_m = (float)s.omega_m;
    for (int k = 0; k < kQ; ++k) {
        const double eg = ex(k) * s.params.g[0] + ey(k) * s.params.g[1] + ez(k) * s.params.g[2];
        p.c.force[k] = (float)(3.0 * weight(k) * eg);
    }
    for (int d = 0; d < 3; ++d) p.c.half_g[d] = (float)(0.5 * s.params.g[d]);
    p.c.shift = 0.0f;
    return p;
}

template <typename T>
int run_steps(Solver &s, int64_t n)
{
    if (s.n_fluid == 0) {
        s.steps += n;
        return LBM_OK;
    }
    StepArgs<T> p = make_args<T>(s);
    const unsigned grid = (unsigned)(s.n_pad / kBlock);
    for (int64_t t = 0; t < n; ++t) {
        p.c.shift = t == 0 ? (float)s.drho_shift : 0.0f;
        if ((s.steps & 1) == 0) k_step_even<T, kEvenBlocksPerSM><<<grid, kBlock, 0, s.stream>>>(p);
        else if (s.odd_rows) k_step_odd<T, true, kOddBlocksPerSM><<<grid, kBlock, 0, s.stream>>>(p);
        else k_step_odd<T, false, kOddBlocksPerSM><<<grid, kBlock, 0, s.stream>>>(p);
        ++s.steps;
    }
    if (n > 0) s.drho_shift = 0.0;
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

template <typename T>
int run_init(Solver &s, const float *u0)
{
    s.steps = 0;
    s.drho_shift = 0.0;
    if (s.n_fluid == 0) return LBM_OK;
    const StepArgs<T> p = make_args<T>(s);
    k_init<T><<<(unsigned)(s.n_pad / kBlock), kBlock, 0, s.stream>>>(p, s.fluid_cell, u0, s.n_cells);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // namespace

Coef make_coef(const Solver &s)
{
    return make_args<float>(const_cast<Solver &>(s)).c;
}

int launch_init(Solver &s, const float *dev_u0)
{
    switch (s.params.storage) {
    case LBM_F32: return run_init<float>(s, dev_u0);
    case LBM_F16: return run_init<__half>(s, dev_u0);
    case LBM_BF16: return run_init<__nv_bfloat16>(s, dev_u0);
    }
    return LBM_EINVAL;
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

}  // namespace lbm
