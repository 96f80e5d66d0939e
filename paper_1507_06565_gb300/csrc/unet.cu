// unet.cu -- a 3-D convolutional U-Net that maps the signed-distance field of
// a geometry to its steady velocity field, used to warm-start the LBM
// (Eq. (equilibrium) evaluated at the predicted u0).  The paper has no learned
// component; the converged LBM stays the arbiter of the prediction's error.
//
// Architecture (fixed): 4 levels of two 3x3x3 convolutions + ReLU with
// 16/32/64/128 channels, 2x2x2 average pooling, nearest x2 upsampling with the
// upsampled tensor and the skip tensor concatenated (in that order), and a
// 1x1x1 head to the 3 velocity components.  Convolutions pad circularly in x
// and y (the periodic directions) and with zeros in z (the walls).  Input
// channels: [sdf, z feature in [-1,1], 14 zeros].
//
// Numerics: activations, activation gradients and the working copies of the
// weights are bf16 (layout [voxel][channel]); every contraction accumulates in
// fp32 on the tensor cores; master weights, weight gradients and the Adam
// moments are fp32.  The 3x3x3 convolution is an implicit GEMM (M = voxels,
// N = output channels, K = 27 taps x input channels) on tcgen05 with a TMEM
// accumulator; its backward with respect to the input is the same kernel with
// the weights flipped in the taps and transposed in the channels (the adjoint
// of a circular/zero-padded convolution).  The weight gradient contracts over
// voxels on tcgen05 as well, one tap and voxel chunk per CTA, and adds the
// partial sums atomically.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.h"

namespace unet {

using bf16 = __nv_bfloat16;

constexpr int kTaps = 27;
constexpr int kIn = 16;       // input channels after padding
constexpr int kOut = 3;       // velocity components
constexpr int kW[4] = {16, 32, 64, 128};   // host-side channel widths
constexpr int kW0 = 16;                      // first level (used in device code)

struct Dims {
    int n, d, h, w;
    __host__ __device__ int64_t voxels() const { return (int64_t)n * d * h * w; }
};

// Voxel v shifted by tap t (dz, dy, dx = t/9-1, t/3%3-1, t%3-1): circular in
// y and x, -1 when z leaves the box.
__device__ __forceinline__ int64_t tap_neighbour(const Dims &g, int64_t v, int t)
{
    const int x = (int)(v % g.w);
    int64_t r = v / g.w;
    const int y = (int)(r % g.h);
    r /= g.h;
    const int z = (int)(r % g.d);
    const int64_t n = r / g.d;
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int zz = z + dz;
    if (zz < 0 || zz >= g.d) return -1;
    int yy = y + dy, xx = x + dx;
    yy = yy < 0 ? yy + g.h : (yy >= g.h ? yy - g.h : yy);
    xx = xx < 0 ? xx + g.w : (xx >= g.w ? xx - g.w : xx);
    return ((n * g.d + zz) * g.h + yy) * g.w + xx;
}

// ---------------------------------------------------------------------------
// 3x3x3 convolution as implicit GEMM (forward, and backward w.r.t. the input)
// ---------------------------------------------------------------------------
struct ConvArgs {
    const bf16 *in0;
    int ci0;            // channels of in0 (multiple of 16)
    const bf16 *in1;
    int ci1;            // channels of in1 (0: none); the input is [in0, in1]
    const bf16 *w;      // [27][co][ci]
    const float *bias;  // [co] or null
    bf16 *out0;
    int co0;            // output channels [0, co0) -> out0 (row length co0)
    bf16 *out1;
    int co1;            // [co0, co0 + co1) -> out1 (row length co1)
    int relu;
    Dims g;
};

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) contractions of the U-Net: the 3x3x3 convolution
// (forward and input gradient) and its weight gradient.  Both accumulate in
// TMEM (M = 128 lanes x N fp32 columns) from bf16 operands in shared memory,
// without swizzle, in 8x8 core matrices of 16-byte rows; a descriptor's
// leading offset is the stride between core matrices along K and its stride
// offset the stride between 8-row (8-element) groups along M or N, as a
// self-checking probe of single MMAs (K-major and MN-major, M = 128)
// confirmed.
//
// Pipelines (128 threads, 2-4 shared-memory stages).  Barrier-free (weight
// gradient): every thread gathers its share of step it with cp.async into
// stage it % stages; when its copies of step j = it - (stages - 1) have
// landed it fences them to the async proxy and arrives on full[j % stages]
// (128 arrivals complete a phase).  Thread 0 waits on full, issues the step's
// MMAs and commits them to empty[j % stages]; a thread refills a stage only
// after waiting on its empty barrier.  Two-stage with CTA barriers
// (convolution): see pipeline_sync.  Every wait is bounded; one that runs out
// sets *status (reported by unet_backward as LBM_ETIMEOUT) and the CTA still
// frees its TMEM.
// ---------------------------------------------------------------------------
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (sm_100 family): start, leading offset,
// stride offset, all >> 4; version bit 46; base offset 0; no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, N/8 at
// bit 17, M/16 at bit 24; mn_major sets both operands MN-major (bits 15, 16)
__device__ __forceinline__ uint32_t idesc(int m, int n, bool mn_major)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (mn_major ? (3u << 15) : 0u) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void wait_groups(int n)
{
    if (n >= 3) asm volatile("cp.async.wait_group 3;\n" ::: "memory");
    else if (n == 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, bool acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                     tmem),
                 "l"(ad), "l"(bd), "r"(id), "r"(acc ? 1u : 0u));
}

__device__ __forceinline__ void commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// bounded wait: false (and *status set) if the phase did not complete
__device__ __forceinline__ bool wait(uint64_t *mbar, uint32_t parity, int *status)
{
    const uint32_t a = smem_u32(mbar);
    for (int it = 0; it < (1 << 24); ++it)
        if (try_wait(a, parity)) return true;
    atomicExch(status, 1);
    return false;
}

__device__ __forceinline__ void arrive(uint64_t *mbar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(mbar)) : "memory");
}

constexpr int kMaxStages = 4;

// Shared set-up: TMEM columns and the full/empty barriers.
struct Ctx {
    uint64_t *full, *empty;
    uint32_t tmem;
};

__device__ __forceinline__ void setup(uint32_t *tmem_slot, uint64_t *full, uint64_t *empty, int stages, int ncols)
{
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < stages; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full[q])), "r"(128));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[q])));
        }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// The producer/consumer loop.  fill(it, s) issues this thread's cp.async
// copies of step it into stage s (no commit); issue(j, s) issues step j's MMAs
// (thread 0 only).  Returns true (on every thread) when all MMAs completed.
template <class Fill, class Issue>
__device__ __forceinline__ bool pipeline(int iters, int stages, uint64_t *full, uint64_t *empty, int *status,
                                         Fill fill, Issue issue)
{
    const int lag = stages - 1;
    bool ok = true;
    for (int it = 0; it < iters + lag && ok; ++it) {
        if (it < iters) {
            const int s = it % stages;
            // the MMAs of step it - stages read this stage; they were issued
            // at step it - 1 of thread 0
            if (it >= stages) ok = wait(&empty[s], (uint32_t)((it / stages - 1) & 1), status);
            if (!ok) break;
            fill(it, s);
        }
        commit_group();   // one group per step (empty while draining)
        if (it >= lag) {
            const int j = it - lag, s = j % stages;
            wait_groups(lag);   // this thread's copies of step j have landed
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            arrive(&full[s]);
            if (threadIdx.x == 0) {
                ok = wait(&full[s], (uint32_t)((j / stages) & 1), status);
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    issue(j, s);
                    commit(&empty[s]);
                }
            }
        }
    }
    wait_groups(0);
    int w = ok ? 1 : 0;
    if (threadIdx.x == 0 && ok) {
        // the last commit tracks every MMA issued before it
        const int l = iters - 1;
        w = wait(&empty[l % stages], (uint32_t)((l / stages) & 1), status) ? 1 : 0;
    }
    ok = __syncthreads_and(w) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return ok;
}

// Two-stage variant with CTA barriers: the whole CTA gathers step it, waits
// for its copies of step it - 1, and thread 0 issues that step after a
// barrier.  Used by the convolution, where it measured faster than the
// barrier-free loop (its steps are short and its producer shares uniform).
template <class Fill, class Issue>
__device__ __forceinline__ bool pipeline_sync(int iters, uint64_t *empty, int *status, Fill fill, Issue issue)
{
    bool ok = true;
    for (int it = 0; it < iters; ++it) {
        const int s = it & 1;
        if (it >= 2) {
            // thread 0 waits for the MMAs that last read stage s; the barrier
            // hands its verdict to the whole CTA
            int w = 1;
            if (threadIdx.x == 0) w = wait(&empty[s], (uint32_t)(((it - 2) >> 1) & 1), status) ? 1 : 0;
            ok = __syncthreads_and(w) != 0;
            if (!ok) break;
        }
        fill(it, s);
        commit_group();
        if (it >= 1) {
            wait_groups(1);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                issue(it - 1, (it - 1) & 1);
                commit(&empty[(it - 1) & 1]);
            }
        }
    }
    wait_groups(0);
    int w = ok ? 1 : 0;
    if (ok) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            const int l = iters - 1;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            issue(l, l & 1);
            commit(&empty[l & 1]);
            // the last commit tracks every MMA issued before it
            w = wait(&empty[l & 1], (uint32_t)((l >> 1) & 1), status) ? 1 : 0;
        }
    } else {
        __syncthreads();
    }
    ok = __syncthreads_and(w) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return ok;
}

__device__ __forceinline__ void teardown(uint32_t tmem, int ncols)
{
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

// 16 fp32 accumulator columns c0..c0+15 of lane 32w + (thread's lane)
__device__ __forceinline__ void load16(uint32_t tmem, int warp, int c0, uint32_t r[16])
{
    const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// voxel v -> (n, z, y, x) and the tap-t neighbour (-1 outside z); 32-bit
// arithmetic (the host keeps voxel counts below 2^31)
__device__ __forceinline__ int32_t tap_nb(const Dims &g, int32_t v, int dz, int dy, int dx)
{
    const int x = v % g.w;
    int32_t r = v / g.w;
    const int y = r % g.h;
    r /= g.h;
    const int z = r % g.d;
    const int32_t n = r / g.d;
    const int zz = z + dz;
    if (zz < 0 || zz >= g.d) return -1;
    int yy = y + dy, xx = x + dx;
    yy = yy < 0 ? yy + g.h : (yy >= g.h ? yy - g.h : yy);
    xx = xx < 0 ? xx + g.w : (xx >= g.w ? xx - g.w : xx);
    return ((n * g.d + zz) * g.h + yy) * g.w + xx;
}

// Position of voxel v, decomposed once, for the tap neighbours of one voxel.
struct VoxPos {
    int32_t v;
    int x, y, z;
};

__device__ __forceinline__ VoxPos vox_pos(const Dims &g, int32_t v)
{
    VoxPos p;
    p.v = v;
    p.x = v % g.w;
    const int32_t r = v / g.w;
    p.y = r % g.h;
    p.z = (r / g.h) % g.d;
    return p;
}

// tap_nb from a decomposed position: offsets and wrap corrections only
__device__ __forceinline__ int32_t tap_nb(const Dims &g, const VoxPos &p, int dz, int dy, int dx)
{
    const int zz = p.z + dz;
    if (zz < 0 || zz >= g.d) return -1;
    const int32_t plane = g.h * g.w;
    int32_t off = dz * plane + dy * g.w + dx;
    const int yy = p.y + dy, xx = p.x + dx;
    off += yy < 0 ? plane : (yy >= g.h ? -plane : 0);
    off += xx < 0 ? g.w : (xx >= g.w ? -g.w : 0);
    return p.v + off;
}

}  // namespace tc

constexpr int kTcM = 128;

// ---------------------------------------------------------------------------
// Convolution: one CTA computes 128 voxels x all N = co output channels.  K
// runs over the 27 taps and chunks of KC input channels (the largest of 64,
// 32, 16 dividing ci); a step gathers 1 or 3 taps: A = 128 voxels x KC channels
// of the tap's neighbours (circular in x, y; zero in z and past the end), B =
// N x KC weights, both K-major (core (row/8, k/8) at (row/8)*SBO + (k/8)*128,
// SBO = KC/8 * 128).  Thread t gathers row t of A and a share of B.  The
// epilogue reads TMEM with tcgen05.ld (warp w owns voxels 32w..32w+31), adds
// the bias, applies ReLU and stores bf16.  The input gradient is the same
// kernel with the weights flipped in the taps and transposed in the channels.
// Its steps run through the two-stage pipeline with CTA barriers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_conv3_tc(ConvArgs a, int kc, int tp, int ncols, int stages, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[tc::kMaxStages], empty[tc::kMaxStages];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ci = a.ci0 + a.ci1, n = a.co0 + a.co1;
    const int32_t V = (int32_t)a.g.voxels();
    const int32_t m0 = (int32_t)blockIdx.x * kTcM;
    // a step gathers tp taps: tp A sub-tiles, then tp B sub-tiles
    const uint32_t a_bytes = (uint32_t)kTcM * kc * 2, b_bytes = (uint32_t)n * kc * 2;
    const uint32_t stage_bytes = (uint32_t)tp * (a_bytes + b_bytes), sbo = (uint32_t)(kc / 8) * 128u;
    const uint32_t base = tc::smem_u32(smem);
    tc::setup(&tmem_slot, full, empty, stages, ncols);
    const uint32_t tmem = tmem_slot;
    const int32_t v = m0 + tid;
    const bool vin = v < V;
    const tc::VoxPos pos = tc::vox_pos(a.g, vin ? v : 0);
    const int chunks = ci / kc, iters = (kTaps / tp) * chunks;
    const uint32_t id = tc::idesc(kTcM, n, false);
    const uint32_t row_off = (uint32_t)(tid >> 3) * sbo + (uint32_t)(tid & 7) * 16u;

    auto fill = [&](int it, int s) {
        const int tg = it / chunks, c0 = (it % chunks) * kc;
        for (int q = 0; q < tp; ++q) {
            const int t = tg * tp + q;
            const uint32_t sa = base + (uint32_t)s * stage_bytes + (uint32_t)q * a_bytes;
            const uint32_t sb = base + (uint32_t)s * stage_bytes + (uint32_t)tp * a_bytes + (uint32_t)q * b_bytes;
            const int32_t nb = vin ? tc::tap_nb(a.g, pos, t / 9 - 1, (t / 3) % 3 - 1, t % 3 - 1) : -1;
            const bool valid = nb >= 0;
            for (int j = 0; j < kc / 8; ++j) {
                const int c = c0 + 8 * j;
                const bf16 *src =
                    c < a.ci0 ? a.in0 + (int64_t)nb * a.ci0 + c : a.in1 + (int64_t)nb * a.ci1 + (c - a.ci0);
                tc::cp16(sa + row_off + (uint32_t)j * 128u, valid ? (const void *)src : (const void *)a.in0, valid);
            }
            for (int e = tid; e < n * (kc / 8); e += 128) {
                const int r = e / (kc / 8), j = e % (kc / 8);
                const bf16 *src = a.w + ((int64_t)t * n + r) * ci + c0 + 8 * j;
                tc::cp16(sb + (uint32_t)(r >> 3) * sbo + (uint32_t)j * 128u + (uint32_t)(r & 7) * 16u, src, true);
            }
        }
    };
    auto issue = [&](int it, int s) {
        for (int q = 0; q < tp; ++q) {
            const uint32_t sa = base + (uint32_t)s * stage_bytes + (uint32_t)q * a_bytes;
            const uint32_t sb = base + (uint32_t)s * stage_bytes + (uint32_t)tp * a_bytes + (uint32_t)q * b_bytes;
            for (int j = 0; j < kc / 16; ++j)
                tc::mma(tmem, tc::desc(sa + (uint32_t)j * 256u, 128u, sbo),
                        tc::desc(sb + (uint32_t)j * 256u, 128u, sbo), id, it > 0 || q > 0 || j > 0);
        }
    };
    const bool ok = tc::pipeline_sync(iters, empty, status, fill, issue);
    if (ok) {
        const int32_t row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < n; c0 += 16) {
            uint32_t r[16];
            tc::load16(tmem, warp, c0, r);
            if (row < V) {
                uint32_t packed[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 + 2 * j;
                    float y0 = __uint_as_float(r[2 * j]) + (a.bias ? a.bias[c] : 0.0f);
                    float y1 = __uint_as_float(r[2 * j + 1]) + (a.bias ? a.bias[c + 1] : 0.0f);
                    if (a.relu) {
                        y0 = fmaxf(y0, 0.0f);
                        y1 = fmaxf(y1, 0.0f);
                    }
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(y0, y1);
                    packed[j] = *reinterpret_cast<const uint32_t *>(&pr);
                }
                // 16 channels lie in one of the two outputs (co0 is a multiple of 16)
                bf16 *dst = c0 < a.co0 ? a.out0 + (int64_t)row * a.co0 + c0 : a.out1 + (int64_t)row * a.co1 + (c0 - a.co0);
                uint4 *d4 = reinterpret_cast<uint4 *>(dst);
                d4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                d4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
    }
    tc::teardown(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Weight gradient dW[t][o][c] += sum_v dY[v][o] X(v + off_t)[c]: one CTA per
// (voxel chunk, tap) computes D = dY^T X_t with M = 128 rows (o < co used),
// N = ci, K = the chunk's voxels in steps of kWgStepVox, and adds D to dW with
// fp32 atomics.  Both operands are MN-major: for each voxel, A holds dY's co
// channels (a plain row of dY) and B the neighbour's ci channels; element
// (mn, k) at (mn/8)*SBO + (k/8)*128 + (k%8)*16 + (mn%8)*2 with SBO =
// kWgStepVox * 16.  Only the co/8 groups of A that exist are written: the MMA
// also reads rows co..127, which land in the following shared memory (held
// inside the allocation by a tail pad) and reach only accumulator rows that
// are never read.
// ---------------------------------------------------------------------------
struct WgradArgs {
    const bf16 *dy;
    int co;
    const bf16 *in0;
    int ci0;
    const bf16 *in1;
    int ci1;
    float *dw;          // [27][co][ci] fp32 (accumulated)
    Dims g;
    int chunk;          // voxels per CTA (a multiple of kWgStepVox)
};

constexpr int kWgStepVox = 64;
constexpr uint32_t kWgSbo = kWgStepVox * 16;              // bytes per 8-element MN group
constexpr uint32_t kWgTail = (kTcM / 8) * kWgSbo;          // over-read room for A

__global__ void __launch_bounds__(128) k_wgrad_tc(WgradArgs a, int ncols, int stages, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[tc::kMaxStages], empty[tc::kMaxStages];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int co = a.co, ci = a.ci0 + a.ci1;
    const int32_t V = (int32_t)a.g.voxels();
    const int t = (int)(blockIdx.x % kTaps);
    const int32_t v_begin = (int32_t)(blockIdx.x / kTaps) * a.chunk;
    const uint32_t a_bytes = (uint32_t)(co / 8) * kWgSbo, b_bytes = (uint32_t)(ci / 8) * kWgSbo;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const uint32_t base = tc::smem_u32(smem);
    tc::setup(&tmem_slot, full, empty, stages, ncols);
    const uint32_t tmem = tmem_slot;
    const uint32_t id = tc::idesc(kTcM, ci, true);
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int iters = a.chunk / kWgStepVox;
    // thread t handles voxel k = t % 64 of each step, pieces part, part + 2, ...
    const int k = tid % kWgStepVox, part = tid / kWgStepVox;
    const uint32_t k_off = (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 16u;

    auto fill = [&](int it, int s) {
        const uint32_t sa = base + (uint32_t)s * stage_bytes, sb = sa + a_bytes;
        const int32_t v = v_begin + it * kWgStepVox + k;
        const bool vin = v < V;
        for (int mg = part; mg < co / 8; mg += 2)
            tc::cp16(sa + (uint32_t)mg * kWgSbo + k_off,
                     vin ? (const void *)(a.dy + (int64_t)v * co + 8 * mg) : (const void *)a.dy, vin);
        const int32_t nb = vin ? tc::tap_nb(a.g, v, dz, dy, dx) : -1;
        const bool valid = nb >= 0;
        for (int ng = part; ng < ci / 8; ng += 2) {
            const int c = 8 * ng;
            const bf16 *src = c < a.ci0 ? a.in0 + (int64_t)nb * a.ci0 + c : a.in1 + (int64_t)nb * a.ci1 + (c - a.ci0);
            tc::cp16(sb + (uint32_t)ng * kWgSbo + k_off, valid ? (const void *)src : (const void *)a.in0, valid);
        }
    };
    auto issue = [&](int it, int s) {
        const uint32_t sa = base + (uint32_t)s * stage_bytes, sb = sa + a_bytes;
        for (int j = 0; j < kWgStepVox / 16; ++j)
            tc::mma(tmem, tc::desc(sa + (uint32_t)j * 256u, 128u, kWgSbo), tc::desc(sb + (uint32_t)j * 256u, 128u, kWgSbo),
                    id, it > 0 || j > 0);
    };
    const bool ok = tc::pipeline(iters, stages, full, empty, status, fill, issue);
    if (ok && warp * 32 < co) {
        const int o = warp * 32 + lane;
        for (int c0 = 0; c0 < ci; c0 += 16) {
            uint32_t r[16];
            tc::load16(tmem, warp, c0, r);
            if (o < co) {
                float *dst = a.dw + ((int64_t)t * co + o) * ci + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) atomicAdd(dst + j, __uint_as_float(r[j]));
            }
        }
    }
    tc::teardown(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Weight gradient with the taps stacked along M.  By the adjoint shift,
// dW[t][o][c] = sum_u dY[u - off_t][o] X[u][c]; with rows (t, o) one M = 128
// tile holds T = 128 / co taps, so no accumulator row is wasted (co = 16 in a
// plain dY^T X_t tile would use 16 of its 128 rows), X rows (B, N = ci, MN-major)
// are plain copies shared by every tap, and only dY is gathered, shifted by
// -off_t (circular in x and y, zero beyond z).  A CTA owns a chunk of voxels
// (grid x) and G consecutive tiles (grid y, G ci <= 512 TMEM columns, one
// accumulator of ci columns per tile); K runs over the chunk in steps of
// kWsStep voxels through the barrier-free pipeline, and the epilogue adds each
// tile's rows to dW[t][o][.] with fp32 atomics.
// ---------------------------------------------------------------------------
struct WstackArgs {
    const bf16 *dy;
    int co;
    const bf16 *x0;
    int ci0;
    const bf16 *x1;
    int ci1;    // the input is [x0, x1] (x1: ci1 = 0 for none)
    float *dw;   // [27][co][ci] fp32 (accumulated)
    Dims g;
    int chunk;   // voxels per CTA (a multiple of kWsStep)
    int tiles;   // tiles per CTA
};

constexpr int kWsStep = 32;
constexpr uint32_t kWsSbo = kWsStep * 16;                  // bytes per 8-element MN group
constexpr uint32_t kWsTileBytes = (kTcM / 8) * kWsSbo;      // one A tile (128 rows)

__global__ void __launch_bounds__(128) k_wgrad_stack(WstackArgs a, int ncols, int stages, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[tc::kMaxStages], empty[tc::kMaxStages];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int co = a.co, ci = a.ci0 + a.ci1, T = kTcM / co;
    const int n_tiles = (kTaps + T - 1) / T;
    const int tile0 = (int)blockIdx.y * a.tiles;
    const int G = min(a.tiles, n_tiles - tile0);
    const int32_t V = (int32_t)a.g.voxels();
    const int32_t v_begin = (int32_t)blockIdx.x * a.chunk;
    const uint32_t b_bytes = (uint32_t)(ci / 8) * kWsSbo;
    const uint32_t stage_bytes = (uint32_t)a.tiles * kWsTileBytes + b_bytes;
    const uint32_t base = tc::smem_u32(smem);
    tc::setup(&tmem_slot, full, empty, stages, ncols);
    const uint32_t tmem = tmem_slot;
    const uint32_t id = tc::idesc(kTcM, ci, true);
    const int iters = a.chunk / kWsStep;
    const int k = tid % kWsStep, part = tid / kWsStep;   // the step's voxel k; 4 parts share its pieces
    const uint32_t k_off = (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 16u;
    const int pieces_o = co / 8;

    auto fill = [&](int it, int s) {
        const uint32_t st0 = base + (uint32_t)s * stage_bytes, sb = st0 + (uint32_t)a.tiles * kWsTileBytes;
        const int32_t u = v_begin + it * kWsStep + k;
        const bool uin = u < V;
        const tc::VoxPos pos = tc::vox_pos(a.g, uin ? u : 0);
        for (int q = part; q < ci / 8; q += 4) {
            const int c = 8 * q;
            const bf16 *src = c < a.ci0 ? a.x0 + (int64_t)u * a.ci0 + c : a.x1 + (int64_t)u * a.ci1 + (c - a.ci0);
            tc::cp16(sb + (uint32_t)q * kWsSbo + k_off, uin ? (const void *)src : (const void *)a.x0, uin);
        }
        for (int j = 0; j < G; ++j) {
            const uint32_t sa = st0 + (uint32_t)j * kWsTileBytes;
            for (int e = part; e < 16; e += 4) {   // T taps x co/8 pieces = 16 MN groups
                const int tl = e / pieces_o, p = e % pieces_o;
                const int t = (tile0 + j) * T + tl;
                int32_t nb = -1;
                if (uin && t < kTaps) nb = tc::tap_nb(a.g, pos, 1 - t / 9, 1 - (t / 3) % 3, 1 - t % 3);
                const bool valid = nb >= 0;
                tc::cp16(sa + (uint32_t)e * kWsSbo + k_off,
                         valid ? (const void *)(a.dy + (int64_t)nb * co + 8 * p) : (const void *)a.dy, valid);
            }
        }
    };
    auto issue = [&](int it, int s) {
        const uint32_t st0 = base + (uint32_t)s * stage_bytes, sb = st0 + (uint32_t)a.tiles * kWsTileBytes;
        for (int j = 0; j < G; ++j)
            for (int jj = 0; jj < kWsStep / 16; ++jj)
                tc::mma(tmem + (uint32_t)(j * ci), tc::desc(st0 + (uint32_t)j * kWsTileBytes + (uint32_t)jj * 256u, 128u, kWsSbo),
                        tc::desc(sb + (uint32_t)jj * 256u, 128u, kWsSbo), id, it > 0 || jj > 0);
    };
    const bool ok = tc::pipeline(iters, stages, full, empty, status, fill, issue);
    if (ok) {
        const int row = warp * 32 + lane, tl = row / co, o = row % co;
        for (int j = 0; j < G; ++j) {
            const int t = (tile0 + j) * T + tl;
            for (int c0 = 0; c0 < ci; c0 += 16) {
                uint32_t r[16];
                tc::load16(tmem, warp, j * ci + c0, r);
                if (t < kTaps) {
                    float *dst = a.dw + ((int64_t)t * co + o) * ci + c0;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) atomicAdd(dst + jj, __uint_as_float(r[jj]));
                }
            }
        }
    }
    tc::teardown(tmem, ncols);
}

// bias gradient: db[o] += sum_v dY[v][o]
__global__ void k_bias_grad(const bf16 *__restrict__ dy, int co, int64_t V, float *__restrict__ db)
{
    extern __shared__ float part[];
    const int o = threadIdx.x % co, lanes = blockDim.x / co, l = threadIdx.x / co;
    float s = 0.0f;
    if (threadIdx.x < lanes * co)
        for (int64_t v = (int64_t)blockIdx.x * lanes + l; v < V; v += (int64_t)gridDim.x * lanes)
            s += __bfloat162float(dy[v * co + o]);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < co) {
        float tot = 0.0f;
        for (int k = 0; k < lanes; ++k) tot += part[k * co + threadIdx.x];
        atomicAdd(db + threadIdx.x, tot);
    }
}

// ---------------------------------------------------------------------------
// elementwise pieces
// ---------------------------------------------------------------------------
// input channels [sdf, z feature, zeros] as bf16 [voxel][16]
__global__ void k_make_input(const float *__restrict__ sdf, Dims g, bf16 *__restrict__ x)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.voxels()) return;
    const int z = (int)((v / ((int64_t)g.w * g.h)) % g.d);
    const float zf = g.d > 1 ? -1.0f + 2.0f * (float)z / (float)(g.d - 1) : 0.0f;
    bf16 *row = x + v * kIn;
    row[0] = __float2bfloat16_rn(sdf[v]);
    row[1] = __float2bfloat16_rn(zf);
    for (int c = 2; c < kIn; ++c) row[c] = __float2bfloat16_rn(0.0f);
}

// out = scale * sum of the 8 children (2x2x2 average pooling with scale 1/8)
__global__ void k_pool(const bf16 *__restrict__ in, Dims gi, int c, float scale, bf16 *__restrict__ out)
{
    const Dims go{gi.n, gi.d / 2, gi.h / 2, gi.w / 2};
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= go.voxels() * c) return;
    const int ch = (int)(e % c);
    int64_t v = e / c;
    const int x = (int)(v % go.w);
    v /= go.w;
    const int y = (int)(v % go.h);
    v /= go.h;
    const int z = (int)(v % go.d);
    const int64_t n = v / go.d;
    float s = 0.0f;
    for (int k = 0; k < 8; ++k) {
        const int64_t vi = ((n * gi.d + 2 * z + (k >> 2)) * gi.h + 2 * y + ((k >> 1) & 1)) * gi.w + 2 * x + (k & 1);
        s += __bfloat162float(in[vi * c + ch]);
    }
    out[e] = __float2bfloat16_rn(scale * s);
}

// out (+)= scale * parent (nearest-neighbour x2 upsampling)
__global__ void k_upsample(const bf16 *__restrict__ in, Dims go, int c, float scale, int accumulate,
                           bf16 *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= go.voxels() * c) return;
    const int ch = (int)(e % c);
    int64_t v = e / c;
    const int x = (int)(v % go.w);
    v /= go.w;
    const int y = (int)(v % go.h);
    v /= go.h;
    const int z = (int)(v % go.d);
    const int64_t n = v / go.d;
    const Dims gi{go.n, go.d / 2, go.h / 2, go.w / 2};
    const int64_t vi = ((n * gi.d + z / 2) * gi.h + y / 2) * gi.w + x / 2;
    float r = scale * __bfloat162float(in[vi * c + ch]);
    if (accumulate) r += __bfloat162float(out[e]);
    out[e] = __float2bfloat16_rn(r);
}

// dy *= (y > 0)
__global__ void k_relu_back(bf16 *__restrict__ dy, const bf16 *__restrict__ y, int64_t n)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !(__bfloat162float(y[e]) > 0.0f)) dy[e] = __float2bfloat16_rn(0.0f);
}

// head: out[v][o] = b[o] + sum_c W[o][c] x[v][c]; writes the normalised output
// (fp32 [voxel][3]) and scale * output in the LBM layout [n][3][nz][ny][nx]
__global__ void k_head(const bf16 *__restrict__ x, const float *__restrict__ w, const float *__restrict__ b, Dims g,
                       float scale, float *__restrict__ out_norm, float *__restrict__ out_field)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.voxels()) return;
    const int64_t per = (int64_t)g.d * g.h * g.w;
    const int64_t n = v / per, cell = v % per;
    for (int o = 0; o < kOut; ++o) {
        float s = b[o];
        for (int c = 0; c < kW0; ++c) s += __bfloat162float(__float2bfloat16_rn(w[o * kW0 + c])) * __bfloat162float(x[v * kW0 + c]);
        out_norm[v * kOut + o] = s;
        if (out_field) out_field[(n * kOut + o) * per + cell] = scale * s;
    }
}

// loss and head backward: dout = 2 (out - tscale * target) / (3 V);
// dx[v][c] = sum_o W[o][c] dout[v][o]; head weight/bias gradients and the
// loss (sum of squares) accumulate per block.
__global__ void __launch_bounds__(256, 2) k_head_back(const bf16 *__restrict__ x, const float *__restrict__ w,
                                                   const float *__restrict__ out_norm, const float *__restrict__ target,
                                                   float tscale, Dims g, bf16 *__restrict__ dx, float *__restrict__ dw,
                                                   float *__restrict__ db, double *__restrict__ loss)
{
    // per-thread partial sums over a grid-stride loop, then warp shuffles,
    // then one shared-memory add per warp and one global add per block
    __shared__ float sw[kOut * 16 + kOut];
    __shared__ float wb[kOut * 16];   // the head weights as the forward used them (bf16)
    __shared__ double sl;
    if (threadIdx.x < kOut * 16 + kOut) sw[threadIdx.x] = 0.0f;
    if (threadIdx.x < kOut * 16) wb[threadIdx.x] = __bfloat162float(__float2bfloat16_rn(w[threadIdx.x]));
    if (threadIdx.x == 0) sl = 0.0;
    __syncthreads();
    float pw[kOut * 16 + kOut];
#pragma unroll
    for (int e = 0; e < kOut * 16 + kOut; ++e) pw[e] = 0.0f;
    double l = 0.0;
    const int64_t V = g.voxels(), per = (int64_t)g.d * g.h * g.w;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = v / per, cell = v % per;
        float d[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) {
            const float diff = out_norm[v * kOut + o] - tscale * target[(n * kOut + o) * per + cell];
            l += (double)diff * diff;
            d[o] = 2.0f * diff / (float)(kOut * V);
            pw[kOut * 16 + o] += d[o];
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float xc = __bfloat162float(x[v * 16 + c]);
            float sacc = 0.0f;
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
                sacc += wb[o * 16 + c] * d[o];
                pw[o * 16 + c] += d[o] * xc;
            }
            dx[v * 16 + c] = __float2bfloat16_rn(sacc);
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < kOut * 16 + kOut; ++e) {
        float t = pw[e];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) atomicAdd(&sw[e], t);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if (lane == 0) atomicAdd(&sl, l);
    __syncthreads();
    if (threadIdx.x < kOut * 16) atomicAdd(dw + threadIdx.x, sw[threadIdx.x]);
    else if (threadIdx.x < kOut * 16 + kOut) atomicAdd(db + threadIdx.x - kOut * 16, sw[threadIdx.x]);
    if (threadIdx.x == 0) atomicAdd(loss, sl);
}

// fp32 master weights -> bf16 working copies: forward [t][o][c] and the
// backward-data layout [t][c][o] flipped in the taps (t -> 26 - t)
__global__ void k_weights_bf16(const float *__restrict__ w, int co, int ci, bf16 *__restrict__ wf, bf16 *__restrict__ wb)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)kTaps * co * ci) return;
    const int c = (int)(e % ci);
    const int o = (int)((e / ci) % co);
    const int t = (int)(e / ((int64_t)ci * co));
    const bf16 v = __float2bfloat16_rn(w[e]);
    wf[e] = v;
    wb[((int64_t)(kTaps - 1 - t) * ci + c) * co + o] = v;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = gr[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Layer {
    int co, ci;
    int64_t w_off, b_off;   // offsets (floats) in the flat parameter vector
    bf16 *wf = nullptr, *wb = nullptr;
};

enum { ENC1A, ENC1B, ENC2A, ENC2B, ENC3A, ENC3B, BOTTA, BOTTB, DEC3A, DEC3B, DEC2A, DEC2B, DEC1A, DEC1B, NLAYERS };

struct Net {
    Dims g[4];                     // dims per level
    std::vector<Layer> layers;
    int64_t head_w = 0, head_b = 0, n_params = 0;
    cudaStream_t st = nullptr;
    char *ws = nullptr;
    size_t ws_need = 0;
    int64_t adam_t = 0;
    // fp32 buffers
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *out_norm = nullptr;
    double *loss = nullptr;
    int *status = nullptr;         // set by a tensor-core wait that ran out
    // activations (bf16) and their gradients
    bf16 *in = nullptr;
    bf16 *act[NLAYERS] = {};
    bf16 *dact[NLAYERS] = {};
    bf16 *p1 = nullptr, *p2 = nullptr, *p3 = nullptr, *dp1 = nullptr, *dp2 = nullptr, *dp3 = nullptr;
    bf16 *u1 = nullptr, *u2 = nullptr, *u3 = nullptr, *du1 = nullptr, *du2 = nullptr, *du3 = nullptr;
};

static int64_t layout(Net &net, bool assign)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = lbm::align_up(off + (bytes ? bytes : 1), 256);
        return assign ? net.ws + at : nullptr;
    };
    const int64_t P = net.n_params;
    net.params = (float *)take(P * 4);
    net.grads = (float *)take(P * 4);
    net.m = (float *)take(P * 4);
    net.v = (float *)take(P * 4);
    for (Layer &L : net.layers) {
        L.wf = (bf16 *)take((size_t)kTaps * L.co * L.ci * 2);
        L.wb = (bf16 *)take((size_t)kTaps * L.co * L.ci * 2);
    }
    net.out_norm = (float *)take((size_t)net.g[0].voxels() * kOut * 4);
    net.loss = (double *)take(8);
    net.status = (int *)take(4);
    const int lvl[NLAYERS] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
    net.in = (bf16 *)take((size_t)net.g[0].voxels() * kIn * 2);
    for (int l = 0; l < NLAYERS; ++l) {
        const size_t b = (size_t)net.g[lvl[l]].voxels() * net.layers[l].co * 2;
        net.act[l] = (bf16 *)take(b);
        net.dact[l] = (bf16 *)take(b);
    }
    net.p1 = (bf16 *)take((size_t)net.g[1].voxels() * kW[0] * 2);
    net.dp1 = (bf16 *)take((size_t)net.g[1].voxels() * kW[0] * 2);
    net.p2 = (bf16 *)take((size_t)net.g[2].voxels() * kW[1] * 2);
    net.dp2 = (bf16 *)take((size_t)net.g[2].voxels() * kW[1] * 2);
    net.p3 = (bf16 *)take((size_t)net.g[3].voxels() * kW[2] * 2);
    net.dp3 = (bf16 *)take((size_t)net.g[3].voxels() * kW[2] * 2);
    net.u3 = (bf16 *)take((size_t)net.g[2].voxels() * kW[3] * 2);
    net.du3 = (bf16 *)take((size_t)net.g[2].voxels() * kW[3] * 2);
    net.u2 = (bf16 *)take((size_t)net.g[1].voxels() * kW[2] * 2);
    net.du2 = (bf16 *)take((size_t)net.g[1].voxels() * kW[2] * 2);
    net.u1 = (bf16 *)take((size_t)net.g[0].voxels() * kW[1] * 2);
    net.du1 = (bf16 *)take((size_t)net.g[0].voxels() * kW[1] * 2);
    return (int64_t)off;
}

static unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

#define UNET_TRY(x)                                    \
    do {                                               \
        if ((x) != cudaSuccess) return LBM_ECUDA;      \
    } while (0)

// Shared memory of the tensor-core kernels: stages are added (2..4) while
// they fit in kTcStepSmem; one stage of the largest layer (co = 192, KC = 64)
// is 40 KB, so two of them (80 KB) stay within kTcMaxSmem.
constexpr int kTcMaxSmem = 96 * 1024;
constexpr int kTcStepSmem = 64 * 1024;

static int launch_conv(const ConvArgs &a, cudaStream_t st, int *status)
{
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem) != cudaSuccess)
            return LBM_ECUDA;
        attr = true;
    }
    const int ci = a.ci0 + a.ci1, co = a.co0 + a.co1;
    if (ci % 16 != 0 || co % 16 != 0 || co > 256 || (a.co1 > 0 && a.co0 % 16 != 0) ||
        a.g.voxels() >= ((int64_t)1 << 31))
        return LBM_EINVAL;
    const int kc = ci % 64 == 0 ? 64 : (ci % 32 == 0 ? 32 : 16);
    int ncols = 32;
    while (ncols < co) ncols <<= 1;
    // two stages of 3 taps when they fit in 48 KB, else of 1 tap.  Measured on
    // the 64x64x128 training batch: the barrier-free loop, 3-4 stages and
    // 9-tap steps were all slower (they cost resident CTAs or add per-step
    // work); the gathers, not the tensor cores, bound this kernel.
    const size_t per_tap = (size_t)kTcM * kc * 2 + (size_t)co * kc * 2;
    const int tp = 2 * 3 * per_tap <= (size_t)48 * 1024 ? 3 : 1;
    const int stages = 2;
    k_conv3_tc<<<blocks(a.g.voxels(), kTcM), 128, stages * tp * per_tap, st>>>(a, kc, tp, ncols, stages, status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

// Weight gradient on the tensor cores: one CTA per (voxel chunk, tap) on grid
// x; chunks of 128..4096 voxels (a power of two) so that the grid keeps ~16
// CTAs per SM busy.  dw (fp32 [27][co][ci]) is accumulated into.
static int launch_wgrad(const bf16 *dy, int co, const bf16 *in0, int ci0, const bf16 *in1, int ci1, float *dw,
                        const Dims &g, cudaStream_t st, int *status)
{
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem) != cudaSuccess)
            return LBM_ECUDA;
        attr = true;
    }
    const int ci = ci0 + ci1;
    const int64_t V = g.voxels();
    if (co > kTcM || co % 16 != 0 || ci % 16 != 0 || ci > 256 || V >= ((int64_t)1 << 31)) return LBM_EINVAL;
    if (co == 16) {
        // taps stacked along M (8 taps per tile): measured 1.5-1.8x faster
        // than one padded tile per tap for the 16-channel layers, and slower
        // for 32-128 output channels, where a tap already fills 2-8 of the
        // tile's 8-row groups
        static bool sattr = false;
        if (!sattr) {
            if (cudaFuncSetAttribute(k_wgrad_stack, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem) !=
                cudaSuccess)
                return LBM_ECUDA;
            sattr = true;
        }
        const int T = kTcM / co, n_tiles = (kTaps + T - 1) / T;
        int tiles = std::min(n_tiles, std::min(4, 512 / ci));
        const int groups = (n_tiles + tiles - 1) / tiles;
        tiles = (n_tiles + groups - 1) / groups;   // even split over the groups
        int ncols = 32;
        while (ncols < tiles * ci) ncols <<= 1;
        int chunk = 4096;
        while (chunk > 256 && ((V + chunk - 1) / chunk) * groups < 4 * 152) chunk >>= 1;
        const size_t stage = (size_t)tiles * kWsTileBytes + (size_t)(ci / 8) * kWsSbo;
        int stages = 3;
        while (stages > 2 && stages * stage > (size_t)kTcMaxSmem) --stages;
        WstackArgs wa{dy, co, in0, ci0, in1, ci1, dw, g, chunk, tiles};
        const dim3 grid((unsigned)((V + chunk - 1) / chunk), (unsigned)groups);
        k_wgrad_stack<<<grid, 128, stages * stage, st>>>(wa, ncols, stages, status);
        return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
    }
    int chunk = 4096;
    while (chunk > 128 && (int64_t)kTaps * ((V + chunk - 1) / chunk) < 16 * 152) chunk >>= 1;
    WgradArgs wa{dy, co, in0, ci0, in1, ci1, dw, g, chunk};
    int ncols = 32;
    while (ncols < ci) ncols <<= 1;
    const size_t stage = (size_t)(co / 8 + ci / 8) * kWgSbo;
    int stages = tc::kMaxStages;
    while (stages > 2 && stages * stage + kWgTail > (size_t)kTcStepSmem) --stages;
    k_wgrad_tc<<<(unsigned)(blocks(V, chunk) * kTaps), 128, stages * stage + kWgTail, st>>>(wa, ncols, stages, status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static int conv(Net &net, int l, const bf16 *in0, int ci0, const bf16 *in1, int ci1, const Dims &g)
{
    const Layer &L = net.layers[l];
    ConvArgs a{in0, ci0, in1, ci1, L.wf, net.params + L.b_off, net.act[l], L.co, nullptr, 0, 1, g};
    return launch_conv(a, net.st, net.status);
}

// backward of conv layer l: mask by ReLU, weight/bias gradients, and (unless
// dx0 is null) the input gradient split into [dx0 (ci0), dx1 (ci1)]
static int conv_back(Net &net, int l, const bf16 *in0, int ci0, const bf16 *in1, int ci1, bf16 *dx0, bf16 *dx1,
                     const Dims &g)
{
    Layer &L = net.layers[l];
    const int64_t V = g.voxels();
    k_relu_back<<<blocks(V * L.co), 256, 0, net.st>>>(net.dact[l], net.act[l], V * L.co);
    {
        const int rc = launch_wgrad(net.dact[l], L.co, in0, ci0, in1, ci1, net.grads + L.w_off, g, net.st, net.status);
        if (rc != LBM_OK) return rc;
    }
    const int lanes = 256 / L.co;
    k_bias_grad<<<(unsigned)std::min<int64_t>(1024, blocks(V, lanes)), lanes * L.co, lanes * L.co * 4, net.st>>>(
        net.dact[l], L.co, V, net.grads + L.b_off);
    if (dx0) {
        // input gradient: the forward kernel with flipped, transposed weights
        ConvArgs a{net.dact[l], L.co, nullptr, 0, L.wb, nullptr, dx0, ci0, dx1, ci1, 0, g};
        const int rc = launch_conv(a, net.st, net.status);
        if (rc != LBM_OK) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static int refresh_weights(Net &net)
{
    for (const Layer &L : net.layers)
        k_weights_bf16<<<blocks((int64_t)kTaps * L.co * L.ci), 256, 0, net.st>>>(net.params + L.w_off, L.co, L.ci, L.wf,
                                                                                L.wb);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static int forward(Net &net, const float *sdf, float *out, float scale)
{
    const Dims *g = net.g;
    k_make_input<<<blocks(g[0].voxels()), 256, 0, net.st>>>(sdf, g[0], net.in);
    int rc = conv(net, ENC1A, net.in, kIn, nullptr, 0, g[0]);
    rc |= conv(net, ENC1B, net.act[ENC1A], kW[0], nullptr, 0, g[0]);
    k_pool<<<blocks(g[1].voxels() * kW[0]), 256, 0, net.st>>>(net.act[ENC1B], g[0], kW[0], 0.125f, net.p1);
    rc |= conv(net, ENC2A, net.p1, kW[0], nullptr, 0, g[1]);
    rc |= conv(net, ENC2B, net.act[ENC2A], kW[1], nullptr, 0, g[1]);
    k_pool<<<blocks(g[2].voxels() * kW[1]), 256, 0, net.st>>>(net.act[ENC2B], g[1], kW[1], 0.125f, net.p2);
    rc |= conv(net, ENC3A, net.p2, kW[1], nullptr, 0, g[2]);
    rc |= conv(net, ENC3B, net.act[ENC3A], kW[2], nullptr, 0, g[2]);
    k_pool<<<blocks(g[3].voxels() * kW[2]), 256, 0, net.st>>>(net.act[ENC3B], g[2], kW[2], 0.125f, net.p3);
    rc |= conv(net, BOTTA, net.p3, kW[2], nullptr, 0, g[3]);
    rc |= conv(net, BOTTB, net.act[BOTTA], kW[3], nullptr, 0, g[3]);
    k_upsample<<<blocks(g[2].voxels() * kW[3]), 256, 0, net.st>>>(net.act[BOTTB], g[2], kW[3], 1.0f, 0, net.u3);
    rc |= conv(net, DEC3A, net.u3, kW[3], net.act[ENC3B], kW[2], g[2]);
    rc |= conv(net, DEC3B, net.act[DEC3A], kW[2], nullptr, 0, g[2]);
    k_upsample<<<blocks(g[1].voxels() * kW[2]), 256, 0, net.st>>>(net.act[DEC3B], g[1], kW[2], 1.0f, 0, net.u2);
    rc |= conv(net, DEC2A, net.u2, kW[2], net.act[ENC2B], kW[1], g[1]);
    rc |= conv(net, DEC2B, net.act[DEC2A], kW[1], nullptr, 0, g[1]);
    k_upsample<<<blocks(g[0].voxels() * kW[1]), 256, 0, net.st>>>(net.act[DEC2B], g[0], kW[1], 1.0f, 0, net.u1);
    rc |= conv(net, DEC1A, net.u1, kW[1], net.act[ENC1B], kW[0], g[0]);
    rc |= conv(net, DEC1B, net.act[DEC1A], kW[0], nullptr, 0, g[0]);
    k_head<<<blocks(g[0].voxels()), 256, 0, net.st>>>(net.act[DEC1B], net.params + net.head_w, net.params + net.head_b,
                                                      g[0], scale, net.out_norm, out);
    if (rc != LBM_OK) return LBM_ECUDA;
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static int backward(Net &net, const float *target, float tscale)
{
    const Dims *g = net.g;
    UNET_TRY(cudaMemsetAsync(net.grads, 0, net.n_params * 4, net.st));
    UNET_TRY(cudaMemsetAsync(net.loss, 0, 8, net.st));
    k_head_back<<<(unsigned)std::min<int64_t>(4 * 152, blocks(g[0].voxels())), 256, 0, net.st>>>(net.act[DEC1B], net.params + net.head_w, net.out_norm,
                                                           target, tscale, g[0], net.dact[DEC1B], net.grads + net.head_w,
                                                           net.grads + net.head_b, net.loss);
    int rc = conv_back(net, DEC1B, net.act[DEC1A], kW[0], nullptr, 0, net.dact[DEC1A], nullptr, g[0]);
    rc |= conv_back(net, DEC1A, net.u1, kW[1], net.act[ENC1B], kW[0], net.du1, net.dact[ENC1B], g[0]);
    k_pool<<<blocks(g[1].voxels() * kW[1]), 256, 0, net.st>>>(net.du1, g[0], kW[1], 1.0f, net.dact[DEC2B]);
    rc |= conv_back(net, DEC2B, net.act[DEC2A], kW[1], nullptr, 0, net.dact[DEC2A], nullptr, g[1]);
    rc |= conv_back(net, DEC2A, net.u2, kW[2], net.act[ENC2B], kW[1], net.du2, net.dact[ENC2B], g[1]);
    k_pool<<<blocks(g[2].voxels() * kW[2]), 256, 0, net.st>>>(net.du2, g[1], kW[2], 1.0f, net.dact[DEC3B]);
    rc |= conv_back(net, DEC3B, net.act[DEC3A], kW[2], nullptr, 0, net.dact[DEC3A], nullptr, g[2]);
    rc |= conv_back(net, DEC3A, net.u3, kW[3], net.act[ENC3B], kW[2], net.du3, net.dact[ENC3B], g[2]);
    k_pool<<<blocks(g[3].voxels() * kW[3]), 256, 0, net.st>>>(net.du3, g[2], kW[3], 1.0f, net.dact[BOTTB]);
    rc |= conv_back(net, BOTTB, net.act[BOTTA], kW[3], nullptr, 0, net.dact[BOTTA], nullptr, g[3]);
    rc |= conv_back(net, BOTTA, net.p3, kW[2], nullptr, 0, net.dp3, nullptr, g[3]);
    k_upsample<<<blocks(g[2].voxels() * kW[2]), 256, 0, net.st>>>(net.dp3, g[2], kW[2], 0.125f, 1, net.dact[ENC3B]);
    rc |= conv_back(net, ENC3B, net.act[ENC3A], kW[2], nullptr, 0, net.dact[ENC3A], nullptr, g[2]);
    rc |= conv_back(net, ENC3A, net.p2, kW[1], nullptr, 0, net.dp2, nullptr, g[2]);
    k_upsample<<<blocks(g[1].voxels() * kW[1]), 256, 0, net.st>>>(net.dp2, g[1], kW[1], 0.125f, 1, net.dact[ENC2B]);
    rc |= conv_back(net, ENC2B, net.act[ENC2A], kW[1], nullptr, 0, net.dact[ENC2A], nullptr, g[1]);
    rc |= conv_back(net, ENC2A, net.p1, kW[0], nullptr, 0, net.dp1, nullptr, g[1]);
    k_upsample<<<blocks(g[0].voxels() * kW[0]), 256, 0, net.st>>>(net.dp1, g[0], kW[0], 0.125f, 1, net.dact[ENC1B]);
    rc |= conv_back(net, ENC1B, net.act[ENC1A], kW[0], nullptr, 0, net.dact[ENC1A], nullptr, g[0]);
    rc |= conv_back(net, ENC1A, net.in, kIn, nullptr, 0, nullptr, nullptr, g[0]);
    if (rc != LBM_OK) return LBM_ECUDA;
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // namespace unet

struct unet_net : public unet::Net {};

using namespace unet;

extern "C" {

int unet_create(int32_t n, int32_t nz, int32_t ny, int32_t nx, unet_net **out)
{
    if (!out || n < 1 || nz < 8 || ny < 8 || nx < 8 || nz % 8 || ny % 8 || nx % 8) return LBM_EINVAL;
    if ((int64_t)n * nz * ny * nx >= ((int64_t)1 << 31)) return LBM_EINVAL;
    unet_net *net = new (std::nothrow) unet_net();
    if (!net) return LBM_ENOMEM;
    for (int l = 0; l < 4; ++l) net->g[l] = Dims{n, nz >> l, ny >> l, nx >> l};
    const int shapes[NLAYERS][2] = {{kW[0], kIn},          {kW[0], kW[0]}, {kW[1], kW[0]},         {kW[1], kW[1]},
                                    {kW[2], kW[1]},        {kW[2], kW[2]}, {kW[3], kW[2]},         {kW[3], kW[3]},
                                    {kW[2], kW[3] + kW[2]}, {kW[2], kW[2]}, {kW[1], kW[2] + kW[1]}, {kW[1], kW[1]},
                                    {kW[0], kW[1] + kW[0]}, {kW[0], kW[0]}};
    int64_t off = 0;
    for (int l = 0; l < NLAYERS; ++l) {
        Layer L;
        L.co = shapes[l][0];
        L.ci = shapes[l][1];
        L.w_off = off;
        off += (int64_t)kTaps * L.co * L.ci;
        L.b_off = off;
        off += L.co;
        net->layers.push_back(L);
    }
    net->head_w = off;
    off += kOut * kW[0];
    net->head_b = off;
    off += kOut;
    net->n_params = off;
    net->ws_need = (size_t)layout(*net, false);
    *out = net;
    return LBM_OK;
}

int unet_param_count(const unet_net *net, int64_t *n)
{
    if (!net || !n) return LBM_EINVAL;
    *n = net->n_params;
    return LBM_OK;
}

int unet_workspace_size(const unet_net *net, size_t *bytes)
{
    if (!net || !bytes) return LBM_EINVAL;
    *bytes = net->ws_need;
    return LBM_OK;
}

int unet_bind(unet_net *net, void *dev_ws, size_t bytes, void *stream)
{
    if (!net || !dev_ws || ((uintptr_t)dev_ws & 255u)) return LBM_EINVAL;
    if (bytes < net->ws_need) return LBM_ESIZE;
    net->ws = (char *)dev_ws;
    net->st = (cudaStream_t)stream;
    layout(*net, true);
    UNET_TRY(cudaMemsetAsync(net->m, 0, net->n_params * 4, net->st));
    UNET_TRY(cudaMemsetAsync(net->v, 0, net->n_params * 4, net->st));
    UNET_TRY(cudaMemsetAsync(net->status, 0, 4, net->st));
    net->adam_t = 0;
    return LBM_OK;
}

int unet_set_params(unet_net *net, const float *dev_params)
{
    if (!net || !net->ws || !dev_params) return LBM_EINVAL;
    UNET_TRY(cudaMemcpyAsync(net->params, dev_params, net->n_params * 4, cudaMemcpyDeviceToDevice, net->st));
    return refresh_weights(*net);
}

int unet_get_params(unet_net *net, float *dev_params)
{
    if (!net || !net->ws || !dev_params) return LBM_EINVAL;
    UNET_TRY(cudaMemcpyAsync(dev_params, net->params, net->n_params * 4, cudaMemcpyDeviceToDevice, net->st));
    return LBM_OK;
}

int unet_get_grads(unet_net *net, float *dev_grads)
{
    if (!net || !net->ws || !dev_grads) return LBM_EINVAL;
    UNET_TRY(cudaMemcpyAsync(dev_grads, net->grads, net->n_params * 4, cudaMemcpyDeviceToDevice, net->st));
    return LBM_OK;
}

int unet_forward(unet_net *net, const float *dev_sdf, float *dev_u, float out_scale)
{
    if (!net || !net->ws || !dev_sdf) return LBM_EINVAL;
    return unet::forward(*net, dev_sdf, dev_u, out_scale);
}

int unet_backward(unet_net *net, const float *dev_target, float target_scale, double *host_loss)
{
    if (!net || !net->ws || !dev_target) return LBM_EINVAL;
    int rc = unet::backward(*net, dev_target, target_scale);
    if (rc != LBM_OK) return rc;
    if (host_loss) {
        double s = 0.0;
        int stalled = 0;
        UNET_TRY(cudaMemcpyAsync(&s, net->loss, 8, cudaMemcpyDeviceToHost, net->st));
        UNET_TRY(cudaMemcpyAsync(&stalled, net->status, 4, cudaMemcpyDeviceToHost, net->st));
        UNET_TRY(cudaStreamSynchronize(net->st));
        if (stalled) return LBM_ETIMEOUT;
        *host_loss = s / (double)(kOut * net->g[0].voxels());
    }
    return LBM_OK;
}

int unet_adam_step(unet_net *net, float lr, float beta1, float beta2, float eps)
{
    if (!net || !net->ws || !(lr > 0.0f)) return LBM_EINVAL;
    net->adam_t += 1;
    const float c1 = 1.0f - (float)std::pow((double)beta1, (double)net->adam_t);
    const float c2 = 1.0f - (float)std::pow((double)beta2, (double)net->adam_t);
    k_adam<<<blocks(net->n_params), 256, 0, net->st>>>(net->params, net->grads, net->m, net->v, net->n_params, lr, beta1,
                                                      beta2, eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    return refresh_weights(*net);
}

void unet_destroy(unet_net *net) { delete net; }

int unet_conv3d(const uint16_t *dev_x, int32_t ci, const uint16_t *dev_w, const float *dev_bias, uint16_t *dev_y,
                int32_t co, int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t relu, int32_t *dev_status,
                void *stream)
{
    if (!dev_x || !dev_w || !dev_y || !dev_status || n < 1 || nz < 1 || ny < 1 || nx < 1) return LBM_EINVAL;
    const Dims g{n, nz, ny, nx};
    ConvArgs a{(const bf16 *)dev_x, ci, nullptr, 0, (const bf16 *)dev_w, dev_bias, (bf16 *)dev_y, co, nullptr, 0,
               relu ? 1 : 0, g};
    return launch_conv(a, (cudaStream_t)stream, dev_status);
}

int unet_conv3d_wgrad(const uint16_t *dev_dy, int32_t co, const uint16_t *dev_x, int32_t ci, float *dev_dw,
                      int32_t n, int32_t nz, int32_t ny, int32_t nx, int32_t *dev_status, void *stream)
{
    if (!dev_dy || !dev_x || !dev_dw || !dev_status || n < 1 || nz < 1 || ny < 1 || nx < 1) return LBM_EINVAL;
    const Dims g{n, nz, ny, nx};
    return launch_wgrad((const bf16 *)dev_dy, co, (const bf16 *)dev_x, ci, nullptr, 0, dev_dw, g, (cudaStream_t)stream,
                        dev_status);
}

}  // extern "C"
