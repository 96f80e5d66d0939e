// lbm_static_scratch.cu -- a plane-average entry point that allocates nothing.
//
// lbm_plane_average() keeps its per-plane sums in the solver's workspace, which
// the caller allocates.  Some callers cannot allocate device memory at all: a
// host application whose device memory is owned by its own pool allocator
// (where a library-side cudaMalloc is forbidden or would escape its
// accounting), or a monitoring loop that must never stall (cudaMalloc and
// cudaFree synchronise the device).  lbm_plane_average_static() serves them:
// it reads a dense velocity field and solid mask the caller already has and
// keeps its scratch in a fixed array compiled into this library.
//
// The scratch lives in device global memory of every GPU that loads the
// library, for as long as the library stays loaded.  Host code cannot use the
// array's name as a device address, so its address is looked up with
// cudaGetSymbolAddress on the first call made in each device context (the
// primary context of the current device, as the runtime uses it).  The cache
// is keyed on the context's unique id: after a cudaDeviceReset the module is
// loaded again into a new context, where the array may sit elsewhere, and the
// next call looks it up afresh.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kStaticThreads = 256;

// Per-plane results (superficial mean, intrinsic mean, porosity) of the last
// call, shared by every call on the device.
__device__ __align__(256) static double g_plane_scratch[3 * LBM_STATIC_MAX_PLANES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchSlot {
    unsigned long long ctx_id = 0;   // 0: never looked up
    double *ptr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];

__device__ double static_block_sum(double v)
{
    __shared__ double part[kStaticThreads / 32];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < kStaticThreads / 32 ? part[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

// One block per z plane over the dense field; every plane entry is written,
// so nothing in the scratch needs clearing between calls.
__global__ void __launch_bounds__(kStaticThreads) k_plane_average_dense(const float *__restrict__ ux,
                                                                       const uint8_t *__restrict__ solid,
                                                                       int64_t plane, double *__restrict__ out)
{
    const int z = blockIdx.x;
    const float *u = ux + (int64_t)z * plane;
    const uint8_t *m = solid + (int64_t)z * plane;
    double s = 0.0, n = 0.0;
    for (int64_t c = threadIdx.x; c < plane; c += kStaticThreads)
        if (!m[c]) {
            s += (double)u[c];
            n += 1.0;
        }
    s = static_block_sum(s);
    n = static_block_sum(n);
    if (threadIdx.x == 0) {
        out[3 * z + 0] = s / (double)plane;
        out[3 * z + 1] = n > 0.0 ? s / n : 0.0;
        out[3 * z + 2] = n / (double)plane;
    }
}

// Unique id of the current CUDA context (0 when none is current or the driver
// does not provide the query).  The driver functions are reached through the
// runtime's entry-point lookup, so the library needs no link to libcuda.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch in the current device context: looked up on
// the first call in that context and kept for the next ones.
int scratch_for_current_device(double **ptr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchSlot &slot = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (id == 0 || slot.ctx_id != id || !slot.ptr) {
        // the lookup also makes the device's primary context current
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_plane_scratch) != cudaSuccess || !p) return LBM_ECUDA;
        slot.ptr = (double *)p;
        slot.ctx_id = current_context_id();
    }
    *ptr = slot.ptr;
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_plane_average_static(const float *dev_ux, const uint8_t *dev_solid, int32_t nx, int32_t ny,
                                        int32_t nz, double *host_out, void *stream)
{
    using namespace lbm;
    if (!dev_ux || !dev_solid || !host_out || nx < 1 || ny < 1 || nz < 1) return LBM_EINVAL;
    if (nz > LBM_STATIC_MAX_PLANES) {
        std::fprintf(stderr, "lbm_plane_average_static: nz = %d exceeds the fixed scratch of %d planes\n", nz,
                     LBM_STATIC_MAX_PLANES);
        return LBM_EINVAL;
    }
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    k_plane_average_dense<<<(unsigned)nz, kStaticThreads, 0, st>>>(dev_ux, dev_solid, (int64_t)nx * ny, scratch);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (cudaMemcpyAsync(host_out, scratch, sizeof(double) * 3 * (size_t)nz, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return LBM_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
