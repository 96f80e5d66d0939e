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
// array's name as a device address, so its address is looked up once per
// device with cudaGetSymbolAddress (on the first call made on that device).
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
double *g_scratch_ptr[kMaxDevices] = {nullptr};

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

// Device address of the scratch on the current device, looked up once.
int scratch_for_current_device(double **ptr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_plane_scratch) != cudaSuccess || !p) return LBM_ECUDA;
        g_scratch_ptr[dev] = (double *)p;
    }
    *ptr = g_scratch_ptr[dev];
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
