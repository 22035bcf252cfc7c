// mmr_render_static: render without allocating device memory.
//
// The depth-id scratch of this entry point is a file-scope __device__ array.
// This file is its own device module (the library is linked without
// relocatable device code), and under CUDA's lazy module loading, the default,
// a module is loaded on a device when it is first used there: the array's
// 32 MiB are reserved by the first call on each device (its
// cudaGetSymbolAddress), not when the library is loaded, and stay reserved
// until the process exits.  Host code cannot use the array's name as a device
// address (on the host it names a stand-in object), so the address is looked
// up once per device with cudaGetSymbolAddress while that device is current,
// cached, and passed to the kernels as a plain pointer.  The cache assumes the
// device's primary context lives as long as the process: after a
// cudaDeviceReset the cached address is stale.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/mmr.h"
#include "mmr_device.cuh"
#include "mmr_internal.h"

namespace mmr {

constexpr uint64_t kStaticMaxPixels = MMR_STATIC_MAX_PIXELS;

static __device__ __align__(256) unsigned long long g_static_keys[kStaticMaxPixels];

__global__ void static_clear_kernel(unsigned long long *__restrict__ keys, uint32_t npx)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += stride)
        keys[p] = kEmptyKey;
}

__global__ void static_resolve_kernel(const unsigned long long *__restrict__ keys, uint32_t *__restrict__ rgba,
                                      uint32_t npx, uint32_t color, uint32_t background)
{
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += stride)
        rgba[p] = keys[p] == kEmptyKey ? background : color;
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
unsigned long long *g_static_ptr[kMaxDevices] = {};

// Device address of g_static_keys on the current device (looked up once).
cudaError_t static_keys_on_current_device(unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_keys);
        if (e != cudaSuccess)
            return e;
        g_static_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

mmr_status static_fail(mmr_status s, const char *msg)
{
    set_process_error(msg);
    return s;
}

}  // namespace
}  // namespace mmr

extern "C" mmr_status mmr_render_static(const void *dev_points, uint64_t n, int dtype, const float m[16],
                                        float znear, float zfar, int width, int height, uint32_t color,
                                        uint32_t background, uint32_t *dev_rgba, void *stream)
{
    using namespace mmr;
    if (!dev_points || !m || !dev_rgba)
        return static_fail(MMR_ERR_INVALID_ARG, "mmr_render_static: NULL pointer");
    if (n == 0 || n >= (1ull << 32))
        return static_fail(MMR_ERR_INVALID_ARG, "mmr_render_static: n outside 1..2^32-1");
    if (dtype != MMR_F32x3 && dtype != MMR_F16x3 && dtype != MMR_BF16x3)
        return static_fail(MMR_ERR_INVALID_ARG, "mmr_render_static: unknown dtype");
    if (width < 1 || height < 1 || (uint64_t)width * (uint64_t)height > kStaticMaxPixels)
        return static_fail(MMR_ERR_INVALID_ARG,
                           "mmr_render_static: width*height must be 1..MMR_STATIC_MAX_PIXELS (4194304)");
    if (!mmr::depth_range_ok(znear, zfar))
        return static_fail(MMR_ERR_INVALID_ARG, "mmr_render_static: need 2^-64 <= znear < zfar <= 2^64");
    if (reinterpret_cast<uintptr_t>(dev_points) % 16 != 0)
        return static_fail(MMR_ERR_INVALID_ARG, "mmr_render_static: dev_points must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(dev_rgba) % 4 != 0)
        return static_fail(MMR_ERR_INVALID_ARG, "mmr_render_static: dev_rgba must be 4-byte aligned");
    unsigned long long *keys = nullptr;
    cudaError_t e = static_keys_on_current_device(&keys);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        snprintf(msg, sizeof msg,
                 "mmr_render_static: loading the 32 MiB scratch array on this device (cudaGetSymbolAddress) "
                 "failed: %s", cudaGetErrorString(e));
        return static_fail(e == cudaErrorMemoryAllocation ? MMR_ERR_OOM : MMR_ERR_CUDA, msg);
    }
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t npx = (uint32_t)((uint64_t)width * (uint64_t)height);
    const int grid_px = (int)std::min<uint64_t>((npx + 255) / 256, (uint64_t)sms * 8);

    static_clear_kernel<<<grid_px, 256, 0, s>>>(keys, npx);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        PointParams P{};
        for (int k = 0; k < 4; ++k) {
            P.cam.rx[k] = m[k];
            P.cam.ry[k] = m[4 + k];
            P.cam.rw[k] = m[12 + k];
        }
        P.cam.znear = znear;
        P.cam.zfar = zfar;
        P.keys = keys;
        P.W = width;
        P.H = height;
        P.fW = (float)width;
        P.fH = (float)height;
        P.halfW = 0.5f * (float)width;
        P.halfH = 0.5f * (float)height;
        P.id_base = 0;
        LaunchShape ls;
        ls.sm_count = sms;
        // render only: the point buffer is read, never written
        e = launch_points(dtype, dev_points, nullptr, (uint32_t)n, P, false, true, ls, s);
    }
    if (e == cudaSuccess) {
        static_resolve_kernel<<<grid_px, 256, 0, s>>>(keys, dev_rgba, npx, color, background);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "mmr_render_static: kernel launch failed: %s", cudaGetErrorString(e));
        return static_fail(MMR_ERR_CUDA, msg);
    }
    return MMR_OK;
}
