// Kernels of the single-cloud path: fused displace + project + splat over the
// points (grid-stride over 48-byte point groups), and resolve + clear over
// the pixels.
#include <cuda_runtime.h>

#include "mmr_device.cuh"
#include "mmr_internal.h"
#include "mmr_points.cuh"
#include "mmr_resolve.cuh"

namespace mmr {

template <int DT, bool kDisplace, bool kSplat>
__global__ void points_kernel(void *__restrict__ pos, uint32_t n, PointParams P)
{
    const uint32_t groups = groups_of<DT>(n);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride)
        process_group<DT, kDisplace, kSplat>(pos, n, g, P);
}

// Resolve + clear: four pixels per thread, grid-stride; the ragged tail
// (npx not a multiple of 4) goes to the first threads.
__global__ void resolve_kernel(const unsigned long long *__restrict__ keys,
                               unsigned long long *__restrict__ next_keys,
                               uint32_t *__restrict__ rgba, const uint32_t *__restrict__ colors,
                               uint32_t npx, uint32_t color, uint32_t background)
{
    const uint32_t quads = npx / 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t q = t; q < quads; q += stride)
        resolve_quad(keys, next_keys, rgba, colors, q, color, background);
    if (quads * 4 + t < npx)
        resolve_pixel(keys, next_keys, rgba, colors, quads * 4 + t, color, background);
}

// ---------------------------------------------------------------- launchers

static int grid_for(uint64_t work_items, const LaunchShape &ls)
{
    if (ls.ctas_per_sm > 0)
        return ls.sm_count * ls.ctas_per_sm;
    uint64_t blocks = (work_items + ls.threads - 1) / ls.threads;
    if (blocks < 1)
        blocks = 1;
    if (blocks > 0x7fffffffull)
        blocks = 0x7fffffffull;
    return (int)blocks;
}

template <int DT>
static cudaError_t launch_points_dt(void *pos, uint32_t n, const PointParams &P, bool displace,
                                    bool splat, const LaunchShape &ls, cudaStream_t s)
{
    const uint64_t groups = groups_of<DT>(n);
    const int grid = grid_for(groups, ls);
    if (displace && splat)
        points_kernel<DT, true, true><<<grid, ls.threads, 0, s>>>(pos, n, P);
    else if (displace)
        points_kernel<DT, true, false><<<grid, ls.threads, 0, s>>>(pos, n, P);
    else
        points_kernel<DT, false, true><<<grid, ls.threads, 0, s>>>(pos, n, P);
    return cudaGetLastError();
}

cudaError_t launch_points(int dtype, void *pos, uint32_t n, const PointParams &P, bool displace,
                          bool splat, const LaunchShape &ls, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    switch (dtype) {
    case kF32: return launch_points_dt<kF32>(pos, n, P, displace, splat, ls, s);
    case kF16: return launch_points_dt<kF16>(pos, n, P, displace, splat, ls, s);
    case kBF16: return launch_points_dt<kBF16>(pos, n, P, displace, splat, ls, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resolve(const unsigned long long *keys, unsigned long long *next_keys,
                           uint32_t *rgba, const uint32_t *colors, uint32_t npx, uint32_t color,
                           uint32_t background, const LaunchShape &ls, cudaStream_t s)
{
    const uint64_t quads = npx / 4;
    int grid = grid_for(quads > 0 ? quads : 1, ls);
    resolve_kernel<<<grid, ls.threads, 0, s>>>(keys, next_keys, rgba, colors, npx, color, background);
    return cudaGetLastError();
}

}  // namespace mmr
