// The single-cloud resolve: depth-id keys into the RGBA8 framebuffer, and the
// other depth-id buffer cleared for the next frame, in one pass over the
// pixels (stores only in the chunks a frame touched, mmr_resolve.cuh).
#include <algorithm>

#include <cuda_runtime.h>

#include "mmr_device.cuh"
#include "mmr_internal.h"
#include "mmr_launch.cuh"
#include "mmr_resolve.cuh"

namespace mmr {

// Resolve + clear: four pixels per thread, whole warps grid-stride (a warp
// takes 32 consecutive quads, two chunks); the ragged tail (npx not a
// multiple of 4) goes to the first threads, always repainted and cleared.
// Keys are read everywhere; colours are stored and the other buffer cleared
// only in chunks that this frame or the previous one touched (FrameChunks).
// Measured against repainting and clearing every pixel, same box: 2^22-point
// 1920x1080 orbit 10.9 -> 8.9 us, 64M-point 16-cluster 3840x2160 frame
// 22.9 -> 17.8 us, identical frames.
__global__ void resolve_kernel(const unsigned long long *__restrict__ keys,
                               unsigned long long *__restrict__ next_keys,
                               uint32_t *__restrict__ rgba, Palette pal, uint32_t npx, FrameChunks F)
{
    enter_dependent_grid();
    const uint32_t quads = npx / 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t q0 = t - lane; q0 < quads; q0 += stride) {
        const uint32_t q = q0 + lane;
        bool dirty = false;
        if (q < quads) {
            const ulonglong2 k01 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q);
            const ulonglong2 k23 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q + 1);
            dirty = (k01.x & k01.y & k23.x & k23.y) != kEmptyKey;
            const bool prev = F.full || __ldg(F.prev + (q >> kChunkQuadShift)) == F.prev_tag;
            if (dirty || prev) {
                const uint4 c = make_uint4(key_colour(k01.x, pal), key_colour(k01.y, pal), key_colour(k23.x, pal),
                                           key_colour(k23.y, pal));
                __stcs(reinterpret_cast<uint4 *>(rgba) + q, c);
            }
            if (prev) {
                const ulonglong2 e = make_ulonglong2(kEmptyKey, kEmptyKey);
                reinterpret_cast<ulonglong2 *>(next_keys)[2 * q] = e;
                reinterpret_cast<ulonglong2 *>(next_keys)[2 * q + 1] = e;
            }
        }
        // lanes 0 and 16 tag their half-warp's chunk when any of its quads holds a key
        const unsigned touched = __ballot_sync(0xffffffffu, dirty);
        if ((lane & 15u) == 0 && ((touched >> lane) & 0xffffu) != 0)
            F.cur[q >> kChunkQuadShift] = F.cur_tag;
    }
    if (quads * 4 + t < npx)
        resolve_pixel(keys, next_keys, rgba, pal, quads * 4 + t);
}

// Host mirror update: whole warps over 32 consecutive quads (two chunks, as
// in the resolve).  A chunk is copied when the latest frame tagged it or the
// mirror still holds a point there (held), and then held becomes "tagged":
// what the mirror holds afterwards.  Every lane of a half warp reads held
// before its first lane rewrites it.  Stores to the mapped host memory are
// 16 bytes per lane, 512 contiguous bytes per warp.
__global__ void mirror_kernel(const uint32_t *__restrict__ rgba, uint32_t *__restrict__ host, uint32_t npx,
                              const uint32_t *__restrict__ tags, uint32_t tag, unsigned char *__restrict__ held,
                              int full, unsigned long long *bytes)
{
    const uint32_t quads = npx / 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t copied = 0;
    for (uint32_t q0 = t - lane; q0 < quads; q0 += stride) {
        const uint32_t q = q0 + lane;
        const uint32_t chunk = q >> kChunkQuadShift;
        bool touched = false, copy = false;
        if (q < quads) {
            touched = tags[chunk] == tag;
            copy = full || touched || held[chunk] != 0;
            if (copy)
                reinterpret_cast<uint4 *>(host)[q] = __ldcs(reinterpret_cast<const uint4 *>(rgba) + q);
        }
        __syncwarp();
        if ((lane & 15u) == 0 && q < quads)
            held[chunk] = touched ? 1 : 0;
        copied += copy ? 16u : 0u;
    }
    if (quads * 4 + t < npx) {
        host[quads * 4 + t] = rgba[quads * 4 + t];
        copied += 4u;
    }
    copied = __reduce_add_sync(0xffffffffu, copied);
    if (lane == 0 && copied)
        atomicAdd(bytes, (unsigned long long)copied);
}

cudaError_t launch_mirror(const uint32_t *rgba, uint32_t *host, uint32_t npx, const uint32_t *tags, uint32_t tag,
                          unsigned char *held, int full, unsigned long long *bytes, cudaStream_t s)
{
    const uint64_t quads = npx / 4;
    const int grid = (int)std::max<uint64_t>(1, (quads + 255) / 256);
    mirror_kernel<<<grid, 256, 0, s>>>(rgba, host, npx, tags, tag, held, full, bytes);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const unsigned long long *keys, unsigned long long *next_keys, uint32_t *rgba,
                           const Palette &pal, uint32_t npx, const FrameChunks &F, cudaStream_t s)
{
    // pure streaming: one quad per thread, 256 threads, whatever the point kernel's shape.
    const uint64_t quads = npx / 4;
    const int grid = (int)std::max<uint64_t>(1, (quads + 255) / 256);
    return launch_dependent(resolve_kernel, grid, 256, s, keys, next_keys, rgba, pal, npx, F);
}

}  // namespace mmr
