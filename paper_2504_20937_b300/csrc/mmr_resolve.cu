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

// Host mirror update, one lane per chunk: a warp reads the tags and `held`
// bytes of 32 consecutive chunks (one coalesced access each), decides which
// to copy (the latest frame tagged it, or the mirror still holds a point
// there: held) and sets held to "tagged", what the mirror holds afterwards;
// then the whole warp copies the chosen chunks, two at a time, 16 lanes of
// 16 bytes on each 256-byte chunk.  The pixels past the last whole quad
// (npx not a multiple of 4) are left out of the chunk tags by the resolve, so
// they are copied every time.  A warp adds the bytes it wrote to *bytes.
__global__ void mirror_kernel(const uint32_t *__restrict__ rgba, uint32_t *__restrict__ host, uint32_t npx,
                              const uint32_t *__restrict__ tags, uint32_t tag, unsigned char *__restrict__ held,
                              int full, unsigned long long *bytes)
{
    const uint32_t quads = npx / 4;
    const uint32_t chunks = (quads + 15) / 16;      // chunks holding at least one whole quad
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t copied = 0;
    for (uint32_t c0 = warp * 32; c0 < chunks; c0 += warps * 32) {
        const uint32_t c = c0 + lane;
        bool copy = false;
        if (c < chunks) {
            const bool touched = tags[c] == tag;
            copy = full || touched || held[c] != 0;
            held[c] = touched ? 1 : 0;
        }
        unsigned todo = __ballot_sync(0xffffffffu, copy);
        while (todo) {
            const uint32_t a = __ffs(todo) - 1;
            todo &= todo - 1;
            uint32_t b = 32;
            if (todo) {
                b = __ffs(todo) - 1;
                todo &= todo - 1;
            }
            const uint32_t mine = lane < 16 ? a : b;
            if (mine < 32) {
                const uint32_t q = (c0 + mine) * 16 + (lane & 15u);
                if (q < quads) {
                    reinterpret_cast<uint4 *>(host)[q] = __ldcs(reinterpret_cast<const uint4 *>(rgba) + q);
                    copied += 16u;
                }
            }
        }
    }
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
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
    // one warp per 32 chunks, 256 threads per block
    const uint64_t chunks = ((uint64_t)npx / 4 + 15) / 16;
    const int grid = (int)std::max<uint64_t>(1, (chunks + 255) / 256);
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
