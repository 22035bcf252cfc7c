// Resolve of depth-id keys into RGBA8, shared by the single-cloud and
// batched resolve kernels.  Empty key -> background; else colors[id] when a
// colour buffer is bound, or the default colour.  The other depth-id buffer
// (the one the next frame splats into) is reset to all-ones in the same pass.
#pragma once

#include "mmr_device.cuh"

namespace mmr {

__device__ __forceinline__ uint32_t key_colour(unsigned long long k, const uint32_t *__restrict__ colors,
                                               uint32_t color, uint32_t background)
{
    if (k == kEmptyKey)
        return background;
    return colors ? __ldg(colors + (uint32_t)(k & 0xffffffffu)) : color;
}

// Four pixels starting at 4q: two 16-byte key loads, one 16-byte RGBA store,
// two 16-byte clears.
__device__ __forceinline__ void resolve_quad(const unsigned long long *__restrict__ keys,
                                             unsigned long long *__restrict__ next_keys,
                                             uint32_t *__restrict__ rgba, const uint32_t *__restrict__ colors,
                                             uint32_t q, uint32_t color, uint32_t background)
{
    const ulonglong2 k01 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q);
    const ulonglong2 k23 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q + 1);
    const uint4 c = make_uint4(key_colour(k01.x, colors, color, background),
                               key_colour(k01.y, colors, color, background),
                               key_colour(k23.x, colors, color, background),
                               key_colour(k23.y, colors, color, background));
    __stcs(reinterpret_cast<uint4 *>(rgba) + q, c);
    const ulonglong2 e = make_ulonglong2(kEmptyKey, kEmptyKey);
    reinterpret_cast<ulonglong2 *>(next_keys)[2 * q] = e;
    reinterpret_cast<ulonglong2 *>(next_keys)[2 * q + 1] = e;
}

__device__ __forceinline__ void resolve_pixel(const unsigned long long *__restrict__ keys,
                                              unsigned long long *__restrict__ next_keys,
                                              uint32_t *__restrict__ rgba, const uint32_t *__restrict__ colors,
                                              uint32_t p, uint32_t color, uint32_t background)
{
    rgba[p] = key_colour(keys[p], colors, color, background);
    next_keys[p] = kEmptyKey;
}

}  // namespace mmr
