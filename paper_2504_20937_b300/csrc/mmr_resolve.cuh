// Resolve of depth-id keys into RGBA8, shared by the single-cloud and
// batched resolve kernels.  Empty key -> background.  Otherwise, in order of
// precedence: colormap[index[id]] when an index buffer is bound (an index at
// or beyond ncolors takes the default colour), colors[id] when a per-point
// colour buffer is bound, else the default colour.  The other depth-id buffer
// (the one the next frame splats into) is reset to all-ones in the same pass.
#pragma once

#include "mmr_device.cuh"

namespace mmr {

struct Palette {
    const uint32_t *colors;    // per-point RGBA8, or null
    const uint32_t *index;     // per-point colormap index, or null
    const uint32_t *colormap;  // ncolors RGBA8 entries
    uint32_t ncolors;
    uint32_t color;            // default colour
    uint32_t background;
};

__device__ __forceinline__ uint32_t key_colour(unsigned long long k, const Palette &pal)
{
    if (k == kEmptyKey)
        return pal.background;
    const uint32_t id = (uint32_t)(k & 0xffffffffu);
    if (pal.index) {
        const uint32_t c = __ldg(pal.index + id);
        return c < pal.ncolors ? __ldg(pal.colormap + c) : pal.color;
    }
    return pal.colors ? __ldg(pal.colors + id) : pal.color;
}

// Four pixels starting at 4q: two 16-byte key loads, one 16-byte RGBA store,
// two 16-byte clears.
__device__ __forceinline__ void resolve_quad(const unsigned long long *__restrict__ keys,
                                             unsigned long long *__restrict__ next_keys,
                                             uint32_t *__restrict__ rgba, const Palette &pal, uint32_t q)
{
    const ulonglong2 k01 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q);
    const ulonglong2 k23 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q + 1);
    const uint4 c = make_uint4(key_colour(k01.x, pal), key_colour(k01.y, pal), key_colour(k23.x, pal),
                               key_colour(k23.y, pal));
    __stcs(reinterpret_cast<uint4 *>(rgba) + q, c);
    const ulonglong2 e = make_ulonglong2(kEmptyKey, kEmptyKey);
    reinterpret_cast<ulonglong2 *>(next_keys)[2 * q] = e;
    reinterpret_cast<ulonglong2 *>(next_keys)[2 * q + 1] = e;
}

// Frame chunks of the single-cloud resolve: runs of 64 consecutive pixels
// (16 quads), one 32-bit tag per chunk and depth-id buffer.  A resolve tags
// every chunk in which its frame left a key with the frame's number.  The
// next resolve, which clears that buffer for the frame after it, clears and
// repaints only the chunks carrying the previous frame's number: elsewhere
// the buffer holds no key, and the framebuffer already holds background
// (painted by an earlier resolve and untouched since), unless this frame
// puts a point there.  Skipping those stores changes no pixel.
constexpr uint32_t kChunkQuadShift = 4;      // 16 quads = 64 pixels per chunk

struct FrameChunks {
    const uint32_t *prev;   // tags of the buffer being cleared (left by the previous frame's resolve)
    uint32_t *cur;          // tags of the buffer being resolved
    uint32_t prev_tag;      // the previous frame's number
    uint32_t cur_tag;       // this frame's number
    uint32_t full;          // non-zero: repaint and clear every chunk (first frame, new background)
};

__device__ __forceinline__ void resolve_pixel(const unsigned long long *__restrict__ keys,
                                              unsigned long long *__restrict__ next_keys,
                                              uint32_t *__restrict__ rgba, const Palette &pal, uint32_t p)
{
    rgba[p] = key_colour(keys[p], pal);
    next_keys[p] = kEmptyKey;
}

}  // namespace mmr
