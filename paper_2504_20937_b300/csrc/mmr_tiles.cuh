// Screen-tile depth bounds for dense clouds, and the warp-aggregated splat.
//
// Depth bounds.  The frame is cut into 8x8-pixel tiles.  A first pass over a
// slice of the points splats them as usual and marks every tile in which one
// of them won an atomic (SplatMarkTiles).  A small kernel then takes, for
// each marked tile, the largest depth (clip-w bits) among the tile's current
// keys (tile_bound_kernel); a tile with an empty pixel gets no bound (the
// empty key's depth bits are all ones).  Keys only decrease while a frame is
// drawn, so every key of the tile stays at or below
// (bound << 32 | 0xffffffff) for the rest of the frame, and a later point
// whose depth bits exceed the bound cannot win any pixel of the tile: the
// second pass drops it without reading the depth-id buffer
// (SplatBelowTileBound).  Bounds are tagged with the frame's tag, so entries
// left from earlier frames are never used and nothing has to be cleared
// between frames.  The result is the same per-pixel minimum as the direct
// splat; only the number of depth-buffer reads changes.
#pragma once

#include "mmr_device.cuh"

namespace mmr {

constexpr uint32_t kTileShift = 3;      // 8x8-pixel tiles

struct TileBounds {
    uint32_t *mark;                     // per tile: the tag of the last frame that marked it
    uint32_t *list;                     // tiles marked this frame, in marking order
    uint32_t *count;                    // number of entries in list
    unsigned long long *bound;          // per tile: (tag << 32) | largest depth bits of its keys
    uint32_t tag;                       // this frame's tag (never 0)
    uint32_t tiles_w;                   // tiles per row
    uint32_t tiles;                     // tiles of the frame: the list's capacity
};

__device__ __forceinline__ uint32_t tile_of(uint32_t ix, uint32_t iy, uint32_t tiles_w)
{
    return (iy >> kTileShift) * tiles_w + (ix >> kTileShift);
}

// First pass: the direct splat, and a mark on the tile of every point that
// performs an atomic.  The first point to mark a tile in this frame (the one
// whose exchange returns another tag) appends the tile to the list, so a
// tile is listed at most once per frame and, as the second pass of every
// frame empties the list, it never outgrows the tile count; the append is
// bounded by the capacity all the same.  A stale L1 copy of a mark costs at
// most one more exchange.
struct SplatMarkTiles {
    static constexpr bool kWarpWide = false;
    TileBounds T;

    __device__ __forceinline__ void on_entry() const {}

    __device__ __forceinline__ void operator()(const PointParams &P, bool, uint32_t ix, uint32_t iy,
                                               unsigned long long key) const
    {
        unsigned long long *k = P.keys + iy * (uint32_t)P.W + ix;
        if (key < __ldca(k)) {
            atomicMin(k, key);
            const uint32_t t = tile_of(ix, iy, T.tiles_w);
            if (__ldca(T.mark + t) != T.tag && atomicExch(T.mark + t, T.tag) != T.tag) {
                const uint32_t slot = atomicAdd(T.count, 1u);
                if (slot < T.tiles)
                    T.list[slot] = t;
            }
        }
    }
};

// Second pass: a point deeper than its tile's bound is dropped; the others
// take the direct splat.  The bound entries were written by the preceding
// kernel, and L1 holds no line across kernel launches, so the read sees them.
// The first thread of the grid also empties the tile list for the next frame
// (its entries were used by the bound kernel, which has completed).
struct SplatBelowTileBound {
    static constexpr bool kWarpWide = false;
    TileBounds T;

    __device__ __forceinline__ void on_entry() const
    {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            *T.count = 0;
    }

    __device__ __forceinline__ void operator()(const PointParams &P, bool, uint32_t ix, uint32_t iy,
                                               unsigned long long key) const
    {
        const unsigned long long b = __ldca(T.bound + tile_of(ix, iy, T.tiles_w));
        if ((uint32_t)(b >> 32) == T.tag && (uint32_t)(key >> 32) > (uint32_t)b)
            return;
        splat_key(P.keys, iy * (uint32_t)P.W + ix, key);
    }
};

// Warp-aggregated splat: the lanes of a warp whose points fall on the same
// pixel (__match_any_sync) elect the one with the smallest key (two 32-bit
// minimum reductions: depth bits, then the id among the lanes at that
// depth; ids are unique, so exactly one lane is elected), and only that lane
// takes the depth test and the atomic.  The minimum is order-free, so the
// frame is the same.
struct SplatWarpAggregated {
    static constexpr bool kWarpWide = true;

    __device__ __forceinline__ void on_entry() const {}

    __device__ __forceinline__ void operator()(const PointParams &P, bool ok, uint32_t ix, uint32_t iy,
                                               unsigned long long key) const
    {
        const unsigned valid = __ballot_sync(__activemask(), ok);
        if (!ok)
            return;
        const uint32_t px = iy * (uint32_t)P.W + ix;
        const unsigned peers = __match_any_sync(valid, px);
        const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
        const uint32_t min_hi = __reduce_min_sync(peers, hi);
        const uint32_t min_lo = __reduce_min_sync(peers, hi == min_hi ? lo : 0xffffffffu);
        if (hi == min_hi && lo == min_lo)
            splat_key(P.keys, px, key);
    }
};

// One warp per listed tile (grid-stride over warps): the largest depth bits
// among the tile's keys, stored with this frame's tag.  Lane l reads row
// l / 4, columns 2 (l % 4) and 2 (l % 4) + 1 of the tile.  Pixels outside the
// frame are left out: no point projects there.
__device__ __forceinline__ void tile_bound_body(const unsigned long long *__restrict__ keys, int W, int H,
                                                const TileBounds &T)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t count = min(*T.count, T.tiles);
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += warps) {
        const uint32_t t = T.list[i];
        const uint32_t x = (t % T.tiles_w) * 8u + 2u * (lane & 3u);
        const uint32_t y = (t / T.tiles_w) * 8u + (lane >> 2);
        uint32_t m = 0u;
        if (y < (uint32_t)H) {
            const unsigned long long *row = keys + (uint64_t)y * (uint32_t)W;
            const uint32_t d0 = x < (uint32_t)W ? (uint32_t)(__ldcg(row + x) >> 32) : 0u;
            const uint32_t d1 = x + 1 < (uint32_t)W ? (uint32_t)(__ldcg(row + x + 1) >> 32) : 0u;
            m = max(d0, d1);
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0)
            T.bound[t] = ((unsigned long long)T.tag << 32) | m;
    }
}

}  // namespace mmr
