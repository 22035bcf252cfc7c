// Disc markers (the paper's front-facing disc markers, mmr_set_marker):
// the splat of one projected point into every pixel of its disc.  Kept apart
// from mmr_device.cuh so that the 1-px point kernels do not depend on it.
#pragma once

#include "mmr_device.cuh"

namespace mmr {

// Disc marker of radius r pixels (the paper's front-facing disc markers):
// the key goes to every pixel whose centre lies within r of (sx, sy), with
// dx = (px + 1/2) - sx, dy = (py + 1/2) - sy and dx*dx + dy*dy <= r*r in FP32
// in that order; that test alone decides.  Candidates: a pixel that passes
// has RN(dx*dx) <= RN(r*r), so |dx| <= r (1 + 2^-23) and
// |px + 1/2 - sx| <= r + r 2^-22 <= r + 2^-16 (r <= 64).  The candidate
// columns are the integers in [sx - 1/2 - r - 1/16, sx - 1/2 + r + 1/16]
// (rows likewise), clipped to the frame.  For |sx| < 2^18 each bound is three
// FP32 operations on values below 2^19, each off by at most 2^-6, so the
// computed interval still holds every pixel that can pass; a point farther
// out is more than 2^17 pixels from any frame (width <= 32768) and its
// interval is empty either way.  NaN bounds convert to 0 and fail the test.
struct DiscBox {
    int x0, x1, y0, y1;      // candidate columns x0..x1 and rows y0..y1 (empty when x0 > x1 or y0 > y1)
};

__device__ __forceinline__ DiscBox disc_box(float sx, float sy, const PointParams &P)
{
    constexpr float kMargin = 0.0625f;
    const float cx = __fsub_rn(sx, 0.5f), cy = __fsub_rn(sy, 0.5f);
    DiscBox b;
    b.x0 = max(__float2int_ru(__fsub_rn(__fsub_rn(cx, P.disc_r), kMargin)), 0);
    b.x1 = min(__float2int_rd(__fadd_rn(__fadd_rn(cx, P.disc_r), kMargin)), P.W - 1);
    b.y0 = max(__float2int_ru(__fsub_rn(__fsub_rn(cy, P.disc_r), kMargin)), 0);
    b.y1 = min(__float2int_rd(__fadd_rn(__fadd_rn(cy, P.disc_r), kMargin)), P.H - 1);
    return b;
}

__device__ __forceinline__ void splat_disc(float sx, float sy, unsigned long long key, const PointParams &P,
                                           const DiscBox &box)
{
    const int x0 = box.x0, x1 = box.x1, y0 = box.y0, y1 = box.y1;
    // Candidates go four at a time: their tests, then their four depth reads
    // together, then the compares and atomics.  One at a time, each read would
    // wait for the previous pixel's atomic (the compiler cannot move a read
    // above an atomic that may touch the same key), serialising the latencies.
    for (int py = y0; py <= y1; ++py) {
        const float dy = __fsub_rn(__fadd_rn((float)py, 0.5f), sy);
        const float dy2 = __fmul_rn(dy, dy);
        unsigned long long *row = P.keys + (uint32_t)py * (uint32_t)P.W;
        for (int px = x0; px <= x1; px += 4) {
            bool in[4];
            unsigned long long cur[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = px + k;
                const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), sx);
                in[k] = x <= x1 && __fadd_rn(__fmul_rn(dx, dx), dy2) <= P.disc_r2;
                cur[k] = in[k] ? __ldca(row + x) : 0ull;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (in[k] && key < cur[k])
                    atomicMin(row + px + k, key);
        }
    }
}

__device__ __forceinline__ void splat_disc(float sx, float sy, unsigned long long key, const PointParams &P)
{
    splat_disc(sx, sy, key, P, disc_box(sx, sy, P));
}

// Depth bounds for disc markers, on 32x32-pixel tiles of the whole frame:
// after a first pass over a slice of the points, disc_tile_bound_body stores
// for every tile the largest depth bits of its keys (all ones when a pixel
// is still empty), tagged with the frame's tag.  A later disc whose depth
// bits exceed the bound of every tile its candidate box touches would lose
// on every pixel it covers (each of them lies in one of those tiles, whose
// keys only decrease), so it is skipped whole.
constexpr int kDiscTileShift = 5;

struct DiscBounds {
    unsigned long long *bound;  // per tile: (tag << 32) | largest depth bits
    uint32_t tag;               // this frame's tag (never 0)
    uint32_t tiles_w, tiles_h;
};

__device__ __forceinline__ bool disc_behind_bounds(const DiscBox &b, uint32_t depth_bits, const DiscBounds &T)
{
    if (b.x0 > b.x1 || b.y0 > b.y1)
        return true;                                     // covers no pixel of the frame
    for (int ty = b.y0 >> kDiscTileShift; ty <= (b.y1 >> kDiscTileShift); ++ty)
        for (int tx = b.x0 >> kDiscTileShift; tx <= (b.x1 >> kDiscTileShift); ++tx) {
            const unsigned long long v = __ldca(T.bound + (uint32_t)ty * T.tiles_w + (uint32_t)tx);
            if ((uint32_t)(v >> 32) != T.tag || depth_bits <= (uint32_t)v)
                return false;
        }
    return true;
}

// The discs of a warp that survived the culling, splatted one at a time by
// the whole warp: every lane calls this (mine = whether its disc is to be
// drawn, with that disc's centre, key and candidate box), each surviving
// disc's parameters are broadcast from its lane, and the lanes share the
// disc's candidate pixels, consecutive lanes on consecutive pixels of a row
// (coalesced depth reads).  Candidate t of a box w pixels wide is at row
// floor(t / w), taken as the high half of t * ceil(2^32 / w), which equals
// floor(t / w) for t < 2^32 / w (here t < 129 * 129).  The pixel test is
// splat_disc's, in the same FP32 operations and order.
__device__ __forceinline__ void splat_discs_by_warp(bool mine, float sx, float sy, unsigned long long key,
                                                    const DiscBox &b, const PointParams &P)
{
    const unsigned full = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned todo = __ballot_sync(full, mine);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const float dsx = __shfl_sync(full, sx, src), dsy = __shfl_sync(full, sy, src);
        const unsigned long long dkey = __shfl_sync(full, key, src);
        const int x0 = __shfl_sync(full, b.x0, src), x1 = __shfl_sync(full, b.x1, src);
        const int y0 = __shfl_sync(full, b.y0, src), y1 = __shfl_sync(full, b.y1, src);
        const uint32_t w = (uint32_t)(x1 - x0 + 1), npx = w * (uint32_t)(y1 - y0 + 1);
        const uint64_t m = ((1ull << 32) + w - 1) / w;
        for (uint32_t t = lane; t < npx; t += 32) {
            const uint32_t row = (uint32_t)(((uint64_t)t * m) >> 32);
            const int px = x0 + (int)(t - row * w), py = y0 + (int)row;
            const float dy = __fsub_rn(__fadd_rn((float)py, 0.5f), dsy);
            const float dx = __fsub_rn(__fadd_rn((float)px, 0.5f), dsx);
            if (__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= P.disc_r2) {
                unsigned long long *k = P.keys + (uint32_t)py * (uint32_t)P.W + (uint32_t)px;
                if (dkey < __ldca(k))
                    atomicMin(k, dkey);
            }
        }
    }
}

// One warp per tile, grid-stride over all tiles: lane l takes column l of
// each of the tile's rows.  Pixels outside the frame are left out: no disc
// reaches them (candidate boxes are clipped to the frame), and every tile
// holds at least one pixel of the frame.
__device__ __forceinline__ void disc_tile_bound_body(const unsigned long long *__restrict__ keys, int W, int H,
                                                     const DiscBounds &T)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t tiles = T.tiles_w * T.tiles_h;
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles; t += warps) {
        const uint32_t x = (t % T.tiles_w) * 32u + lane;
        const uint32_t y0 = (t / T.tiles_w) * 32u;
        const uint32_t y1 = min(y0 + 32u, (uint32_t)H);
        uint32_t m = 0u;
        if (x < (uint32_t)W)
            for (uint32_t y = y0; y < y1; ++y)
                m = max(m, (uint32_t)(__ldcg(keys + (uint64_t)y * (uint32_t)W + x) >> 32));
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0)
            T.bound[t] = ((unsigned long long)T.tag << 32) | m;
    }
}

}  // namespace mmr
