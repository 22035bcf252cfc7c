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
__device__ __forceinline__ void splat_disc(float sx, float sy, unsigned long long key, const PointParams &P)
{
    constexpr float kMargin = 0.0625f;
    const float cx = __fsub_rn(sx, 0.5f), cy = __fsub_rn(sy, 0.5f);
    const int x0 = max(__float2int_ru(__fsub_rn(__fsub_rn(cx, P.disc_r), kMargin)), 0);
    const int x1 = min(__float2int_rd(__fadd_rn(__fadd_rn(cx, P.disc_r), kMargin)), P.W - 1);
    const int y0 = max(__float2int_ru(__fsub_rn(__fsub_rn(cy, P.disc_r), kMargin)), 0);
    const int y1 = min(__float2int_rd(__fadd_rn(__fadd_rn(cy, P.disc_r), kMargin)), P.H - 1);
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

}  // namespace mmr
