// Per-thread point processing shared by the single-cloud and batched
// kernels.  Each thread owns a group of points whose storage is exactly 48
// bytes (4 FP32 points or 8 16-bit points), read and written as three
// 16-byte vectors, so a warp moves 1536 contiguous bytes per direction.
// Positions are streamed (evict-first) so the depth-id buffer, which is the
// data reused within a frame, keeps its place in L2.
#pragma once

#include "mmr_device.cuh"

namespace mmr {

template <int DT>
struct Group;

template <>
struct Group<kF32> {
    static constexpr int kPoints = 4;
};

template <>
struct Group<kF16> {
    static constexpr int kPoints = 8;
};

template <>
struct Group<kBF16> {
    static constexpr int kPoints = 8;
};

// How a projected point reaches the depth-id buffer.  A point kernel body
// calls its splat policy for every point that projected into the frame, with
// the pixel's column and row and the key; a policy whose kWarpWide is true is
// called for every point, with ok = whether it projected (all lanes of a warp
// call it together, which warp-level policies rely on).  A kernel calls
// on_entry() once per thread before its first point.  The default policy is
// the depth-tested splat of mmr_device.cuh.
struct SplatDirect {
    static constexpr bool kWarpWide = false;

    __device__ __forceinline__ void on_entry() const {}

    __device__ __forceinline__ void operator()(const PointParams &P, bool, uint32_t ix, uint32_t iy,
                                               unsigned long long key) const
    {
        splat_key(P.keys, iy * (uint32_t)P.W + ix, key);
    }
};

// One projected point through a splat policy (see above).
template <typename Splat>
__device__ __forceinline__ void splat_point(const Splat &splat, const PointParams &P, bool in_range, float x,
                                            float y, float z, uint32_t id)
{
    uint32_t ix = 0, iy = 0;
    float cw = 0.0f;
    if constexpr (Splat::kWarpWide) {
        const bool ok = in_range && project_pixel(x, y, z, P, ix, iy, cw);
        splat(P, ok, ix, iy, depth_key(cw, id));
    } else {
        if (in_range && project_pixel(x, y, z, P, ix, iy, cw))
            splat(P, true, ix, iy, depth_key(cw, id));
    }
}

// Two points through a splat policy, projected together (project_pixel2);
// the same calls, in the same order, as splat_point on each.
template <typename Splat>
__device__ __forceinline__ void splat_pair(const Splat &splat, const PointParams &P, bool in_a, float xa, float ya,
                                           float za, uint32_t ida, bool in_b, float xb, float yb, float zb,
                                           uint32_t idb)
{
    bool oka, okb;
    uint32_t ixa, iya, ixb, iyb;
    float cwa, cwb;
    project_pixel2(xa, ya, za, xb, yb, zb, P, oka, ixa, iya, cwa, okb, ixb, iyb, cwb);
    oka = oka && in_a;
    okb = okb && in_b;
    if constexpr (Splat::kWarpWide) {
        splat(P, oka, ixa, iya, depth_key(cwa, ida));
        splat(P, okb, ixb, iyb, depth_key(cwb, idb));
    } else {
        if (oka)
            splat(P, true, ixa, iya, depth_key(cwa, ida));
        if (okb)
            splat(P, true, ixb, iyb, depth_key(cwb, idb));
    }
}

template <int DT>
__device__ __forceinline__ float load_coord(const void *pos, uint64_t k)
{
    if constexpr (DT == kF32)
        return reinterpret_cast<const float *>(pos)[k];
    else
        return widen<DT>(reinterpret_cast<const uint16_t *>(pos)[k]);
}

template <int DT>
__device__ __forceinline__ void store_coord(void *pos, uint64_t k, float f)
{
    if constexpr (DT == kF32)
        reinterpret_cast<float *>(pos)[k] = f;
    else
        reinterpret_cast<uint16_t *>(pos)[k] = narrow<DT>(f);
}

// Storage rounding of a freshly displaced coordinate: what the buffer will
// hold, widened back to FP32, is what gets projected, so rendering the
// buffer later gives the same frame.
template <int DT>
__device__ __forceinline__ float storage_round(float f)
{
    if constexpr (DT == kF32)
        return f;
    else
        return widen<DT>(narrow<DT>(f));
}

// The ragged tail: points i0 .. n-1 of the last, partial group, with scalar
// accesses (the vector path would read past n).  Reads src, writes dst
// (the same buffer for an in-place step).  One thread does this, so it
// always takes the direct splat.
template <int DT, bool kDisplace, bool kSplat>
__device__ __forceinline__ void process_tail(const void *src, void *dst, uint32_t n, uint32_t i0,
                                             const PointParams &P)
{
    for (uint32_t i = i0; i < n; ++i) {
        float x = load_coord<DT>(src, 3ull * i);
        float y = load_coord<DT>(src, 3ull * i + 1);
        float z = load_coord<DT>(src, 3ull * i + 2);
        if constexpr (kDisplace) {
            displace_point(x, y, z, i, P);
            x = storage_round<DT>(x);
            y = storage_round<DT>(y);
            z = storage_round<DT>(z);
            store_coord<DT>(dst, 3ull * i, x);
            store_coord<DT>(dst, 3ull * i + 1, y);
            store_coord<DT>(dst, 3ull * i + 2, z);
        }
        if constexpr (kSplat) {
            uint32_t px;
            unsigned long long key;
            if (project_key(x, y, z, P.id_base + i, P, px, key))
                splat_key(P.keys, px, key);
        }
    }
}

// Group g (48 bytes) as three 16-byte streamed (evict-first) accesses.
__device__ __forceinline__ void load_words(const void *pos, uint32_t g, uint4 (&q)[3])
{
    const uint4 *p4 = reinterpret_cast<const uint4 *>(pos) + 3ull * g;
    q[0] = __ldcs(p4 + 0);
    q[1] = __ldcs(p4 + 1);
    q[2] = __ldcs(p4 + 2);
}

__device__ __forceinline__ void store_words(void *pos, uint32_t g, const uint4 (&q)[3])
{
    uint4 *p4 = reinterpret_cast<uint4 *>(pos) + 3ull * g;
    __stcs(p4 + 0, q[0]);
    __stcs(p4 + 1, q[1]);
    __stcs(p4 + 2, q[2]);
}

// The points of one 48-byte group held as three 16-byte words (as loaded
// from global or shared memory): displace in place and/or splat the first
// `count` points (count == G except in the ragged last group).
template <int DT>
__device__ __forceinline__ float word_coord(const uint4 (&q)[3], int k)
{
    if constexpr (DT == kF32)
        return __uint_as_float(reinterpret_cast<const uint32_t *>(q)[k]);
    else
        return widen<DT>(reinterpret_cast<const uint16_t *>(q)[k]);
}

template <int DT>
__device__ __forceinline__ void set_word_coord(uint4 (&q)[3], int k, float f)
{
    if constexpr (DT == kF32)
        reinterpret_cast<uint32_t *>(q)[k] = __float_as_uint(f);
    else
        reinterpret_cast<uint16_t *>(q)[k] = narrow<DT>(f);
}

// A full 16-bit group in two phases that keep only the packed words live
// between them: displace (widen, move, narrow once into the word) and, after
// the caller has stored the words, project and splat (widen again).  The 24
// widened coordinates never occupy registers together, so the 16-bit kernel
// fits 40 registers without spilling.
template <int DT>
__device__ __forceinline__ void displace_packed(uint4 (&q)[3], uint32_t i0, const PointParams &P)
{
    static_assert(DT != kF32, "16-bit groups only");
    constexpr int G = Group<DT>::kPoints;
#pragma unroll
    for (int j = 0; j < G; ++j) {
        float x = word_coord<DT>(q, 3 * j), y = word_coord<DT>(q, 3 * j + 1), z = word_coord<DT>(q, 3 * j + 2);
        displace_point(x, y, z, i0 + j, P);
        set_word_coord<DT>(q, 3 * j, x);
        set_word_coord<DT>(q, 3 * j + 1, y);
        set_word_coord<DT>(q, 3 * j + 2, z);
    }
}

template <int DT, typename Splat = SplatDirect>
__device__ __forceinline__ void splat_packed(const uint4 (&q)[3], uint32_t i0, const PointParams &P,
                                             const Splat &splat = Splat{})
{
    static_assert(DT != kF32, "16-bit groups only");
    constexpr int G = Group<DT>::kPoints;
#pragma unroll
    for (int j = 0; j < G; ++j)
        splat_point(splat, P, true, word_coord<DT>(q, 3 * j), word_coord<DT>(q, 3 * j + 1),
                    word_coord<DT>(q, 3 * j + 2), P.id_base + i0 + j);
}

// kPairs (FP32): displace and project the points two at a time on packed
// FP32 pairs (displace_pair, project_pixel2): fewer instructions, more
// registers.
template <int DT, bool kDisplace, bool kSplat, typename Splat = SplatDirect, bool kPairs = false>
__device__ __forceinline__ void process_words(uint4 (&q)[3], uint32_t i0, uint32_t count, const PointParams &P,
                                              const Splat &splat = Splat{})
{
    constexpr int G = Group<DT>::kPoints;
    float v[3 * G];
#pragma unroll
    for (int k = 0; k < 3 * G; ++k)
        v[k] = word_coord<DT>(q, k);
    if constexpr (kDisplace && kPairs && DT == kF32) {
        // two points at a time (displace_pair); a point past `count` is displaced but not kept
#pragma unroll
        for (int j = 0; j < G; j += 2) {
            float w[6] = {v[3 * j], v[3 * j + 1], v[3 * j + 2], v[3 * j + 3], v[3 * j + 4], v[3 * j + 5]};
            displace_pair(w[0], w[1], w[2], i0 + j, w[3], w[4], w[5], i0 + j + 1, P);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                if ((uint32_t)(j + c / 3) < count) {
                    v[3 * j + c] = w[c];
                    set_word_coord<DT>(q, 3 * j + c, w[c]);
                }
            }
        }
    } else if constexpr (kDisplace) {
#pragma unroll
        for (int j = 0; j < G; ++j) {       // constant indices keep q and v in registers
            if ((uint32_t)j < count) {
                displace_point(v[3 * j], v[3 * j + 1], v[3 * j + 2], i0 + j, P);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    v[3 * j + c] = storage_round<DT>(v[3 * j + c]);
                    set_word_coord<DT>(q, 3 * j + c, v[3 * j + c]);
                }
            }
        }
    }
    if constexpr (kSplat) {
        if constexpr (kPairs) {
#pragma unroll
            for (int j = 0; j < G; j += 2)
                splat_pair(splat, P, (uint32_t)j < count, v[3 * j], v[3 * j + 1], v[3 * j + 2], P.id_base + i0 + j,
                           (uint32_t)j + 1 < count, v[3 * j + 3], v[3 * j + 4], v[3 * j + 5],
                           P.id_base + i0 + j + 1);
        } else {
#pragma unroll
            for (int j = 0; j < G; ++j)
                splat_point(splat, P, (uint32_t)j < count, v[3 * j], v[3 * j + 1], v[3 * j + 2],
                            P.id_base + i0 + j);
        }
    }
}

// Groups covering n points, the last one possibly partial.  The sum is taken
// in 64 bits: n may be as large as 2^32 - 1, where n + G - 1 would wrap.
template <int DT>
__host__ __device__ constexpr uint32_t groups_of(uint32_t n)
{
    return (uint32_t)(((uint64_t)n + Group<DT>::kPoints - 1) / Group<DT>::kPoints);
}

}  // namespace mmr
