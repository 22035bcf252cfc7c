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

template <int DT>
__device__ __forceinline__ void load_group(const void *pos, uint32_t g, float *v)
{
    const uint4 *p4 = reinterpret_cast<const uint4 *>(pos) + 3ull * g;
    uint4 q[3];
    q[0] = __ldcs(p4 + 0);
    q[1] = __ldcs(p4 + 1);
    q[2] = __ldcs(p4 + 2);
    if constexpr (DT == kF32) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(q);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            v[k] = __uint_as_float(w[k]);
    } else {
        const uint16_t *h = reinterpret_cast<const uint16_t *>(q);
#pragma unroll
        for (int k = 0; k < 24; ++k)
            v[k] = widen<DT>(h[k]);
    }
}

template <int DT>
__device__ __forceinline__ void store_group(void *pos, uint32_t g, const float *v)
{
    uint4 q[3];
    if constexpr (DT == kF32) {
        uint32_t *w = reinterpret_cast<uint32_t *>(q);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            w[k] = __float_as_uint(v[k]);
    } else {
        uint16_t *h = reinterpret_cast<uint16_t *>(q);
#pragma unroll
        for (int k = 0; k < 24; ++k)
            h[k] = narrow<DT>(v[k]);
    }
    uint4 *p4 = reinterpret_cast<uint4 *>(pos) + 3ull * g;
    __stcs(p4 + 0, q[0]);
    __stcs(p4 + 1, q[1]);
    __stcs(p4 + 2, q[2]);
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

// One thread's share of a point buffer: group g (G points, 48 bytes), or
// the ragged tail of fewer than G points with scalar accesses.
template <int DT, bool kDisplace, bool kSplat>
__device__ __forceinline__ void process_group(void *__restrict__ pos, uint32_t n, uint32_t g,
                                              const PointParams &P)
{
    constexpr int G = Group<DT>::kPoints;
    const uint32_t full = n / G;
    const uint32_t i0 = g * G;
    if (g < full) {
        float v[3 * G];
        load_group<DT>(pos, g, v);
        if constexpr (kDisplace) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                displace_point(v[3 * j], v[3 * j + 1], v[3 * j + 2], i0 + j, P);
                v[3 * j + 0] = storage_round<DT>(v[3 * j + 0]);
                v[3 * j + 1] = storage_round<DT>(v[3 * j + 1]);
                v[3 * j + 2] = storage_round<DT>(v[3 * j + 2]);
            }
            store_group<DT>(pos, g, v);
        }
        if constexpr (kSplat) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                uint32_t px;
                unsigned long long key;
                if (project_key(v[3 * j], v[3 * j + 1], v[3 * j + 2], P.id_base + i0 + j, P, px, key))
                    splat_key(P.keys, px, key);
            }
        }
    } else {
        for (uint32_t i = i0; i < n; ++i) {
            float x = load_coord<DT>(pos, 3ull * i);
            float y = load_coord<DT>(pos, 3ull * i + 1);
            float z = load_coord<DT>(pos, 3ull * i + 2);
            if constexpr (kDisplace) {
                displace_point(x, y, z, i, P);
                x = storage_round<DT>(x);
                y = storage_round<DT>(y);
                z = storage_round<DT>(z);
                store_coord<DT>(pos, 3ull * i, x);
                store_coord<DT>(pos, 3ull * i + 1, y);
                store_coord<DT>(pos, 3ull * i + 2, z);
            }
            if constexpr (kSplat) {
                uint32_t px;
                unsigned long long key;
                if (project_key(x, y, z, P.id_base + i, P, px, key))
                    splat_key(P.keys, px, key);
            }
        }
    }
}

template <int DT>
__host__ __device__ constexpr uint32_t groups_of(uint32_t n)
{
    return (n + Group<DT>::kPoints - 1) / Group<DT>::kPoints;
}

}  // namespace mmr
