// Kernels of the single-cloud path: fused displace + project + splat over the
// points, and resolve + clear over the pixels.
//
// Point kernel layout: each thread owns a group of points whose storage is
// exactly 48 bytes (4 FP32 points or 8 16-bit points), read and written as
// three 16-byte vectors, so a warp moves 1536 contiguous bytes per direction.
// Positions are streamed (evict-first) so the depth-id buffer, which is the
// data reused within a frame, keeps its place in L2.
#include <cuda_runtime.h>

#include "mmr_device.cuh"
#include "mmr_internal.h"

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

template <int DT, bool kDisplace, bool kSplat>
__global__ void points_kernel(void *__restrict__ pos, uint32_t n, PointParams P)
{
    constexpr int G = Group<DT>::kPoints;
    const uint32_t full = n / G;
    const uint32_t groups = (n + G - 1) / G;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const uint32_t i0 = g * G;
        float v[3 * G];
        if (g < full) {
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
            // ragged tail: fewer than G points, scalar accesses
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
}

// Resolve + clear: four pixels per thread.  RGBA = background for an empty
// key, else colors[id] (or the default colour); the other depth-id buffer,
// which the next frame splats into, is reset to all-ones in the same pass.
__global__ void resolve_kernel(const unsigned long long *__restrict__ keys,
                               unsigned long long *__restrict__ next_keys,
                               uint32_t *__restrict__ rgba, const uint32_t *__restrict__ colors,
                               uint32_t npx, uint32_t color, uint32_t background)
{
    const uint32_t quads = npx / 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += stride) {
        const ulonglong2 k01 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q);
        const ulonglong2 k23 = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q + 1);
        const unsigned long long k[4] = {k01.x, k01.y, k23.x, k23.y};
        uint32_t c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k[j] == kEmptyKey)
                c[j] = background;
            else
                c[j] = colors ? __ldg(colors + (uint32_t)(k[j] & 0xffffffffu)) : color;
        }
        __stcs(reinterpret_cast<uint4 *>(rgba) + q, make_uint4(c[0], c[1], c[2], c[3]));
        const ulonglong2 e = make_ulonglong2(kEmptyKey, kEmptyKey);
        reinterpret_cast<ulonglong2 *>(next_keys)[2 * q] = e;
        reinterpret_cast<ulonglong2 *>(next_keys)[2 * q + 1] = e;
    }
    // ragged tail (npx not a multiple of 4): handled by the first threads
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t p = quads * 4 + t;
    if (p < npx) {
        const unsigned long long k = keys[p];
        rgba[p] = k == kEmptyKey ? background
                                 : (colors ? colors[(uint32_t)(k & 0xffffffffu)] : color);
        next_keys[p] = kEmptyKey;
    }
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
    const uint64_t groups = (n + Group<DT>::kPoints - 1) / Group<DT>::kPoints;
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
