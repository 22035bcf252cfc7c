// Kernels of the single-cloud path: fused displace + project + splat over the
// points (grid-stride over 48-byte point groups); the resolve is in
// mmr_resolve.cu.
#include <algorithm>
#include <type_traits>

#include <cuda_runtime.h>

#include "mmr_device.cuh"
#include "mmr_disc.cuh"
#include "mmr_internal.h"
#include "mmr_launch.cuh"
#include "mmr_points.cuh"
#include "mmr_resolve.cuh"
#include "mmr_tiles.cuh"
#include "mmr_tma.cuh"

namespace mmr {

// Grid-stride over the 48-byte point groups g_begin .. g_end - 1.  On FP32
// storage each thread prefetches its next group into registers before working
// on the current one, so a load is always in flight while the thread computes.
// Positions are read from src and the displaced ones written to dst: the same
// buffer for an in-place step, the other ping-pong buffer otherwise.  Groups
// at or past n / G hold the ragged tail (only the last group can).
template <int DT, bool kDisplace, bool kSplat, typename Splat>
__device__ __forceinline__ void points_body(const void *src, void *dst, uint32_t n, uint32_t g_begin,
                                            uint32_t g_end, const PointParams &P, const Splat &splat)
{
    constexpr int G = Group<DT>::kPoints;
    constexpr bool kPrefetch = (DT == kF32);
    const uint32_t full = min(n / G, g_end);
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t g = g_begin + blockIdx.x * blockDim.x + threadIdx.x;
    uint4 next[3];
    if (kPrefetch && g < full)
        load_words(src, g, next);
    while (g < g_end) {
        const uint32_t gn = g + stride;
        if (g < full) {
            uint4 q[3];
            if constexpr (kPrefetch) {
                q[0] = next[0];
                q[1] = next[1];
                q[2] = next[2];
                if (gn < full)
                    load_words(src, gn, next);
            } else {
                load_words(src, g, q);
            }
            if constexpr (DT == kF32) {
                process_words<DT, kDisplace, kSplat, Splat, true>(q, g * G, G, P, splat);
                if constexpr (kDisplace)
                    store_words(dst, g, q);
            } else {
                // stored before the splat (measured slower for FP32: 417 -> 427 us on the 64M-point 4K frame)
                if constexpr (kDisplace) {
                    displace_packed<DT>(q, g * G, P);
                    store_words(dst, g, q);
                }
                if constexpr (kSplat)
                    splat_packed<DT>(q, g * G, P, splat);
            }
        } else {
            process_tail<DT, kDisplace, kSplat>(src, dst, n, g * G, P);
        }
        g = gn;
    }
}

// FP32 storage.  Points are projected two at a time on packed FP32 pairs
// (project_pixel2): 62 registers uncapped; under a cap of 60 the compiler
// finds 55 without spilling (at 56 it spills 8 bytes).  Measured on the
// 64M-point 16-cluster 4K frame against the one-point projection at 47
// registers, on one box: 444.5 -> 408.9 us (cap 56: 408.0 us with the spill,
// cap 64: 414.3 us); the 2^22-point 1080p frame 43.8 -> 42.9 us.  Pairing the
// displacement's offsets too (displace_pair), still 55 registers: 408.5 ->
// 405.0 us and 43.1 -> 42.3 us on another box.
// Groups g_begin .. g_end - 1; `splat` is the splat policy (mmr_points.cuh,
// mmr_tiles.cuh).
template <bool kDisplace, bool kSplat, typename Splat>
__global__ void __maxnreg__(60) points_kernel(const void *src, void *dst, uint32_t n, uint32_t g_begin, uint32_t g_end,
                              PointParams P, Splat splat)
{
    enter_dependent_grid();
    splat.on_entry();
    points_body<kF32, kDisplace, kSplat>(src, dst, n, g_begin, g_end, P, splat);
}

// 16-bit storage.  A group holds 8 points, twice the work per load, so the
// prefetch's 12 registers are better spent on resident warps.  Without it, and
// with only the packed words live between displacement and splat, the kernel
// fits a cap of 40 registers (48 warps per SM) without spilling; 36 spills.
// The displace-only form (host round trip) keeps 48: at 40 it spills 4 bytes.
// Measured on the 64M-point 4K frame against 48 registers with all widened
// coordinates kept: binary16 348.4 -> 347.1 us, bfloat16 355.6 -> 351.7 us.
// A register cap, unlike a launch bound, leaves every block size up to 1024
// valid.
template <int DT, bool kDisplace, bool kSplat, typename Splat>
__global__ void __maxnreg__(kSplat ? 40 : 48) points_kernel_narrow(const void *src, void *dst, uint32_t n,
                                                                   uint32_t g_begin, uint32_t g_end, PointParams P,
                                                                   Splat splat)
{
    enter_dependent_grid();
    splat.on_entry();
    points_body<DT, kDisplace, kSplat>(src, dst, n, g_begin, g_end, P, splat);
}

// The depth bounds of the tiles the first pass marked (mmr_tiles.cuh).
__global__ void tile_bound_kernel(const unsigned long long *__restrict__ keys, int W, int H, TileBounds T)
{
    enter_dependent_grid();
    tile_bound_body(keys, W, H, T);
}

// Disc markers: as points_kernel (one thread per 48-byte group, groups
// g_begin .. g_end - 1), each point splatted as a disc of radius P.disc_r
// pixels instead of one pixel, by its own thread.
template <int DT, bool kDisplace>
__global__ void points_disc_kernel(const void *src, void *dst, uint32_t n, uint32_t g_begin, uint32_t g_end,
                                   PointParams P)
{
    enter_dependent_grid();
    constexpr int G = Group<DT>::kPoints;
    const uint32_t full = n / G;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = g_begin + blockIdx.x * blockDim.x + threadIdx.x; g < g_end; g += stride) {
        const uint32_t i0 = g * G;
        const uint32_t count = min((uint32_t)G, n - i0);
        uint4 q[3];
        float v[3 * G];
        if (g < full) {
            load_words(src, g, q);
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                v[k] = word_coord<DT>(q, k);
        } else {
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                v[k] = (uint32_t)(k / 3) < count ? load_coord<DT>(src, 3ull * i0 + k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if ((uint32_t)j >= count)
                continue;
            if constexpr (kDisplace) {
                displace_point(v[3 * j], v[3 * j + 1], v[3 * j + 2], i0 + j, P);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    v[3 * j + c] = storage_round<DT>(v[3 * j + c]);
            }
            float sx, sy, cw;
            if (project_screen(v[3 * j], v[3 * j + 1], v[3 * j + 2], P, sx, sy, cw))
                splat_disc(sx, sy, depth_key(cw, P.id_base + i0 + j), P);
        }
        if constexpr (kDisplace) {
            if (g < full) {
#pragma unroll
                for (int k = 0; k < 3 * G; ++k)
                    set_word_coord<DT>(q, k, v[k]);
                store_words(dst, g, q);
            } else {
#pragma unroll
                for (int k = 0; k < 3 * G; ++k)
                    if ((uint32_t)k < 3 * count)
                        store_coord<DT>(dst, 3ull * i0 + k, v[k]);
            }
        }
    }
}

// The culled disc pass: as points_disc_kernel, but the grid-stride loop
// advances whole warps together (lane l of a warp takes group base + l, lanes
// past g_end take no points), so every lane of a warp is present when the
// discs that survive the tile bounds are splatted by the whole warp
// (splat_discs_by_warp).  Discs behind their tiles' bounds are dropped.
template <int DT, bool kDisplace>
__global__ void points_disc_culled_kernel(const void *src, void *dst, uint32_t n, uint32_t g_begin, uint32_t g_end,
                                          PointParams P, DiscBounds T)
{
    enter_dependent_grid();
    constexpr int G = Group<DT>::kPoints;
    const uint32_t full = n / G;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t gw = g_begin + blockIdx.x * blockDim.x + (threadIdx.x & ~31u); gw < g_end; gw += stride) {
        const uint32_t g = gw + lane;
        const uint32_t i0 = g * G;
        const uint32_t count = g < g_end ? min((uint32_t)G, n - i0) : 0u;
        uint4 q[3];
        float v[3 * G];
        if (g < full && g < g_end) {
            load_words(src, g, q);
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                v[k] = word_coord<DT>(q, k);
        } else {
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                v[k] = (uint32_t)(k / 3) < count ? load_coord<DT>(src, 3ull * i0 + k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const bool in = (uint32_t)j < count;
            if constexpr (kDisplace) {
                if (in) {
                    displace_point(v[3 * j], v[3 * j + 1], v[3 * j + 2], i0 + j, P);
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        v[3 * j + c] = storage_round<DT>(v[3 * j + c]);
                }
            }
            float sx = 0.0f, sy = 0.0f, cw = 0.0f;
            bool draw = in && project_screen(v[3 * j], v[3 * j + 1], v[3 * j + 2], P, sx, sy, cw);
            DiscBox box{1, 0, 1, 0};
            if (draw) {
                box = disc_box(sx, sy, P);
                draw = !disc_behind_bounds(box, __float_as_uint(cw), T);
            }
            splat_discs_by_warp(draw, sx, sy, depth_key(cw, P.id_base + i0 + j), box, P);
        }
        if constexpr (kDisplace) {
            if (g < full && g < g_end) {
#pragma unroll
                for (int k = 0; k < 3 * G; ++k)
                    set_word_coord<DT>(q, k, v[k]);
                store_words(dst, g, q);
            } else {
#pragma unroll
                for (int k = 0; k < 3 * G; ++k)
                    if ((uint32_t)k < 3 * count)
                        store_coord<DT>(dst, 3ull * i0 + k, v[k]);
            }
        }
    }
}

// The depth bounds of every 32x32 tile, for the culled disc pass.
__global__ void disc_tile_bound_kernel(const unsigned long long *__restrict__ keys, int W, int H, DiscBounds T)
{
    enter_dependent_grid();
    disc_tile_bound_body(keys, W, H, T);
}

template <int DT, bool kCull>
static cudaError_t launch_disc_range(const void *src, void *dst, uint32_t n, uint32_t g_begin, uint32_t g_end,
                                     const PointParams &P, bool displace, const DiscBounds &T, cudaStream_t s)
{
    const uint64_t groups = g_end - g_begin;
    const int grid = (int)std::max<uint64_t>(1, (groups + 63) / 64);
    if constexpr (kCull) {
        if (displace)
            return launch_dependent(points_disc_culled_kernel<DT, true>, grid, 64, s, src, dst, n, g_begin, g_end, P,
                                    T);
        return launch_dependent(points_disc_culled_kernel<DT, false>, grid, 64, s, src, dst, n, g_begin, g_end, P, T);
    } else {
        if (displace)
            return launch_dependent(points_disc_kernel<DT, true>, grid, 64, s, src, dst, n, g_begin, g_end, P);
        return launch_dependent(points_disc_kernel<DT, false>, grid, 64, s, src, dst, n, g_begin, g_end, P);
    }
}

template <int DT>
static cudaError_t launch_disc_dt(const void *src, void *dst, uint32_t n, const PointParams &P, bool displace,
                                  const DiscBounds *T, int bound_shift, int sm_count, cudaStream_t s)
{
    const uint32_t groups = groups_of<DT>(n);
    if (!T)
        return launch_disc_range<DT, false>(src, dst, n, 0, groups, P, displace, DiscBounds{}, s);
    const uint32_t ga = groups >> bound_shift;
    cudaError_t e = launch_disc_range<DT, false>(src, dst, n, 0, ga, P, displace, *T, s);
    if (e != cudaSuccess)
        return e;
    const uint64_t tiles = (uint64_t)T->tiles_w * T->tiles_h;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((tiles + 7) / 8, (uint64_t)sm_count * 16));
    e = launch_dependent(disc_tile_bound_kernel, grid, 256, s, (const unsigned long long *)P.keys, P.W, P.H, *T);
    if (e != cudaSuccess)
        return e;
    return launch_disc_range<DT, true>(src, dst, n, ga, groups, P, displace, *T, s);
}

cudaError_t launch_points_disc(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                               bool displace, const DiscBounds *T, int bound_shift, int sm_count, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    switch (dtype) {
    case kF32: return launch_disc_dt<kF32>(src, dst, n, P, displace, T, bound_shift, sm_count, s);
    case kF16: return launch_disc_dt<kF16>(src, dst, n, P, displace, T, bound_shift, sm_count, s);
    case kBF16: return launch_disc_dt<kBF16>(src, dst, n, P, displace, T, bound_shift, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

// Persistent, TMA-staged variant of points_kernel.  The point buffer is cut
// into tiles of kThreads 48-byte groups (12 KB at 256 threads); CTA b owns
// tiles b, b + grid, b + 2 grid, ...  Thread 0 keeps kStages tiles in flight
// with 1D bulk copies into shared memory, each completing on its own
// mbarrier.  Every thread reads its group from shared memory (16-byte
// accesses at a 48-byte stride: conflict-free), updates it in place and
// splats; thread 0 then bulk-stores the tile back and refills the stage with
// the CTA's next tile.  Global memory is touched only by whole-tile bulk
// copies, so loads and stores are fully coalesced and many kilobytes per SM
// are in flight.  Requires the buffer padded to whole groups (the library's
// own allocations are).  Waits give up after kWaitCycles; the CTA then
// raises *err and returns without storing.
constexpr long long kWaitCycles = 1ll << 31;
constexpr int kTmaStages = 4;

template <int kThreads>
constexpr uint32_t tma_smem_bytes()
{
    return kTmaStages * kThreads * 48u + kTmaStages * 8u;
}

template <int DT, bool kDisplace, bool kSplat, int kThreads>
__global__ void __launch_bounds__(kThreads) points_tma_kernel(const void *src, void *dst, uint32_t n, PointParams P,
                                                              uint32_t *__restrict__ err)
{
    constexpr int G = Group<DT>::kPoints;
    constexpr uint32_t kTileBytes = kThreads * 48u;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kTmaStages * kTileBytes);
    const uint32_t tid = threadIdx.x;
    const uint32_t total_groups = groups_of<DT>(n);
    const uint32_t tiles = (total_groups + kThreads - 1) / kThreads;
    if (blockIdx.x >= tiles)
        return;
    const uint32_t my_tiles = (tiles - 1 - blockIdx.x) / gridDim.x + 1;
    const char *gsrc = static_cast<const char *>(src);
    char *gdst = static_cast<char *>(dst);
    auto tile_of = [&](uint32_t k) { return blockIdx.x + k * gridDim.x; };
    auto bytes_of = [&](uint32_t tile) { return min((uint32_t)kThreads, total_groups - tile * kThreads) * 48u; };

    if (tid == 0) {
        for (int st = 0; st < kTmaStages; ++st)
            mbar_init(smem_addr(&bars[st]), 1);
        mbar_init_fence();
        for (uint32_t k = 0; k < my_tiles && k < (uint32_t)kTmaStages; ++k) {
            const uint32_t tile = tile_of(k), bytes = bytes_of(tile), bar = smem_addr(&bars[k]);
            mbar_arrive_expect_tx(bar, bytes);
            bulk_load(smem_addr(smem + k * kTileBytes), gsrc + (size_t)tile * kTileBytes, bytes, bar);
        }
    }
    __syncthreads();

    for (uint32_t k = 0; k < my_tiles; ++k) {
        const uint32_t st = k % kTmaStages;
        const uint32_t tile = tile_of(k);
        unsigned char *stage = smem + st * kTileBytes;
        const bool ok = mbar_wait_bounded(smem_addr(&bars[st]), (k / kTmaStages) & 1u, kWaitCycles);
        const uint32_t g = tile * kThreads + tid;
        if (ok && g < total_groups) {
            uint4 q[3];
            uint4 *mine = reinterpret_cast<uint4 *>(stage + tid * 48u);
            q[0] = mine[0];
            q[1] = mine[1];
            q[2] = mine[2];
            const uint32_t i0 = g * G;
            process_words<DT, kDisplace, kSplat>(q, i0, min((uint32_t)G, n - i0), P);
            if constexpr (kDisplace) {
                mine[0] = q[0];
                mine[1] = q[1];
                mine[2] = q[2];
            }
        }
        if constexpr (kDisplace)
            fence_proxy_async_smem();
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(err, 1u);
                if constexpr (kDisplace)
                    bulk_wait_all();
            }
            return;
        }
        if (tid == 0) {
            if constexpr (kDisplace) {
                bulk_store(gdst + (size_t)tile * kTileBytes, smem_addr(stage), bytes_of(tile));
                bulk_commit();
            }
            const uint32_t kn = k + kTmaStages;
            if (kn < my_tiles) {
                if constexpr (kDisplace)
                    bulk_wait_read_all();       // the store has left the stage
                const uint32_t tn = tile_of(kn), bytes = bytes_of(tn), bar = smem_addr(&bars[st]);
                mbar_arrive_expect_tx(bar, bytes);
                bulk_load(smem_addr(stage), gsrc + (size_t)tn * kTileBytes, bytes, bar);
            }
        }
    }
    if constexpr (kDisplace) {
        if (tid == 0)
            bulk_wait_all();
    }
}

// Self-test of the bounded wait used by the TMA kernel: wait on an mbarrier
// that nothing ever arrives on, give up after max_cycles and report it the
// same way the point kernel does.
__global__ void bounded_wait_selftest_kernel(long long max_cycles, uint32_t *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(smem_addr(&bar), 0, max_cycles);
    if (!__syncthreads_and(ok) && threadIdx.x == 0)
        atomicOr(err, 1u);
}

cudaError_t launch_bounded_wait_selftest(long long max_cycles, uint32_t *err, cudaStream_t s)
{
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(max_cycles, err);
    return cudaGetLastError();
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

template <int DT, typename Splat>
static cudaError_t launch_points_range(const void *src, void *dst, uint32_t n, uint32_t g_begin, uint32_t g_end,
                                       const PointParams &P, bool displace, bool splat_on, const Splat &splat,
                                       const LaunchShape &ls, cudaStream_t s)
{
    const int grid = grid_for(g_end - g_begin, ls);
    if constexpr (!std::is_same<Splat, SplatDirect>::value) {
        // the other policies only ever run with displacement and splat, or splat alone
        if (!splat_on)
            return cudaErrorInvalidValue;
    }
    if constexpr (DT == kF32) {
        if (displace && splat_on)
            return launch_dependent(points_kernel<true, true, Splat>, grid, ls.threads, s, src, dst, n, g_begin, g_end,
                                    P, splat);
        if constexpr (std::is_same<Splat, SplatDirect>::value) {
            if (displace)
                return launch_dependent(points_kernel<true, false, Splat>, grid, ls.threads, s, src, dst, n, g_begin,
                                        g_end, P, splat);
        }
        return launch_dependent(points_kernel<false, true, Splat>, grid, ls.threads, s, src, dst, n, g_begin, g_end,
                                P, splat);
    } else {
        if (displace && splat_on)
            return launch_dependent(points_kernel_narrow<DT, true, true, Splat>, grid, ls.threads, s, src, dst, n,
                                    g_begin, g_end, P, splat);
        if constexpr (std::is_same<Splat, SplatDirect>::value) {
            if (displace)
                return launch_dependent(points_kernel_narrow<DT, true, false, Splat>, grid, ls.threads, s, src, dst,
                                        n, g_begin, g_end, P, splat);
        }
        return launch_dependent(points_kernel_narrow<DT, false, true, Splat>, grid, ls.threads, s, src, dst, n,
                                g_begin, g_end, P, splat);
    }
}

template <int DT>
static cudaError_t launch_points_dt(const void *src, void *dst, uint32_t n, const PointParams &P, bool displace,
                                    bool splat, const LaunchShape &ls, cudaStream_t s)
{
    const uint32_t groups = groups_of<DT>(n);
    if (splat && ls.kernel == kKernelWarpAgg)
        return launch_points_range<DT>(src, dst, n, 0, groups, P, displace, true, SplatWarpAggregated{}, ls, s);
    return launch_points_range<DT>(src, dst, n, 0, groups, P, displace, splat, SplatDirect{}, ls, s);
}

// Depth-bounded frame: the first groups_a groups with the marking splat, the
// bound kernel over the marked tiles, then the remaining groups with the
// bounded splat.
template <int DT>
static cudaError_t launch_points_bounded_dt(const void *src, void *dst, uint32_t n, const PointParams &P,
                                            bool displace, const TileBounds &T, uint32_t tiles,
                                            const LaunchShape &ls, cudaStream_t s)
{
    const uint32_t groups = groups_of<DT>(n);
    const uint32_t ga = groups >> ls.bound_shift;
    cudaError_t e = launch_points_range<DT>(src, dst, n, 0, ga, P, displace, true, SplatMarkTiles{T}, ls, s);
    if (e != cudaSuccess)
        return e;
    // one warp per marked tile: the grid covers every tile in the worst case, capped at 16 CTAs per SM
    const int warps_per_cta = 8;
    const uint64_t need = ((uint64_t)tiles + warps_per_cta - 1) / warps_per_cta;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)ls.sm_count * 16));
    e = launch_dependent(tile_bound_kernel, grid, 32 * warps_per_cta, s, (const unsigned long long *)P.keys, P.W, P.H,
                         T);
    if (e != cudaSuccess)
        return e;
    return launch_points_range<DT>(src, dst, n, ga, groups, P, displace, true, SplatBelowTileBound{T}, ls, s);
}

cudaError_t launch_points_bounded(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                                  bool displace, const TileBounds &T, uint32_t tiles, const LaunchShape &ls,
                                  cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    switch (dtype) {
    case kF32: return launch_points_bounded_dt<kF32>(src, dst, n, P, displace, T, tiles, ls, s);
    case kF16: return launch_points_bounded_dt<kF16>(src, dst, n, P, displace, T, tiles, ls, s);
    case kBF16: return launch_points_bounded_dt<kBF16>(src, dst, n, P, displace, T, tiles, ls, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int DT, bool kD, bool kS, int kT>
static cudaError_t launch_tma_one(const void *src, void *dst, uint32_t n, const PointParams &P, uint32_t *err,
                                  int ctas_per_sm, int sm_count, cudaStream_t s)
{
    constexpr uint32_t smem = tma_smem_bytes<kT>();
    static unsigned long long configured = 0;    // one bit per device ordinal
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured & bit)) {
        e = cudaFuncSetAttribute(points_tma_kernel<DT, kD, kS, kT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess)
            return e;
        configured |= bit;
    }
    const uint64_t tiles = (groups_of<DT>(n) + kT - 1) / kT;
    const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)sm_count * ctas_per_sm);
    points_tma_kernel<DT, kD, kS, kT><<<grid, kT, smem, s>>>(src, dst, n, P, err);
    return cudaGetLastError();
}

template <int DT, int kT>
static cudaError_t launch_tma_dt(const void *src, void *dst, uint32_t n, const PointParams &P, bool displace,
                                 bool splat, uint32_t *err, int ctas_per_sm, int sm_count, cudaStream_t s)
{
    if (displace && splat)
        return launch_tma_one<DT, true, true, kT>(src, dst, n, P, err, ctas_per_sm, sm_count, s);
    if (displace)
        return launch_tma_one<DT, true, false, kT>(src, dst, n, P, err, ctas_per_sm, sm_count, s);
    return launch_tma_one<DT, false, true, kT>(src, dst, n, P, err, ctas_per_sm, sm_count, s);
}

template <int kT>
static cudaError_t launch_tma_threads(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                                     bool displace, bool splat, uint32_t *err, int ctas_per_sm, int sm_count,
                                     cudaStream_t s)
{
    switch (dtype) {
    case kF32: return launch_tma_dt<kF32, kT>(src, dst, n, P, displace, splat, err, ctas_per_sm, sm_count, s);
    case kF16: return launch_tma_dt<kF16, kT>(src, dst, n, P, displace, splat, err, ctas_per_sm, sm_count, s);
    case kBF16: return launch_tma_dt<kBF16, kT>(src, dst, n, P, displace, splat, err, ctas_per_sm, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_points_tma(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                              bool displace, bool splat, uint32_t *err, const LaunchShape &ls, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    const int ctas = ls.ctas_per_sm > 0 ? ls.ctas_per_sm : 1;
    switch (ls.threads) {
    case 128: return launch_tma_threads<128>(dtype, src, dst, n, P, displace, splat, err, ctas, ls.sm_count, s);
    case 256: return launch_tma_threads<256>(dtype, src, dst, n, P, displace, splat, err, ctas, ls.sm_count, s);
    case 512: return launch_tma_threads<512>(dtype, src, dst, n, P, displace, splat, err, ctas, ls.sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_points(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P, bool displace,
                          bool splat, const LaunchShape &ls, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    switch (dtype) {
    case kF32: return launch_points_dt<kF32>(src, dst, n, P, displace, splat, ls, s);
    case kF16: return launch_points_dt<kF16>(src, dst, n, P, displace, splat, ls, s);
    case kBF16: return launch_points_dt<kBF16>(src, dst, n, P, displace, splat, ls, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mmr
