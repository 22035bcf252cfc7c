// Host-side declarations shared by the libmmr translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace mmr {

// NVTX range around a host call, so profiler timelines show which library
// call enqueued which kernels.  Header-only NVTX: no cost without a tool.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct PointParams;
struct Palette;
struct TileBounds;
struct FrameChunks;

// Point-kernel variants (the values of mmr_set_launch's `kernel`).
enum : int {
    kKernelGrid = 0,         // grid-stride, direct depth-tested splat
    kKernelTma = 1,          // persistent, TMA-staged
    kKernelDepthBound = 2,   // grid-stride in two passes with per-tile depth bounds (mmr_tiles.cuh)
    kKernelWarpAgg = 3,      // grid-stride, warp-aggregated splat
};

struct LaunchShape {
    int threads = 256;       // threads per block
    int ctas_per_sm = 0;     // 0: one thread per work item; else a persistent grid
    int sm_count = 148;
    int kernel = kKernelGrid;
    int bound_shift = 0;     // depth-bound variants: the first pass takes groups >> bound_shift groups (0: the
                             // library's choice)
};

// Point kernels read positions from src and write displaced ones to dst
// (src == dst for an in-place step).
cudaError_t launch_points(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P, bool displace,
                          bool splat, const LaunchShape &ls, cudaStream_t s);

// Depth-bounded point phase (kKernelDepthBound): the first
// groups >> ls.bound_shift point groups with the marking splat, the bounds of
// the marked tiles, the remaining groups with the bounded splat; three
// launches.  `tiles` is the number of tiles of the frame (the list's size).
cudaError_t launch_points_bounded(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                                  bool displace, const TileBounds &T, uint32_t tiles, const LaunchShape &ls,
                                  cudaStream_t s);

// Disc markers of radius P.disc_r pixels (grid-stride, 64 threads).  With
// T, in two passes around the depth bounds of T's 32x32 tiles: the first
// groups >> bound_shift groups, the bounds of every tile, then the other
// groups with discs behind their tiles' bounds skipped; three launches.
struct DiscBounds;
cudaError_t launch_points_disc(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                               bool displace, const DiscBounds *T, int bound_shift, int sm_count, cudaStream_t s);

// TMA-staged persistent variant (threads 128, 256 or 512; grid =
// sm_count * ctas_per_sm CTAs).  The buffer must be padded to whole 48-byte
// groups.  A timed-out wait sets *err (device word) to a non-zero value.
cudaError_t launch_points_tma(int dtype, const void *src, void *dst, uint32_t n, const PointParams &P,
                              bool displace, bool splat, uint32_t *err, const LaunchShape &ls, cudaStream_t s);

// One CTA that waits on an mbarrier nothing arrives on, for max_cycles, then
// sets *err like a point kernel whose bulk copy never completed.
cudaError_t launch_bounded_wait_selftest(long long max_cycles, uint32_t *err, cudaStream_t s);

// Resolve keys into rgba and clear next_keys, storing only in the chunks
// that F says this frame or the previous one touched (mmr_resolve.cuh).
cudaError_t launch_resolve(const unsigned long long *keys, unsigned long long *next_keys, uint32_t *rgba,
                           const Palette &pal, uint32_t npx, const FrameChunks &F, cudaStream_t s);

// Host mirror: write into `host` (mapped pinned memory, npx uint32) the quads
// of every 64-pixel chunk the frame numbered `tag` touched (chunk tags
// `tags`) or the mirror still holds a point in (`held`, one byte per chunk,
// updated), or of every chunk when `full`; the ragged tail pixels always.
// Adds the bytes written to *bytes.
cudaError_t launch_mirror(const uint32_t *rgba, uint32_t *host, uint32_t npx, const uint32_t *tags, uint32_t tag,
                          unsigned char *held, int full, unsigned long long *bytes, cudaStream_t s);

// Displacement amplitudes the kernels accept: 0, or [2^-100, 1] (so that
// amplitude * 2^-23 is a normal float and the scaling is exact).
inline bool amplitude_ok(float a) { return a == 0.0f || (a >= 0x1p-100f && a <= 1.0f); }

// Message returned by mmr_last_error(NULL) on this thread.
void set_process_error(const char *msg);

// All-pairs gravity step parameters.
struct NbodyParams {
    float G;
    float eps2;
    float dt;
};

// One N-body step reading pin, writing pout and vel, splatting the new
// positions into P.keys (FP32 positions, n bodies).  `partial` is scratch of
// nbody_chunks(n) * n float4 (the per-chunk sums).
uint32_t nbody_chunks(uint32_t n);
cudaError_t launch_nbody(const float *pin, float *pout, float *vel, const float *mass, float4 *partial, uint32_t n,
                         const NbodyParams &B, const PointParams &P, cudaStream_t s);

// The depth ranges a camera may use: 2^-64 <= znear < zfar <= 2^64 as FP32
// values.  Kernels draw only points with znear < clip w < zfar, and on that
// range of w their perspective divide (perspective_divide, one shared
// reciprocal with Markstein's correction) gives every pixel that IEEE
// division gives.
inline bool depth_range_ok(float znear, float zfar)
{
    return znear >= 0x1p-64f && zfar > znear && zfar <= 0x1p64f;
}

// FP64 camera -> FP32 clip matrix (row-major 4x4); returns false on invalid input.
bool build_clip_matrix(const double eye[3], const double target[3], const double up[3],
                       double fovy_deg, double aspect, double znear, double zfar, float out[16]);

}  // namespace mmr
