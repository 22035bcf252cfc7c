// Batched clouds (include/mmr.h, mmr_batch_*): many independent clouds of
// uneven size, each with its own camera and framebuffer, advanced and
// rendered by one persistent launch per frame.
//
// Work is cut into items: a point item is up to `chunk_groups` 48-byte point
// groups of one cloud (displace, project, splat), a pixel item up to
// 4*chunk_groups quads of one cloud's framebuffer (resolve, clear the other
// depth-id buffer).  Persistent CTAs take items in list order from one
// counter, so a 1e3-point cloud and a 1e6-point cloud cost in proportion to
// their size and no CTA idles on a small cloud.  The list holds every
// cloud's point items in order, and a cloud's pixel items once about one
// resident grid's worth of later point items precede them: by the time they
// are taken the cloud's points are normally done, and the bandwidth-bound
// resolve runs beside other clouds' latency-bound point items (on the
// 256-cloud scene the keys still come back from DRAM; the gain is that
// overlap).  A pixel item waits (bounded) for its cloud's count of
// unfinished point items to reach zero; every point item it waits on was
// taken earlier by a running CTA and never waits itself, so the wait ends.
// A device-side frame counter selects the Philox step, the camera slot and
// the depth-id buffer, so a captured frame replays as a CUDA graph with no
// host update.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mmr.h"
#include "mmr_device.cuh"
#include "mmr_internal.h"
#include "mmr_points.cuh"
#include "mmr_resolve.cuh"
#include "mmr_worklist.h"

namespace mmr {

struct CloudDev {
    void *pos;
    unsigned long long *keys[2];
    uint32_t *rgba;
    uint32_t n;
    uint32_t npx;
    int W, H;
    float fW, fH, halfW, halfH;
    uint32_t seed_lo, seed_hi, cloud;
    float amplitude;
    uint32_t color, background;
    uint32_t *tags[2];          // per depth-id buffer: one tag per 64-pixel chunk (FrameChunks)
};


struct BatchTables {
    const CloudDev *clouds;
    const Cam *cams;            // [slots][count]
    const uint2 *items;         // hand-out order
    uint32_t n_items;
    uint32_t chunk_groups;
    uint32_t chunk_quads;
    uint32_t count;
    uint32_t slots;
    uint32_t first_step;
    uint32_t spin_limit;        // polls before a pixel item gives up waiting
    uint32_t *frame;            // device frame counter, then the repaint flag (non-zero: the next frame repaints
                                // and clears every pixel; the advance kernel resets it)
    uint32_t *next;             // next item to hand out, zeroed before every frame
    uint32_t *remaining;        // [count] unfinished point items per cloud, reset before every frame
    uint32_t *err;              // bit 0: a bounded wait gave up
    struct ItemParams *params;  // [count] this frame's parameters of each cloud
    long long pos_shift;        // bytes added to every cloud's position pointer (render from a copy)
};

// A cloud's parameters for one frame, built once per frame for all clouds
// and copied by every point item into shared memory, 4 bytes per thread.
struct ItemParams {
    PointParams P;
    void *pos;
    uint32_t n;
    uint32_t pad;
};

__global__ void batch_params_kernel(BatchTables T)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= T.count)
        return;
    const uint32_t frame = *T.frame;
    const CloudDev &cl = T.clouds[c];
    ItemParams I;
    PointParams &P = I.P;
    P.cam = T.cams[(size_t)(frame % T.slots) * T.count + c];
    P.keys = cl.keys[frame & 1];
    P.W = cl.W;
    P.H = cl.H;
    P.fW = cl.fW;
    P.fH = cl.fH;
    P.halfW = cl.halfW;
    P.halfH = cl.halfH;
    P.seed_lo = cl.seed_lo;
    P.seed_hi = cl.seed_hi;
    P.step = T.first_step + frame;
    P.cloud = cl.cloud;
    P.amplitude = cl.amplitude;
    P.id_base = 0;
    P.disc_r = 0.0f;
    P.disc_r2 = 0.0f;
    philox_prepare(P);
    I.pos = reinterpret_cast<void *>(reinterpret_cast<uintptr_t>(cl.pos) + T.pos_shift);
    I.n = cl.n;
    I.pad = 0;
    T.params[c] = I;
}

// Bounded wait until *count reads 0 (acquire, GPU scope), polling about
// every 64 ns at most `limit` times; on giving up sets bit 0 of *err and
// returns false.
__device__ __forceinline__ bool wait_until_zero(const uint32_t *count, uint32_t limit, uint32_t *err)
{
    for (uint32_t k = 0;; ++k) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
        if (v == 0)
            return true;
        if (k >= limit) {
            atomicOr(err, 1u);
            return false;
        }
        __nanosleep(64);
    }
}

// At most 512 threads per block (a bound the autotuner stays well below).
constexpr int kBatchMaxThreads = 512;

// Resolve + clear of four pixels with the keys read from L2 (ld.global.cg):
// this SM's L1 may still hold lines of this cloud's keys from its own early
// depth tests, older than the atomics that followed.  As in the single-cloud
// resolve (FrameChunks), colours are stored and the other buffer cleared
// only in 64-pixel chunks that this frame or the previous one touched; a
// quad holding a key tags its chunk with this frame's number (lanes of a
// warp storing the same tag to the same word make one store).
__device__ __forceinline__ void resolve_quad_l2(const unsigned long long *keys, unsigned long long *next_keys,
                                                uint32_t *rgba, const Palette &pal, uint32_t q, FrameChunks F)
{
    const ulonglong2 k01 = __ldcg(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q);
    const ulonglong2 k23 = __ldcg(reinterpret_cast<const ulonglong2 *>(keys) + 2 * q + 1);
    const bool dirty = (k01.x & k01.y & k23.x & k23.y) != kEmptyKey;
    const uint32_t chunk = q >> kChunkQuadShift;
    const bool prev = F.full || __ldg(F.prev + chunk) == F.prev_tag;
    if (dirty || prev) {
        const uint4 c = make_uint4(key_colour(k01.x, pal), key_colour(k01.y, pal), key_colour(k23.x, pal),
                                   key_colour(k23.y, pal));
        __stcs(reinterpret_cast<uint4 *>(rgba) + q, c);
    }
    if (prev) {
        const ulonglong2 e = make_ulonglong2(kEmptyKey, kEmptyKey);
        reinterpret_cast<ulonglong2 *>(next_keys)[2 * q] = e;
        reinterpret_cast<ulonglong2 *>(next_keys)[2 * q + 1] = e;
    }
    if (dirty)
        F.cur[chunk] = F.cur_tag;
}

// One frame of every cloud.  A point item copies its cloud's parameters from
// the frame's table into shared memory, 4 bytes per thread, and every thread
// reads them there (held in registers by each thread they cost some 30
// registers and halve the resident warps).  A CTA takes its next item while
// it works on a point item, or after a pixel item's wait: an item is never
// held by a CTA that is waiting.  Measured on the 256-cloud scene against one
// thread building the parameters per item and the next item taken after the
// current one: 0.770 -> 0.748 ms per frame.  The host round trip runs it twice
// per frame: displace only (pixel items skipped), then render only from the
// copied positions.  FP32 runs under a cap of 40 registers (8 bytes spilled;
// uncapped the chunk bookkeeping of the pixel items takes it to 52): 0.606 ->
// 0.587 ms per frame, tuned shape 256 threads, 8 CTAs per SM, 2048 groups per
// item (a cap of 48: 0.591 ms).  The 16-bit bodies keep up to 64, as before.
// Either cap, times kBatchMaxThreads threads, fits the register file.
template <int DT, bool kDisplace, bool kSplat>
__global__ void __maxnreg__(DT == kF32 ? 40 : 64) batch_frame_kernel(BatchTables T)
{
    constexpr uint32_t G = Group<DT>::kPoints;
    __shared__ ItemParams sI;
    __shared__ uint32_t s_next, s_ok;
    const int buf = *T.frame & 1;
    if (threadIdx.x == 0)
        s_next = atomicAdd(T.next, 1u);
    __syncthreads();
    uint32_t it = s_next;
    while (it < T.n_items) {
        const uint2 w = T.items[it];
        const uint32_t cloud = w.x & ~kPixelItem;
        uint32_t nxt = 0;
        if (w.x & kPixelItem) {
            if (threadIdx.x == 0) {
                if constexpr (kSplat) {
                    s_ok = wait_until_zero(T.remaining + cloud, T.spin_limit, T.err);
                    __threadfence();
                }
                nxt = atomicAdd(T.next, 1u);    // taken only after the wait: a held item never waits behind one
            }
            __syncthreads();
            if (kSplat && s_ok) {
                const CloudDev &cl = T.clouds[cloud];
                const unsigned long long *keys = cl.keys[buf];
                unsigned long long *nk = cl.keys[buf ^ 1];
                const uint32_t quads = cl.npx / 4;
                const uint32_t end = min(w.y + T.chunk_quads, quads);
                const Palette pal{nullptr, nullptr, nullptr, 0u, cl.color, cl.background};
                // frame numbers are the counter + 1, so the previous frame's is the counter; after a wrap
                // old tags can only match too often, which costs stores, never a pixel
                const uint32_t frame = T.frame[0];
                const FrameChunks F{cl.tags[buf ^ 1], cl.tags[buf], frame, frame + 1u, T.frame[1]};
#pragma unroll 1
                for (uint32_t q = w.y + threadIdx.x; q < end; q += blockDim.x)
                    resolve_quad_l2(keys, nk, cl.rgba, pal, q, F);
                if (end == quads && quads * 4 + threadIdx.x < cl.npx) {     // the ragged tail
                    const uint32_t p = quads * 4 + threadIdx.x;
                    cl.rgba[p] = key_colour(__ldcg(keys + p), pal);
                    nk[p] = kEmptyKey;
                }
            }
            if (threadIdx.x == 0)
                s_next = nxt;
            __syncthreads();
        } else {
            if (threadIdx.x == 0)
                nxt = atomicAdd(T.next, 1u);    // this item never waits, so the next one is taken now
            const uint32_t *src = reinterpret_cast<const uint32_t *>(T.params + cloud);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sI);
            for (uint32_t k = threadIdx.x; k < sizeof(ItemParams) / 4; k += blockDim.x)
                dst[k] = src[k];
            __syncthreads();
            const uint32_t n = sI.n;
            void *pos = sI.pos;
            const uint32_t full = n / G;
            const uint32_t end = min(w.y + T.chunk_groups, groups_of<DT>(n));
            for (uint32_t g = w.y + threadIdx.x; g < end; g += blockDim.x) {
                if (g < full) {
                    uint4 q[3];
                    load_words(pos, g, q);
                    process_words<DT, kDisplace, kSplat>(q, g * G, G, sI.P);
                    if constexpr (kDisplace)
                        store_words(pos, g, q);
                } else {
                    process_tail<DT, kDisplace, kSplat>(pos, pos, n, g * G, sI.P);
                }
            }
            if (threadIdx.x == 0)
                s_next = nxt;
            __syncthreads();                     // every thread's atomics and stores precede the count below
            if (kSplat && threadIdx.x == 0) {
                __threadfence();
                atomicSub(T.remaining + cloud, 1u);
            }
        }
        it = s_next;
    }
}

// Failure-path self-test of the pixel items' wait: one thread waits on a
// count that nothing decrements and gives up after `limit` polls.
__global__ void batch_wait_selftest_kernel(const uint32_t *never_zero, uint32_t limit, uint32_t *err)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        wait_until_zero(never_zero, limit, err);
}

// After every frame: the next frame number, and no forced repaint.
__global__ void batch_advance_kernel(uint32_t *frame)
{
    frame[0] += 1u;
    frame[1] = 0u;
}

}  // namespace mmr

struct mmr_batch {
    int device = 0;
    int count = 0;
    int dtype = 0;
    int slots = 1;
    uint64_t budget = 0;
    uint64_t held = 0;
    mmr::LaunchShape launch;
    uint32_t chunk_groups = 256;

    std::vector<mmr_cloud_desc> desc;
    std::vector<uint64_t> pos_off;   // byte offset of each cloud's positions
    std::vector<uint64_t> px_off;    // pixel offset of each cloud's framebuffer
    uint64_t pos_bytes = 0;
    uint64_t total_px = 0;

    void *pos_base = nullptr;
    unsigned long long *keys_base[2] = {nullptr, nullptr};
    uint32_t *rgba_base = nullptr;
    uint32_t *tags_base = nullptr;       // chunk tags: [2][total_chunks]
    std::vector<uint64_t> chunk_off;     // first chunk tag of each cloud
    uint64_t total_chunks = 0;
    mmr::CloudDev *d_clouds = nullptr;
    mmr::Cam *d_cams = nullptr;
    uint2 *d_items = nullptr;        // work list in hand-out order
    uint64_t item_bytes = 0;
    uint32_t n_items = 0;
    int grid = 1;                    // resident CTAs of the persistent launch
    uint32_t *d_frame = nullptr;         // [0] frame counter, [1] repaint flag
    uint32_t *d_work = nullptr;      // [0] next item, [1] error bits, [2] self-test count (never zero)
    uint32_t *d_remaining = nullptr; // [count] unfinished point items per cloud, then [count] their full counts
    mmr::ItemParams *d_params = nullptr;
    void *rt_host = nullptr;         // host round trip: host copy of the positions (pinned or pageable)
    int rt_host_pinned = -1;
    void *rt_device = nullptr;       // and the device buffer the copy comes back to

    std::vector<mmr::Cam> cams;      // host copy [slots][count]
    std::vector<uint8_t> cam_set;
    mmr::Cam *staging = nullptr;     // pinned staging for camera uploads
    cudaEvent_t staging_done = nullptr;
    bool cams_dirty = false;

    uint32_t frames = 0;             // frames enqueued
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;

    char err[512] = "";
};

namespace {

thread_local char g_batch_error[512] = "";

mmr_status bfail(mmr_batch *b, mmr_status s, const char *fmt, ...)
{
    char *dst = b ? b->err : g_batch_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return s;
}

mmr_status bcuda(mmr_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, MMR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

mmr_status balloc(mmr_batch *b, void **p, uint64_t bytes, const char *what)
{
    *p = nullptr;
    if (b->budget && b->held + bytes > b->budget)
        return bfail(b, MMR_ERR_BUDGET, "%s: %llu bytes would exceed the budget (%llu of %llu held)", what,
                     (unsigned long long)bytes, (unsigned long long)b->held, (unsigned long long)b->budget);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return bfail(b, e == cudaErrorMemoryAllocation ? MMR_ERR_OOM : MMR_ERR_CUDA, "%s: cudaMalloc(%llu): %s",
                     what, (unsigned long long)bytes, cudaGetErrorString(e));
    }
    b->held += bytes;
    return MMR_OK;
}

void bfree(mmr_batch *b, void **p, uint64_t bytes)
{
    if (*p) {
        cudaFree(*p);
        b->held -= bytes;
        *p = nullptr;
    }
}

uint64_t point_bytes(uint64_t n, int dtype) { return n * (dtype == MMR_F32x3 ? 12u : 6u); }

uint32_t groups_for(uint64_t n, int dtype)
{
    const uint64_t g = dtype == MMR_F32x3 ? 4 : 8;
    return (uint32_t)((n + g - 1) / g);
}

uint32_t chunk_quads(const mmr_batch *b) { return 4u * b->chunk_groups; }

// Resident CTAs of the persistent launch for the current shape: CTAs per SM
// as set, or as many as fit (0).
cudaError_t resident_grid(const mmr_batch *b, int *grid)
{
    int per_sm = b->launch.ctas_per_sm;
    if (per_sm <= 0) {
        cudaError_t e;
        switch (b->dtype) {
        case MMR_F32x3:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mmr::batch_frame_kernel<mmr::kF32, true, true>,
                                                              b->launch.threads, 0);
            break;
        case MMR_F16x3:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mmr::batch_frame_kernel<mmr::kF16, true, true>,
                                                              b->launch.threads, 0);
            break;
        default:
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mmr::batch_frame_kernel<mmr::kBF16, true, true>,
                                                              b->launch.threads, 0);
            break;
        }
        if (e != cudaSuccess)
            return e;
    }
    *grid = std::max(1, per_sm) * b->launch.sm_count;
    return cudaSuccess;
}

// (Re)build the work list for the current chunk size and launch shape.  A
// cloud's pixel items follow its last point item once `grid` further point
// items have been listed: by then the point items taken before them have
// normally finished (measured on the 256-cloud scene: a lag of 0.5 to 4
// grids all within 1.5% of the best, 0 to 0.15 grids up to 15% slower, all
// pixel items at the end 6% slower).
mmr_status build_items(mmr_batch *b)
{
    int grid = 1;
    cudaError_t e = resident_grid(b, &grid);
    if (e != cudaSuccess)
        return bcuda(b, e, "occupancy query");
    std::vector<uint32_t> groups(b->count), quads(b->count), per_cloud;
    for (int c = 0; c < b->count; ++c) {
        groups[c] = groups_for(b->desc[c].n, b->dtype);
        quads[c] = (uint32_t)(((uint64_t)b->desc[c].width * b->desc[c].height) / 4);
    }
    static_assert(sizeof(mmr::WorkItem) == sizeof(uint2), "a work item is uploaded as a uint2");
    const std::vector<mmr::WorkItem> items =
        mmr::build_work_list(groups, quads, b->chunk_groups, chunk_quads(b), (uint64_t)grid, per_cloud);
    std::vector<uint32_t> counts(per_cloud);                 // [count] live counts, then [count] full counts
    counts.insert(counts.end(), per_cloud.begin(), per_cloud.end());
    bfree(b, (void **)&b->d_items, b->item_bytes);
    b->n_items = 0;                  // until the new list is in place a frame hands out nothing
    b->item_bytes = items.size() * sizeof(uint2);
    mmr_status st = balloc(b, (void **)&b->d_items, b->item_bytes, "work list");
    if (st != MMR_OK)
        return st;
    e = cudaMemcpy(b->d_items, items.data(), b->item_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_remaining, counts.data(), counts.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return bcuda(b, e, "work list upload");
    b->n_items = (uint32_t)items.size();
    b->grid = grid;
    return MMR_OK;
}

// Polls before a pixel item gives up waiting (about a second).
constexpr uint32_t kSpinLimit = 1u << 24;

mmr::BatchTables tables(const mmr_batch *b)
{
    mmr::BatchTables T;
    T.clouds = b->d_clouds;
    T.cams = b->d_cams;
    T.items = b->d_items;
    T.n_items = b->n_items;
    T.chunk_groups = b->chunk_groups;
    T.chunk_quads = chunk_quads(b);
    T.count = (uint32_t)b->count;
    T.slots = (uint32_t)b->slots;
    T.first_step = 0;
    T.spin_limit = kSpinLimit;
    T.frame = b->d_frame;
    T.next = b->d_work;
    T.remaining = b->d_remaining;
    T.err = b->d_work + 1;
    T.params = b->d_params;
    T.pos_shift = 0;
    return T;
}

mmr_status upload_cameras(mmr_batch *b, cudaStream_t s)
{
    if (!b->cams_dirty)
        return MMR_OK;
    cudaError_t e = cudaEventSynchronize(b->staging_done);   // previous upload has left the staging buffer
    if (e != cudaSuccess)
        return bcuda(b, e, "camera staging wait");
    memcpy(b->staging, b->cams.data(), b->cams.size() * sizeof(mmr::Cam));
    e = cudaMemcpyAsync(b->d_cams, b->staging, b->cams.size() * sizeof(mmr::Cam), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaEventRecord(b->staging_done, s);
    if (e != cudaSuccess)
        return bcuda(b, e, "camera upload");
    b->cams_dirty = false;
    return MMR_OK;
}

enum class Pass { kFrame, kDisplace, kRender };

template <int DT>
cudaError_t launch_pass(const mmr_batch *b, cudaStream_t s, const mmr::BatchTables &T, Pass pass)
{
    switch (pass) {
    case Pass::kFrame: mmr::batch_frame_kernel<DT, true, true><<<b->grid, b->launch.threads, 0, s>>>(T); break;
    case Pass::kDisplace: mmr::batch_frame_kernel<DT, true, false><<<b->grid, b->launch.threads, 0, s>>>(T); break;
    default: mmr::batch_frame_kernel<DT, false, true><<<b->grid, b->launch.threads, 0, s>>>(T); break;
    }
    return cudaGetLastError();
}

// Enqueue one pass over the work list on s: reset the hand-out counter and
// the per-cloud counts, build every cloud's parameters for the frame (its
// positions `shift` bytes from its own buffer), one persistent launch.
cudaError_t enqueue_pass(const mmr_batch *b, cudaStream_t s, Pass pass, long long shift)
{
    mmr::BatchTables T = tables(b);
    T.pos_shift = shift;
    cudaError_t e = cudaMemsetAsync(b->d_work, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_remaining, b->d_remaining + b->count, sizeof(uint32_t) * b->count,
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return e;
    mmr::batch_params_kernel<<<(b->count + 127) / 128, 128, 0, s>>>(T);
    switch (b->dtype) {
    case MMR_F32x3: return launch_pass<mmr::kF32>(b, s, T, pass);
    case MMR_F16x3: return launch_pass<mmr::kF16>(b, s, T, pass);
    default: return launch_pass<mmr::kBF16>(b, s, T, pass);
    }
}

// Enqueue one frame on s (one pass, then advance the frame counter); no host
// synchronisation.
cudaError_t enqueue_frame(const mmr_batch *b, cudaStream_t s)
{
    cudaError_t e = enqueue_pass(b, s, Pass::kFrame, 0);
    if (e != cudaSuccess)
        return e;
    mmr::batch_advance_kernel<<<1, 1, 0, s>>>(b->d_frame);
    return cudaGetLastError();
}

mmr_status cameras_ready(mmr_batch *b, bool all_slots)
{
    const int first = all_slots ? 0 : (int)(b->frames % (uint32_t)b->slots);
    const int last = all_slots ? b->slots : first + 1;
    for (int s = first; s < last; ++s)
        for (int c = 0; c < b->count; ++c)
            if (!b->cam_set[(size_t)s * b->count + c])
                return bfail(b, MMR_ERR_STATE, "camera of cloud %d, slot %d not set", c, s);
    return MMR_OK;
}

void drop_graph(mmr_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

}  // namespace

extern "C" {

const char *mmr_batch_last_error(const mmr_batch *b) { return b ? b->err : g_batch_error; }

mmr_status mmr_batch_destroy(mmr_batch *b)
{
    if (!b)
        return MMR_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    bfree(b, &b->pos_base, b->pos_bytes);
    bfree(b, (void **)&b->keys_base[0], b->total_px * 8);
    bfree(b, (void **)&b->keys_base[1], b->total_px * 8);
    bfree(b, (void **)&b->rgba_base, b->total_px * 4);
    bfree(b, (void **)&b->d_clouds, (uint64_t)b->count * sizeof(mmr::CloudDev));
    bfree(b, (void **)&b->d_cams, b->cams.size() * sizeof(mmr::Cam));
    bfree(b, (void **)&b->d_items, b->item_bytes);
    bfree(b, (void **)&b->d_frame, 8);
    bfree(b, (void **)&b->tags_base, 2 * 4 * b->total_chunks);
    bfree(b, (void **)&b->d_work, 3 * sizeof(uint32_t));
    bfree(b, (void **)&b->d_remaining, 2 * sizeof(uint32_t) * (uint64_t)b->count);
    bfree(b, (void **)&b->d_params, sizeof(mmr::ItemParams) * (uint64_t)b->count);
    bfree(b, &b->rt_device, b->pos_bytes);
    if (b->rt_host) {
        if (b->rt_host_pinned == 1)
            cudaFreeHost(b->rt_host);
        else
            free(b->rt_host);
    }
    if (b->staging)
        cudaFreeHost(b->staging);
    if (b->staging_done)
        cudaEventDestroy(b->staging_done);
    if (b->capture_stream)
        cudaStreamDestroy(b->capture_stream);
    delete b;
    return MMR_OK;
}

mmr_status mmr_batch_create(int count, const mmr_cloud_desc *clouds, int dtype, int camera_slots,
                            uint64_t budget_bytes, mmr_batch **out)
{
    if (!out || !clouds)
        return bfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_batch_create: NULL argument");
    *out = nullptr;
    if (count < 1 || count > 65536 || camera_slots < 1 || camera_slots > 4096)
        return bfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_batch_create: count %d or camera_slots %d out of range",
                     count, camera_slots);
    if (dtype != MMR_F32x3 && dtype != MMR_F16x3 && dtype != MMR_BF16x3)
        return bfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_batch_create: unknown dtype %d", dtype);
    for (int c = 0; c < count; ++c) {
        const mmr_cloud_desc &d = clouds[c];
        if (d.n == 0 || d.n >= (1ull << 32) || d.width < 1 || d.height < 1 || d.width > 32768 ||
            d.height > 32768 || !mmr::amplitude_ok(d.amplitude))
            return bfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_batch_create: cloud %d has an invalid descriptor", c);
    }
    mmr_batch *b = new (std::nothrow) mmr_batch();
    if (!b)
        return bfail(nullptr, MMR_ERR_OOM, "mmr_batch_create: host allocation failed");
    b->count = count;
    b->dtype = dtype;
    b->slots = camera_slots;
    b->budget = budget_bytes;
    b->desc.assign(clouds, clouds + count);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->launch.sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bfail(nullptr, MMR_ERR_CUDA, "mmr_batch_create: no usable CUDA device: %s", cudaGetErrorString(e));
        delete b;
        return MMR_ERR_CUDA;
    }
    b->launch.threads = 64;
    b->launch.ctas_per_sm = 0;
    // layout: positions 256-byte aligned per cloud and padded to 48-byte groups
    for (int c = 0; c < count; ++c) {
        b->pos_off.push_back(b->pos_bytes);
        const uint64_t bytes = (point_bytes(clouds[c].n, dtype) + 47) / 48 * 48;
        b->pos_bytes += (bytes + 255) / 256 * 256;
        b->px_off.push_back(b->total_px);
        const uint64_t px = (uint64_t)clouds[c].width * clouds[c].height;
        b->total_px += (px + 31) / 32 * 32;             // keeps every framebuffer 256-byte aligned
        b->chunk_off.push_back(b->total_chunks);
        b->total_chunks += (px + 63) / 64;
    }
    b->cams.assign((size_t)camera_slots * count, mmr::Cam{});
    b->cam_set.assign((size_t)camera_slots * count, 0);
    mmr_status st = balloc(b, &b->pos_base, b->pos_bytes, "batch positions");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->keys_base[0], b->total_px * 8, "batch depth-id buffers 0");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->keys_base[1], b->total_px * 8, "batch depth-id buffers 1");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->rgba_base, b->total_px * 4, "batch framebuffers");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->tags_base, 2 * 4 * b->total_chunks, "batch chunk tags");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->d_clouds, (uint64_t)count * sizeof(mmr::CloudDev), "cloud table");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->d_cams, b->cams.size() * sizeof(mmr::Cam), "camera table");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->d_frame, 8, "frame counter and repaint flag");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->d_work, 3 * sizeof(uint32_t), "work counters");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->d_remaining, 2 * sizeof(uint32_t) * (uint64_t)count, "per-cloud counts");
    if (st == MMR_OK)
        st = balloc(b, (void **)&b->d_params, sizeof(mmr::ItemParams) * (uint64_t)count, "per-cloud parameters");
    if (st == MMR_OK) {
        const uint32_t init[3] = {0u, 0u, 1u};
        e = cudaMemcpy(b->d_work, init, sizeof init, cudaMemcpyHostToDevice);
        st = e == cudaSuccess ? build_items(b) : bcuda(b, e, "mmr_batch_create: work counters");
    }
    if (st == MMR_OK) {
        std::vector<mmr::CloudDev> host(count);
        for (int c = 0; c < count; ++c) {
            const mmr_cloud_desc &d = clouds[c];
            mmr::CloudDev &h = host[c];
            h.pos = (char *)b->pos_base + b->pos_off[c];
            h.keys[0] = b->keys_base[0] + b->px_off[c];
            h.keys[1] = b->keys_base[1] + b->px_off[c];
            h.rgba = b->rgba_base + b->px_off[c];
            h.tags[0] = b->tags_base + b->chunk_off[c];
            h.tags[1] = b->tags_base + b->total_chunks + b->chunk_off[c];
            h.n = (uint32_t)d.n;
            h.npx = (uint32_t)((uint64_t)d.width * d.height);
            h.W = d.width;
            h.H = d.height;
            h.fW = (float)d.width;
            h.fH = (float)d.height;
            h.halfW = 0.5f * (float)d.width;
            h.halfH = 0.5f * (float)d.height;
            h.seed_lo = (uint32_t)(d.seed & 0xffffffffu);
            h.seed_hi = (uint32_t)(d.seed >> 32);
            h.cloud = d.cloud;
            h.amplitude = d.amplitude;
            h.color = d.color;
            h.background = d.background;
        }
        e = cudaMemcpy(b->d_clouds, host.data(), host.size() * sizeof(mmr::CloudDev), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemset(b->pos_base, 0, b->pos_bytes);
        if (e == cudaSuccess)
            e = cudaMemset(b->keys_base[0], 0xff, b->total_px * 8);
        if (e == cudaSuccess)
            e = cudaMemset(b->keys_base[1], 0xff, b->total_px * 8);
        if (e == cudaSuccess)
            e = cudaMemset(b->rgba_base, 0, b->total_px * 4);
        if (e == cudaSuccess)
            e = cudaMemset(b->tags_base, 0, 2 * 4 * b->total_chunks);
        if (e == cudaSuccess) {
            const uint32_t fr[2] = {0u, 1u};        // frame 0, repaint everything
            e = cudaMemcpy(b->d_frame, fr, sizeof fr, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&b->staging, b->cams.size() * sizeof(mmr::Cam));
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b->staging_done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
        if (e != cudaSuccess)
            st = bcuda(b, e, "mmr_batch_create: set-up");
    }
    if (st != MMR_OK) {
        snprintf(g_batch_error, sizeof g_batch_error, "%s", b->err);
        mmr_batch_destroy(b);
        return st;
    }
    g_batch_error[0] = 0;
    *out = b;
    return MMR_OK;
}

mmr_status mmr_batch_points(mmr_batch *b, int cloud, void **dev_ptr)
{
    if (!b || !dev_ptr || cloud < 0 || cloud >= (b ? b->count : 0))
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_points: bad argument");
    *dev_ptr = (char *)b->pos_base + b->pos_off[cloud];
    return MMR_OK;
}

mmr_status mmr_batch_set_camera(mmr_batch *b, int cloud, int slot, const double eye[3], const double target[3],
                                const double up[3], double fovy_deg, double znear, double zfar)
{
    if (!b || !eye || !target || !up || cloud < 0 || cloud >= b->count || slot < 0 || slot >= b->slots)
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_set_camera: bad argument");
    if (!(fovy_deg > 0.0 && fovy_deg < 180.0) || !(znear > 0.0) || !(zfar > znear) || !std::isfinite(zfar) ||
        !mmr::depth_range_ok((float)znear, (float)zfar))
        return bfail(b, MMR_ERR_INVALID_ARG,
                     "mmr_batch_set_camera: need 0 < fovy < 180, 2^-64 <= znear < zfar <= 2^64");
    float m[16];
    const double aspect = (double)b->desc[cloud].width / (double)b->desc[cloud].height;
    if (!mmr::build_clip_matrix(eye, target, up, fovy_deg, aspect, znear, zfar, m))
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_set_camera: eye == target or up parallel to view");
    mmr::Cam &cam = b->cams[(size_t)slot * b->count + cloud];
    for (int k = 0; k < 4; ++k) {
        cam.rx[k] = m[k];
        cam.ry[k] = m[4 + k];
        cam.rw[k] = m[12 + k];
    }
    cam.znear = (float)znear;
    cam.zfar = (float)zfar;
    b->cam_set[(size_t)slot * b->count + cloud] = 1;
    b->cams_dirty = true;
    return MMR_OK;
}

mmr_status mmr_batch_set_launch(mmr_batch *b, int threads, int ctas_per_sm, int chunk_groups)
{
    if (!b)
        return MMR_ERR_INVALID_ARG;
    if (threads < 32 || threads > mmr::kBatchMaxThreads || threads % 32 || ctas_per_sm < 0 || ctas_per_sm > 64 ||
        chunk_groups < 1 || chunk_groups > 65536)
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_set_launch: out of range");
    b->launch.threads = threads;
    b->launch.ctas_per_sm = ctas_per_sm;
    b->chunk_groups = (uint32_t)chunk_groups;
    drop_graph(b);
    cudaError_t e = cudaDeviceSynchronize();         // the old work list may still be in use
    if (e != cudaSuccess)
        return bcuda(b, e, "mmr_batch_set_launch: sync");
    return build_items(b);                           // chunk size and resident grid set the list
}

mmr_status mmr_batch_step_and_render(mmr_batch *b, void *stream)
{
    mmr::NvtxRange nvtx("mmr_batch_step_and_render");
    if (!b)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = cameras_ready(b, false);
    if (st != MMR_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = upload_cameras(b, s);
    if (st != MMR_OK)
        return st;
    cudaError_t e = enqueue_frame(b, s);
    if (e != cudaSuccess)
        return bcuda(b, e, "batch frame launch");
    b->frames += 1;
    return MMR_OK;
}

mmr_status mmr_batch_step_and_render_roundtrip(mmr_batch *b, void *stream, int pinned_host)
{
    mmr::NvtxRange nvtx("mmr_batch_step_and_render_roundtrip");
    if (!b)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = cameras_ready(b, false);
    if (st != MMR_OK)
        return st;
    const int want_pinned = pinned_host ? 1 : 0;
    if (b->rt_host && b->rt_host_pinned != want_pinned) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess)
            return bcuda(b, e, "batch round trip: sync before switching host buffer");
        if (b->rt_host_pinned == 1)
            cudaFreeHost(b->rt_host);
        else
            free(b->rt_host);
        b->rt_host = nullptr;
    }
    if (!b->rt_host) {
        if (want_pinned) {
            cudaError_t e = cudaMallocHost(&b->rt_host, b->pos_bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b->rt_host = nullptr;
                return bfail(b, MMR_ERR_OOM, "batch round trip: pinned host allocation failed: %s",
                             cudaGetErrorString(e));
            }
        } else {
            b->rt_host = malloc(b->pos_bytes);
            if (!b->rt_host)
                return bfail(b, MMR_ERR_OOM, "batch round trip: host allocation failed");
        }
        b->rt_host_pinned = want_pinned;
    }
    if (!b->rt_device) {
        st = balloc(b, &b->rt_device, b->pos_bytes, "batch round-trip device copy");
        if (st != MMR_OK)
            return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = upload_cameras(b, s);
    if (st != MMR_OK)
        return st;
    cudaError_t e = enqueue_pass(b, s, Pass::kDisplace, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->rt_host, b->pos_base, b->pos_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->rt_device, b->rt_host, b->pos_bytes, cudaMemcpyHostToDevice, s);
    const long long shift = (long long)((uintptr_t)b->rt_device - (uintptr_t)b->pos_base);
    if (e == cudaSuccess)
        e = enqueue_pass(b, s, Pass::kRender, shift);
    if (e == cudaSuccess) {
        mmr::batch_advance_kernel<<<1, 1, 0, s>>>(b->d_frame);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return bcuda(b, e, "batch round-trip frame");
    b->frames += 1;
    return MMR_OK;
}

mmr_status mmr_batch_run_graph(mmr_batch *b, int frames, void *stream)
{
    mmr::NvtxRange nvtx("mmr_batch_run_graph");
    if (!b || frames < 0)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = cameras_ready(b, true);
    if (st != MMR_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = upload_cameras(b, s);
    if (st != MMR_OK)
        return st;
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return bcuda(b, e, "graph capture begin");
        cudaError_t le = enqueue_frame(b, b->capture_stream);
        e = cudaStreamEndCapture(b->capture_stream, &g);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (g)
                cudaGraphDestroy(g);
            return bcuda(b, le != cudaSuccess ? le : e, "graph capture");
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return bcuda(b, e, "graph instantiate");
        }
    }
    for (int f = 0; f < frames; ++f) {
        cudaError_t e = cudaGraphLaunch(b->graph, s);
        if (e != cudaSuccess)
            return bcuda(b, e, "graph launch");
        b->frames += 1;
    }
    return MMR_OK;
}

mmr_status mmr_batch_autotune(mmr_batch *b, void *stream, int frames_per_config, int *threads, int *ctas_per_sm,
                              int *chunk_groups, float *best_ms)
{
    if (!b || frames_per_config < 1 || frames_per_config > 1000)
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_autotune: bad argument");
    mmr_status st = cameras_ready(b, true);
    if (st != MMR_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    void *saved = nullptr;
    st = balloc(b, &saved, b->pos_bytes, "autotune position snapshot");
    if (st != MMR_OK)
        return st;
    const uint32_t saved_frames = b->frames;
    const mmr::LaunchShape saved_launch = b->launch;
    const uint32_t saved_chunk = b->chunk_groups;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(saved, b->pos_base, b->pos_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t1);
    st = e == cudaSuccess ? upload_cameras(b, s) : bcuda(b, e, "autotune set-up");
    // chunks are whole multiples of the block, so no thread of a CTA idles
    const int cand_threads[] = {64, 128, 256};
    const int cand_mult[] = {1, 2, 4, 8};
    const int cand_ctas[] = {0, 4, 8};
    float best = 1e30f;
    int bt = saved_launch.threads, bc = saved_launch.ctas_per_sm, bg = (int)saved_chunk;
    for (int th : cand_threads) {
        if (st != MMR_OK)
            break;
        for (int m : cand_mult) {
            if (st != MMR_OK)
                break;
            for (int ct : cand_ctas) {
                const int cg = th * m;
                st = mmr_batch_set_launch(b, th, ct, cg);
                if (st != MMR_OK)
                    break;
                e = enqueue_frame(b, s);                         // warm-up frame
                if (e == cudaSuccess)
                    e = cudaEventRecord(t0, s);
                for (int f = 0; f < frames_per_config && e == cudaSuccess; ++f)
                    e = enqueue_frame(b, s);
                if (e == cudaSuccess)
                    e = cudaEventRecord(t1, s);
                if (e == cudaSuccess)
                    e = cudaEventSynchronize(t1);
                float ms = 0.0f;
                if (e == cudaSuccess)
                    e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) {
                    st = bcuda(b, e, "autotune timing");
                    break;
                }
                ms /= (float)frames_per_config;
                if (ms < best) {
                    best = ms;
                    bt = th;
                    bc = ct;
                    bg = cg;
                }
            }
        }
    }
    // restore the simulation state whatever happened above
    cudaError_t re = cudaMemcpyAsync(b->pos_base, saved, b->pos_bytes, cudaMemcpyDeviceToDevice, s);
    if (re == cudaSuccess)
        re = cudaMemsetAsync(b->keys_base[0], 0xff, b->total_px * 8, s);
    if (re == cudaSuccess)
        re = cudaMemsetAsync(b->keys_base[1], 0xff, b->total_px * 8, s);
    if (re == cudaSuccess)
        re = cudaMemsetAsync(b->rgba_base, 0, b->total_px * 4, s);
    if (re == cudaSuccess)
        re = cudaStreamSynchronize(s);
    if (re == cudaSuccess) {
        const uint32_t fr[2] = {saved_frames, 1u};   // the cleared buffers: the next frame repaints everything
        re = cudaMemcpy(b->d_frame, fr, sizeof fr, cudaMemcpyHostToDevice);
    }
    b->frames = saved_frames;
    bfree(b, &saved, b->pos_bytes);
    if (t0)
        cudaEventDestroy(t0);
    if (t1)
        cudaEventDestroy(t1);
    if (re != cudaSuccess)
        return bcuda(b, re, "autotune restore");
    if (st != MMR_OK) {
        mmr_batch_set_launch(b, saved_launch.threads, saved_launch.ctas_per_sm, (int)saved_chunk);
        return st;
    }
    st = mmr_batch_set_launch(b, bt, bc, bg);
    if (st != MMR_OK)
        return st;
    if (threads)
        *threads = bt;
    if (ctas_per_sm)
        *ctas_per_sm = bc;
    if (chunk_groups)
        *chunk_groups = bg;
    if (best_ms)
        *best_ms = best;
    return MMR_OK;
}

mmr_status mmr_batch_check_device(mmr_batch *b)
{
    if (!b)
        return MMR_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    uint32_t err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&err, b->d_work + 1, sizeof err, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && err)
        e = cudaMemset(b->d_work + 1, 0, sizeof err);
    if (e != cudaSuccess)
        return bcuda(b, e, "mmr_batch_check_device");
    if (err)
        return bfail(b, MMR_ERR_TIMEOUT, "mmr_batch_check_device: a pixel item gave up waiting for its cloud's "
                                         "point items; that frame is incomplete");
    return MMR_OK;
}

mmr_status mmr_batch_selftest_bounded_wait(mmr_batch *b, uint32_t max_polls, void *stream)
{
    if (!b || max_polls < 1 || max_polls > kSpinLimit)
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_selftest_bounded_wait: max_polls must be 1..2^24");
    mmr::batch_wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(b->d_work + 2, max_polls, b->d_work + 1);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MMR_OK : bcuda(b, e, "mmr_batch_selftest_bounded_wait");
}

mmr_status mmr_batch_frame_ptr(mmr_batch *b, int cloud, const uint32_t **rgba, const uint64_t **depth_id)
{
    if (!b || cloud < 0 || cloud >= b->count)
        return bfail(b, MMR_ERR_INVALID_ARG, "mmr_batch_frame_ptr: bad argument");
    const int latest = b->frames ? (int)((b->frames - 1) & 1u) : 1;
    if (rgba)
        *rgba = b->rgba_base + b->px_off[cloud];
    if (depth_id)
        *depth_id = reinterpret_cast<const uint64_t *>(b->keys_base[latest] + b->px_off[cloud]);
    return MMR_OK;
}

mmr_status mmr_batch_frames(const mmr_batch *b, uint32_t *frames)
{
    if (!b || !frames)
        return MMR_ERR_INVALID_ARG;
    *frames = b->frames;
    return MMR_OK;
}

mmr_status mmr_batch_device_bytes(const mmr_batch *b, uint64_t *bytes)
{
    if (!b || !bytes)
        return MMR_ERR_INVALID_ARG;
    *bytes = b->held;
    return MMR_OK;
}

}  // extern "C"
