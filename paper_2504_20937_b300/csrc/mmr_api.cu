// libmmr C ABI: context, point allocation, camera, frames (see include/mmr.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "../../include/mmr.h"
#include "mmr_device.cuh"
#include "mmr_internal.h"
#include "mmr_disc.cuh"
#include "mmr_resolve.cuh"
#include "mmr_tiles.cuh"

namespace {

thread_local char g_create_error[512] = "";

}  // namespace

struct mmr_ctx {
    int device = 0;
    int W = 0, H = 0;
    uint64_t budget = 0;          // 0 = unlimited
    uint64_t held = 0;            // device bytes held
    mmr::LaunchShape launch;

    unsigned long long *keys[2] = {nullptr, nullptr};
    int splat_buf = 0;            // key buffer the next frame splats into
    int latest_buf = 0;           // key buffer holding the latest frame
    uint32_t *rgba = nullptr;
    uint32_t *d_err = nullptr;    // device error word (bounded waits that gave up), at the start of the control
                                  // block that also holds the frame-chunk tags
    uint64_t ctrl_bytes = 0;
    uint32_t *chunk_tags[2] = {nullptr, nullptr};  // per depth-id buffer: one tag per 64-pixel chunk (FrameChunks)
    uint32_t frame_no = 0;        // number of the latest resolved frame (1, 2, ...)
    uint32_t buf_frame[2] = {0, 0};   // number of the frame last resolved from each depth-id buffer
    bool repaint_all = true;      // the next resolve repaints and clears every pixel

    // host mirror of the framebuffer (mmr_alloc_host_mirror): mapped pinned host memory, and on the device one
    // byte per chunk (does the mirror hold a point there) after an 8-byte count of the bytes written
    uint32_t *mirror = nullptr;           // host pointer
    uint32_t *mirror_dev = nullptr;       // its device alias
    unsigned char *mirror_mem = nullptr;  // count, then the chunk bytes
    bool mirror_full = true;              // the next mirror update writes every pixel
    bool mirror_pending = false;          // a mirror update may still read the framebuffer
    cudaEvent_t frame_done = nullptr;     // recorded after every resolve once the mirror exists
    cudaEvent_t mirror_done = nullptr;    // recorded after every mirror update

    void *buf[2] = {nullptr, nullptr};   // point buffers; buf[1] only with ping-pong
    int visible = 0;                     // the buffer holding the current state (rendered)
    uint64_t n = 0;
    int dtype = 0;
    uint64_t point_bytes = 0;
    uint32_t *colors = nullptr;
    float *nb_vel = nullptr;             // N-body workload: velocities (3n) and masses (n)
    float *nb_mass = nullptr;
    float4 *nb_partial = nullptr;        // per-chunk partial sums (scratch)
    uint32_t *index = nullptr;           // indexed colour: colormap[index[id]]
    uint32_t *colormap = nullptr;
    uint32_t ncolors = 0;

    // screen-tile depth bounds (MMR_KERNEL_DEPTH_BOUND), allocated on first use: one block of
    // 16 bytes per 8x8 tile (mark, list, bound) plus the list's count
    unsigned char *tiles_mem = nullptr;
    uint64_t tiles = 0;
    uint32_t tiles_w = 0;
    uint32_t tile_tag = 0;
    int last_frame_kernels = 0;    // kernels the latest frame launched

    // round-trip baseline buffers (allocated on first use)
    void *rt_device = nullptr;
    void *rt_host = nullptr;
    int rt_host_pinned = -1;

    mmr::Cam cam{};
    bool have_cam = false;
    float matrix[16] = {};

    uint64_t seed = 0;
    uint32_t cloud = 0;
    float amplitude = 0.0f;
    uint32_t step = 0;
    uint32_t color = 0xFFFFFFFFu;
    uint32_t background = 0u;
    float disc_r = 0.0f;          // 0: 1-px points; else disc markers of this radius (pixels)

    // per-kernel timing: a ring of event triples (before the point phase, between it and the resolve, after
    // the resolve), one triple per frame, so a caller can enqueue many frames and read their times afterwards
    bool timing = false;
    uint32_t timed_frames = 0;                 // frames timed since timing was switched on
    cudaEvent_t *ring = nullptr;               // kTimingRing * 3 events
    cudaEvent_t *ev = nullptr;                 // the triple of the frame being enqueued

    char err[512] = "";
};

namespace {

constexpr uint32_t kTimingRing = MMR_TIMING_RING;

mmr_status fail(mmr_ctx *c, mmr_status s, const char *fmt, ...)
{
    char *dst = c ? c->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return s;
}

mmr_status cuda_fail(mmr_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, MMR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// Test hook: MMR_FAIL_ALLOC_AFTER=k makes every device allocation after the
// first k in this process report out-of-memory (host-side, no device fault).
bool injected_alloc_failure()
{
    static long long count = 0;
    const char *v = getenv("MMR_FAIL_ALLOC_AFTER");
    if (!v || !*v)
        return false;
    return count++ >= atoll(v);
}

mmr_status dev_alloc(mmr_ctx *c, void **p, uint64_t bytes, const char *what)
{
    *p = nullptr;
    if (c->budget && c->held + bytes > c->budget)
        return fail(c, MMR_ERR_BUDGET, "%s: %llu bytes would exceed the budget (%llu of %llu held)",
                    what, (unsigned long long)bytes, (unsigned long long)c->held,
                    (unsigned long long)c->budget);
    if (injected_alloc_failure())
        return fail(c, MMR_ERR_OOM, "%s: injected allocation failure", what);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, e == cudaErrorMemoryAllocation ? MMR_ERR_OOM : MMR_ERR_CUDA,
                    "%s: cudaMalloc(%llu) failed: %s", what, (unsigned long long)bytes,
                    cudaGetErrorString(e));
    }
    c->held += bytes;
    return MMR_OK;
}

void dev_free(mmr_ctx *c, void **p, uint64_t bytes)
{
    if (*p) {
        cudaFree(*p);
        c->held -= bytes;
        *p = nullptr;
    }
}

uint64_t frame_px(const mmr_ctx *c) { return (uint64_t)c->W * (uint64_t)c->H; }

uint64_t bytes_per_point(int dtype) { return dtype == MMR_F32x3 ? 12u : 6u; }

// Storage is padded to whole 48-byte groups so the vector path never reads
// past the allocation.
uint64_t storage_bytes(uint64_t n, int dtype)
{
    const uint64_t raw = n * bytes_per_point(dtype);
    return (raw + 47) / 48 * 48;
}

mmr::PointParams point_params(const mmr_ctx *c)
{
    mmr::PointParams P{};
    P.cam = c->cam;
    P.keys = c->keys[c->splat_buf];
    P.W = c->W;
    P.H = c->H;
    P.fW = (float)c->W;
    P.fH = (float)c->H;
    P.halfW = 0.5f * (float)c->W;
    P.halfH = 0.5f * (float)c->H;
    P.seed_lo = (uint32_t)(c->seed & 0xffffffffu);
    P.seed_hi = (uint32_t)(c->seed >> 32);
    P.step = c->step;
    P.cloud = c->cloud;
    P.amplitude = c->amplitude;
    P.id_base = 0;
    P.disc_r = c->disc_r;
    P.disc_r2 = c->disc_r * c->disc_r;
    mmr::philox_prepare(P);
    return P;
}

mmr::Palette palette(const mmr_ctx *c)
{
    return mmr::Palette{c->colors, c->index, c->colormap, c->ncolors, c->color, c->background};
}

mmr_status check_frame_ready(mmr_ctx *c, bool need_cam)
{
    if (!c->buf[0])
        return fail(c, MMR_ERR_STATE, "no points allocated (call mmr_alloc_points first)");
    if (need_cam && !c->have_cam)
        return fail(c, MMR_ERR_STATE, "no camera set (call mmr_set_camera or mmr_set_matrix first)");
    return MMR_OK;
}

bool uses_tma(const mmr::LaunchShape &ls) { return ls.kernel == MMR_KERNEL_TMA; }

uint64_t tile_bytes(uint64_t tiles) { return 16 * tiles + 16; }

// Control block: the 4-byte device error word, padded to 16 bytes, then the
// chunk tags of both depth-id buffers.
uint64_t frame_chunks_of(const mmr_ctx *c) { return (frame_px(c) + 63) / 64; }
uint64_t control_bytes(const mmr_ctx *c) { return 16 + 2 * 4 * frame_chunks_of(c); }

// The chunk bookkeeping of the resolve that turns depth-id buffer `cur` into
// the framebuffer and clears the other one.  Frame numbers run 1, 2, ...; tags
// start at 0, which matches the "previous frame" of both buffers before any
// frame, so the first resolve clears everything.  Before the numbers would
// repeat the tags are cleared on the stream and counting starts again.
mmr::FrameChunks frame_chunks(mmr_ctx *c, int cur, cudaStream_t s, cudaError_t *e)
{
    *e = cudaSuccess;
    if (c->frame_no == 0xffffffffu) {
        *e = cudaMemsetAsync(c->chunk_tags[0], 0, 2 * 4 * frame_chunks_of(c), s);
        c->frame_no = 0;
        c->buf_frame[0] = c->buf_frame[1] = 0;
        c->repaint_all = true;
    }
    return mmr::FrameChunks{c->chunk_tags[cur ^ 1], c->chunk_tags[cur], c->buf_frame[cur ^ 1], c->frame_no + 1,
                            c->repaint_all ? 1u : 0u};
}

// After the resolve of buffer `cur` is enqueued.
void frame_resolved(mmr_ctx *c, int cur)
{
    c->frame_no += 1;
    c->buf_frame[cur] = c->frame_no;
    c->repaint_all = false;
}

uint64_t mirror_mem_bytes(const mmr_ctx *c) { return 8 + frame_chunks_of(c); }

// Before a resolve on s: a mirror update still reading the framebuffer it
// rewrites must finish first.
cudaError_t before_resolve(mmr_ctx *c, cudaStream_t s)
{
    if (!c->mirror_pending)
        return cudaSuccess;
    c->mirror_pending = false;
    return cudaStreamWaitEvent(s, c->mirror_done, 0);
}

// After a resolve on s: the point a mirror update on another stream waits for.
cudaError_t after_resolve(mmr_ctx *c, cudaStream_t s)
{
    return c->mirror ? cudaEventRecord(c->frame_done, s) : cudaSuccess;
}

// The depth-bound path pays for disc markers where many discs cover each
// pixel: at least kDiscCoverMin on average (n pi r^2 / pixels), for clouds of
// at least 2^20 points.  Measured on the 2^22-point 1080p orbit (direct ->
// bounded, first pass 1/8): r = 2, 25 discs per pixel, 0.154 -> 0.263 ms;
// r = 4, 100 per pixel, 0.42 -> 0.23 ms; r = 8, 400, 1.52 -> 0.35 ms; r = 16,
// 1600, 5.86 -> 0.96 ms (0.80 ms with a first pass of 1/16).  For 1-px points
// it is chosen only explicitly: on the 64M-point 16-cluster 4K frame it cost
// 8% in FP32 and 9% in binary16, at every first-pass share tried.
constexpr double kDiscCoverMin = 64.0;

double discs_per_pixel(const mmr_ctx *c)
{
    return (double)c->n * 3.14159265358979 * c->disc_r * c->disc_r / (double)frame_px(c);
}

// The first pass's share, 2^-shift: as set by mmr_set_depth_bound_split,
// else 1/16 for discs covering each pixel a thousand times or more and 1/8
// otherwise (the fastest of 1/4 .. 1/64 measured at r = 4, 8 and 16).
int bound_shift(const mmr_ctx *c)
{
    if (c->launch.bound_shift > 0)
        return c->launch.bound_shift;
    return c->disc_r > 0.0f && discs_per_pixel(c) >= 1024.0 ? 4 : 3;
}

bool uses_depth_bound(const mmr_ctx *c)
{
    if (c->launch.kernel == MMR_KERNEL_DEPTH_BOUND)
        return true;
    if (c->launch.kernel != MMR_KERNEL_AUTO || c->n < (1ull << 20))
        return false;
    if (c->disc_r > 0.0f)
        return discs_per_pixel(c) >= kDiscCoverMin;
    return false;     // 1-px points: the direct splat
}

// The tile arrays of the depth-bound path, allocated (zero-filled: no tile
// marked, no bound, an empty list) the first time a frame needs them.
mmr_status ensure_tiles(mmr_ctx *c)
{
    if (c->tiles_mem)
        return MMR_OK;
    const uint64_t tw = ((uint64_t)c->W + 7) / 8, th = ((uint64_t)c->H + 7) / 8;
    mmr_status st = dev_alloc(c, (void **)&c->tiles_mem, tile_bytes(tw * th), "tile depth bounds");
    if (st != MMR_OK)
        return st;
    cudaError_t e = cudaMemset(c->tiles_mem, 0, tile_bytes(tw * th));
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dev_free(c, (void **)&c->tiles_mem, tile_bytes(tw * th));
        return cuda_fail(c, e, "clearing the tile depth bounds");
    }
    c->tiles = tw * th;
    c->tiles_w = (uint32_t)tw;
    c->tile_tag = 0;
    return MMR_OK;
}

// This frame's view of the tile arrays, with a fresh tag.  Tags run 1, 2, ...;
// when the 32-bit tag wraps the arrays are cleared on the stream, so no entry
// of an earlier frame can carry the new tag.
mmr::TileBounds next_tile_bounds(mmr_ctx *c, cudaStream_t s, cudaError_t *e)
{
    *e = cudaSuccess;
    if (++c->tile_tag == 0) {
        *e = cudaMemsetAsync(c->tiles_mem, 0, tile_bytes(c->tiles), s);
        c->tile_tag = 1;
    }
    mmr::TileBounds T{};
    T.mark = reinterpret_cast<uint32_t *>(c->tiles_mem);
    T.list = T.mark + c->tiles;
    T.bound = reinterpret_cast<unsigned long long *>(c->tiles_mem + 8 * c->tiles);
    T.count = reinterpret_cast<uint32_t *>(c->tiles_mem + 16 * c->tiles);
    T.tag = c->tile_tag;
    T.tiles_w = c->tiles_w;
    T.tiles = (uint32_t)c->tiles;
    return T;
}

// The point phase of a frame: the disc kernel for disc markers, the TMA-staged
// persistent kernel or the depth-bounded passes when chosen, else the
// grid-stride kernel (direct or warp-aggregated splat).  Sets the number of
// kernels launched.
cudaError_t launch_point_kernel(mmr_ctx *c, const void *src, void *dst, const mmr::PointParams &P, bool displace,
                                bool splat, cudaStream_t s)
{
    c->last_frame_kernels = 1;
    if (splat && c->disc_r > 0.0f) {
        if (uses_depth_bound(c) && c->tiles_mem) {
            cudaError_t e;
            const mmr::TileBounds fine = next_tile_bounds(c, s, &e);
            if (e != cudaSuccess)
                return e;
            // the 32x32-tile bounds live in the fine tiles' bound array, which is more than large enough
            mmr::DiscBounds T{fine.bound, fine.tag, (uint32_t)((c->W + 31) / 32), (uint32_t)((c->H + 31) / 32)};
            c->last_frame_kernels = 3;
            return mmr::launch_points_disc(c->dtype, src, dst, (uint32_t)c->n, P, displace, &T, bound_shift(c),
                                           c->launch.sm_count, s);
        }
        return mmr::launch_points_disc(c->dtype, src, dst, (uint32_t)c->n, P, displace, nullptr, 0,
                                       c->launch.sm_count, s);
    }
    if (uses_tma(c->launch))
        return mmr::launch_points_tma(c->dtype, src, dst, (uint32_t)c->n, P, displace, splat, c->d_err, c->launch,
                                      s);
    if (splat && uses_depth_bound(c) && c->tiles_mem) {
        cudaError_t e;
        const mmr::TileBounds T = next_tile_bounds(c, s, &e);
        if (e != cudaSuccess)
            return e;
        c->last_frame_kernels = 3;
        mmr::LaunchShape ls = c->launch;
        ls.bound_shift = bound_shift(c);
        return mmr::launch_points_bounded(c->dtype, src, dst, (uint32_t)c->n, P, displace, T, (uint32_t)c->tiles, ls,
                                          s);
    }
    mmr::LaunchShape ls = c->launch;
    if (ls.kernel != MMR_KERNEL_WARP_AGG)
        ls.kernel = MMR_KERNEL_GRID;
    return mmr::launch_points(c->dtype, src, dst, (uint32_t)c->n, P, displace, splat, ls, s);
}

// Render the positions in `src` into the splat key buffer (displacing them
// into `dst` first when `displace`), then resolve and flip key buffers.
mmr_status frame(mmr_ctx *c, const void *src, void *dst, bool displace, cudaStream_t s)
{
    if (uses_depth_bound(c)) {
        mmr_status st = ensure_tiles(c);
        if (st != MMR_OK)
            return st;
    }
    mmr::PointParams P = point_params(c);
    if (c->timing) {
        c->ev = c->ring + 3 * (c->timed_frames % kTimingRing);
        cudaEventRecord(c->ev[0], s);
    }
    cudaError_t e = launch_point_kernel(c, src, dst, P, displace, true, s);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "point kernel launch");
    if (c->timing)
        cudaEventRecord(c->ev[1], s);
    const int cur = c->splat_buf;
    const mmr::FrameChunks F = frame_chunks(c, cur, s, &e);
    if (e == cudaSuccess)
        e = before_resolve(c, s);
    if (e == cudaSuccess)
        e = mmr::launch_resolve(c->keys[cur], c->keys[cur ^ 1], c->rgba, palette(c), (uint32_t)frame_px(c), F, s);
    if (e == cudaSuccess)
        e = after_resolve(c, s);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "resolve kernel launch");
    frame_resolved(c, cur);
    if (c->timing) {
        cudaEventRecord(c->ev[2], s);
        c->timed_frames += 1;
    }
    c->last_frame_kernels += 1;
    c->latest_buf = cur;
    c->splat_buf = cur ^ 1;
    if (displace)
        c->step += 1;
    return MMR_OK;
}

}  // namespace

namespace mmr {

void set_process_error(const char *msg) { snprintf(g_create_error, sizeof g_create_error, "%s", msg); }

bool build_clip_matrix(const double eye[3], const double target[3], const double up[3],
                       double fovy_deg, double aspect, double znear, double zfar, float out[16])
{
    // View: forward f = normalize(target - eye), side s = normalize(f x up),
    // true up u = s x f.  Perspective: g = cot(fovy/2).  M = P * V in FP64.
    double f[3] = {target[0] - eye[0], target[1] - eye[1], target[2] - eye[2]};
    const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0.0) || !std::isfinite(fl))
        return false;
    for (double &v : f)
        v /= fl;
    double s[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    const double sl = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (!(sl > 0.0) || !std::isfinite(sl))
        return false;   // up parallel to the view direction
    for (double &v : s)
        v /= sl;
    const double u[3] = {s[1] * f[2] - s[2] * f[1], s[2] * f[0] - s[0] * f[2], s[0] * f[1] - s[1] * f[0]};
    auto dot = [](const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    const double view[4][4] = {
        {s[0], s[1], s[2], -dot(s, eye)},
        {u[0], u[1], u[2], -dot(u, eye)},
        {-f[0], -f[1], -f[2], dot(f, eye)},
        {0.0, 0.0, 0.0, 1.0},
    };
    const double kPi = 3.14159265358979323846;
    const double g = 1.0 / std::tan(0.5 * fovy_deg * (kPi / 180.0));
    const double proj[4][4] = {
        {g / aspect, 0.0, 0.0, 0.0},
        {0.0, g, 0.0, 0.0},
        {0.0, 0.0, (zfar + znear) / (znear - zfar), 2.0 * zfar * znear / (znear - zfar)},
        {0.0, 0.0, -1.0, 0.0},
    };
    for (int r = 0; r < 4; ++r)
        for (int col = 0; col < 4; ++col) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k)
                acc += proj[r][k] * view[k][col];
            out[4 * r + col] = (float)acc;
        }
    return true;
}

}  // namespace mmr

// ============================================================== C ABI

extern "C" {

const char *mmr_status_string(mmr_status s)
{
    switch (s) {
    case MMR_OK: return "ok";
    case MMR_ERR_INVALID_ARG: return "invalid argument";
    case MMR_ERR_OOM: return "out of memory";
    case MMR_ERR_BUDGET: return "over device-memory budget";
    case MMR_ERR_CUDA: return "CUDA error";
    case MMR_ERR_STATE: return "call out of order";
    case MMR_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

const char *mmr_last_error(const mmr_ctx *ctx) { return ctx ? ctx->err : g_create_error; }

mmr_status mmr_create_ex(int width, int height, uint64_t budget_bytes, mmr_ctx **out)
{
    if (!out)
        return fail(nullptr, MMR_ERR_INVALID_ARG, "mmr_create: out is NULL");
    *out = nullptr;
    if (width < 1 || height < 1 || width > 32768 || height > 32768)
        return fail(nullptr, MMR_ERR_INVALID_ARG, "mmr_create: size %dx%d outside 1..32768", width, height);
    mmr_ctx *c = new (std::nothrow) mmr_ctx();
    if (!c)
        return fail(nullptr, MMR_ERR_OOM, "mmr_create: host allocation failed");
    c->W = width;
    c->H = height;
    c->budget = budget_bytes;
    c->launch.threads = 64;           // fastest measured shape (grid-stride, one thread per group)
    c->launch.ctas_per_sm = 0;
    c->launch.kernel = MMR_KERNEL_AUTO;   // depth bounds for dense disc markers, else the grid-stride kernel
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->launch.sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(nullptr, MMR_ERR_CUDA, "mmr_create: no usable CUDA device: %s", cudaGetErrorString(e));
        delete c;
        return MMR_ERR_CUDA;
    }
    const uint64_t npx = frame_px(c);
    mmr_status st = dev_alloc(c, (void **)&c->keys[0], npx * 8, "depth-id buffer 0");
    if (st == MMR_OK)
        st = dev_alloc(c, (void **)&c->keys[1], npx * 8, "depth-id buffer 1");
    if (st == MMR_OK)
        st = dev_alloc(c, (void **)&c->rgba, npx * 4, "RGBA framebuffer");
    c->ctrl_bytes = control_bytes(c);
    if (st == MMR_OK)
        st = dev_alloc(c, (void **)&c->d_err, c->ctrl_bytes, "device error word and frame-chunk tags");
    if (st == MMR_OK) {
        c->chunk_tags[0] = c->d_err + 4;
        c->chunk_tags[1] = c->chunk_tags[0] + frame_chunks_of(c);
        if (const char *v = getenv("MMR_FIRST_FRAME_NUMBER"))      // test hook: start near the wrap of the numbers
            c->frame_no = (uint32_t)strtoul(v, nullptr, 0);
        e = cudaMemset(c->d_err, 0, c->ctrl_bytes);
        if (e == cudaSuccess)
            e = cudaMemset(c->keys[0], 0xff, npx * 8);
        if (e == cudaSuccess)
            e = cudaMemset(c->keys[1], 0xff, npx * 8);
        if (e == cudaSuccess)
            e = cudaMemset(c->rgba, 0, npx * 4);
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
        if (e != cudaSuccess)
            st = cuda_fail(c, e, "mmr_create: clearing buffers");
    }
    if (st != MMR_OK) {
        snprintf(g_create_error, sizeof g_create_error, "%s", c->err);
        mmr_destroy(c);
        return st;
    }
    g_create_error[0] = 0;
    *out = c;
    return MMR_OK;
}

mmr_status mmr_create(int width, int height, mmr_ctx **out) { return mmr_create_ex(width, height, 0, out); }

mmr_status mmr_destroy(mmr_ctx *ctx)
{
    if (!ctx)
        return MMR_OK;
    cudaDeviceSynchronize();
    dev_free(ctx, (void **)&ctx->keys[0], frame_px(ctx) * 8);
    dev_free(ctx, (void **)&ctx->keys[1], frame_px(ctx) * 8);
    dev_free(ctx, (void **)&ctx->rgba, frame_px(ctx) * 4);
    dev_free(ctx, (void **)&ctx->d_err, ctx->ctrl_bytes);
    dev_free(ctx, &ctx->buf[0], storage_bytes(ctx->n, ctx->dtype));
    dev_free(ctx, &ctx->buf[1], storage_bytes(ctx->n, ctx->dtype));
    dev_free(ctx, (void **)&ctx->colors, ctx->n * 4);
    dev_free(ctx, (void **)&ctx->index, ctx->n * 4);
    dev_free(ctx, (void **)&ctx->nb_vel, ctx->n * 12);
    dev_free(ctx, (void **)&ctx->nb_mass, ctx->n * 4);
    dev_free(ctx, (void **)&ctx->nb_partial, (uint64_t)mmr::nbody_chunks((uint32_t)ctx->n) * ctx->n * 16);
    dev_free(ctx, (void **)&ctx->colormap, (uint64_t)ctx->ncolors * 4);
    dev_free(ctx, &ctx->rt_device, storage_bytes(ctx->n, ctx->dtype));
    dev_free(ctx, (void **)&ctx->tiles_mem, tile_bytes(ctx->tiles));
    if (ctx->rt_host) {
        if (ctx->rt_host_pinned == 1)
            cudaFreeHost(ctx->rt_host);
        else
            free(ctx->rt_host);
    }
    dev_free(ctx, (void **)&ctx->mirror_mem, mirror_mem_bytes(ctx));
    if (ctx->mirror)
        cudaFreeHost(ctx->mirror);
    if (ctx->frame_done)
        cudaEventDestroy(ctx->frame_done);
    if (ctx->mirror_done)
        cudaEventDestroy(ctx->mirror_done);
    if (ctx->ring) {
        for (uint32_t k = 0; k < 3 * kTimingRing; ++k)
            if (ctx->ring[k])
                cudaEventDestroy(ctx->ring[k]);
        delete[] ctx->ring;
    }
    delete ctx;
    return MMR_OK;
}

static mmr_status alloc_point_buffers(mmr_ctx *ctx, uint64_t n, int dtype, int count, const char *who)
{
    if (n == 0 || n >= (1ull << 32))
        return fail(ctx, MMR_ERR_INVALID_ARG, "%s: n=%llu outside 1..2^32-1", who, (unsigned long long)n);
    if (dtype != MMR_F32x3 && dtype != MMR_F16x3 && dtype != MMR_BF16x3)
        return fail(ctx, MMR_ERR_INVALID_ARG, "%s: unknown dtype %d", who, dtype);
    if (ctx->buf[0])
        return fail(ctx, MMR_ERR_STATE, "%s: this context already has points", who);
    const uint64_t bytes = storage_bytes(n, dtype);
    for (int k = 0; k < count; ++k) {
        mmr_status st = dev_alloc(ctx, &ctx->buf[k], bytes, k ? "second point buffer" : "point buffer");
        cudaError_t e = st == MMR_OK ? cudaMemset(ctx->buf[k], 0, bytes) : cudaSuccess;
        if (st == MMR_OK && e == cudaSuccess)
            e = cudaDeviceSynchronize();
        if (st != MMR_OK || e != cudaSuccess) {
            if (st == MMR_OK)
                st = cuda_fail(ctx, e, "clearing points");
            dev_free(ctx, &ctx->buf[0], bytes);
            dev_free(ctx, &ctx->buf[1], bytes);
            return st;
        }
    }
    ctx->n = n;
    ctx->dtype = dtype;
    ctx->point_bytes = n * bytes_per_point(dtype);
    ctx->visible = 0;
    return MMR_OK;
}

mmr_status mmr_alloc_points(mmr_ctx *ctx, uint64_t n, int dtype, void **dev_ptr)
{
    if (!ctx || !dev_ptr)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_alloc_points: NULL argument");
    *dev_ptr = nullptr;
    mmr_status st = alloc_point_buffers(ctx, n, dtype, 1, "mmr_alloc_points");
    if (st == MMR_OK)
        *dev_ptr = ctx->buf[0];
    return st;
}

mmr_status mmr_alloc_pingpong(mmr_ctx *ctx, uint64_t n, int dtype, void **dev_a, void **dev_b)
{
    if (!ctx || !dev_a || !dev_b)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_alloc_pingpong: NULL argument");
    *dev_a = *dev_b = nullptr;
    mmr_status st = alloc_point_buffers(ctx, n, dtype, 2, "mmr_alloc_pingpong");
    if (st == MMR_OK) {
        *dev_a = ctx->buf[0];
        *dev_b = ctx->buf[1];
    }
    return st;
}

mmr_status mmr_set_visible(mmr_ctx *ctx, int which)
{
    if (!ctx || (which != 0 && which != 1))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_visible: which must be 0 or 1");
    if (!ctx->buf[which])
        return fail(ctx, MMR_ERR_STATE, "mmr_set_visible: buffer %d not allocated (use mmr_alloc_pingpong)", which);
    ctx->visible = which;
    return MMR_OK;
}

mmr_status mmr_get_visible(const mmr_ctx *ctx, int *which)
{
    if (!ctx || !which)
        return MMR_ERR_INVALID_ARG;
    *which = ctx->visible;
    return MMR_OK;
}

mmr_status mmr_step_and_render_pingpong(mmr_ctx *ctx, void *stream)
{
    mmr::NvtxRange nvtx("mmr_step_and_render_pingpong");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = check_frame_ready(ctx, true);
    if (st != MMR_OK)
        return st;
    if (!ctx->buf[1])
        return fail(ctx, MMR_ERR_STATE, "mmr_step_and_render_pingpong: no second buffer (use mmr_alloc_pingpong)");
    const int r = ctx->visible;
    st = frame(ctx, ctx->buf[r], ctx->buf[r ^ 1], true, (cudaStream_t)stream);
    if (st == MMR_OK)
        ctx->visible = r ^ 1;
    return st;
}

mmr_status mmr_alloc_nbody(mmr_ctx *ctx, float **dev_vel, float **dev_mass)
{
    if (!ctx || !dev_vel || !dev_mass)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_alloc_nbody: NULL argument");
    *dev_vel = nullptr;
    *dev_mass = nullptr;
    if (!ctx->buf[1] || ctx->dtype != MMR_F32x3)
        return fail(ctx, MMR_ERR_STATE, "mmr_alloc_nbody: needs FP32 ping-pong buffers (mmr_alloc_pingpong)");
    if (ctx->nb_vel)
        return fail(ctx, MMR_ERR_STATE, "mmr_alloc_nbody: already allocated");
    const uint64_t partial_bytes = (uint64_t)mmr::nbody_chunks((uint32_t)ctx->n) * ctx->n * 16;
    mmr_status st = dev_alloc(ctx, (void **)&ctx->nb_vel, ctx->n * 12, "N-body velocities");
    if (st == MMR_OK)
        st = dev_alloc(ctx, (void **)&ctx->nb_mass, ctx->n * 4, "N-body masses");
    if (st == MMR_OK)
        st = dev_alloc(ctx, (void **)&ctx->nb_partial, partial_bytes, "N-body partial sums");
    if (st != MMR_OK) {
        dev_free(ctx, (void **)&ctx->nb_vel, ctx->n * 12);
        dev_free(ctx, (void **)&ctx->nb_mass, ctx->n * 4);
        return st;
    }
    cudaError_t e = cudaMemset(ctx->nb_vel, 0, ctx->n * 12);
    if (e == cudaSuccess)
        e = cudaMemset(ctx->nb_mass, 0, ctx->n * 4);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_alloc_nbody: clearing");
    *dev_vel = ctx->nb_vel;
    *dev_mass = ctx->nb_mass;
    return MMR_OK;
}

mmr_status mmr_nbody_step_and_render(mmr_ctx *ctx, float G, float eps2, float dt, void *stream)
{
    mmr::NvtxRange nvtx("mmr_nbody_step_and_render");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = check_frame_ready(ctx, true);
    if (st != MMR_OK)
        return st;
    if (!ctx->nb_vel)
        return fail(ctx, MMR_ERR_STATE, "mmr_nbody_step_and_render: call mmr_alloc_nbody first");
    if (!std::isfinite(G) || !(eps2 > 0.0f) || !std::isfinite(eps2) || !std::isfinite(dt))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_nbody_step_and_render: need finite G, dt and eps2 > 0");
    cudaStream_t s = (cudaStream_t)stream;
    mmr::PointParams P = point_params(ctx);
    const mmr::NbodyParams B{G, eps2, dt};
    const int r = ctx->visible;
    if (ctx->timing) {
        ctx->ev = ctx->ring + 3 * (ctx->timed_frames % kTimingRing);
        cudaEventRecord(ctx->ev[0], s);
    }
    cudaError_t e = mmr::launch_nbody(static_cast<const float *>(ctx->buf[r]), static_cast<float *>(ctx->buf[r ^ 1]),
                                      ctx->nb_vel, ctx->nb_mass, ctx->nb_partial, (uint32_t)ctx->n, B, P, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "N-body kernel launch");
    if (ctx->timing)
        cudaEventRecord(ctx->ev[1], s);
    const int cur = ctx->splat_buf;
    const mmr::FrameChunks F = frame_chunks(ctx, cur, s, &e);
    if (e == cudaSuccess)
        e = before_resolve(ctx, s);
    if (e == cudaSuccess)
        e = mmr::launch_resolve(ctx->keys[cur], ctx->keys[cur ^ 1], ctx->rgba, palette(ctx), (uint32_t)frame_px(ctx),
                                F, s);
    if (e == cudaSuccess)
        e = after_resolve(ctx, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "resolve kernel launch");
    frame_resolved(ctx, cur);
    if (ctx->timing) {
        cudaEventRecord(ctx->ev[2], s);
        ctx->timed_frames += 1;
    }
    ctx->latest_buf = cur;
    ctx->splat_buf = cur ^ 1;
    ctx->visible = r ^ 1;
    ctx->step += 1;
    return MMR_OK;
}

mmr_status mmr_alloc_indexed_colors(mmr_ctx *ctx, uint32_t ncolors, uint32_t **dev_index, uint32_t **dev_colormap)
{
    if (!ctx || !dev_index || !dev_colormap || ncolors == 0 || ncolors > (1u << 24))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_alloc_indexed_colors: bad argument (1 <= ncolors <= 2^24)");
    *dev_index = nullptr;
    *dev_colormap = nullptr;
    if (!ctx->buf[0])
        return fail(ctx, MMR_ERR_STATE, "mmr_alloc_indexed_colors: allocate points first");
    if (ctx->index)
        return fail(ctx, MMR_ERR_STATE, "mmr_alloc_indexed_colors: already allocated");
    mmr_status st = dev_alloc(ctx, (void **)&ctx->index, ctx->n * 4, "colour index buffer");
    if (st == MMR_OK)
        st = dev_alloc(ctx, (void **)&ctx->colormap, (uint64_t)ncolors * 4, "colormap");
    if (st != MMR_OK) {
        dev_free(ctx, (void **)&ctx->index, ctx->n * 4);
        return st;
    }
    ctx->ncolors = ncolors;
    cudaError_t e = cudaMemset(ctx->index, 0, ctx->n * 4);
    if (e == cudaSuccess)
        e = cudaMemset(ctx->colormap, 0xff, (uint64_t)ncolors * 4);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_alloc_indexed_colors: clearing");
    *dev_index = ctx->index;
    *dev_colormap = ctx->colormap;
    return MMR_OK;
}

mmr_status mmr_alloc_colors(mmr_ctx *ctx, uint32_t **dev_colors)
{
    if (!ctx || !dev_colors)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_alloc_colors: NULL argument");
    *dev_colors = nullptr;
    if (!ctx->buf[0])
        return fail(ctx, MMR_ERR_STATE, "mmr_alloc_colors: allocate points first");
    if (!ctx->colors) {
        mmr_status st = dev_alloc(ctx, (void **)&ctx->colors, ctx->n * 4, "colour buffer");
        if (st != MMR_OK)
            return st;
        cudaError_t e = cudaMemset(ctx->colors, 0xff, ctx->n * 4);
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "mmr_alloc_colors: clearing");
    }
    *dev_colors = ctx->colors;
    return MMR_OK;
}

mmr_status mmr_set_matrix(mmr_ctx *ctx, const float m[16], float znear, float zfar)
{
    if (!ctx || !m)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_matrix: NULL argument");
    if (!mmr::depth_range_ok(znear, zfar))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_matrix: need 2^-64 <= znear < zfar <= 2^64");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(m[k]))
            return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_matrix: non-finite entry %d", k);
    memcpy(ctx->matrix, m, sizeof ctx->matrix);
    for (int k = 0; k < 4; ++k) {
        ctx->cam.rx[k] = m[k];
        ctx->cam.ry[k] = m[4 + k];
        ctx->cam.rw[k] = m[12 + k];
    }
    ctx->cam.znear = znear;
    ctx->cam.zfar = zfar;
    ctx->have_cam = true;
    return MMR_OK;
}

mmr_status mmr_get_matrix(const mmr_ctx *ctx, float m[16])
{
    if (!ctx || !m)
        return MMR_ERR_INVALID_ARG;
    if (!ctx->have_cam)
        return MMR_ERR_STATE;
    memcpy(m, ctx->matrix, sizeof ctx->matrix);
    return MMR_OK;
}

mmr_status mmr_set_camera(mmr_ctx *ctx, const double eye[3], const double target[3],
                          const double up[3], double fovy_deg, double znear, double zfar)
{
    if (!ctx || !eye || !target || !up)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_camera: NULL argument");
    if (!(fovy_deg > 0.0 && fovy_deg < 180.0) || !(znear > 0.0) || !(zfar > znear) || !std::isfinite(zfar) ||
        !mmr::depth_range_ok((float)znear, (float)zfar))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_camera: need 0 < fovy < 180, 2^-64 <= znear < zfar <= 2^64");
    float m[16];
    if (!mmr::build_clip_matrix(eye, target, up, fovy_deg, (double)ctx->W / (double)ctx->H, znear, zfar, m))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_camera: eye == target or up parallel to view");
    return mmr_set_matrix(ctx, m, (float)znear, (float)zfar);
}

mmr_status mmr_set_sim(mmr_ctx *ctx, uint64_t seed, uint32_t cloud, float amplitude, uint32_t first_step)
{
    if (!ctx)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_sim: NULL ctx");
    if (!mmr::amplitude_ok(amplitude))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_sim: amplitude must be 0 or in [2^-100, 1]");
    ctx->seed = seed;
    ctx->cloud = cloud;
    ctx->amplitude = amplitude;
    ctx->step = first_step;
    return MMR_OK;
}

mmr_status mmr_set_style(mmr_ctx *ctx, uint32_t color, uint32_t background)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    ctx->color = color;
    if (background != ctx->background) {
        ctx->repaint_all = true;      // pixels left as background by earlier frames are repainted
        ctx->mirror_full = true;      // and so are those of the host mirror
    }
    ctx->background = background;
    return MMR_OK;
}

mmr_status mmr_set_marker(mmr_ctx *ctx, float radius_px)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (!(radius_px == 0.0f || (radius_px >= 0.5f && radius_px <= 64.0f)))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_marker: radius must be 0 (1-px points) or in [0.5, 64]");
    ctx->disc_r = radius_px;
    return MMR_OK;
}

mmr_status mmr_set_launch(mmr_ctx *ctx, int threads, int ctas_per_sm, int kernel)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (threads < 32 || threads > 1024 || threads % 32 != 0 || ctas_per_sm < 0 || ctas_per_sm > 64)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_launch: threads %d / ctas_per_sm %d out of range",
                    threads, ctas_per_sm);
    if (kernel < MMR_KERNEL_GRID || kernel > MMR_KERNEL_AUTO)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_launch: unknown kernel %d", kernel);
    if (kernel == MMR_KERNEL_TMA && (ctas_per_sm < 1 || (threads != 128 && threads != 256 && threads != 512)))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_launch: the TMA kernel needs 128/256/512 threads and "
                    "ctas_per_sm >= 1");
    ctx->launch.threads = threads;
    ctx->launch.ctas_per_sm = ctas_per_sm;
    ctx->launch.kernel = kernel;
    return MMR_OK;
}

mmr_status mmr_step_and_render(mmr_ctx *ctx, void *stream)
{
    mmr::NvtxRange nvtx("mmr_step_and_render");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = check_frame_ready(ctx, true);
    if (st != MMR_OK)
        return st;
    void *cur = ctx->buf[ctx->visible];
    return frame(ctx, cur, cur, true, (cudaStream_t)stream);
}

mmr_status mmr_render(mmr_ctx *ctx, void *stream)
{
    mmr::NvtxRange nvtx("mmr_render");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = check_frame_ready(ctx, true);
    if (st != MMR_OK)
        return st;
    return frame(ctx, ctx->buf[ctx->visible], nullptr, false, (cudaStream_t)stream);
}

mmr_status mmr_displace(mmr_ctx *ctx, void *stream)
{
    mmr::NvtxRange nvtx("mmr_displace");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = check_frame_ready(ctx, false);
    if (st != MMR_OK)
        return st;
    mmr::PointParams P = point_params(ctx);
    void *cur = ctx->buf[ctx->visible];
    cudaError_t e = launch_point_kernel(ctx, cur, cur, P, true, false, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "displace kernel launch");
    ctx->step += 1;
    return MMR_OK;
}

mmr_status mmr_step_and_render_roundtrip(mmr_ctx *ctx, void *stream, int pinned_host)
{
    mmr::NvtxRange nvtx("mmr_step_and_render_roundtrip");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    mmr_status st = check_frame_ready(ctx, true);
    if (st != MMR_OK)
        return st;
    const int want_pinned = pinned_host ? 1 : 0;
    const uint64_t bytes = storage_bytes(ctx->n, ctx->dtype);
    if (ctx->rt_host && ctx->rt_host_pinned != want_pinned) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "round-trip: sync before switching host buffer");
        if (ctx->rt_host_pinned == 1)
            cudaFreeHost(ctx->rt_host);
        else
            free(ctx->rt_host);
        ctx->rt_host = nullptr;
    }
    if (!ctx->rt_host) {
        if (want_pinned) {
            cudaError_t e = cudaMallocHost(&ctx->rt_host, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->rt_host = nullptr;
                return fail(ctx, MMR_ERR_OOM, "round-trip: pinned host allocation failed: %s",
                            cudaGetErrorString(e));
            }
        } else {
            ctx->rt_host = malloc(bytes);
            if (!ctx->rt_host)
                return fail(ctx, MMR_ERR_OOM, "round-trip: host allocation failed");
        }
        ctx->rt_host_pinned = want_pinned;
    }
    if (!ctx->rt_device) {
        st = dev_alloc(ctx, &ctx->rt_device, bytes, "round-trip device copy");
        if (st != MMR_OK)
            return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = mmr_displace(ctx, stream);
    if (st != MMR_OK)
        return st;
    cudaError_t e = cudaMemcpyAsync(ctx->rt_host, ctx->buf[ctx->visible], ctx->point_bytes, cudaMemcpyDeviceToHost,
                                    s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->rt_device, ctx->rt_host, ctx->point_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "round-trip copies");
    return frame(ctx, ctx->rt_device, nullptr, false, s);
}

mmr_status mmr_frame_ptr(mmr_ctx *ctx, const uint32_t **rgba, const uint64_t **depth_id)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (rgba)
        *rgba = ctx->rgba;
    if (depth_id)
        *depth_id = reinterpret_cast<const uint64_t *>(ctx->keys[ctx->latest_buf]);
    return MMR_OK;
}

mmr_status mmr_set_depth_bound_split(mmr_ctx *ctx, int first_pass_shift)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (first_pass_shift < 0 || first_pass_shift > 10)
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_set_depth_bound_split: shift %d outside 0..10", first_pass_shift);
    ctx->launch.bound_shift = first_pass_shift;
    return MMR_OK;
}

mmr_status mmr_last_frame_kernels(const mmr_ctx *ctx, int *kernels)
{
    if (!ctx || !kernels)
        return MMR_ERR_INVALID_ARG;
    *kernels = ctx->last_frame_kernels;
    return MMR_OK;
}

mmr_status mmr_get_step(const mmr_ctx *ctx, uint32_t *step)
{
    if (!ctx || !step)
        return MMR_ERR_INVALID_ARG;
    *step = ctx->step;
    return MMR_OK;
}

mmr_status mmr_set_timing(mmr_ctx *ctx, int enable)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (enable && !ctx->ring) {
        ctx->ring = new (std::nothrow) cudaEvent_t[3 * kTimingRing]();
        if (!ctx->ring)
            return fail(ctx, MMR_ERR_OOM, "mmr_set_timing: host allocation failed");
        for (uint32_t k = 0; k < 3 * kTimingRing; ++k) {
            cudaError_t e = cudaEventCreate(&ctx->ring[k]);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "mmr_set_timing: cudaEventCreate");
        }
    }
    ctx->timing = enable != 0;
    ctx->timed_frames = 0;
    return MMR_OK;
}

mmr_status mmr_frame_kernel_ms(mmr_ctx *ctx, uint32_t frames_back, float *point_ms, float *resolve_ms)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (!ctx->timing || frames_back >= ctx->timed_frames || frames_back >= kTimingRing)
        return fail(ctx, MMR_ERR_STATE, "mmr_frame_kernel_ms: timing off, or frame %u back not timed or no longer "
                    "kept (%u timed, %u kept)", frames_back, ctx->timed_frames, kTimingRing);
    const cudaEvent_t *t = ctx->ring + 3 * ((ctx->timed_frames - 1 - frames_back) % kTimingRing);
    cudaError_t e = cudaEventSynchronize(t[2]);
    float a = 0.0f, b = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&a, t[0], t[1]);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&b, t[1], t[2]);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_frame_kernel_ms");
    if (point_ms)
        *point_ms = a;
    if (resolve_ms)
        *resolve_ms = b;
    return MMR_OK;
}

mmr_status mmr_last_kernel_ms(mmr_ctx *ctx, float *point_ms, float *resolve_ms)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (!ctx->timing || ctx->timed_frames == 0)
        return fail(ctx, MMR_ERR_STATE, "mmr_last_kernel_ms: timing off or no timed frame yet");
    return mmr_frame_kernel_ms(ctx, 0, point_ms, resolve_ms);
}

mmr_status mmr_check_device(mmr_ctx *ctx)
{
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    uint32_t word = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(&word, ctx->d_err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_check_device");
    if (word) {
        cudaMemset(ctx->d_err, 0, 4);
        return fail(ctx, MMR_ERR_TIMEOUT, "a kernel gave up waiting for a bulk copy (error word %u)", word);
    }
    return MMR_OK;
}

mmr_status mmr_selftest_bounded_wait(mmr_ctx *ctx, long long max_cycles, void *stream)
{
    if (!ctx || max_cycles < 1 || max_cycles > (1ll << 32))
        return fail(ctx, MMR_ERR_INVALID_ARG, "mmr_selftest_bounded_wait: max_cycles outside 1..2^32");
    cudaError_t e = mmr::launch_bounded_wait_selftest(max_cycles, ctx->d_err, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_selftest_bounded_wait");
    return MMR_OK;
}

mmr_status mmr_device_bytes(const mmr_ctx *ctx, uint64_t *bytes)
{
    if (!ctx || !bytes)
        return MMR_ERR_INVALID_ARG;
    *bytes = ctx->held;
    return MMR_OK;
}

mmr_status mmr_alloc_host_mirror(mmr_ctx *ctx, uint32_t **host_rgba)
{
    if (!ctx || !host_rgba)
        return MMR_ERR_INVALID_ARG;
    if (ctx->mirror) {
        *host_rgba = ctx->mirror;
        return MMR_OK;
    }
    *host_rgba = nullptr;
    mmr_status st = dev_alloc(ctx, (void **)&ctx->mirror_mem, mirror_mem_bytes(ctx), "host mirror chunk state");
    if (st != MMR_OK)
        return st;
    void *h = nullptr, *d = nullptr;
    cudaError_t e = cudaMemset(ctx->mirror_mem, 0, mirror_mem_bytes(ctx));
    if (e == cudaSuccess)
        e = cudaHostAlloc(&h, frame_px(ctx) * 4, cudaHostAllocMapped);
    if (e == cudaSuccess)
        e = cudaHostGetDevicePointer(&d, h, 0);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ctx->frame_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ctx->mirror_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h)
            cudaFreeHost(h);
        if (ctx->frame_done)
            cudaEventDestroy(ctx->frame_done);
        if (ctx->mirror_done)
            cudaEventDestroy(ctx->mirror_done);
        ctx->frame_done = ctx->mirror_done = nullptr;
        dev_free(ctx, (void **)&ctx->mirror_mem, mirror_mem_bytes(ctx));
        return cuda_fail(ctx, e, "mmr_alloc_host_mirror");
    }
    memset(h, 0, frame_px(ctx) * 4);
    ctx->mirror = static_cast<uint32_t *>(h);
    ctx->mirror_dev = static_cast<uint32_t *>(d);
    ctx->mirror_full = true;
    ctx->mirror_pending = false;
    *host_rgba = ctx->mirror;
    return MMR_OK;
}

mmr_status mmr_mirror_frame(mmr_ctx *ctx, void *stream)
{
    mmr::NvtxRange nvtx("mmr_mirror_frame");
    if (!ctx)
        return MMR_ERR_INVALID_ARG;
    if (!ctx->mirror)
        return fail(ctx, MMR_ERR_STATE, "mmr_mirror_frame: no host mirror (call mmr_alloc_host_mirror first)");
    if (ctx->frame_no == 0)
        return fail(ctx, MMR_ERR_STATE, "mmr_mirror_frame: no frame rendered yet");
    const cudaStream_t s = (cudaStream_t)stream;
    const int latest = ctx->latest_buf;
    // resolves record frame_done only once the mirror exists, so the update that fills the whole mirror (the
    // first one, or the first after a background change) synchronises with the device instead of waiting on it
    cudaError_t e = cudaSuccess;
    if (ctx->mirror_full) {
        e = cudaDeviceSynchronize();
    } else {
        e = cudaStreamWaitEvent(s, ctx->frame_done, 0);
        if (e == cudaSuccess && ctx->mirror_pending)      // updates run one after another (they share `held`)
            e = cudaStreamWaitEvent(s, ctx->mirror_done, 0);
    }
    if (e == cudaSuccess)
        e = mmr::launch_mirror(ctx->rgba, ctx->mirror_dev, (uint32_t)frame_px(ctx), ctx->chunk_tags[latest],
                               ctx->buf_frame[latest], ctx->mirror_mem + 8, ctx->mirror_full ? 1 : 0,
                               reinterpret_cast<unsigned long long *>(ctx->mirror_mem), s);
    if (e == cudaSuccess)
        e = cudaEventRecord(ctx->mirror_done, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_mirror_frame");
    ctx->mirror_full = false;
    ctx->mirror_pending = true;
    return MMR_OK;
}

mmr_status mmr_mirror_bytes(mmr_ctx *ctx, uint64_t *bytes)
{
    if (!ctx || !bytes)
        return MMR_ERR_INVALID_ARG;
    if (!ctx->mirror)
        return fail(ctx, MMR_ERR_STATE, "mmr_mirror_bytes: no host mirror");
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpy(&v, ctx->mirror_mem, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "mmr_mirror_bytes");
    *bytes = v;
    return MMR_OK;
}

}  // extern "C"
