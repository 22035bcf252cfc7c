/*
 * mmr.h - C ABI of libmmr: zero-copy displace + render of a device-resident
 * point cloud on one GPU (NVIDIA B300, sm_103a).
 *
 * Usage model (Mimir, Sec. 3.2.1 and Listing 1): the simulation replaces its
 * own device allocation of the visualised data with a library call that
 * returns a plain device pointer; the simulation writes through that pointer
 * and the library renders from the same memory, so the data never leaves the
 * GPU.  The paper's render thread and prepareViews/updateViews critical
 * section (Sec. 3.4, Listing 2) become stream ordering: every call that takes
 * a stream only enqueues work on it, and a frame is valid once that stream
 * has been synchronised.  The paper draws through Vulkan; here projection and
 * a depth-tested splat (1 px, or a disc of a chosen radius) are CUDA kernels
 * writing a framebuffer that stays in device memory.
 *
 * Conventions for every entry point:
 *  - Pointers named dev_* or returned as device pointers are GPU addresses of
 *    the device that was current when mmr_create ran; host arrays are read
 *    during the call only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued, not finished, when the call returns.
 *  - Calls on one context are not thread-safe; distinct contexts are
 *    independent.
 *  - Errors return a negative mmr_status; nothing aborts the process and no
 *    kernel traps.  mmr_last_error(ctx) gives a message for the last failure
 *    on that context.  The status codes and messages are this library's own
 *    convention: the paper specifies no error reporting.
 */
#ifndef MMR_H
#define MMR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MMR_API __attribute__((visibility("default")))
#else
#define MMR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mmr_ctx mmr_ctx;
typedef int mmr_status;

/* Status codes: this library's chosen convention (the paper defines none). */
enum {
    MMR_OK = 0,
    MMR_ERR_INVALID_ARG = -1,  /* a pointer is NULL, a size is 0 or too large, a value out of range */
    MMR_ERR_OOM = -2,          /* a device or pinned-host allocation failed */
    MMR_ERR_BUDGET = -3,       /* the allocation would exceed the context's device-memory budget */
    MMR_ERR_CUDA = -4,         /* a CUDA runtime call or kernel launch failed (message has the text) */
    MMR_ERR_STATE = -5,        /* call out of order (no points yet, no camera yet, already allocated) */
    MMR_ERR_TIMEOUT = -6       /* reserved: a bounded device-side wait gave up */
};

/* Position storage: three packed coordinates per point (x, y, z), array of
 * structures, as the paper's float3 position format (Listing 1).  The 16-bit
 * forms hold binary16 or bfloat16 bit patterns; arithmetic is FP32. */
enum mmr_dtype { MMR_F32x3 = 0, MMR_F16x3 = 1, MMR_BF16x3 = 2 };

/* ---- context -------------------------------------------------------------- */

/* Create a context with a width x height framebuffer on the current device
 * (the paper's createInstance(w, h, &instance), Listing 1).  Allocates the
 * RGBA8 framebuffer (uint32 per pixel, row 0 at the top) and two 64-bit
 * depth-id buffers, all cleared.  1 <= width, height <= 32768.
 * budget_bytes: device-memory cap for everything this context allocates
 * (0 = no cap); an allocation over it fails with MMR_ERR_BUDGET.
 * On failure *out is NULL and nothing stays allocated. */
MMR_API mmr_status mmr_create(int width, int height, mmr_ctx **out);
MMR_API mmr_status mmr_create_ex(int width, int height, uint64_t budget_bytes, mmr_ctx **out);

/* Release every device and host allocation of the context (the points
 * pointer included), as destroying a Mimir handle cleans up the resources
 * created with it (Sec. 3.2.2).  Waits for work the context enqueued to
 * finish.  A NULL ctx is a no-op.  Every pointer the context handed out is
 * invalid after. */
MMR_API mmr_status mmr_destroy(mmr_ctx *ctx);

/* Message of the last failure on ctx ("" if none); for a NULL ctx, the last
 * failure of mmr_create or mmr_render_static in this process.  Valid until
 * the next call on ctx.  Like the status codes, a convention of this library
 * (the paper specifies no error reporting). */
MMR_API const char *mmr_last_error(const mmr_ctx *ctx);
MMR_API const char *mmr_status_string(mmr_status s);

/* ---- data ----------------------------------------------------------------- */

/* Allocate device storage for n points of the given dtype and return its
 * device pointer (the paper's allocLinear, Sec. 3.2.1 / Table 2: same role as
 * cudaMalloc).  The simulation writes positions through *dev_ptr; the
 * library owns the memory: never cudaFree it.  The buffer is 256-byte aligned
 * and zero-filled.  1 <= n < 2^32.  One point buffer per context
 * (MMR_ERR_STATE on a second call). */
MMR_API mmr_status mmr_alloc_points(mmr_ctx *ctx, uint64_t n, int dtype, void **dev_ptr);

/* Allocate an optional per-point colour buffer (n uint32 RGBA8 values, the
 * paper's Color property, Sec. 3.2.2) and return its device pointer.  Once
 * allocated, resolve colours each covered pixel with colors[winning id];
 * without it every point takes the default colour (Sec. 4.1: one colour). */
MMR_API mmr_status mmr_alloc_colors(mmr_ctx *ctx, uint32_t **dev_colors);

/* Ping-pong buffers (the paper's alternating read/write buffers, Sec. 3.4
 * and Listing 2): allocate two point buffers of n points instead of one and
 * return both device pointers (same layout and ownership as
 * mmr_alloc_points; buffer 0 starts visible).  A simulation that reads one
 * state and writes the next uses them in turn; mmr_set_visible picks the
 * buffer mmr_render and mmr_step_and_render use (the paper's
 * toggleVisibility).  MMR_ERR_STATE if the context already has points. */
MMR_API mmr_status mmr_alloc_pingpong(mmr_ctx *ctx, uint64_t n, int dtype, void **dev_a, void **dev_b);
MMR_API mmr_status mmr_set_visible(mmr_ctx *ctx, int which);
MMR_API mmr_status mmr_get_visible(const mmr_ctx *ctx, int *which);

/* Indexed colour (the paper's colour property read through an index buffer,
 * Sec. 3.2.2, Listings 3 and 6): allocate a per-point index buffer (n uint32,
 * zero-filled) and a colormap (ncolors RGBA8, 1..2^24, white) and return both
 * device pointers.  Once allocated, a covered pixel is coloured
 * colormap[index[id]]; an index >= ncolors takes the default colour.  Takes
 * precedence over mmr_alloc_colors. */
MMR_API mmr_status mmr_alloc_indexed_colors(mmr_ctx *ctx, uint32_t ncolors, uint32_t **dev_index,
                                            uint32_t **dev_colormap);

/* ---- view and simulation parameters --------------------------------------- */

/* Camera (the paper's interactive camera, Sec. 1): right-handed look-at from
 * eye to target with the given up vector, times an OpenGL-style perspective
 * with vertical field of view fovy_deg and aspect width/height.  Built in FP64
 * on the host and rounded once to FP32; a point is drawn only when
 * znear < clip w < zfar (clip w is its distance along the view axis).
 * Requires 0 < fovy_deg < 180, 2^-64 <= znear < zfar <= 2^64 (as FP32) and
 * eye != target, else MMR_ERR_INVALID_ARG.  On that depth range the
 * kernels' perspective divide (one shared reciprocal, Markstein's
 * correction) gives every pixel that IEEE division gives. */
MMR_API mmr_status mmr_set_camera(mmr_ctx *ctx, const double eye[3], const double target[3],
                          const double up[3], double fovy_deg, double znear, double zfar);

/* Set the FP32 row-major 4x4 clip matrix directly (rows x, y and w are used)
 * and the depth range; mmr_get_matrix returns the matrix in use.  Requires
 * finite entries and 2^-64 <= znear < zfar <= 2^64, else MMR_ERR_INVALID_ARG. */
MMR_API mmr_status mmr_set_matrix(mmr_ctx *ctx, const float m[16], float znear, float zfar);
MMR_API mmr_status mmr_get_matrix(const mmr_ctx *ctx, float m[16]);

/* Displacement parameters (Sec. 4.1, Brownian motion).  Each step moves every
 * coordinate by amplitude * (2u - 1), u the top 24 bits of a
 * Philox4x32-10 draw with counter (point, step, cloud, 0) and key
 * (seed low, seed high) scaled by 2^-24, then clamps it to [0, 1].  The next
 * step index is first_step.  amplitude is 0 or in [2^-100, 1]. */
MMR_API mmr_status mmr_set_sim(mmr_ctx *ctx, uint64_t seed, uint32_t cloud, float amplitude,
                       uint32_t first_step);

/* Marker shape.  radius_px = 0 (default): each point covers the one pixel it
 * projects into.  0.5 <= radius_px <= 64: front-facing disc markers of the
 * same size for all points (Sec. 4.1): a point covers every pixel whose
 * centre lies within radius_px of its projected position (computed in FP32
 * in a fixed order), all at the point's depth. */
MMR_API mmr_status mmr_set_marker(mmr_ctx *ctx, float radius_px);

/* Default point colour (no colour buffer) and background colour, RGBA8. */
MMR_API mmr_status mmr_set_style(mmr_ctx *ctx, uint32_t color, uint32_t background);

/* Kernel launch shape of the point kernel.
 *  kernel = MMR_KERNEL_GRID: grid-stride over 48-byte point groups with
 *    `threads` per block (a multiple of 32, 32..1024); ctas_per_sm = 0 gives
 *    one thread per group, ctas_per_sm > 0 a persistent grid of
 *    sm_count * ctas_per_sm CTAs.  On FP32 storage every thread of such a
 *    grid prefetches its next group while working on the current one; the
 *    16-bit kernels load each group when they reach it, to stay at 40
 *    registers.  Each point reads its pixel's key and, when it is nearer,
 *    takes a 64-bit atomic minimum.
 *  kernel = MMR_KERNEL_TMA: persistent, TMA-staged (threads 128, 256 or
 *    512; ctas_per_sm >= 1): each CTA keeps 4 tiles of threads*48 bytes in
 *    flight through shared memory with bulk copies.
 *  kernel = MMR_KERNEL_DEPTH_BOUND: the grid-stride kernel in two passes
 *    over the points with screen-tile depth bounds between them, for dense
 *    clouds: the first eighth of the point groups splats as usual and marks
 *    the 8x8-pixel tiles it wrote; a small kernel takes the largest depth of
 *    each marked tile's keys; the rest of the points skip the depth-buffer
 *    read when they lie behind their tile's bound (they could not win any of
 *    its pixels).  Three point-phase launches; 16 bytes per tile of device
 *    memory, allocated at the first such frame.  mmr_set_depth_bound_split
 *    sets the first pass's share of the points to 2^-shift (1..10; 0 for
 *    the library's choice: one eighth, one sixteenth for discs covering
 *    each pixel 1024 times or more), for 1-px points and disc markers alike.
 *  kernel = MMR_KERNEL_WARP_AGG: the grid-stride kernel whose lanes that hit
 *    the same pixel in one step elect their nearest point, which alone reads
 *    the key and takes the atomic.
 *  kernel = MMR_KERNEL_AUTO (the default): MMR_KERNEL_GRID (64 threads, one
 *    thread per group) for 1-px points.
 * Disc markers (mmr_set_marker) use their own grid-stride kernel (64
 * threads).  Under MMR_KERNEL_DEPTH_BOUND, or MMR_KERNEL_AUTO with at least
 * 2^20 points and 64 discs over each pixel on average (n pi r^2 >= 64 w h),
 * it runs in two passes with depth bounds of 32x32-pixel tiles between them:
 * a later disc behind the bounds of every tile it touches is skipped, and
 * the discs that remain are drawn by whole warps, one disc at a time.
 * Results never depend on the shape or the kernel; only speed does. */
enum mmr_kernel {
    MMR_KERNEL_GRID = 0,
    MMR_KERNEL_TMA = 1,
    MMR_KERNEL_DEPTH_BOUND = 2,
    MMR_KERNEL_WARP_AGG = 3,
    MMR_KERNEL_AUTO = 4
};
MMR_API mmr_status mmr_set_launch(mmr_ctx *ctx, int threads, int ctas_per_sm, int kernel);
MMR_API mmr_status mmr_set_depth_bound_split(mmr_ctx *ctx, int first_pass_shift);

/* ---- frames ---------------------------------------------------------------- */

/* One frame of the paper's benchmark (Sec. 4.1): a compute step moves every
 * point by Brownian motion and the new state is drawn, the compute section
 * and the render that follows it being what display / prepareViews +
 * updateViews order (Sec. 3.4, Listing 2).  Here: displace every point
 * (current step), project and depth-splat it (key = bits(clip w) << 32 |
 * point id, per-pixel minimum), then resolve the keys to RGBA8, all enqueued
 * on `stream` in that order.  Displacement and splat are one fused kernel;
 * resolve also clears the other depth-id buffer for the next frame.
 * Advances the step counter.  Requires points and a camera. */
MMR_API mmr_status mmr_step_and_render(mmr_ctx *ctx, void *stream);

/* One frame out of place (ping-pong): read the visible buffer, write the
 * displaced positions into the other one, render them and make that buffer
 * visible.  The visible state and the frame equal those of
 * mmr_step_and_render; the previous state stays untouched in the other
 * buffer.  Requires mmr_alloc_pingpong. */
MMR_API mmr_status mmr_step_and_render_pingpong(mmr_ctx *ctx, void *stream);

/* Second workload: gravitational all-pairs N-body (the paper's N-body
 * sample, Sec. 4.2.3) feeding the same renderer.  mmr_alloc_nbody needs FP32
 * ping-pong buffers (the visible one holds the bodies' positions) and
 * allocates velocities (3n floats, zero) and masses (n floats, zero; write
 * them), plus scratch for per-chunk sums, and returns the velocity and mass
 * device pointers.  mmr_nbody_step_and_render: for every body i, acc = the
 * sum over j of (p_j - p_i) m_j / (|p_j - p_i|^2 + eps2)^(3/2) (FP32, exact
 * sqrt and division), summed in chunks of 1024 consecutive j (each chunk in
 * order, then the chunk sums in order), which stays within the FP32
 * summation error bound of the sequential sum; v += G acc dt, p' = p + v dt
 * written to the other buffer, which is then
 * rendered (1-px splat fused into the same kernel) and made visible.  Needs
 * eps2 > 0 (it also removes the j = i term).  Advances the step counter. */
MMR_API mmr_status mmr_alloc_nbody(mmr_ctx *ctx, float **dev_vel, float **dev_mass);
MMR_API mmr_status mmr_nbody_step_and_render(mmr_ctx *ctx, float G, float eps2, float dt, void *stream);

/* Displace only (advances the step counter). */
MMR_API mmr_status mmr_displace(mmr_ctx *ctx, void *stream);

/* Render only: the simulation already wrote the positions (the paper's
 * updateViews after a user kernel, Listing 2). */
MMR_API mmr_status mmr_render(mmr_ctx *ctx, void *stream);

/* The host round-trip baseline (the paper's RAM-based comparison, abstract
 * and Sec. 4.1): displace on the device, copy the positions device -> host
 * (pinned when pinned_host != 0, else pageable) -> a second device buffer,
 * then render that copy.  Output is identical to mmr_step_and_render.  The
 * extra host and device buffers are allocated on first use and counted
 * against the budget. */
MMR_API mmr_status mmr_step_and_render_roundtrip(mmr_ctx *ctx, void *stream, int pinned_host);

/* Device pointers of the latest frame: RGBA8 (width*height uint32) and its
 * depth-id keys (width*height uint64, all-ones = empty).  This is the device
 * memory a display would read, as the paper's renderer reads the latest state
 * straight from memory shared with the compute side instead of a host copy
 * (Sec. 1, Sec. 3.2.1).  Valid after the stream that rendered the frame is
 * synchronised, until the next frame or mmr_destroy.  Either output pointer
 * may be NULL.  Both buffers are read-only to the caller: each resolve
 * repaints only the runs of 64 pixels that its frame or the one before
 * touched (elsewhere the framebuffer already holds the background), so a
 * pixel the caller changed could stay changed. */
MMR_API mmr_status mmr_frame_ptr(mmr_ctx *ctx, const uint32_t **rgba, const uint64_t **depth_id);

/* Number of kernels the latest frame of this context launched (point phase
 * and resolve), for launch counting in benchmarks. */
MMR_API mmr_status mmr_last_frame_kernels(const mmr_ctx *ctx, int *kernels);

/* Current step counter (index of the next displacement step). */
MMR_API mmr_status mmr_get_step(const mmr_ctx *ctx, uint32_t *step);

/* Per-kernel timing for benchmarks.  When enabled, the library records CUDA
 * events on the frame's stream before the point phase, between it and the
 * resolve and after the resolve of every frame, and keeps them for the last
 * MMR_TIMING_RING frames, so that many frames can be enqueued back to back
 * and timed afterwards.  mmr_frame_kernel_ms waits for the events of the
 * frame `frames_back` frames before the latest (0 = the latest) and returns
 * both durations in milliseconds (either pointer may be NULL);
 * mmr_last_kernel_ms is the latest frame's.  MMR_ERR_STATE if timing is off
 * or that frame was not timed or is no longer kept.  Switching timing on
 * restarts the count.  The events between the point phase and the resolve
 * cost a few microseconds per frame. */
#define MMR_TIMING_RING 4096u
MMR_API mmr_status mmr_set_timing(mmr_ctx *ctx, int enable);
MMR_API mmr_status mmr_frame_kernel_ms(mmr_ctx *ctx, uint32_t frames_back, float *point_ms, float *resolve_ms);
MMR_API mmr_status mmr_last_kernel_ms(mmr_ctx *ctx, float *point_ms, float *resolve_ms);

/* Synchronise the device and report whether a kernel of this context gave
 * up a bounded wait (MMR_ERR_TIMEOUT; the flag is then cleared) since the
 * last check.  A timed-out frame is incomplete; the context stays usable. */
MMR_API mmr_status mmr_check_device(mmr_ctx *ctx);

/* Failure-path self-test: one CTA waits on a barrier that nothing ever
 * completes, gives up after max_cycles SM clock cycles (1..2^32) and raises
 * the context's device error flag, exactly as a point kernel whose bulk copy
 * never arrived would.  mmr_check_device then reports MMR_ERR_TIMEOUT and the
 * context stays usable.  No fault and no unbounded wait is involved. */
MMR_API mmr_status mmr_selftest_bounded_wait(mmr_ctx *ctx, long long max_cycles, void *stream);

/* Device bytes this context holds right now. */
MMR_API mmr_status mmr_device_bytes(const mmr_ctx *ctx, uint64_t *bytes);

/* Host mirror of the framebuffer: width*height RGBA8 pixels (uint32, row 0
 * at the top) of pinned host memory that the context allocates, mapped into
 * the device's address space, and frees in mmr_destroy.  A host counterpart
 * of the paper's display reading the latest frame (Sec. 1): instead of
 * copying the whole framebuffer to the host every frame, mmr_mirror_frame
 * enqueues on `stream` a kernel that writes over the host link only the runs
 * of 64 pixels that differ from what the mirror holds (those the latest
 * frame touched, and those where the mirror still holds a point of an
 * earlier frame; everything after the mirror is allocated or the background
 * colour changes).  Once `stream` is synchronised the mirror equals the
 * latest frame.  The stream may differ from the one that renders: the next
 * frame's resolve waits for the kernel (the resolve rewrites the device
 * framebuffer the kernel reads), so the copy overlaps the next point phase.
 * Give that stream a higher priority than the rendering stream: the kernel's
 * CTAs then start ahead of the next point kernel's instead of after them, and
 * the next resolve does not wait for them (measured on a 3840x2160 frame of
 * 2^26 points: 10 us added per frame instead of 40 us).  Frames may be
 * skipped; the mirror catches up at the next call.  An update
 * that writes every pixel (the first, and the first after a background
 * change) synchronises the device before it is enqueued.  The host must not
 * read the mirror while a mmr_mirror_frame is in flight.
 * mmr_mirror_bytes reports the bytes written to the mirror since it was
 * allocated (synchronises the device).  MMR_ERR_STATE before the mirror
 * exists or before the first frame. */
MMR_API mmr_status mmr_alloc_host_mirror(mmr_ctx *ctx, uint32_t **host_rgba);
MMR_API mmr_status mmr_mirror_frame(mmr_ctx *ctx, void *stream);
MMR_API mmr_status mmr_mirror_bytes(mmr_ctx *ctx, uint64_t *bytes);

/* ---- batched clouds --------------------------------------------------------
 * Many independent clouds, each with its own size, framebuffer, camera and
 * displacement parameters, advanced and rendered together by one persistent
 * launch per frame.  Its CTAs take work items from one list: each cloud's
 * point items (displace, project, splat), and that cloud's pixel items
 * (resolve, clear) placed about one resident grid later, so that streaming
 * pixel work runs beside latency-bound point work.  A pixel item waits,
 * bounded, until its cloud's point items are done; a wait that gives
 * up raises the batch's device error flag (mmr_batch_check_device).  A
 * device-side frame counter picks the Philox step, the camera slot and the
 * depth-id buffer, so one captured frame can be replayed as a CUDA graph
 * with nothing changed on the host.  Each cloud's result is identical to
 * rendering it alone in its own mmr_ctx with the same parameters (the
 * per-pixel minimum does not depend on the order of the work). */
typedef struct mmr_batch mmr_batch;

typedef struct mmr_cloud_desc {
    uint64_t n;            /* points, 1 .. 2^32-1 */
    int width, height;     /* this cloud's framebuffer, 1..32768 each */
    uint64_t seed;         /* Philox key (see mmr_set_sim) */
    uint32_t cloud;        /* Philox counter word 2 */
    float amplitude;       /* displacement amplitude, 0 or [2^-100, 1] */
    uint32_t color;        /* RGBA8 of every point */
    uint32_t background;   /* RGBA8 of empty pixels */
} mmr_cloud_desc;

/* Create a batch of `count` clouds (1..65536) stored as `dtype`, with
 * `camera_slots` cameras per cloud (frame f uses slot f mod camera_slots,
 * 1..4096).  All point buffers live in one device allocation (each cloud's
 * slice 256-byte aligned, zero-filled); every cloud gets two depth-id
 * buffers and an RGBA8 framebuffer.  budget_bytes as in mmr_create_ex.
 * The descriptor array is read during the call only. */
MMR_API mmr_status mmr_batch_create(int count, const mmr_cloud_desc *clouds, int dtype, int camera_slots,
                                    uint64_t budget_bytes, mmr_batch **out);
MMR_API mmr_status mmr_batch_destroy(mmr_batch *b);
MMR_API const char *mmr_batch_last_error(const mmr_batch *b);

/* Device pointer of cloud `cloud`'s positions (n * 3 coordinates, AoS). */
MMR_API mmr_status mmr_batch_points(mmr_batch *b, int cloud, void **dev_ptr);

/* Camera of `cloud` in slot `slot`, as mmr_set_camera with the cloud's own
 * aspect (same argument rules).  Uploaded to the device before the next
 * step or graph replay. */
MMR_API mmr_status mmr_batch_set_camera(mmr_batch *b, int cloud, int slot, const double eye[3],
                                        const double target[3], const double up[3], double fovy_deg,
                                        double znear, double zfar);

/* Launch shape: threads per block (multiple of 32, 32..512), CTAs per SM
 * of the persistent grid (0 = as many as fit), and point groups per item
 * (1..65536; a group is 48 bytes of positions; a pixel item covers 16 pixels
 * per group).  Rebuilds the work list (synchronises the device).  Results
 * never depend on it. */
MMR_API mmr_status mmr_batch_set_launch(mmr_batch *b, int threads, int ctas_per_sm, int chunk_groups);

/* One frame of every cloud: displace + project + splat and resolve + clear
 * (one persistent launch, after resetting the work counters and building
 * every cloud's parameters for the frame), then advance the device frame
 * counter.  Requires every cloud's camera for the slot the frame uses. */
MMR_API mmr_status mmr_batch_step_and_render(mmr_batch *b, void *stream);

/* The same frame by the paper's RAM-based path, for comparison: displace
 * every cloud (one persistent launch, no splat), copy all positions device
 * -> host (pinned when pinned_host != 0, else pageable) -> a second device
 * buffer, render every cloud from that copy (one persistent launch, no
 * displacement), advance the frame counter.  Results are identical to
 * mmr_batch_step_and_render.  The host and device copies (the positions'
 * size each) are allocated on first use and kept until mmr_batch_destroy;
 * the device copy counts against the budget.  Enqueued on `stream`. */
MMR_API mmr_status mmr_batch_step_and_render_roundtrip(mmr_batch *b, void *stream, int pinned_host);

/* `frames` frames by replaying a CUDA graph of one frame (captured on first
 * use and again after mmr_batch_set_launch).  Same results as calling
 * mmr_batch_step_and_render `frames` times. */
MMR_API mmr_status mmr_batch_run_graph(mmr_batch *b, int frames, void *stream);

/* Autotuner: times each candidate launch shape (threads in {64, 128, 256},
 * chunk groups = threads x {1, 2, 4, 8}, CTAs per SM in {0, 4, 8}) over
 * `frames_per_config` frames with CUDA events on `stream`, keeps the fastest
 * and returns it (any output pointer may be NULL).  Positions and the frame
 * counter are saved before and restored after, so the simulation state is
 * unchanged; the frame buffers are cleared.  Allocates a temporary copy of
 * the positions (counted against the budget). */
MMR_API mmr_status mmr_batch_autotune(mmr_batch *b, void *stream, int frames_per_config, int *threads,
                                      int *ctas_per_sm, int *chunk_groups, float *best_ms);

/* Synchronise the device and report whether a pixel item of this batch gave
 * up its bounded wait (MMR_ERR_TIMEOUT; the flag is then cleared) since the
 * last check.  That frame is incomplete; the batch stays usable. */
MMR_API mmr_status mmr_batch_check_device(mmr_batch *b);

/* Failure-path self-test: one thread runs the pixel items' wait on a count
 * that nothing ever decrements, gives up after max_polls polls (1..2^24,
 * about 64 ns apart) and raises the batch's device error flag, as a pixel
 * item whose cloud's point items never finished would.  Enqueued on
 * `stream`; mmr_batch_check_device then reports MMR_ERR_TIMEOUT.  No fault
 * and no unbounded wait is involved. */
MMR_API mmr_status mmr_batch_selftest_bounded_wait(mmr_batch *b, uint32_t max_polls, void *stream);

/* Latest frame of one cloud (device pointers, as mmr_frame_ptr; read-only to
 * the caller for the same reason). */
MMR_API mmr_status mmr_batch_frame_ptr(mmr_batch *b, int cloud, const uint32_t **rgba,
                                       const uint64_t **depth_id);

/* Frames enqueued so far, and device bytes held. */
MMR_API mmr_status mmr_batch_frames(const mmr_batch *b, uint32_t *frames);
MMR_API mmr_status mmr_batch_device_bytes(const mmr_batch *b, uint64_t *bytes);

/* ---- serving: many viewers of one shared cloud -----------------------------
 * A serving engine holds one shared point cloud and up to any number of
 * viewers, each with a private cloud, a camera and a framebuffer.  One call
 * of mmr_serve_tick renders one frame for every active viewer:
 *  - the shared cloud is displaced once (Philox step = tick index) and every
 *    shared point is splatted into every active viewer's buffer in the same
 *    pass, so its positions are read once per tick;
 *  - each viewer's private cloud is displaced (step = that viewer's frame
 *    index) and splatted into its own buffer, all viewers in one launch;
 *  - one resolve launch writes every viewer's RGBA8 frame: shared points in
 *    the shared colour, private points in the viewer's colour, storing only
 *    in runs of 64 pixels that the view's frame or its previous one touched.
 * Point ids in the keys: shared point i -> i, private point j -> shared_n + j.
 * Viewers join and leave between ticks (continuous batching); a join whose
 * buffers would exceed the budget is refused with MMR_ERR_BUDGET and can be
 * retried after others leave.  Frame k of a viewer that joined before tick t0
 * is rendered at tick t0 + k and depends only on (t0 + k, k): it is the same
 * whether the viewer is served alone or with others. */
typedef struct mmr_serve mmr_serve;

/* Engine with a shared cloud of shared_n points (1..2^31-1) stored as dtype,
 * displaced with Philox key `seed`, counter word 2 `cloud`, and amplitude.
 * budget_bytes caps the device memory of the shared cloud and all viewers
 * (0 = no cap). */
MMR_API mmr_status mmr_serve_create(uint64_t shared_n, int dtype, uint64_t seed, uint32_t cloud, float amplitude,
                                    uint64_t budget_bytes, mmr_serve **out);
MMR_API mmr_status mmr_serve_destroy(mmr_serve *s);
MMR_API const char *mmr_serve_last_error(const mmr_serve *s);

/* Device pointer of the shared positions (write them before the first tick). */
MMR_API mmr_status mmr_serve_shared_points(mmr_serve *s, void **dev_ptr);
MMR_API mmr_status mmr_serve_set_shared_color(mmr_serve *s, uint32_t color);

/* Admit a viewer: private cloud of private_n points (zero-filled; write it
 * through mmr_serve_viewer_points before its first tick), a width x height
 * framebuffer, its own Philox key/cloud word/amplitude and colours.  Returns
 * the viewer id in *viewer.  A viewer needs 12 (FP32) or 6 bytes per private
 * point (padded to 48-byte groups) and 20 bytes per pixel, plus 8 bytes per
 * 64 pixels of chunk tags.  MMR_ERR_BUDGET when its buffers do not fit
 * beside those of the active viewers (nothing is allocated then).
 * shared_n + private_n must stay below 2^32.  Buffers kept from viewers
 * that left are reused when their size fits (a buffer at most twice the
 * size needed); they are cleared on the engine's own stream, so a join does
 * not wait for a tick in flight, and the call returns once they are clear. */
MMR_API mmr_status mmr_serve_add_viewer(mmr_serve *s, uint64_t private_n, int width, int height, uint64_t seed,
                                        uint32_t cloud, float amplitude, uint32_t color, uint32_t background,
                                        int *viewer);
MMR_API mmr_status mmr_serve_viewer_points(mmr_serve *s, int viewer, void **dev_ptr);

/* Camera of a viewer for the next tick (as mmr_set_camera, viewer aspect,
 * same argument rules). */
MMR_API mmr_status mmr_serve_set_camera(mmr_serve *s, int viewer, const double eye[3], const double target[3],
                                        const double up[3], double fovy_deg, double znear, double zfar);

/* Remove a viewer once the last enqueued tick has finished.  Its buffers are
 * kept by the engine for later joins (still counted in the device bytes and
 * against the budget); they are freed when a join needs the room under the
 * budget, when an allocation fails, or at mmr_serve_destroy. */
MMR_API mmr_status mmr_serve_remove_viewer(mmr_serve *s, int viewer);

/* One tick on `stream` (every active viewer needs a camera).  The
 * _roundtrip form first sends the shared positions device -> pinned host ->
 * device (the paper's RAM-based comparison); results are identical. */
MMR_API mmr_status mmr_serve_tick(mmr_serve *s, void *stream);
MMR_API mmr_status mmr_serve_tick_roundtrip(mmr_serve *s, void *stream);

/* Latest frame of a viewer (device pointers) and how many frames it has had.
 * Read-only to the caller, as for mmr_frame_ptr: each resolve repaints only
 * the runs of 64 pixels that the view's frame or its previous one touched. */
MMR_API mmr_status mmr_serve_frame_ptr(mmr_serve *s, int viewer, const uint32_t **rgba, const uint64_t **depth_id,
                                       uint32_t *frame_index);

/* Ticks so far, active viewers, device bytes held, kept buffers of departed
 * viewers included (any pointer may be NULL). */
MMR_API mmr_status mmr_serve_status(const mmr_serve *s, uint32_t *tick, int *active_viewers,
                                    uint64_t *device_bytes);

/* CUDA-event timing of each tick's kernels; mmr_serve_last_tick_ms waits for
 * the latest tick and returns its device time. */
MMR_API mmr_status mmr_serve_set_timing(mmr_serve *s, int enable);
MMR_API mmr_status mmr_serve_last_tick_ms(mmr_serve *s, float *ms);

/* ---- rendering without allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc.  Examples: a simulation embedded in a host
 * program whose own memory manager owns the device (a pool or arena that
 * every allocation must go through, with the rest of memory reserved), or a
 * real-time loop that must not allocate per frame because an allocation can
 * synchronise the device and stall it.  Such a caller keeps its positions
 * and its RGBA8 output in memory it already owns and passes both in; the
 * only scratch this call needs, the per-pixel depth-id keys, lives in a
 * fixed-size array inside the library.
 *
 * MMR_STATIC_MAX_PIXELS: capacity of that array, in pixels (8 bytes each,
 * 32 MiB).  The array is device memory of its own code module, which CUDA
 * loads on a device when it is first used there (lazy module loading, the
 * default): the first call of this function on a device reserves the
 * 32 MiB, and the device keeps them until the process exits.  A caller whose
 * memory manager claims the rest of the device should make that first call
 * at start-up, before the claim; if the array cannot be loaded the call
 * fails with MMR_ERR_OOM (or MMR_ERR_CUDA) and the CUDA error text.
 *
 * mmr_render_static: render n points (dtype as mmr_alloc_points; dev_points
 * 16-byte aligned, n*3 coordinates, AoS, read only) with the FP32 row-major
 * clip matrix m (rows x, y and w used; znear < clip w < zfar drawn) into
 * dev_rgba (width*height uint32 RGBA8, row 0 at the top, written): each
 * covered pixel gets `color`, the others `background`.  The frame equals
 * what mmr_set_matrix + mmr_render produce for the same points.
 *  - Allocates nothing: no cudaMalloc, cudaFree or other allocating call.
 *  - width*height above MMR_STATIC_MAX_PIXELS, n outside 1..2^32-1, a NULL
 *    pointer, dev_points not 16-byte aligned, dev_rgba not 4-byte aligned
 *    or a depth range outside 2^-64 <= znear < zfar <= 2^64:
 *    MMR_ERR_INVALID_ARG, nothing launched.
 *  - The first call on a device (with that device current) looks up the
 *    array's device address once and keeps it; make that first call before
 *    any CUDA stream capture that contains this call.  The kept address
 *    assumes the device is not reset (cudaDeviceReset) while the library is
 *    in use.
 *  - Every call on a device shares the one array.  Each call clears the
 *    part it uses before drawing, but calls whose work overlaps on the GPU
 *    (different streams, or threads without ordering between them) race on
 *    it and give wrong frames: order them on one stream.
 *  - Work is enqueued on `stream` (NULL = legacy default stream); the
 *    frame is complete when the stream is synchronised.  Errors are read
 *    with mmr_last_error(NULL). */
#define MMR_STATIC_MAX_PIXELS 4194304u
MMR_API mmr_status mmr_render_static(const void *dev_points, uint64_t n, int dtype, const float m[16],
                                     float znear, float zfar, int width, int height, uint32_t color,
                                     uint32_t background, uint32_t *dev_rgba, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MMR_H */
