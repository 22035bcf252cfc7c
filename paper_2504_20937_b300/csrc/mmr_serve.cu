// Serving engine (include/mmr.h, mmr_serve_*): many concurrent viewers of
// one shared point cloud, each with its own private cloud, camera and
// framebuffer, continuously batched.
//
// One engine tick = one frame for every active viewer:
//  1. the shared cloud is displaced once (step = tick) and, in the same pass,
//     every shared point is projected and depth-splatted into every active
//     viewer's depth-id buffer, so the shared positions are read once per
//     tick however many viewers watch them;
//  2. every active viewer's private cloud is displaced (step = that viewer's
//     frame index) and splatted into its own buffer, all viewers in one
//     chunked launch;
//  3. one resolve launch covers every active viewer's framebuffer.
// Viewers join and leave between ticks; a join is refused when its buffers
// would exceed the engine's device-memory budget (the caller queues it).
// Frame k of a viewer that joined at tick t0 is a pure function of (t0 + k,
// k): the same whether the viewer is served alone or among others.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <iterator>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mmr.h"
#include "mmr_device.cuh"
#include "mmr_internal.h"
#include "mmr_points.cuh"
#include "mmr_resolve.cuh"

namespace mmr {

// Per active viewer, uploaded every tick.
struct ViewDev {
    Cam cam;
    unsigned long long *keys;       // buffer this tick splats into
    unsigned long long *next_keys;  // buffer the resolve clears
    uint32_t *rgba;
    void *pos;                      // private cloud
    uint32_t n;                     // private points
    uint32_t npx;
    int W, H;
    float fW, fH, halfW, halfH;
    uint32_t step;                  // private Philox step (the viewer's frame index)
    uint32_t cloud;                 // private Philox counter word 2
    uint32_t seed_lo, seed_hi;
    float amplitude;
    uint32_t color, shared_color, background;
    uint32_t ph_a, ph_b, ph_c;      // prepared Philox words of the private cloud
    const uint32_t *prev_tags;      // chunk tags of next_keys (FrameChunks), left by this view's previous frame
    uint32_t *cur_tags;             // chunk tags of keys
    uint32_t prev_tag, cur_tag;     // the view's previous and current frame numbers (frames rendered, + 1)
};

struct ServeTables {
    const ViewDev *views;
    uint32_t nviews;
    const uint2 *point_chunks;      // (view, first group) of private clouds
    uint32_t n_point_chunks;
    const uint2 *pixel_chunks;      // (view, first quad)
    uint32_t n_pixel_chunks;
    uint32_t chunk_groups, chunk_quads;
    uint32_t id_base;               // private ids start after the shared ones
};

__device__ __forceinline__ void view_params(const ViewDev &v, PointParams &P)
{
    P.cam = v.cam;
    P.keys = v.keys;
    P.W = v.W;
    P.H = v.H;
    P.fW = v.fW;
    P.fH = v.fH;
    P.halfW = v.halfW;
    P.halfH = v.halfH;
}

// Pass 1: the shared cloud, displaced once and splatted into every view.
// The tick is bound by the latency of the depth tests into many views, so
// resident warps matter: on FP32 storage a cap of 56 registers (from 58)
// gives 9 blocks of 128 threads per SM instead of 8, without spilling.  The
// 16-bit groups hold 24 coordinates across the view loop and need 69; their
// cap of 72 only keeps them there (with no cap the compiler takes 80).
template <int DT>
__global__ void __maxnreg__(DT == kF32 ? 56 : 72)
serve_shared_kernel(void *__restrict__ pos, uint32_t n, PointParams S, ServeTables T)
{
    constexpr int G = Group<DT>::kPoints;
    const uint32_t full = n / G;
    const uint32_t groups = groups_of<DT>(n);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const uint32_t i0 = g * G;
        const uint32_t count = min((uint32_t)G, n - i0);
        uint4 q[3];
        float v[3 * G];
        if (g < full) {
            load_words(pos, g, q);
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                v[k] = word_coord<DT>(q, k);
        } else {
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                v[k] = (uint32_t)(k / 3) < count ? load_coord<DT>(pos, 3ull * i0 + k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if ((uint32_t)j < count) {
                displace_point(v[3 * j], v[3 * j + 1], v[3 * j + 2], i0 + j, S);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    v[3 * j + c] = storage_round<DT>(v[3 * j + c]);
            }
        }
        if (g < full) {
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)
                set_word_coord<DT>(q, k, v[k]);
            store_words(pos, g, q);
        } else {
#pragma unroll
            for (int k = 0; k < 3 * G; ++k)      // constant indices keep v in registers
                if ((uint32_t)k < 3 * count)
                    store_coord<DT>(pos, 3ull * i0 + k, v[k]);
        }
        for (uint32_t w = 0; w < T.nviews; ++w) {
            PointParams P = S;
            view_params(T.views[w], P);
#pragma unroll
            for (int j = 0; j < G; ++j) {
                uint32_t px;
                unsigned long long key;
                if ((uint32_t)j < count && project_key(v[3 * j], v[3 * j + 1], v[3 * j + 2], i0 + j, P, px, key))
                    splat_key(P.keys, px, key);
            }
        }
    }
}

// Pass 2: private clouds, chunked over all views.
template <int DT>
__global__ void __launch_bounds__(256) serve_private_kernel(ServeTables T)
{
    constexpr int G = Group<DT>::kPoints;
    for (uint32_t c = blockIdx.x; c < T.n_point_chunks; c += gridDim.x) {
        const uint2 ch = T.point_chunks[c];
        const ViewDev &vw = T.views[ch.x];
        PointParams P;
        view_params(vw, P);
        P.seed_lo = vw.seed_lo;
        P.seed_hi = vw.seed_hi;
        P.step = vw.step;
        P.cloud = vw.cloud;
        P.amplitude = vw.amplitude;
        P.amplitude_2m23 = vw.amplitude * 0x1p-23f;
        P.id_base = T.id_base;
        P.ph_a = vw.ph_a;
        P.ph_b = vw.ph_b;
        P.ph_c = vw.ph_c;
        const uint32_t n = vw.n;
        const uint32_t full = n / G;
        const uint32_t end = min(ch.y + T.chunk_groups, groups_of<DT>(n));
        for (uint32_t g = ch.y + threadIdx.x; g < end; g += blockDim.x) {
            if (g < full) {
                uint4 q[3];
                load_words(vw.pos, g, q);
                process_words<DT, true, true>(q, g * G, G, P);
                store_words(vw.pos, g, q);
            } else {
                process_tail<DT, true, true>(vw.pos, vw.pos, n, g * G, P);
            }
        }
    }
}

// Pass 3: resolve every view; ids below id_base are shared points.
__global__ void serve_resolve_kernel(ServeTables T)
{
    for (uint32_t c = blockIdx.x; c < T.n_pixel_chunks; c += gridDim.x) {
        const uint2 ch = T.pixel_chunks[c];
        const ViewDev &vw = T.views[ch.x];
        const uint32_t quads = vw.npx / 4;
        const uint32_t end = min(ch.y + T.chunk_quads, quads);
        auto colour = [&](unsigned long long k) {
            if (k == kEmptyKey)
                return vw.background;
            return (uint32_t)(k & 0xffffffffu) < T.id_base ? vw.shared_color : vw.color;
        };
        // colours and clears only in 64-pixel chunks this frame or the view's previous one touched, as in
        // the single-cloud resolve (FrameChunks); a quad holding a key tags its chunk
        for (uint32_t q = ch.y + threadIdx.x; q < end; q += blockDim.x) {
            const ulonglong2 k01 = __ldcs(reinterpret_cast<const ulonglong2 *>(vw.keys) + 2 * q);
            const ulonglong2 k23 = __ldcs(reinterpret_cast<const ulonglong2 *>(vw.keys) + 2 * q + 1);
            const bool dirty = (k01.x & k01.y & k23.x & k23.y) != kEmptyKey;
            const uint32_t chunk = q >> kChunkQuadShift;
            const bool prev = __ldg(vw.prev_tags + chunk) == vw.prev_tag;
            if (dirty || prev)
                __stcs(reinterpret_cast<uint4 *>(vw.rgba) + q,
                       make_uint4(colour(k01.x), colour(k01.y), colour(k23.x), colour(k23.y)));
            if (prev) {
                const ulonglong2 e = make_ulonglong2(kEmptyKey, kEmptyKey);
                reinterpret_cast<ulonglong2 *>(vw.next_keys)[2 * q] = e;
                reinterpret_cast<ulonglong2 *>(vw.next_keys)[2 * q + 1] = e;
            }
            if (dirty)
                vw.cur_tags[chunk] = vw.cur_tag;
        }
        if (end == quads && quads * 4 + threadIdx.x < vw.npx) {
            const uint32_t p = quads * 4 + threadIdx.x;
            vw.rgba[p] = colour(vw.keys[p]);
            vw.next_keys[p] = kEmptyKey;
        }
    }
}

}  // namespace mmr

namespace {

struct Viewer {
    bool active = false;
    uint64_t n = 0;
    int W = 0, H = 0;
    uint64_t seed = 0;
    uint32_t cloud = 0;
    float amplitude = 0.0f;
    uint32_t color = 0xFFFFFFFFu;
    uint32_t background = 0;
    void *pos = nullptr;
    uint64_t pos_bytes = 0;
    unsigned long long *keys[2] = {nullptr, nullptr};
    uint32_t *rgba = nullptr;
    uint64_t cap_pos = 0, cap_keys[2] = {0, 0}, cap_rgba = 0;  // sizes of the buffers held (>= what is used)
    uint64_t bytes = 0;             // everything this viewer needs
    uint32_t frames = 0;            // frames rendered = next private step
    uint32_t joined_tick = 0;
    mmr::Cam cam{};
    bool cam_set = false;
};

}  // namespace

struct mmr_serve {
    int device = 0;
    int sm_count = 148;
    int dtype = 0;
    uint64_t budget = 0, held = 0;
    void *shared_pos = nullptr;
    uint64_t shared_n = 0, shared_bytes = 0;
    uint64_t shared_seed = 0;
    uint32_t shared_cloud = 0;
    float shared_amplitude = 0.0f;
    uint32_t shared_color = 0xFFFFFFFFu;
    uint32_t tick = 0;
    std::vector<Viewer> viewers;
    uint32_t chunk_groups = 256, chunk_quads = 1024;

    // per-tick tables: device copies and a two-deep pinned staging ring
    std::vector<mmr::ViewDev> h_views;
    std::vector<uint2> h_pchunks, h_xchunks;
    mmr::ViewDev *d_views = nullptr;
    uint2 *d_pchunks = nullptr, *d_xchunks = nullptr;
    uint64_t cap_views = 0, cap_pchunks = 0, cap_xchunks = 0;
    unsigned char *staging[2] = {nullptr, nullptr};
    uint64_t staging_cap = 0;
    cudaEvent_t staging_free[2] = {nullptr, nullptr};
    int staging_slot = 0;
    cudaEvent_t tick_done = nullptr;
    bool timing = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};

    // host round-trip baseline buffers
    void *rt_host = nullptr;
    uint64_t rt_cap = 0;

    // Buffers of viewers that left, kept for the next joins (size in bytes -> pointer) instead of being freed:
    // cudaMalloc and cudaFree cost host time on every join and leave, and cudaFree waits for the whole device.
    // They stay counted in `held`; `cached` is their total.  No tick in flight uses them (a leave waits for
    // the last tick).
    std::multimap<uint64_t, void *> cache;
    uint64_t cached = 0;
    cudaStream_t aux = nullptr;     // non-blocking: clears a joining viewer's buffers without waiting for a tick

    char err[512] = "";
};

namespace {

thread_local char g_serve_error[512] = "";

mmr_status sfail(mmr_serve *s, mmr_status st, const char *fmt, ...)
{
    char *dst = s ? s->err : g_serve_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return st;
}

mmr_status scuda(mmr_serve *s, cudaError_t e, const char *what)
{
    return sfail(s, MMR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

mmr_status salloc(mmr_serve *s, void **p, uint64_t bytes, const char *what, bool budgeted = true)
{
    *p = nullptr;
    if (budgeted && s->budget && s->held + bytes > s->budget)
        return sfail(s, MMR_ERR_BUDGET, "%s: %llu bytes would exceed the budget (%llu of %llu held)", what,
                     (unsigned long long)bytes, (unsigned long long)s->held, (unsigned long long)s->budget);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return sfail(s, e == cudaErrorMemoryAllocation ? MMR_ERR_OOM : MMR_ERR_CUDA, "%s: cudaMalloc(%llu): %s",
                     what, (unsigned long long)bytes, cudaGetErrorString(e));
    }
    if (budgeted)
        s->held += bytes;
    return MMR_OK;
}

void sfree(mmr_serve *s, void **p, uint64_t bytes, bool budgeted = true)
{
    if (*p) {
        cudaFree(*p);
        if (budgeted)
            s->held -= bytes;
        *p = nullptr;
    }
}

// Free cached buffers, largest first, until `need` more bytes fit the budget (all of them for UINT64_MAX).
void trim_cache(mmr_serve *s, uint64_t need)
{
    while (!s->cache.empty() && (need == UINT64_MAX || (s->budget && s->held + need > s->budget))) {
        auto it = std::prev(s->cache.end());
        cudaFree(it->second);
        s->held -= it->first;
        s->cached -= it->first;
        s->cache.erase(it);
    }
}

// A viewer buffer of at least `bytes`: the smallest cached one of at most
// twice that size, else a new allocation (after trimming the cache to fit
// the budget, and once more after an out-of-memory failure).  *cap gets the
// buffer's size.
mmr_status vtake(mmr_serve *s, void **p, uint64_t bytes, uint64_t *cap, const char *what)
{
    auto it = s->cache.lower_bound(bytes);
    if (it != s->cache.end() && it->first <= 2 * bytes) {
        *p = it->second;
        *cap = it->first;
        s->cached -= it->first;
        s->cache.erase(it);
        return MMR_OK;
    }
    trim_cache(s, bytes);
    mmr_status st = salloc(s, p, bytes, what);
    if (st == MMR_ERR_OOM && !s->cache.empty()) {
        trim_cache(s, UINT64_MAX);
        st = salloc(s, p, bytes, what);
    }
    if (st == MMR_OK)
        *cap = bytes;
    return st;
}

// Return a viewer buffer to the cache.
void vgive(mmr_serve *s, void **p, uint64_t *cap)
{
    if (*p) {
        s->cache.emplace(*cap, *p);
        s->cached += *cap;
    }
    *p = nullptr;
    *cap = 0;
}

// A viewer's depth-id buffers each end with the buffer's chunk tags, one
// 32-bit word per 64 pixels; all zero at the join, which is what the first
// frame (number 1) takes as its "previous frame", so it repaints everything.
uint64_t tag_bytes(uint64_t npx) { return (npx + 63) / 64 * 4; }

uint32_t *view_tags(const Viewer &v, int b)
{
    return reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(v.keys[b]) + (uint64_t)v.W * v.H * 8);
}

uint64_t padded_point_bytes(uint64_t n, int dtype)
{
    const uint64_t raw = n * (dtype == MMR_F32x3 ? 12u : 6u);
    return (raw + 47) / 48 * 48;
}

uint32_t groups_for(uint64_t n, int dtype) { return (uint32_t)((n + (dtype == MMR_F32x3 ? 3 : 7)) / (dtype == MMR_F32x3 ? 4 : 8)); }

// Grow a device table to at least `bytes` (outside the budget: tables are
// tiny and belong to the engine, not to a viewer).
mmr_status ensure(mmr_serve *s, void **p, uint64_t *cap, uint64_t bytes, const char *what)
{
    if (*cap >= bytes && *p)
        return MMR_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return scuda(s, e, what);
    sfree(s, p, *cap, false);
    uint64_t want = std::max<uint64_t>(bytes, 2 * *cap);
    mmr_status st = salloc(s, p, want, what, false);
    if (st == MMR_OK)
        *cap = want;
    return st;
}

// Build this tick's tables on the host and copy them to the device on s.
mmr_status upload_tables(mmr_serve *S, cudaStream_t s, mmr::ServeTables &T)
{
    S->h_views.clear();
    S->h_pchunks.clear();
    S->h_xchunks.clear();
    for (size_t id = 0; id < S->viewers.size(); ++id) {
        Viewer &v = S->viewers[id];
        if (!v.active)
            continue;
        const uint32_t w = (uint32_t)S->h_views.size();
        mmr::ViewDev d{};
        d.cam = v.cam;
        const int buf = (int)(v.frames & 1u);
        d.keys = v.keys[buf];
        d.next_keys = v.keys[buf ^ 1];
        d.cur_tags = view_tags(v, buf);
        d.prev_tags = view_tags(v, buf ^ 1);
        d.cur_tag = v.frames + 1u;    // after a wrap old tags can only match too often: extra stores, same pixels
        d.prev_tag = v.frames;
        d.rgba = v.rgba;
        d.pos = v.pos;
        d.n = (uint32_t)v.n;
        d.npx = (uint32_t)((uint64_t)v.W * v.H);
        d.W = v.W;
        d.H = v.H;
        d.fW = (float)v.W;
        d.fH = (float)v.H;
        d.halfW = 0.5f * (float)v.W;
        d.halfH = 0.5f * (float)v.H;
        d.step = v.frames;
        d.cloud = v.cloud;
        d.seed_lo = (uint32_t)(v.seed & 0xffffffffu);
        d.seed_hi = (uint32_t)(v.seed >> 32);
        d.amplitude = v.amplitude;
        d.color = v.color;
        d.shared_color = S->shared_color;
        d.background = v.background;
        mmr::PointParams tmp{};
        tmp.seed_lo = d.seed_lo;
        tmp.seed_hi = d.seed_hi;
        tmp.step = d.step;
        tmp.cloud = d.cloud;
        mmr::philox_prepare(tmp);
        d.ph_a = tmp.ph_a;
        d.ph_b = tmp.ph_b;
        d.ph_c = tmp.ph_c;
        S->h_views.push_back(d);
        const uint32_t groups = groups_for(v.n, S->dtype);
        for (uint32_t g = 0; g < groups; g += S->chunk_groups)
            S->h_pchunks.push_back(make_uint2(w, g));
        const uint32_t quads = d.npx / 4;
        uint32_t q = 0;
        do {
            S->h_xchunks.push_back(make_uint2(w, q));
            q += S->chunk_quads;
        } while (q < quads);
    }
    const uint64_t bv = S->h_views.size() * sizeof(mmr::ViewDev);
    const uint64_t bp = S->h_pchunks.size() * sizeof(uint2);
    const uint64_t bx = S->h_xchunks.size() * sizeof(uint2);
    mmr_status st = ensure(S, (void **)&S->d_views, &S->cap_views, bv, "view table");
    if (st == MMR_OK)
        st = ensure(S, (void **)&S->d_pchunks, &S->cap_pchunks, bp, "private chunk table");
    if (st == MMR_OK)
        st = ensure(S, (void **)&S->d_xchunks, &S->cap_xchunks, bx, "pixel chunk table");
    if (st != MMR_OK)
        return st;
    const uint64_t total = bv + bp + bx;
    if (S->staging_cap < total) {
        cudaError_t e = cudaDeviceSynchronize();
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            if (S->staging[k])
                cudaFreeHost(S->staging[k]);
            S->staging[k] = nullptr;
            e = cudaMallocHost((void **)&S->staging[k], std::max<uint64_t>(total, 2 * S->staging_cap));
        }
        if (e != cudaSuccess)
            return scuda(S, e, "staging allocation");
        S->staging_cap = std::max<uint64_t>(total, 2 * S->staging_cap);
    }
    const int k = S->staging_slot;
    S->staging_slot ^= 1;
    cudaError_t e = cudaEventSynchronize(S->staging_free[k]);   // the copy two ticks ago has read it
    if (e != cudaSuccess)
        return scuda(S, e, "staging wait");
    unsigned char *h = S->staging[k];
    memcpy(h, S->h_views.data(), bv);
    memcpy(h + bv, S->h_pchunks.data(), bp);
    memcpy(h + bv + bp, S->h_xchunks.data(), bx);
    if (bv)
        e = cudaMemcpyAsync(S->d_views, h, bv, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && bp)
        e = cudaMemcpyAsync(S->d_pchunks, h + bv, bp, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && bx)
        e = cudaMemcpyAsync(S->d_xchunks, h + bv + bp, bx, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaEventRecord(S->staging_free[k], s);
    if (e != cudaSuccess)
        return scuda(S, e, "table upload");
    T.views = S->d_views;
    T.nviews = (uint32_t)S->h_views.size();
    T.point_chunks = S->d_pchunks;
    T.n_point_chunks = (uint32_t)S->h_pchunks.size();
    T.pixel_chunks = S->d_xchunks;
    T.n_pixel_chunks = (uint32_t)S->h_xchunks.size();
    T.chunk_groups = S->chunk_groups;
    T.chunk_quads = S->chunk_quads;
    T.id_base = (uint32_t)S->shared_n;
    return MMR_OK;
}

template <int DT>
cudaError_t launch_tick(mmr_serve *S, const mmr::ServeTables &T, cudaStream_t s, void *shared_pos)
{
    mmr::PointParams P{};
    P.seed_lo = (uint32_t)(S->shared_seed & 0xffffffffu);
    P.seed_hi = (uint32_t)(S->shared_seed >> 32);
    P.step = S->tick;
    P.cloud = S->shared_cloud;
    P.amplitude = S->shared_amplitude;
    P.id_base = 0;
    mmr::philox_prepare(P);
    const uint64_t groups = groups_for(S->shared_n, S->dtype);
    const int grid = (int)std::max<uint64_t>(1, (groups + 127) / 128);
    if (S->dtype == MMR_F32x3)
        mmr::serve_shared_kernel<mmr::kF32><<<grid, 128, 0, s>>>(shared_pos, (uint32_t)S->shared_n, P, T);
    else if (S->dtype == MMR_F16x3)
        mmr::serve_shared_kernel<mmr::kF16><<<grid, 128, 0, s>>>(shared_pos, (uint32_t)S->shared_n, P, T);
    else
        mmr::serve_shared_kernel<mmr::kBF16><<<grid, 128, 0, s>>>(shared_pos, (uint32_t)S->shared_n, P, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || T.nviews == 0)
        return e;
    if (T.n_point_chunks) {
        const int gp = (int)std::min<uint32_t>(T.n_point_chunks, (uint32_t)S->sm_count * 8);
        if (S->dtype == MMR_F32x3)
            mmr::serve_private_kernel<mmr::kF32><<<gp, 256, 0, s>>>(T);
        else if (S->dtype == MMR_F16x3)
            mmr::serve_private_kernel<mmr::kF16><<<gp, 256, 0, s>>>(T);
        else
            mmr::serve_private_kernel<mmr::kBF16><<<gp, 256, 0, s>>>(T);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    mmr::serve_resolve_kernel<<<(int)std::min<uint32_t>(T.n_pixel_chunks, (uint32_t)S->sm_count * 8), 256, 0, s>>>(T);
    return cudaGetLastError();
}

void release_viewer(mmr_serve *S, Viewer &v)
{
    vgive(S, &v.pos, &v.cap_pos);
    vgive(S, (void **)&v.keys[0], &v.cap_keys[0]);
    vgive(S, (void **)&v.keys[1], &v.cap_keys[1]);
    vgive(S, (void **)&v.rgba, &v.cap_rgba);
    v = Viewer{};
}

}  // namespace

extern "C" {

const char *mmr_serve_last_error(const mmr_serve *s) { return s ? s->err : g_serve_error; }

mmr_status mmr_serve_destroy(mmr_serve *s)
{
    if (!s)
        return MMR_OK;
    cudaDeviceSynchronize();
    for (Viewer &v : s->viewers)
        if (v.active)
            release_viewer(s, v);
    trim_cache(s, UINT64_MAX);
    if (s->aux)
        cudaStreamDestroy(s->aux);
    sfree(s, &s->shared_pos, s->shared_bytes);
    sfree(s, (void **)&s->d_views, s->cap_views, false);
    sfree(s, (void **)&s->d_pchunks, s->cap_pchunks, false);
    sfree(s, (void **)&s->d_xchunks, s->cap_xchunks, false);
    for (int k = 0; k < 2; ++k) {
        if (s->staging[k])
            cudaFreeHost(s->staging[k]);
        if (s->staging_free[k])
            cudaEventDestroy(s->staging_free[k]);
    }
    if (s->tick_done)
        cudaEventDestroy(s->tick_done);
    for (cudaEvent_t &e : s->ev)
        if (e)
            cudaEventDestroy(e);
    if (s->rt_host)
        cudaFreeHost(s->rt_host);
    delete s;
    return MMR_OK;
}

mmr_status mmr_serve_create(uint64_t shared_n, int dtype, uint64_t seed, uint32_t cloud, float amplitude,
                            uint64_t budget_bytes, mmr_serve **out)
{
    if (!out)
        return sfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_serve_create: out is NULL");
    *out = nullptr;
    if (shared_n == 0 || shared_n >= (1ull << 31))
        return sfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_serve_create: shared_n outside 1..2^31-1");
    if (dtype != MMR_F32x3 && dtype != MMR_F16x3 && dtype != MMR_BF16x3)
        return sfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_serve_create: unknown dtype %d", dtype);
    if (!mmr::amplitude_ok(amplitude))
        return sfail(nullptr, MMR_ERR_INVALID_ARG, "mmr_serve_create: amplitude must be 0 or in [2^-100, 1]");
    mmr_serve *s = new (std::nothrow) mmr_serve();
    if (!s)
        return sfail(nullptr, MMR_ERR_OOM, "mmr_serve_create: host allocation failed");
    s->dtype = dtype;
    s->budget = budget_bytes;
    s->shared_n = shared_n;
    s->shared_seed = seed;
    s->shared_cloud = cloud;
    s->shared_amplitude = amplitude;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sfail(nullptr, MMR_ERR_CUDA, "mmr_serve_create: no usable CUDA device: %s", cudaGetErrorString(e));
        delete s;
        return MMR_ERR_CUDA;
    }
    s->shared_bytes = padded_point_bytes(shared_n, dtype);
    mmr_status st = salloc(s, &s->shared_pos, s->shared_bytes, "shared cloud");
    if (st == MMR_OK) {
        e = cudaMemset(s->shared_pos, 0, s->shared_bytes);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&s->staging_free[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&s->tick_done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
        if (e != cudaSuccess)
            st = scuda(s, e, "mmr_serve_create: set-up");
    }
    if (st != MMR_OK) {
        snprintf(g_serve_error, sizeof g_serve_error, "%s", s->err);
        mmr_serve_destroy(s);
        return st;
    }
    *out = s;
    return MMR_OK;
}

mmr_status mmr_serve_shared_points(mmr_serve *s, void **dev_ptr)
{
    if (!s || !dev_ptr)
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_shared_points: NULL argument");
    *dev_ptr = s->shared_pos;
    return MMR_OK;
}

mmr_status mmr_serve_set_shared_color(mmr_serve *s, uint32_t color)
{
    if (!s)
        return MMR_ERR_INVALID_ARG;
    s->shared_color = color;
    return MMR_OK;
}

mmr_status mmr_serve_add_viewer(mmr_serve *s, uint64_t private_n, int width, int height, uint64_t seed,
                                uint32_t cloud, float amplitude, uint32_t color, uint32_t background, int *viewer)
{
    if (!s || !viewer)
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_add_viewer: NULL argument");
    *viewer = -1;
    if (private_n == 0 || s->shared_n + private_n >= (1ull << 32) || width < 1 || height < 1 || width > 32768 ||
        height > 32768 || !mmr::amplitude_ok(amplitude))
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_add_viewer: invalid viewer description");
    const uint64_t npx = (uint64_t)width * height;
    Viewer v;
    v.n = private_n;
    v.W = width;
    v.H = height;
    v.seed = seed;
    v.cloud = cloud;
    v.amplitude = amplitude;
    v.color = color;
    v.background = background;
    v.pos_bytes = padded_point_bytes(private_n, s->dtype);
    v.bytes = v.pos_bytes + npx * 20 + 2 * tag_bytes(npx);
    const uint64_t in_use = s->held - s->cached;      // cached buffers can always be given up
    if (s->budget && in_use + v.bytes > s->budget)   // refuse before touching the allocator
        return sfail(s, MMR_ERR_BUDGET, "mmr_serve_add_viewer: %llu bytes would exceed the budget (%llu of %llu "
                     "in use)", (unsigned long long)v.bytes, (unsigned long long)in_use,
                     (unsigned long long)s->budget);
    mmr_status st = vtake(s, &v.pos, v.pos_bytes, &v.cap_pos, "private cloud");
    if (st == MMR_OK)
        st = vtake(s, (void **)&v.keys[0], npx * 8 + tag_bytes(npx), &v.cap_keys[0], "viewer depth-id buffer 0");
    if (st == MMR_OK)
        st = vtake(s, (void **)&v.keys[1], npx * 8 + tag_bytes(npx), &v.cap_keys[1], "viewer depth-id buffer 1");
    if (st == MMR_OK)
        st = vtake(s, (void **)&v.rgba, npx * 4, &v.cap_rgba, "viewer framebuffer");
    if (st == MMR_OK) {
        // The buffers are new or come from a viewer whose last tick has finished, so clearing them on the
        // engine's own stream needs no wait for the tick in flight; the call returns once they are clear.
        cudaError_t e = cudaMemsetAsync(v.pos, 0, v.pos_bytes, s->aux);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(v.keys[0], 0xff, npx * 8, s->aux);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(v.keys[1], 0xff, npx * 8, s->aux);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(view_tags(v, 0), 0, tag_bytes(npx), s->aux);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(view_tags(v, 1), 0, tag_bytes(npx), s->aux);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(v.rgba, 0, npx * 4, s->aux);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s->aux);
        if (e != cudaSuccess)
            st = scuda(s, e, "mmr_serve_add_viewer: clearing");
    }
    if (st != MMR_OK) {
        char msg[512];
        snprintf(msg, sizeof msg, "%s", s->err);
        v.active = true;
        release_viewer(s, v);
        snprintf(s->err, sizeof s->err, "%s", msg);
        return st;
    }
    v.active = true;
    v.joined_tick = s->tick;
    int id = -1;
    for (size_t k = 0; k < s->viewers.size(); ++k)
        if (!s->viewers[k].active) {
            id = (int)k;
            break;
        }
    if (id < 0) {
        id = (int)s->viewers.size();
        s->viewers.push_back(Viewer{});
    }
    s->viewers[id] = v;
    *viewer = id;
    return MMR_OK;
}

static Viewer *viewer_at(mmr_serve *s, int id)
{
    if (!s || id < 0 || (size_t)id >= s->viewers.size() || !s->viewers[id].active)
        return nullptr;
    return &s->viewers[id];
}

mmr_status mmr_serve_viewer_points(mmr_serve *s, int viewer, void **dev_ptr)
{
    Viewer *v = viewer_at(s, viewer);
    if (!v || !dev_ptr)
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_viewer_points: no such viewer");
    *dev_ptr = v->pos;
    return MMR_OK;
}

mmr_status mmr_serve_set_camera(mmr_serve *s, int viewer, const double eye[3], const double target[3],
                                const double up[3], double fovy_deg, double znear, double zfar)
{
    Viewer *v = viewer_at(s, viewer);
    if (!v || !eye || !target || !up)
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_set_camera: bad argument");
    if (!(fovy_deg > 0.0 && fovy_deg < 180.0) || !(znear > 0.0) || !(zfar > znear) || !std::isfinite(zfar) ||
        !mmr::depth_range_ok((float)znear, (float)zfar))
        return sfail(s, MMR_ERR_INVALID_ARG,
                     "mmr_serve_set_camera: need 0 < fovy < 180, 2^-64 <= znear < zfar <= 2^64");
    float m[16];
    if (!mmr::build_clip_matrix(eye, target, up, fovy_deg, (double)v->W / (double)v->H, znear, zfar, m))
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_set_camera: eye == target or up parallel to view");
    for (int k = 0; k < 4; ++k) {
        v->cam.rx[k] = m[k];
        v->cam.ry[k] = m[4 + k];
        v->cam.rw[k] = m[12 + k];
    }
    v->cam.znear = (float)znear;
    v->cam.zfar = (float)zfar;
    v->cam_set = true;
    return MMR_OK;
}

mmr_status mmr_serve_remove_viewer(mmr_serve *s, int viewer)
{
    Viewer *v = viewer_at(s, viewer);
    if (!v)
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_remove_viewer: no such viewer");
    cudaError_t e = cudaEventSynchronize(s->tick_done);      // no tick in flight still uses its buffers
    if (e != cudaSuccess)
        return scuda(s, e, "mmr_serve_remove_viewer: wait for the last tick");
    release_viewer(s, *v);
    return MMR_OK;
}

static mmr_status serve_tick(mmr_serve *s, void *stream, int roundtrip)
{
    mmr::NvtxRange nvtx(roundtrip ? "mmr_serve_tick_roundtrip" : "mmr_serve_tick");
    if (!s)
        return MMR_ERR_INVALID_ARG;
    for (size_t k = 0; k < s->viewers.size(); ++k)
        if (s->viewers[k].active && !s->viewers[k].cam_set)
            return sfail(s, MMR_ERR_STATE, "viewer %d has no camera", (int)k);
    cudaStream_t st = (cudaStream_t)stream;
    mmr::ServeTables T{};
    mmr_status r = upload_tables(s, st, T);
    if (r != MMR_OK)
        return r;
    if (s->timing)
        cudaEventRecord(s->ev[0], st);
    void *render_pos = s->shared_pos;
    if (roundtrip) {
        // the paper's RAM-based comparison for the shared cloud: positions go
        // device -> host -> device every tick before they are drawn
        if (s->rt_cap < s->shared_bytes) {
            cudaError_t e = cudaDeviceSynchronize();
            if (s->rt_host)
                cudaFreeHost(s->rt_host);
            s->rt_host = nullptr;
            if (e == cudaSuccess)
                e = cudaMallocHost(&s->rt_host, s->shared_bytes);
            if (e != cudaSuccess)
                return scuda(s, e, "round-trip host buffer");
            s->rt_cap = s->shared_bytes;
        }
        cudaError_t e = cudaMemcpyAsync(s->rt_host, s->shared_pos, s->shared_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->shared_pos, s->rt_host, s->shared_bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess)
            return scuda(s, e, "round-trip copies");
    }
    cudaError_t e;
    if (s->dtype == MMR_F32x3)
        e = launch_tick<mmr::kF32>(s, T, st, render_pos);
    else if (s->dtype == MMR_F16x3)
        e = launch_tick<mmr::kF16>(s, T, st, render_pos);
    else
        e = launch_tick<mmr::kBF16>(s, T, st, render_pos);
    if (e != cudaSuccess)
        return scuda(s, e, "tick launch");
    if (s->timing)
        cudaEventRecord(s->ev[1], st);
    e = cudaEventRecord(s->tick_done, st);
    if (e != cudaSuccess)
        return scuda(s, e, "tick event");
    s->tick += 1;
    for (Viewer &v : s->viewers)
        if (v.active)
            v.frames += 1;
    return MMR_OK;
}

mmr_status mmr_serve_tick(mmr_serve *s, void *stream) { return serve_tick(s, stream, 0); }

mmr_status mmr_serve_tick_roundtrip(mmr_serve *s, void *stream) { return serve_tick(s, stream, 1); }

mmr_status mmr_serve_frame_ptr(mmr_serve *s, int viewer, const uint32_t **rgba, const uint64_t **depth_id,
                               uint32_t *frame_index)
{
    Viewer *v = viewer_at(s, viewer);
    if (!v)
        return sfail(s, MMR_ERR_INVALID_ARG, "mmr_serve_frame_ptr: no such viewer");
    if (rgba)
        *rgba = v->rgba;
    if (depth_id)
        *depth_id = reinterpret_cast<const uint64_t *>(v->keys[v->frames ? ((v->frames - 1) & 1u) : 1]);
    if (frame_index)
        *frame_index = v->frames;
    return MMR_OK;
}

mmr_status mmr_serve_status(const mmr_serve *s, uint32_t *tick, int *active_viewers, uint64_t *device_bytes)
{
    if (!s)
        return MMR_ERR_INVALID_ARG;
    if (tick)
        *tick = s->tick;
    if (active_viewers) {
        int a = 0;
        for (const Viewer &v : s->viewers)
            a += v.active ? 1 : 0;
        *active_viewers = a;
    }
    if (device_bytes)
        *device_bytes = s->held;
    return MMR_OK;
}

mmr_status mmr_serve_set_timing(mmr_serve *s, int enable)
{
    if (!s)
        return MMR_ERR_INVALID_ARG;
    for (cudaEvent_t &e : s->ev)
        if (enable && !e && cudaEventCreate(&e) != cudaSuccess)
            return sfail(s, MMR_ERR_CUDA, "mmr_serve_set_timing: cudaEventCreate");
    s->timing = enable != 0;
    return MMR_OK;
}

mmr_status mmr_serve_last_tick_ms(mmr_serve *s, float *ms)
{
    if (!s || !ms)
        return MMR_ERR_INVALID_ARG;
    if (!s->timing)
        return sfail(s, MMR_ERR_STATE, "timing is off");
    cudaError_t e = cudaEventSynchronize(s->ev[1]);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(ms, s->ev[0], s->ev[1]);
    if (e != cudaSuccess)
        return scuda(s, e, "mmr_serve_last_tick_ms");
    return MMR_OK;
}

}  // extern "C"
