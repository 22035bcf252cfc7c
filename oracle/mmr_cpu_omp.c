/* CPU baseline on all host cores, for measurement only (not the oracle).
 *
 * The paper runs its sample simulations on the CPU with OpenMP as well as
 * on the GPU (Sec. 4); this file times the benchmark's frame (Sec. 4.1:
 * Brownian displacement of every point, then a depth-tested render) the
 * same way, so the GPU path has a multi-core CPU figure beside the
 * single-threaded oracle.  Only bench.py's CPU legs and tests/ load it.
 *
 * Every point and pixel is computed by the oracle's own routines (linked
 * from mmr_oracle.c); this file only spreads them over threads:
 *  - displacement: each thread displaces a contiguous range of points
 *    through orc_displace_ids_f32, with the ids of that range;
 *  - splat: each thread projects its points with orc_project_f32 and
 *    lowers the pixel's key with a compare-and-swap minimum on the one
 *    shared depth-id buffer.  A minimum is order-free, so the frame is the
 *    oracle's bit for bit.  (Per-thread buffers merged at the end would cost
 *    threads x W x H per frame, more than the splat itself at 1080p.)
 *  - clear and resolve: split over the pixels.
 */
#include <stdint.h>
#include <stdlib.h>

#include <omp.h>

void orc_displace_ids_f32(float *pos, const uint32_t *ids, uint64_t m, uint64_t seed,
                          uint32_t cloud, uint32_t step, float a);
int orc_project_f32(const float M[16], float x, float y, float z, int W, int H,
                    float znear, float zfar, uint32_t *px, float *w_out, float ndc[2]);
void orc_resolve(const uint64_t *keybuf, uint64_t npx, const uint32_t *colors, uint32_t color,
                 uint32_t background, uint32_t *rgba);

enum { kIdsPerCall = 4096 };

static uint32_t f32_bits_omp(float f)
{
    union { float f; uint32_t u; } v;
    v.f = f;
    return v.u;
}

static void atomic_min_u64(uint64_t *p, uint64_t key)
{
    uint64_t cur = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (key < cur &&
           !__atomic_compare_exchange_n(p, &cur, key, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
    }
}

/* Threads the frame uses when `threads` <= 0: OpenMP's default (the host's
 * cores unless OMP_NUM_THREADS says otherwise). */
int cpu_omp_threads(int threads)
{
    return threads > 0 ? threads : omp_get_max_threads();
}

/* One FP32 frame: displace (step `step`), clear, splat, resolve with one
 * colour; the same arguments and results as orc_frame_f32 without a colour
 * buffer.  Returns the number of threads used. */
int cpu_omp_frame_f32(float *pos, uint64_t n, uint64_t seed, uint32_t cloud, uint32_t step, float a,
                      const float M[16], int W, int H, float znear, float zfar, uint32_t color,
                      uint32_t background, uint64_t *keybuf, uint32_t *rgba, int threads)
{
    const int T = cpu_omp_threads(threads);
    const uint64_t npx = (uint64_t)W * (uint64_t)H;
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int nt = omp_get_num_threads();
        const uint64_t lo = n * (uint64_t)t / (uint64_t)nt;
        const uint64_t hi = n * (uint64_t)(t + 1) / (uint64_t)nt;
        uint32_t ids[kIdsPerCall];
        for (uint64_t i0 = lo; i0 < hi; i0 += kIdsPerCall) {
            const uint64_t m = hi - i0 < kIdsPerCall ? hi - i0 : kIdsPerCall;
            for (uint64_t j = 0; j < m; ++j)
                ids[j] = (uint32_t)(i0 + j);
            orc_displace_ids_f32(pos + 3 * i0, ids, m, seed, cloud, step, a);
        }
        const uint64_t plo = npx * (uint64_t)t / (uint64_t)nt;
        const uint64_t phi = npx * (uint64_t)(t + 1) / (uint64_t)nt;
        for (uint64_t p = plo; p < phi; ++p)
            keybuf[p] = ~(uint64_t)0;
#pragma omp barrier
        for (uint64_t i = lo; i < hi; ++i) {
            uint32_t px;
            float cw;
            if (!orc_project_f32(M, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], W, H, znear, zfar, &px, &cw, 0))
                continue;
            atomic_min_u64(keybuf + px, ((uint64_t)f32_bits_omp(cw) << 32) | (uint64_t)(uint32_t)i);
        }
#pragma omp barrier
        orc_resolve(keybuf + plo, phi - plo, 0, color, background, rgba + plo);
    }
    return T;
}
