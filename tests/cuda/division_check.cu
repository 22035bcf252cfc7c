// Test-only checks of the perspective divide of the point kernels
// (perspective_divide in mmr_device.cuh) against CUDA's IEEE division
// __fdiv_rn.  Built by tests/test_division_gpu.py with the product's flags.
//
// div_significands: for divisors b = 1.m (all 2^23 significands from
//   b_begin) and `count` dividends a = 1.m' spread over [1, 2), compares
//   nx and ny of perspective_divide(a, -a, b) with __fdiv_rn(a, b) and
//   __fdiv_rn(-a, b) bit for bit.  With count = 2^23 this covers every
//   significand pair.
// div_rcp_scaling: the hardware reciprocal estimate of 1.m * 2^j equals
//   the one of 1.m times 2^-j for every significand and j in [-64, 64].
// div_random: random (a, b) with b over [2^-64, 2^64] (the clip w range
//   that camera validation allows) and |a / b| over [2^-40, 2^70]; inside the
//   exact band 2^-26 <= |a/b| <= 2^60 the quotient must equal __fdiv_rn;
//   below it |q| <= 2^-25, above it |q| > 2^59 or not finite.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../paper_2504_20937_b300/csrc/mmr_device.cuh"

namespace {

__device__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ void record(unsigned long long *bad, uint32_t *first, float a, float b)
{
    atomicAdd(bad, 1ull);
    if (atomicCAS(first, 0u, 1u) == 0u) {
        first[1] = __float_as_uint(a);
        first[2] = __float_as_uint(b);
    }
}

__global__ void significands_kernel(uint32_t b_begin, uint32_t b_count, uint32_t count, uint32_t step,
                                    unsigned long long *bad, uint32_t *first)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b_count || b_begin + t >= (1u << 23))
        return;
    const float b = __uint_as_float(0x3f800000u | (b_begin + t));
    for (uint32_t j = 0; j < count; ++j) {
        const uint32_t m = (j * step + (step > 1 ? mix32((b_begin + t) * 977u + j) % step : 0u)) & 0x7fffffu;
        const float a = __uint_as_float(0x3f800000u | m);
        float nx, ny;
        mmr::perspective_divide(a, -a, b, nx, ny);
        if (__float_as_uint(nx) != __float_as_uint(__fdiv_rn(a, b)) ||
            __float_as_uint(ny) != __float_as_uint(__fdiv_rn(-a, b)))
            record(bad, first, a, b);
    }
}

__global__ void rcp_scaling_kernel(unsigned long long *bad, uint32_t *first)
{
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (1u << 23))
        return;
    float y1;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(__uint_as_float(0x3f800000u | m)));
    const int e1 = (int)((__float_as_uint(y1) >> 23) & 0xff);
    for (int j = -64; j <= 64; ++j) {
        const float b = __uint_as_float(((uint32_t)(127 + j) << 23) | m);
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(b));
        const uint32_t want = (__float_as_uint(y1) & 0x807fffffu) | ((uint32_t)(e1 - j) << 23);
        if (__float_as_uint(y) != want)
            record(bad, first, 0.0f, b);
    }
}

__global__ void random_kernel(uint32_t seed, uint32_t iters, unsigned long long *bad, uint32_t *first,
                              unsigned long long *exact_count)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long exact = 0;
    for (uint32_t j = 0; j < iters; ++j) {
        const uint32_t h1 = mix32(seed ^ (t * 0x9e3779b9u + j * 0x85ebca6bu));
        const uint32_t h2 = mix32(h1 + 0x68e31da4u);
        const uint32_t h3 = mix32(h2 + 0xb5297a4du);
        const int eb = (int)(h1 % 129u) - 64;                     // b in [2^-64, 2^65)
        const int eq = (int)(h3 % 111u) - 40;                     // |a/b| around 2^eq
        const float b = __uint_as_float(((uint32_t)(127 + eb) << 23) | (h2 & 0x7fffffu));
        const int ea = eb + eq;
        if (ea < -126 || ea > 127 || b > 0x1p64f)
            continue;
        const float a = __uint_as_float((h1 & 0x80000000u) | ((uint32_t)(127 + ea) << 23) | (h3 >> 9));
        float nx, ny;
        mmr::perspective_divide(a, a, b, nx, ny);
        const float ieee = __fdiv_rn(a, b);
        const float mag = fabsf(ieee);
        bool ok;
        if (mag >= 0x1p-26f && mag <= 0x1p60f) {
            ok = __float_as_uint(nx) == __float_as_uint(ieee);
            ++exact;
        } else if (mag < 0x1p-26f) {
            ok = fabsf(nx) <= 0x1p-25f;
        } else {
            ok = !(fabsf(nx) <= 0x1p59f);                           // huge, infinite or NaN
        }
        if (!ok || __float_as_uint(nx) != __float_as_uint(ny))
            record(bad, first, a, b);
    }
    atomicAdd(exact_count, exact);
}

int finish(unsigned long long *d_bad, uint32_t *d_first, unsigned long long *bad, uint32_t *first)
{
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(bad, d_bad, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(first, d_first, 12, cudaMemcpyDeviceToHost);
    cudaFree(d_bad);
    cudaFree(d_first);
    return e == cudaSuccess ? 0 : (int)e;
}

int start(unsigned long long **d_bad, uint32_t **d_first)
{
    cudaError_t e = cudaMalloc(d_bad, 16);
    if (e == cudaSuccess)
        e = cudaMalloc(d_first, 12);
    if (e == cudaSuccess)
        e = cudaMemset(*d_bad, 0, 16);
    if (e == cudaSuccess)
        e = cudaMemset(*d_first, 0, 12);
    return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace

// count: dividends per divisor, a power of two <= 2^23.  bad: mismatches;
// first: (flag, a bits, b bits) of one mismatch.  Returns a CUDA error code.
extern "C" int div_significands(uint32_t count, unsigned long long *bad, uint32_t *first)
{
    if (count == 0 || count > (1u << 23) || (count & (count - 1)) != 0)
        return -1;
    unsigned long long *d_bad;
    uint32_t *d_first;
    int st = start(&d_bad, &d_first);
    if (st)
        return st;
    const uint32_t step = (1u << 23) / count;
    // slices of 2^15 divisors keep every launch well under a second
    const uint32_t slice = 1u << 15;
    for (uint32_t b0 = 0; b0 < (1u << 23); b0 += slice) {
        significands_kernel<<<slice / 256, 256>>>(b0, slice, count, step, d_bad, d_first);
        if (cudaPeekAtLastError() != cudaSuccess)
            break;
        if (count > (1u << 16) && cudaDeviceSynchronize() != cudaSuccess)
            break;
    }
    return finish(d_bad, d_first, bad, first);
}

extern "C" int div_rcp_scaling(unsigned long long *bad, uint32_t *first)
{
    unsigned long long *d_bad;
    uint32_t *d_first;
    int st = start(&d_bad, &d_first);
    if (st)
        return st;
    rcp_scaling_kernel<<<(1u << 23) / 256, 256>>>(d_bad, d_first);
    return finish(d_bad, d_first, bad, first);
}

// exact: how many sampled pairs fell in the exact band.
extern "C" int div_random(uint32_t seed, uint32_t iters, unsigned long long *bad, uint32_t *first,
                          unsigned long long *exact)
{
    unsigned long long *d_bad;
    uint32_t *d_first;
    int st = start(&d_bad, &d_first);
    if (st)
        return st;
    random_kernel<<<148 * 16, 256>>>(seed, iters, d_bad, d_first, d_bad + 1);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(exact, d_bad + 1, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaFree(d_bad);
        cudaFree(d_first);
        return (int)e;
    }
    return finish(d_bad, d_first, bad, first);
}
