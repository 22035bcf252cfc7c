// Second workload: gravitational all-pairs N-body (the paper's N-body
// sample, Sec. 4.2.3), feeding the same renderer.  Written from the physics:
// softened Newtonian gravity; for body i the terms over j,
//   d = p_j - p_i, r2 = ((dx dx + dy dy) + dz dz) + eps2, inv = 1 / sqrt(r2),
//   t_j = d (m_j ((inv inv) inv)),
// are summed in chunks of kNbodyChunk consecutive j (each chunk in order,
// then the chunk sums in chunk order), then v' = v + (G acc) dt and
// p' = p + v' dt; every operation is an IEEE round-to-nearest FP32
// operation (exact sqrt and division), so the result does not depend on the
// launch shape.
//
// Pass 1 gives one thread to every (body, chunk) pair, so even a few
// thousand bodies fill the GPU: each CTA stages tiles of the chunk's bodies
// (positions and masses, structure of arrays) in shared memory and every
// thread reads them by broadcast, keeping its partial sum in registers.
// Pass 2 adds a body's chunk sums in order, integrates, writes the new
// position into the other ping-pong buffer (every body must read every old
// position, so the update cannot be in place) and depth-splats it.
#include <algorithm>

#include <cuda_runtime.h>

#include "mmr_device.cuh"
#include "mmr_internal.h"

namespace mmr {

constexpr uint32_t kNbodyChunk = 1024;
constexpr int kNbodyTile = 128;

__global__ void __launch_bounds__(kNbodyTile) nbody_partial_kernel(const float *__restrict__ pin,
                                                                   const float *__restrict__ mass, uint32_t n,
                                                                   float eps2, float4 *__restrict__ partial)
{
    __shared__ float tx[kNbodyTile], ty[kNbodyTile], tz[kNbodyTile], tm[kNbodyTile];
    const uint32_t i = blockIdx.x * kNbodyTile + threadIdx.x;
    const uint32_t c0 = blockIdx.y * kNbodyChunk;
    const uint32_t c1 = min(c0 + kNbodyChunk, n);
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    if (i < n) {
        px = pin[3ull * i];
        py = pin[3ull * i + 1];
        pz = pin[3ull * i + 2];
    }
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (uint32_t t = c0; t < c1; t += kNbodyTile) {
        const uint32_t j = t + threadIdx.x;
        if (j < c1) {
            tx[threadIdx.x] = pin[3ull * j];
            ty[threadIdx.x] = pin[3ull * j + 1];
            tz[threadIdx.x] = pin[3ull * j + 2];
            tm[threadIdx.x] = mass[j];
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)kNbodyTile, c1 - t);
        if (i < n) {
#pragma unroll 4
            for (uint32_t k = 0; k < cnt; ++k) {
                const float dx = __fsub_rn(tx[k], px);
                const float dy = __fsub_rn(ty[k], py);
                const float dz = __fsub_rn(tz[k], pz);
                const float r2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                                                     __fmul_rn(dz, dz)), eps2);
                const float inv = __fdiv_rn(1.0f, __fsqrt_rn(r2));
                const float s = __fmul_rn(tm[k], __fmul_rn(__fmul_rn(inv, inv), inv));
                sx = __fadd_rn(sx, __fmul_rn(dx, s));
                sy = __fadd_rn(sy, __fmul_rn(dy, s));
                sz = __fadd_rn(sz, __fmul_rn(dz, s));
            }
        }
        __syncthreads();
    }
    if (i < n)
        partial[(size_t)blockIdx.y * n + i] = make_float4(sx, sy, sz, 0.0f);
}

__global__ void nbody_finalize_kernel(const float *__restrict__ pin, float *__restrict__ pout,
                                      float *__restrict__ vel, const float4 *__restrict__ partial, uint32_t n,
                                      uint32_t chunks, NbodyParams B, PointParams P)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    for (uint32_t c = 0; c < chunks; ++c) {
        const float4 q = partial[(size_t)c * n + i];
        ax = __fadd_rn(ax, q.x);
        ay = __fadd_rn(ay, q.y);
        az = __fadd_rn(az, q.z);
    }
    const float px = pin[3ull * i], py = pin[3ull * i + 1], pz = pin[3ull * i + 2];
    const float vx = __fadd_rn(vel[3ull * i], __fmul_rn(__fmul_rn(B.G, ax), B.dt));
    const float vy = __fadd_rn(vel[3ull * i + 1], __fmul_rn(__fmul_rn(B.G, ay), B.dt));
    const float vz = __fadd_rn(vel[3ull * i + 2], __fmul_rn(__fmul_rn(B.G, az), B.dt));
    vel[3ull * i] = vx;
    vel[3ull * i + 1] = vy;
    vel[3ull * i + 2] = vz;
    const float qx = __fadd_rn(px, __fmul_rn(vx, B.dt));
    const float qy = __fadd_rn(py, __fmul_rn(vy, B.dt));
    const float qz = __fadd_rn(pz, __fmul_rn(vz, B.dt));
    pout[3ull * i] = qx;
    pout[3ull * i + 1] = qy;
    pout[3ull * i + 2] = qz;
    uint32_t px_idx;
    unsigned long long key;
    if (project_key(qx, qy, qz, P.id_base + i, P, px_idx, key))
        splat_key(P.keys, px_idx, key);
}

uint32_t nbody_chunks(uint32_t n) { return (n + kNbodyChunk - 1) / kNbodyChunk; }

cudaError_t launch_nbody(const float *pin, float *pout, float *vel, const float *mass, float4 *partial, uint32_t n,
                         const NbodyParams &B, const PointParams &P, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    const uint32_t chunks = nbody_chunks(n);
    const dim3 grid1((n + kNbodyTile - 1) / kNbodyTile, chunks);
    nbody_partial_kernel<<<grid1, kNbodyTile, 0, s>>>(pin, mass, n, B.eps2, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    nbody_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(pin, pout, vel, partial, n, chunks, B, P);
    return cudaGetLastError();
}

}  // namespace mmr
