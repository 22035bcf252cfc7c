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

// One term t_j, in the fixed order above.
__device__ __forceinline__ void nbody_term(float4 b, float px, float py, float pz, float eps2, float &tx, float &ty,
                                           float &tz)
{
    const float dx = __fsub_rn(b.x, px);
    const float dy = __fsub_rn(b.y, py);
    const float dz = __fsub_rn(b.z, pz);
    const float r2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)), eps2);
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(r2));
    const float s = __fmul_rn(b.w, __fmul_rn(__fmul_rn(inv, inv), inv));
    tx = __fmul_rn(dx, s);
    ty = __fmul_rn(dy, s);
    tz = __fmul_rn(dz, s);
}

// Terms of bodies a and b (two consecutive j) at once on packed FP32 pairs:
// every element is the IEEE operation of nbody_term (subtraction as the
// addition of the exact negation; each product that feeds an addition an
// fma with -0, so the assembler cannot fuse it); the square root and the
// division stay scalar.
__device__ __forceinline__ void nbody_term_pair(float4 a, float4 b, F2 NPX, F2 NPY, F2 NPZ, F2 EPS2, float &txa,
                                                float &tya, float &tza, float &txb, float &tyb, float &tzb)
{
    const F2 DX = f2_add(f2(a.x, b.x), NPX);
    const F2 DY = f2_add(f2(a.y, b.y), NPY);
    const F2 DZ = f2_add(f2(a.z, b.z), NPZ);
    const F2 R2 = f2_add(f2_add(f2_add(f2_product(DX, DX), f2_product(DY, DY)), f2_product(DZ, DZ)), EPS2);
    float ra, rb;
    f2_split(R2, ra, rb);
    const F2 INV = f2(__fdiv_rn(1.0f, __fsqrt_rn(ra)), __fdiv_rn(1.0f, __fsqrt_rn(rb)));
    const F2 S = f2_mul(f2(a.w, b.w), f2_mul(f2_mul(INV, INV), INV));
    f2_split(f2_product(DX, S), txa, txb);
    f2_split(f2_product(DY, S), tya, tyb);
    f2_split(f2_product(DZ, S), tza, tzb);
}

// Each tile holds (x, y, z, m) of kNbodyTile bodies, so a term reads one
// 16-byte word of shared memory.  Terms are computed two at a time
// (nbody_term_pair) and added to the sums one after another in j order.
__global__ void __launch_bounds__(kNbodyTile) nbody_partial_kernel(const float *__restrict__ pin,
                                                                   const float *__restrict__ mass, uint32_t n,
                                                                   float eps2, float4 *__restrict__ partial)
{
    __shared__ float4 tile[kNbodyTile];
    const uint32_t i = blockIdx.x * kNbodyTile + threadIdx.x;
    const uint32_t c0 = blockIdx.y * kNbodyChunk;
    const uint32_t c1 = min(c0 + kNbodyChunk, n);
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    if (i < n) {
        px = pin[3ull * i];
        py = pin[3ull * i + 1];
        pz = pin[3ull * i + 2];
    }
    const F2 NPX = f2(-px, -px), NPY = f2(-py, -py), NPZ = f2(-pz, -pz), EPS2 = f2(eps2, eps2);
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (uint32_t t = c0; t < c1; t += kNbodyTile) {
        const uint32_t j = t + threadIdx.x;
        if (j < c1)
            tile[threadIdx.x] = make_float4(pin[3ull * j], pin[3ull * j + 1], pin[3ull * j + 2], mass[j]);
        __syncthreads();
        const uint32_t cnt = min((uint32_t)kNbodyTile, c1 - t);
        if (i < n) {
            uint32_t k = 0;
#pragma unroll 2
            for (; k + 1 < cnt; k += 2) {
                float txa, tya, tza, txb, tyb, tzb;
                nbody_term_pair(tile[k], tile[k + 1], NPX, NPY, NPZ, EPS2, txa, tya, tza, txb, tyb, tzb);
                sx = __fadd_rn(__fadd_rn(sx, txa), txb);
                sy = __fadd_rn(__fadd_rn(sy, tya), tyb);
                sz = __fadd_rn(__fadd_rn(sz, tza), tzb);
            }
            if (k < cnt) {
                float tx, ty, tz;
                nbody_term(tile[k], px, py, pz, eps2, tx, ty, tz);
                sx = __fadd_rn(sx, tx);
                sy = __fadd_rn(sy, ty);
                sz = __fadd_rn(sz, tz);
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
