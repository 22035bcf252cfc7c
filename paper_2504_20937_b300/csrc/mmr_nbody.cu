// Second workload: gravitational all-pairs N-body (the paper's N-body
// sample, Sec. 4.2.3), feeding the same renderer.  Written from the physics:
// softened Newtonian gravity, for body i summed over j = 0 .. n-1 in order,
//   d = p_j - p_i, r2 = ((dx dx + dy dy) + dz dz) + eps2, inv = 1 / sqrt(r2),
//   s = m_j ((inv inv) inv), acc += d s,
// then v' = v + (G acc) dt and p' = p + v' dt, every operation an IEEE
// round-to-nearest FP32 operation (exact sqrt and division), so the result
// does not depend on the launch shape.
//
// Each CTA stages tiles of B bodies (positions and masses, structure of
// arrays) in shared memory; every thread reads them by broadcast and keeps
// its own sum in registers, in the same j order as a sequential loop.  Old
// positions are read from one ping-pong buffer and new ones written to the
// other, because every body reads every other body's old position.  The new
// position is projected and depth-splatted in the same kernel.
#include <algorithm>

#include <cuda_runtime.h>

#include "mmr_device.cuh"
#include "mmr_internal.h"

namespace mmr {

constexpr int kNbodyTile = 256;

__global__ void __launch_bounds__(kNbodyTile) nbody_kernel(const float *__restrict__ pin, float *__restrict__ pout,
                                                           float *__restrict__ vel, const float *__restrict__ mass,
                                                           uint32_t n, NbodyParams B, PointParams P)
{
    __shared__ float tx[kNbodyTile], ty[kNbodyTile], tz[kNbodyTile], tm[kNbodyTile];
    const uint32_t i = blockIdx.x * kNbodyTile + threadIdx.x;
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    if (i < n) {
        px = pin[3ull * i];
        py = pin[3ull * i + 1];
        pz = pin[3ull * i + 2];
    }
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    for (uint32_t t = 0; t < n; t += kNbodyTile) {
        const uint32_t j = t + threadIdx.x;
        if (j < n) {
            tx[threadIdx.x] = pin[3ull * j];
            ty[threadIdx.x] = pin[3ull * j + 1];
            tz[threadIdx.x] = pin[3ull * j + 2];
            tm[threadIdx.x] = mass[j];
        }
        __syncthreads();
        const uint32_t cnt = min((uint32_t)kNbodyTile, n - t);
        if (i < n) {
#pragma unroll 4
            for (uint32_t k = 0; k < cnt; ++k) {
                const float dx = __fsub_rn(tx[k], px);
                const float dy = __fsub_rn(ty[k], py);
                const float dz = __fsub_rn(tz[k], pz);
                const float r2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                                                     __fmul_rn(dz, dz)), B.eps2);
                const float inv = __fdiv_rn(1.0f, __fsqrt_rn(r2));
                const float s = __fmul_rn(tm[k], __fmul_rn(__fmul_rn(inv, inv), inv));
                ax = __fadd_rn(ax, __fmul_rn(dx, s));
                ay = __fadd_rn(ay, __fmul_rn(dy, s));
                az = __fadd_rn(az, __fmul_rn(dz, s));
            }
        }
        __syncthreads();
    }
    if (i >= n)
        return;
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

cudaError_t launch_nbody(const float *pin, float *pout, float *vel, const float *mass, uint32_t n,
                         const NbodyParams &B, const PointParams &P, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    const int grid = (int)((n + kNbodyTile - 1) / kNbodyTile);
    nbody_kernel<<<grid, kNbodyTile, 0, s>>>(pin, pout, vel, mass, n, B, P);
    return cudaGetLastError();
}

}  // namespace mmr
