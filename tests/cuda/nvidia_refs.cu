// Test-only: NVIDIA's own device implementations, called on the GPU so the
// tests can pin the CPU oracle against them (cuRAND's Philox4x32-10 and the
// CUDA binary16 / bfloat16 round-to-nearest conversions).  Not part of the
// library; built by the tests into tests/_build/.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

__global__ void philox_ref_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

__global__ void narrow_ref_kernel(uint32_t start, uint32_t count, uint16_t *f16, uint16_t *bf16)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        const float x = __uint_as_float(start + i);
        f16[i] = __half_as_ushort(__float2half_rn(x));
        bf16[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    }
}

extern "C" int nvref_philox(const void *ctr, const void *key, void *out, int n)
{
    philox_ref_kernel<<<(n + 255) / 256, 256>>>(static_cast<const uint4 *>(ctr), static_cast<const uint2 *>(key),
                                                static_cast<uint4 *>(out), n);
    return (int)cudaDeviceSynchronize();
}

extern "C" int nvref_narrow(uint32_t start, uint32_t count, void *f16, void *bf16)
{
    narrow_ref_kernel<<<(count + 255) / 256, 256>>>(start, count, static_cast<uint16_t *>(f16),
                                                    static_cast<uint16_t *>(bf16));
    return (int)cudaDeviceSynchronize();
}
