// Test helper: cuRAND's device Philox-4x32-10 block function over arrays of
// (counter, key), used to pin the oracle's Philox on the GPU.
#include <curand_kernel.h>
#include <stdint.h>

__global__ void philox_ref_kernel(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    uint4 r = curand_Philox4x32_10(c, k);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

extern "C" int philox_ref(const uint32_t* ctr_dev, const uint32_t* key_dev, uint32_t* out_dev, int n) {
    philox_ref_kernel<<<(n + 255) / 256, 256>>>(ctr_dev, key_dev, out_dev, n);
    return (int)cudaDeviceSynchronize();
}
