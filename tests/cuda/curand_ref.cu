// Test helper (not part of the library): Philox4x32-10 outputs of cuRAND's
// own device function, called for each (counter, key) pair, to check the
// library's Philox against it.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint4* ctr, const uint2* key, uint4* out, unsigned long long n) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_ref_philox(const void* ctr, const void* key, void* out, unsigned long long n) {
    k_curand_philox<<<256, 256>>>((const uint4*)ctr, (const uint2*)key, (uint4*)out, n);
    return (int)cudaDeviceSynchronize();
}
