// Test-only: Philox4x32-10 draws of the library's device function next to
// cuRAND's device-API Philox4_32_10 for the same (counter, key).
//
// cuRAND: curand_init(seed, subsequence, offset) keys the generator with
// (seed & 0xffffffff, seed >> 32) and starts at the 128-bit counter
// (offset / 4) + subsequence * 2^64; curand4() returns the four words of that
// counter. So counter (c0, c1, c2, c3) is subsequence = c2 | c3 << 32 and
// offset = 4 * (c0 | c1 << 32).
#include <curand_kernel.h>

#include "../../paper_2205_01313_gb300/csrc/cupso_device.cuh"

__global__ void draws(const uint4* ctr, int n, uint32_t k0, uint32_t k1, uint4* own, uint4* ref) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    own[i] = cupso::philox4x32_10(c, k0, k1);
    curandStatePhilox4_32_10_t st;
    const unsigned long long seed = (unsigned long long)k0 | ((unsigned long long)k1 << 32);
    const unsigned long long sub = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    const unsigned long long off = 4ull * ((unsigned long long)c.x | ((unsigned long long)c.y << 32));
    curand_init(seed, sub, off, &st);
    ref[i] = curand4(&st);
}

extern "C" int philox_check(const unsigned* ctr_host, int n, unsigned k0, unsigned k1, unsigned* own_host,
                            unsigned* ref_host) {
    uint4 *c = nullptr, *a = nullptr, *b = nullptr;
    const size_t bytes = sizeof(uint4) * (size_t)n;
    if (cudaMalloc(&c, bytes) != cudaSuccess || cudaMalloc(&a, bytes) != cudaSuccess ||
        cudaMalloc(&b, bytes) != cudaSuccess)
        return 1;
    cudaMemcpy(c, ctr_host, bytes, cudaMemcpyHostToDevice);
    draws<<<(n + 127) / 128, 128>>>(c, n, k0, k1, a, b);
    cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(own_host, a, bytes, cudaMemcpyDeviceToHost);
    cudaMemcpy(ref_host, b, bytes, cudaMemcpyDeviceToHost);
    cudaFree(c);
    cudaFree(a);
    cudaFree(b);
    return e == cudaSuccess ? 0 : 2;
}
