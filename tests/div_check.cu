// Checks div_normal (the step kernels' division for normal positive operands)
// against the IEEE division on n seeded log-uniform operand pairs.
#include <cstdint>
#include <cuda_runtime.h>
#include "lbm_math.cuh"

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float logu(uint64_t r, float lo_exp, float hi_exp) {
    const float u = (float)(r >> 40) * (1.0f / 16777216.0f);
    return exp2f(lo_exp + (hi_exp - lo_exp) * u);
}
__global__ void k_check(long long n, unsigned long long seed, unsigned long long* bad,
                        unsigned* max_ulp) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint64_t r1 = mix64(seed + 2 * i), r2 = mix64(seed + 2 * i + 1);
        float x = logu(r1, -10.f, 10.f), y = logu(r2, -10.f, 10.f);
        if (r1 & 1) x = -x;
        const float a = lbmk::div_normal(x, y), b = __fdiv_rn(x, y);
        const int d = __float_as_int(a) - __float_as_int(b);
        const unsigned ad = d < 0 ? -d : d;
        if (ad) { atomicAdd(bad, 1ull); atomicMax(max_ulp, ad); }
    }
}
extern "C" int div_check(long long n, unsigned long long seed, unsigned long long* bad,
                         unsigned* max_ulp) {
    unsigned long long* d_bad; unsigned* d_max;
    if (cudaMalloc(&d_bad, 8) || cudaMalloc(&d_max, 4)) return 1;
    cudaMemset(d_bad, 0, 8); cudaMemset(d_max, 0, 4);
    k_check<<<1216, 256>>>(n, seed, d_bad, d_max);
    cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(bad, d_bad, 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(max_ulp, d_max, 4, cudaMemcpyDeviceToHost);
    cudaFree(d_bad); cudaFree(d_max);
    return e == cudaSuccess ? 0 : 2;
}
