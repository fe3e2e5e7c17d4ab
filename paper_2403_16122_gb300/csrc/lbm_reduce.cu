// lbm_reduce.cu -- FP64 reduction of the observable partials (arXiv
// 2403.16122: the global volume, solid, enthalpy and mass sums and the
// mass-source integral of Sections 4.1-4.3, plus the front and velocity
// records). The step kernels leave one partial per tile or strip item and
// observable; this kernel turns them into one record per lattice.
#include "lbm_reduce.h"

namespace lbmk {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double combine(int j, double a, double b) {
    return j == 9 ? fmax(a, b) : a + b;  // slot 9: max |u|
}

// Thread t sums partials t, t + 512, ... of each observable in that order (the
// loads of four rounds in flight together), a fixed xor tree combines the
// sums of a warp, and warp 0 combines the 16 warp sums the same way: the
// result does not depend on scheduling. Each observable's partials are
// contiguous, so a warp's loads are coalesced.
__global__ void __launch_bounds__(kThreads)
reduce_obs_wide(const Inst* __restrict__ insts, const double* __restrict__ partials,
                double* __restrict__ out) {
    __shared__ double red[kObs][kWarps];
    const Inst& I = insts[blockIdx.x];
    const int begin = I.part_begin, end = I.part_end, stride = I.part_stride;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double acc[kObs];
#pragma unroll
    for (int j = 0; j < kObs; ++j) acc[j] = 0.0;
#pragma unroll 4
    for (int p = begin + t; p < end; p += kThreads) {
#pragma unroll
        for (int j = 0; j < kObs; ++j)
            acc[j] = combine(j, acc[j], partials[(long long)j * stride + p]);
    }
#pragma unroll
    for (int j = 0; j < kObs; ++j) {
        double v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = combine(j, v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[j][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < kObs; ++j) {
            double v = lane < kWarps ? red[j][lane] : 0.0;  // 0 is neutral for slot 9 too
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = combine(j, v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) out[(long long)blockIdx.x * kObs + j] = v;
        }
    }
}

}  // namespace

cudaError_t launch_reduce_obs(const Inst* d_inst, int n_inst, const double* d_partials,
                              double* d_obs, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    reduce_obs_wide<<<n_inst, kThreads, 0, s>>>(d_inst, d_partials, d_obs);
    return cudaGetLastError();
}

}  // namespace lbmk
