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
// contiguous, so a warp's loads are coalesced. The per-slot running sums of
// mdot (every step since the start) are summed the same way into the
// lattice's freezing record, which also keeps the first observed step whose
// solidified fraction reached kFreezeFraction.
__global__ void __launch_bounds__(kThreads)
reduce_obs_wide(const Inst* __restrict__ insts, const double* __restrict__ partials,
                double* __restrict__ out, double* __restrict__ frz, long long step) {
    constexpr int kSums = kObs + 1;  // the observables, then the mdot running sums
    __shared__ double red[kSums][kWarps];
    const Inst& I = insts[blockIdx.x];
    const int begin = I.part_begin, end = I.part_end, stride = I.part_stride;
    const double* macc = I.macc;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double acc[kSums];
#pragma unroll
    for (int j = 0; j < kSums; ++j) acc[j] = 0.0;
#pragma unroll 4
    for (int p = begin + t; p < end; p += kThreads) {
#pragma unroll
        for (int j = 0; j < kObs; ++j)
            acc[j] = combine(j, acc[j], partials[(long long)j * stride + p]);
        if (macc) acc[kObs] += macc[p];
    }
#pragma unroll
    for (int j = 0; j < kSums; ++j) {
        double v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = combine(j, v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[j][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
        double tot[kSums];
#pragma unroll
        for (int j = 0; j < kSums; ++j) {
            double v = lane < kWarps ? red[j][lane] : 0.0;  // 0 is neutral for slot 9 too
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = combine(j, v, __shfl_xor_sync(0xffffffffu, v, o));
            tot[j] = v;
            if (lane == 0 && j < kObs) out[(long long)blockIdx.x * kObs + j] = v;
        }
        if (lane == 0 && frz) {
            double* r = frz + (long long)blockIdx.x * kFrz;
            const double X = tot[LBM_OBS_VOLUME] > 0.0 ? tot[LBM_OBS_SOLID] / tot[LBM_OBS_VOLUME] : 0.0;
            r[LBM_FRZ_STEP] = (double)step;
            r[LBM_FRZ_MDOT_INTEGRAL] = tot[kObs];
            if (r[LBM_FRZ_FREEZE_STEP] < 0.0 && X >= kFreezeFraction) r[LBM_FRZ_FREEZE_STEP] = (double)step;
            r[LBM_FRZ_SOLID_FRACTION] = X;
        }
    }
}

}  // namespace

cudaError_t launch_reduce_obs(const Inst* d_inst, int n_inst, const double* d_partials,
                              double* d_obs, double* d_frz, long long step, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    reduce_obs_wide<<<n_inst, kThreads, 0, s>>>(d_inst, d_partials, d_obs, d_frz, step);
    return cudaGetLastError();
}

}  // namespace lbmk
