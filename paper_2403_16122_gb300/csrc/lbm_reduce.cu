// lbm_reduce.cu -- FP64 reduction of the observable partials (arXiv
// 2403.16122: the global volume, solid, enthalpy and mass sums and the
// mass-source integral of Sections 4.1-4.3, plus the front and velocity
// records). The step kernels leave one partial per tile or strip item and
// observable; this kernel turns them into one record per lattice.
//
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so a
// lattice's partials are spread over several CTAs (kPer each) instead of one
// SM, and each CTA spends as few FP64 additions as a fixed tree allows; the
// last CTA of a lattice to finish (an atomic count) combines the CTA sums in
// CTA order. Every sum is taken in an order fixed by the partial indices
// alone, so the result does not depend on scheduling.
#include "lbm_reduce.h"

namespace lbmk {
namespace {

constexpr int kPer = 256;             // partials (and threads) per CTA
constexpr int kSums = kObs + 1;       // the observables, then the mdot running sums
constexpr int kGroup = 16;            // first-level group of the in-CTA tree

__device__ __forceinline__ double combine(int j, double a, double b) {
    return j == 9 ? fmax(a, b) : a + b;  // slot 9: max |u|; 0 is neutral for it too
}

// Thread t of CTA b holds partial begin + b * kPer + t (zeros past the end).
// In the CTA: kSums x (kPer / kGroup) threads each sum kGroup consecutive
// values in order, then kSums threads sum those in order; the CTA's kSums
// totals go to scratch. The last CTA of the lattice sums the CTA totals in CTA
// order, writes the observable record and the freezing record, publishes the
// column profile the observable step accumulated (copies it to prof_out and
// zeroes the accumulator for the next observable step) and re-arms the count.
__global__ void __launch_bounds__(kPer)
reduce_obs_split(const Inst* __restrict__ insts, const double* __restrict__ partials,
                 double* __restrict__ out, double* __restrict__ out_host,
                 double* __restrict__ frz, double* __restrict__ scratch,
                 unsigned* __restrict__ counts, long long step) {
    // value q of a row sits at q + q / kGroup: the first-level readers of one
    // warp (one group each) then hit distinct banks
    __shared__ double v[kSums][kPer + kPer / kGroup];
    __shared__ double g1[kSums][kPer / kGroup];
    __shared__ bool last;
    // Programmatic dependent launch: this grid is scheduled while the
    // observable step drains and reads nothing before that step has completed;
    // the next step's grid may be scheduled as soon as every CTA here has
    // started (it waits for this grid in turn). No-ops without the attribute.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int k = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
    const Inst& I = insts[k];
    const int begin = I.part_begin, n = I.part_end - I.part_begin, stride = I.part_stride;
    const int n_cta = n > 0 ? (n + kPer - 1) / kPer : 1;
    if (b >= n_cta) return;  // whole CTA, before any barrier or count
    const int p = b * kPer + t;
    const bool in = p < n;
#pragma unroll
    for (int j = 0; j < kObs; ++j)
        v[j][t + t / kGroup] = in ? partials[(long long)j * stride + begin + p] : 0.0;
    v[kObs][t + t / kGroup] = (in && I.macc) ? I.macc[begin + p] : 0.0;
    __syncthreads();
    if (t < kSums * (kPer / kGroup)) {
        const int j = t / (kPer / kGroup), c = t % (kPer / kGroup);
        const double* row = &v[j][c * (kGroup + 1)];
        double s = row[0];
#pragma unroll
        for (int q = 1; q < kGroup; ++q) s = combine(j, s, row[q]);
        g1[j][c] = s;
    }
    __syncthreads();
    // the scratch slots of lattice k: floor(begin / kPer) + k onwards (disjoint
    // across lattices, fewer than max_parts / kPer + n_inst + 1 in all)
    double* const mine = scratch + (long long)(begin / kPer + k) * kSums;
    if (t < kSums) {
        double s = g1[t][0];
#pragma unroll
        for (int c = 1; c < kPer / kGroup; ++c) s = combine(t, s, g1[t][c]);
        mine[(long long)b * kSums + t] = s;
        __threadfence();
    }
    __syncthreads();
    if (t == 0) last = atomicAdd(counts + k, 1u) == (unsigned)(n_cta - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the CTA sums in CTA order (0 is neutral for every slot), staged through
    // v (free again) kCap CTAs at a time so that their loads are in flight
    // together
    constexpr int kCap = kPer + kPer / kGroup;
    double tot = 0.0;
    for (int c0 = 0; c0 < n_cta; c0 += kCap) {
        const int nc = n_cta - c0 < kCap ? n_cta - c0 : kCap;
        for (int q = t; q < nc * kSums; q += kPer)
            v[q % kSums][q / kSums] = __ldcg(mine + (long long)c0 * kSums + q);
        __syncthreads();
        if (t < kSums)
            for (int c = 0; c < nc; ++c) tot = combine(t, tot, v[t][c]);
        __syncthreads();
    }
    if (t < kSums) {
        g1[t][0] = tot;
        if (t < kObs) {
            out[(long long)k * kObs + t] = tot;
            if (out_host) out_host[(long long)k * kObs + t] = tot;
        }
    }
    if (I.prof && I.prof_out) {
        double* const acc = I.prof;
        double* const pub = I.prof_out;
        for (int x0 = 0; x0 < I.nx; x0 += 4 * kPer) {
            double q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int x = x0 + u * kPer + t;
                q[u] = x < I.nx ? __ldcg(acc + x) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int x = x0 + u * kPer + t;
                if (x < I.nx) { pub[x] = q[u]; acc[x] = 0.0; }
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        counts[k] = 0u;  // the next reduction is stream-ordered after this one
        if (frz) {
            double* r = frz + (long long)k * kFrz;
            const double vol = g1[LBM_OBS_VOLUME][0], sol = g1[LBM_OBS_SOLID][0];
            const double X = vol > 0.0 ? sol / vol : 0.0;
            r[LBM_FRZ_STEP] = (double)step;
            r[LBM_FRZ_MDOT_INTEGRAL] = g1[kObs][0];
            if (r[LBM_FRZ_FREEZE_STEP] < 0.0 && X >= kFreezeFraction) r[LBM_FRZ_FREEZE_STEP] = (double)step;
            r[LBM_FRZ_SOLID_FRACTION] = X;
        }
    }
}

}  // namespace

int reduce_slots(int max_parts, int n_inst) { return max_parts / kPer + n_inst + 1; }

cudaError_t launch_reduce_obs(const Inst* d_inst, int n_inst, int max_lattice_parts,
                              const double* d_partials, double* d_obs, double* d_obs_host,
                              double* d_frz, double* d_scratch, unsigned* d_counts,
                              long long step, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    const int per = (max_lattice_parts + kPer - 1) / kPer;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_inst, (unsigned)(per > 0 ? per : 1));
    cfg.blockDim = dim3(kPer);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, reduce_obs_split, d_inst, d_partials, d_obs, d_obs_host, d_frz,
                              d_scratch, d_counts, step);
}

}  // namespace lbmk
