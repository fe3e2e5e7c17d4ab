// lbm_reduce.h -- the per-lattice reduction of the observable partials that
// every lbm_step call ends with (its own translation unit, lbm_reduce.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbmk {

// One record of kObs doubles per lattice (grid = n_inst CTAs) from the
// observable-major partials of its tiles or strip items, summed in a fixed
// order (slot 9 is a maximum), in stream s. d_frz (kFrz doubles per lattice,
// may be null) receives the freezing record of that observable step `step`:
// the running mdot integral of the lattice's slots (Inst::macc), the first
// observed step with solidified fraction >= kFreezeFraction (kept once set;
// -1 before) and the fraction itself.
cudaError_t launch_reduce_obs(const Inst* d_inst, int n_inst, const double* d_partials,
                              double* d_obs, double* d_frz, long long step, cudaStream_t s);

}  // namespace lbmk
