// lbm_reduce.h -- the per-lattice reduction of the observable partials that
// every lbm_step call ends with (its own translation unit, lbm_reduce.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbmk {

// One record of kObs doubles per lattice (grid = n_inst CTAs) from the
// observable-major partials of its tiles or strip items, summed in a fixed
// order (slot 9 is a maximum), in stream s.
cudaError_t launch_reduce_obs(const Inst* d_inst, int n_inst, const double* d_partials,
                              double* d_obs, cudaStream_t s);

}  // namespace lbmk
