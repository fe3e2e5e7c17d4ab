// lbm_reduce.h -- the per-lattice reduction of the observable partials that
// every lbm_step call ends with (its own translation unit, lbm_reduce.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbmk {

// One record of kObs doubles per lattice from the observable-major partials of
// its tiles or strip items, summed in a fixed order (slot 9 is a maximum), in
// stream s (and, when d_obs_host is not null, the same records into that
// device-mapped host memory); grid: n_inst x (CTAs for the largest lattice's
// partials).
// max_lattice_parts: the most partials any one lattice has. d_frz (kFrz
// doubles per lattice, may be null) receives the freezing record of that
// observable step `step`: the running mdot integral of the lattice's slots
// (Inst::macc), the first observed step with solidified fraction >=
// kFreezeFraction (kept once set; -1 before) and the fraction itself. The
// column profile a lattice's observable step added to Inst::prof is copied to
// Inst::prof_out and Inst::prof is zeroed again. d_scratch holds
// reduce_slots(max_parts, n_inst) x (kObs + 1) doubles; d_counts n_inst
// counters, zero before the first launch (each launch leaves them zero).
cudaError_t launch_reduce_obs(const Inst* d_inst, int n_inst, int max_lattice_parts,
                              const double* d_partials, double* d_obs, double* d_obs_host,
                              double* d_frz, double* d_scratch, unsigned* d_counts,
                              long long step, cudaStream_t s);

// Scratch slots (of kObs + 1 doubles) the reduction needs for a handle whose
// lattices have max_parts partials in all.
int reduce_slots(int max_parts, int n_inst);

}  // namespace lbmk
