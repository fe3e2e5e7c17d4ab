// lbm_internal.h -- device-side records and launch entry points shared by the
// kernel and host-API translation units of liblbmfreeze (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbmk {

constexpr int kObs = 11;  // observables per instance (LBM_OBS_COUNT)

// Bits of Inst::flags.
enum : int {
    kPeriodicX = 1 << 0,
    kPeriodicY = 1 << 1,
    kDirXlo = 1 << 2,
    kDirXhi = 1 << 3,
    kDirYlo = 1 << 4,
    kDirYhi = 1 << 5,
    kStMask = 1 << 6,
};

// One lattice as the kernels see it. Populations of set s (0 g, 1 h, 2 f) and
// direction i live in plane 9*s + i; a plane holds ny rows of `pitch`
// elements. In FP32 storage the rest population h_0 is stored shifted by
// -L f_l of the same site and step, which keeps every stored value O(1) (the
// latent part of H is carried by the liquid-fraction plane instead).
struct Inst {
    int nx, ny, pitch, flags;
    long long plane;          // elements per plane
    void* pop[2];             // 27 planes, ping-pong buffers
    float* aux[2];            // 5 planes: f_l, (phi u)_x, (phi u)_y, p, S
    int part_begin, part_end; // observable partials of this lattice's tiles
    // physics, single precision
    float L, Hs, Tm, Cp, Cpref, Tw;
    float omega_g, omega_h;          // 1 / tau
    float kappa, beta, lam_coef;     // lam_coef = 4 / W
    float rho_s, rho_l, rho_g, mu_s, mu_l, mu_g, mdot_coef;
    float tan_w, inv_ramp;
    float normal_eps2;               // squared regularisation of the normal
    float inv_L, inv_Cp;
};

// One CTA's tile: lattice `inst`, origin (x0, y0), extent tw x th, and the
// slot of its observable partials.
struct Tile {
    int inst, x0, y0, tw, th, part;
};

// One warp's work in the strip kernel: lattice `inst`, output columns
// [x0, x0 + 30) (a periodic x axis), rows [y0, y1), observable slot `part`.
struct Item {
    int inst, x0, y0, y1, part, pad[3];
};

// Output columns of one warp strip (the two remaining lanes hold the halo).
constexpr int kStripW = 30;

// Launch one time step over every strip item (one warp each, `warps` warps
// per CTA) in stream s.
cudaError_t launch_step_strip(int warps, int regs, int storage, const Inst* d_inst,
                              const Item* d_items, int n_items, int parity, int obs,
                              double* d_partials, cudaStream_t s);

// Supported strip-kernel variants (warps per CTA, register budget).
bool strip_supported(int warps, int regs);

// Staged strip variants (rows staged through shared memory with cp.async):
// FP32 and FP16 storage, the same (warps, regs) pairs as the plain strip kernel.
bool staged_supported(int warps, int regs, int storage);
// Raise the dynamic shared-memory limit of a staged variant (host call, once
// before its first launch; not a stream operation).
cudaError_t prepare_staged(int warps, int regs, int storage);
cudaError_t launch_step_staged(int warps, int regs, int storage, const Inst* d_inst,
                               const Item* d_items, int n_items, int parity, int obs,
                               double* d_partials, cudaStream_t s);
// Warps of a strip variant (staged != 0: the staged one) resident at once on
// the device; 0 if unsupported.
int strip_resident_warps(int staged, int warps, int regs, int storage);

// Persistent form of the strip step (staged != 0: the row-staged body):
// grid size (CTAs) of one cooperative launch over n_items items, at most what
// the device holds resident at once; 0 if the variant is unsupported. Also
// raises the variant's dynamic shared-memory limit (host call).
int persistent_grid(int staged, int warps, int regs, int storage, int n_items);

// One cooperative launch of `grid` CTAs that advances every item by nsteps
// steps (no observables) starting from buffer parity0, with a device-wide
// barrier between steps on *d_bar (must be zero at launch; the caller resets
// it in the same stream). A barrier wait longer than limit_ns sets *d_err.
cudaError_t launch_step_strip_persistent(int staged, int warps, int regs, int storage, int grid,
                                         const Inst* d_inst, const Item* d_items, int n_items,
                                         int parity0, int nsteps, unsigned* d_bar, int* d_err,
                                         unsigned long long limit_ns, cudaStream_t s);

// One CTA waiting at a barrier that nobody else joins: sets *d_err once
// limit_ns has passed, then returns.
cudaError_t launch_barrier_timeout_probe(unsigned* d_bar, int* d_err,
                                         unsigned long long limit_ns, cudaStream_t s);

// Launch one time step over every tile (grid = n_tiles CTAs) in stream s.
// parity selects the source buffer; obs != 0 also writes per-tile partials.
cudaError_t launch_step(int tx, int ty, int storage, const Inst* d_inst,
                        const Tile* d_tiles, int n_tiles, int parity, int obs,
                        double* d_partials, cudaStream_t s);

// Reduce per-tile partials into one record per lattice (grid = n_inst).
cudaError_t launch_reduce(const Inst* d_inst, int n_inst, const double* d_partials,
                          double* d_obs, cudaStream_t s);

// Double-precision constants of the equilibrium initialisation.
struct InitConst {
    double L, Hs, Hl, Tm, Cp, Cpref, inv_ramp;
};

// Equilibrium initialisation of lattice `inst` (nx*ny sites) from phi0/T0
// (device doubles, nx*ny each) into buffer `parity`.
cudaError_t launch_init(const Inst* d_inst, int inst, int n_sites, int storage,
                        InitConst c, const double* d_phi0, const double* d_T0,
                        int parity, cudaStream_t s);

// One time step of the 32 x 8 tile kernel for a single lattice whose record
// is passed by value (no device tables), with the per-tile observable
// partials in `scratch` (n_tiles * kObs doubles) and the reduced record in
// d_obs (kObs doubles). Buffer 0 of I is the source, buffer 1 the target.
cudaError_t launch_step_noalloc(const Inst& I, int tiles_x, int n_tiles, double* scratch,
                                double* d_obs, cudaStream_t s);

// Physics constants of a lattice record from its problem statement (the
// pointers, pitch and observable slots are left to the caller); *L gets the
// latent heat in double precision.
void inst_from_params(const lbm_params& p, Inst* I, double* L);

// Parameter checks of lbm_workspace_size / lbm_create.
bool params_valid(const lbm_params& p);

// Pitch (elements per row) the library uses for a lattice of width nx.
inline int pitch_for(int nx) { return (nx + 31) / 32 * 32; }

// Supported tile shapes (TX x TY threads, one site per thread).
bool tile_supported(int tx, int ty);

}  // namespace lbmk
