// lbm_internal.h -- device-side records and launch entry points shared by the
// kernel and host-API translation units of liblbmfreeze (not installed).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbmk {

constexpr int kObs = 11;  // observables per instance (LBM_OBS_COUNT)
constexpr int kFrz = LBM_FRZ_COUNT;       // doubles of a lattice's freezing record
constexpr double kFreezeFraction = LBM_FREEZE_FRACTION;

// Bits of Inst::flags.
enum : int {
    kPeriodicX = 1 << 0,
    kPeriodicY = 1 << 1,
    kDirXlo = 1 << 2,
    kDirXhi = 1 << 3,
    kDirYlo = 1 << 4,
    kDirYhi = 1 << 5,
    kStMask = 1 << 6,
    kBuoy = 1 << 7,   // Boussinesq force present
    kPhaseProps = 1 << 8,  // per-phase heat capacity / conductivity
};

// Blocked state layout of one ping-pong buffer of a lattice. Sites are
// numbered site = y * pitch + x with pitch a multiple of 32, so that
// site = 32 * blk + l with blk = y * (pitch / 32) + x / 32 the row block of 32
// sites and l = x % 32 the site's place in it. Every block keeps all the
// values of its 32 sites together (one contiguous run per block, blocks in
// row order), so the values of a row segment share DRAM pages instead of
// lying in 24 or more planes a whole lattice apart.
//   population region (kPopBlock elements of the storage type per block):
//     three chunks by the y component of the direction a population moves
//     along, so that a row's pull takes one contiguous chunk from each of
//     the rows y - 1, y and y + 1:
//       chunk P (c_y = +1: directions 2, 5, 6) at element 0,
//       chunk Z (c_y =  0: directions 1, 3)    at element 288,
//       chunk M (c_y = -1: directions 4, 7, 8) at element 480;
//     inside a chunk of n directions, direction number k (in the order
//     above) keeps its (g, h) pairs at 64 k + 2 l + set and its f at
//     64 n + 32 k + l. Chunks P and M list opposite directions in the same
//     order (4 = opp 2, 7 = opp 5, 8 = opp 6), so a wall's bounce-back reads
//     the opposite chunk of the same row where the pull would read the
//     chunk of the row behind the wall.
//   own-site region (kAuxBlock FP32 values per block):
//     (g_0, h_0 - L f_l, f_0, f_l) at 4 l,
//     ((phi u)_x, (phi u)_y, p, S) at 128 + 4 l,
//     16-bit storage only: (phi_ref, T_ref) at 256 + 2 l.
// h_0 is stored shifted by -L f_l of the same site and step, which keeps every
// stored value O(1) (the latent part of H is carried by f_l instead).
constexpr int kPopElems = 24;
constexpr int kPopBlock = kPopElems * 32;  // population elements per block
constexpr int kAuxBlock = 10 * 32;         // own-site floats per block
constexpr int kChunkP = 0, kChunkZ = 288, kChunkM = 480;  // chunk offsets (elements)

// Chunk of direction i (1..8): its offset, the direction's number k inside
// it and the chunk's number of directions n.
__host__ __device__ constexpr int chunk_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? kChunkP : ((i == 1 || i == 3) ? kChunkZ : kChunkM);
}
__host__ __device__ constexpr int chunk_k(int i) {
    return (i == 2 || i == 1 || i == 4) ? 0 : ((i == 5 || i == 3 || i == 7) ? 1 : 2);
}
__host__ __device__ constexpr int chunk_n(int i) { return (i == 1 || i == 3) ? 2 : 3; }
// Offsets of (g_i, h_i) and f_i inside a block (elements).
__host__ __device__ constexpr int gh_off(int i) { return chunk_of(i) + 64 * chunk_k(i); }
__host__ __device__ constexpr int f_off(int i) {
    return chunk_of(i) + 64 * chunk_n(i) + 32 * chunk_k(i);
}

// The two 16-bit storage types (FP16: 10-bit mantissa, BF16: 7-bit mantissa
// and the FP32 exponent range) behind one set of conversions.
template <typename ST>
struct Bits16;
template <>
struct Bits16<__half> {
    static __host__ __device__ float to_f(__half v) { return __half2float(v); }
    static __host__ __device__ __half from_f(float v) { return __float2half_rn(v); }
    static __host__ __device__ __half from_d(double v) { return __double2half(v); }
    static __host__ __device__ __half from_bits(unsigned short b) { return __ushort_as_half(b); }
    static __host__ __device__ unsigned short bits(__half v) { return __half_as_ushort(v); }
    // two values in one word (lo in the low half), and back, one rounding each
    static __device__ unsigned pack2(float lo, float hi) {
        const __half2 q = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const unsigned*>(&q);
    }
    static __device__ float2 unpack2(unsigned w) {
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    }
    // mixed-precision forms (sm_100 and later): the 16-bit operand converts
    // exactly, the result rounds once
    static __device__ float add_lo(unsigned w, float c) {  // low half of w + c
        float d;
        asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.f16 %0, lo, %2; }"
            : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
    static __device__ float add_hi(unsigned w, float c) {  // high half of w + c
        float d;
        asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.f16 %0, hi, %2; }"
            : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
    // low half of w times 2^-12, plus c
    static __device__ float fma_lo_2m12(unsigned w, float c) {
        float d;
        asm("{ .reg .b16 lo, hi, s; mov.b32 {lo, hi}, %1; mov.b16 s, 0x0C00; fma.rn.f32.f16 %0, lo, s, %2; }"
            : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
};
template <>
struct Bits16<__nv_bfloat16> {
    static __host__ __device__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __host__ __device__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
    static __host__ __device__ __nv_bfloat16 from_d(double v) { return __double2bfloat16(v); }
    static __host__ __device__ __nv_bfloat16 from_bits(unsigned short b) { return __ushort_as_bfloat16(b); }
    static __host__ __device__ unsigned short bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
    static __device__ unsigned pack2(float lo, float hi) {
        const __nv_bfloat162 q = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const unsigned*>(&q);
    }
    static __device__ float2 unpack2(unsigned w) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    }
    static __device__ float add_lo(unsigned w, float c) {
        float d;
        asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.bf16 %0, lo, %2; }"
            : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
    static __device__ float add_hi(unsigned w, float c) {
        float d;
        asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.bf16 %0, hi, %2; }"
            : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
    static __device__ float fma_lo_2m12(unsigned w, float c) {
        float d;
        asm("{ .reg .b16 lo, hi, s; mov.b32 {lo, hi}, %1; mov.b16 s, 0x3980; fma.rn.f32.bf16 %0, lo, s, %2; }"
            : "=f"(d) : "r"(w), "f"(c));
        return d;
    }
};
__host__ __device__ inline int gh_at(int i, int site, int set) {
    return (site >> 5) * kPopBlock + gh_off(i) + 2 * (site & 31) + set;
}
__host__ __device__ inline int f_at(int i, int site) {
    return (site >> 5) * kPopBlock + f_off(i) + (site & 31);
}
__host__ __device__ inline int own0_at(int site, int c) {
    return (site >> 5) * kAuxBlock + 4 * (site & 31) + c;
}
__host__ __device__ inline int own1_at(int site, int c) {
    return (site >> 5) * kAuxBlock + 128 + 4 * (site & 31) + c;
}
__host__ __device__ inline int ref_at(int site, int c) {
    return (site >> 5) * kAuxBlock + 256 + 2 * (site & 31) + c;
}
// Element offset of population (set, i) in the population region (i >= 1).
__host__ __device__ inline int pop_at(int set, int i, int site) {
    return set < 2 ? gh_at(i, site, set) : f_at(i, site);
}
// Carried field k of the own-site region: 0 f_l, 1 (phi u)_x, 2 (phi u)_y,
// 3 p, 4 S, 5 phi_ref, 6 T_ref, 7/8/9 the rest populations g_0, h_0, f_0.
__host__ __device__ inline int aux_at(int k, int site) {
    return k == 0 ? own0_at(site, 3)
                  : (k <= 4 ? own1_at(site, k - 1)
                            : (k <= 6 ? ref_at(site, k - 5) : own0_at(site, k - 7)));
}

// One lattice as the kernels see it (state in the grouped layout above).
struct Inst {
    int nx, ny, pitch, flags;
    long long plane;          // sites per plane
    void* pop[2];             // population regions, ping-pong buffers
    float* aux[2];            // own-site regions
    int part_begin, part_end; // observable partials of this lattice's tiles
    int part_stride;          // partials are observable-major: [kObs][part_stride]
    double* macc;             // per tile / strip item (index `part`): sum of mdot over
                              // its sites, accumulated over every step (null: off)
    double* prof;             // nx doubles: sum over y of f_s per column, added to
                              // by observable steps (zero before each; null: off)
    double* prof_out;         // nx doubles: prof as of the last observable step,
                              // published by the reduction, which re-zeroes prof
    // physics, single precision
    float L, Hs, Tm, Cp, Cpref, Tw;
    float omega_g, omega_h;          // 1 / tau
    float kappa, beta, lam_coef;     // lam_coef = 4 / W
    float rho_s, rho_l, rho_g, mu_s, mu_l, mu_g, mdot_coef;
    float tan_w, inv_ramp;
    float normal_eps2;               // squared regularisation of the normal
    float inv_L, inv_Cp;
    float buoy_x, buoy_y, T_ref;     // F_g = buoy (T - T_ref), buoy = -rho_0 beta g
    float Cp_s, Cp_g;                // heat capacities of solid and gas (liquid: Cp)
    float k_s, k_g;                  // conductivities relative to the liquid's
    float dtau_h;                    // tau_h - 1/2 of the liquid
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

// The strip kernels of one storage type ST, row-staged (STAGED) or loading
// in place, for the supported (warps, regs) pairs; compiled in their own part
// of the kernel library and reached through the dispatchers below.
template <typename ST, bool STAGED>
struct StripPart {
    static cudaError_t launch(int warps, int regs, const Inst* d_inst, const Item* d_items,
                              int n_items, int parity, int obs, double* d_partials,
                              cudaStream_t s);
    static cudaError_t prepare(int warps, int regs);
    static int resident_warps(int warps, int regs);
    static int persist_grid(int warps, int regs, int n_items);
    static cudaError_t persist_launch(int warps, int regs, int grid, const Inst* d_inst,
                                      const Item* d_items, int n_items, int parity0, int nsteps,
                                      unsigned* d_bar, int* d_err, unsigned long long limit_ns,
                                      cudaStream_t s);
};

// The block kernels of one storage type ST (one warp per 32-site column of
// row blocks; lattices periodic in x), for the supported (warps, regs) pairs;
// compiled in their own part of the kernel library. d_err: raised (2) when a
// staged row never completed, then the warp stops.
template <typename ST>
struct BlockPart {
    static cudaError_t launch(int warps, int regs, const Inst* d_inst, const Item* d_items,
                              int n_items, int parity, int obs, double* d_partials, int* d_err,
                              cudaStream_t s);
    static cudaError_t prepare(int warps, int regs);
    static int resident_warps(int warps, int regs);
    static int persist_grid(int warps, int regs, int n_items);
    static cudaError_t persist_launch(int warps, int regs, int grid, const Inst* d_inst,
                                      const Item* d_items, int n_items, int parity0, int nsteps,
                                      unsigned* d_bar, int* d_err, unsigned long long limit_ns,
                                      cudaStream_t s);
};
// Block items: columns [x0, x0 + 32) with x0 a multiple of 32.
constexpr int kBlockW = 32;
bool block_supported(int warps, int regs);
// Raise the dynamic shared-memory limits of a block variant (host call).
cudaError_t prepare_block(int warps, int regs, int storage);
cudaError_t launch_step_block(int warps, int regs, int storage, const Inst* d_inst,
                              const Item* d_items, int n_items, int parity, int obs,
                              double* d_partials, int* d_err, cudaStream_t s);
int block_resident_warps(int warps, int regs, int storage);
int block_persistent_grid(int warps, int regs, int storage, int n_items);
cudaError_t launch_step_block_persistent(int warps, int regs, int storage, int grid,
                                         const Inst* d_inst, const Item* d_items, int n_items,
                                         int parity0, int nsteps, unsigned* d_bar, int* d_err,
                                         unsigned long long limit_ns, cudaStream_t s);

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

// Double-precision constants of the equilibrium initialisation.
struct InitConst {
    double L, Hs, Hl, Tm, Cp, Cpref, inv_ramp;
    double Cp_s, Cp_g;  // per-phase heat capacities (equal to Cp when uniform)
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
