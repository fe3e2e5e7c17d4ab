/*
 * lbm.h -- C-ABI of liblbmfreeze, the GB300 (sm_103a) time step of the
 * phase-field lattice Boltzmann method for freezing with volume change of
 * Huang, Wang, Chai & Shi, "Phase-field based lattice Boltzmann method for
 * containerless freezing" (arXiv 2403.16122).
 *
 * One time step advances three D2Q9 distribution sets together (Section 3):
 *   g  -- conservative Allen-Cahn phase field (Eqs. 21-26),
 *   h  -- total-enthalpy temperature field with the liquid-fraction closure
 *         (Eqs. 8-9, 27-29),
 *   f  -- pressure-based flow with the phase-change mass source and the
 *         solid-region forcing (Eqs. 19-20, 30-36),
 * with the isotropic stencils of Eq. 38 and the wetting ghost layer of
 * Eqs. 39-41. All of a step runs in one fused CUDA kernel per launch.
 *
 * Conventions (shared with every function below):
 *   - Lattice units, dx = dt = 1. A lattice has nx * ny sites; site (x, y)
 *     has host index y * nx + x.
 *   - Host distribution arrays ("pops") hold 27 planes of nx*ny doubles in the
 *     order g_0..g_8, h_0..h_8, f_0..f_8; c_1..c_4 point E, N, W, S and
 *     c_5..c_8 point NE, NW, SW, SE (Eq. 23). They are post-collision values.
 *   - Host carried-field arrays ("aux") hold 5 planes of nx*ny doubles:
 *     f_l (liquid fraction), (phi u)_x, (phi u)_y, p, S of the last
 *     completed step.
 *   - A non-periodic axis has a wall at both ends, half a link outside the
 *     first and last lattice rows/columns.
 *   - Return codes are LBM_OK or one of the negative LBM_E* values; no call
 *     aborts the process. Device faults surface as LBM_ECUDA.
 *
 * Ownership: the caller owns the device workspace passed to lbm_create (the
 * library never allocates device memory) and every host array; host arrays
 * are read or written during the call and never retained. The handle itself
 * is host memory owned by the library until lbm_destroy, with a pinned host
 * mirror of the observable records (11 doubles per lattice) through which
 * lbm_observables and lbm_observables_all copy.
 *
 * Thread safety: a handle is used by one host thread at a time. All device
 * work is queued on the stream given to lbm_create.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK          0
#define LBM_EINVAL     -1  /* invalid argument or parameter set              */
#define LBM_ENOMEM     -2  /* workspace smaller than lbm_workspace_size      */
#define LBM_ECUDA      -3  /* a CUDA call failed (launch, copy or fault)      */
#define LBM_ETIMEOUT   -4  /* a device-side wait gave up (batched launches)  */
#define LBM_EUNSTABLE  -5  /* non-finite fields or |u| > 0.5 at the last     */
                           /* observable step                              */
#define LBM_ESTATE     -6  /* call out of order (e.g. step before init)      */
#define LBM_ETOOLARGE  -7  /* lattice exceeds the fixed scratch of           */
                           /* lbm_step_noalloc                               */

/* Storage format of the distribution sets in device memory. Arithmetic is
   FP32 in every format.
   LBM_STORE_FP32: 27 FP32 planes (h_0 shifted by -L f_l) + 5 FP32 carried
                   planes: 256 bytes moved per lattice update.
   LBM_STORE_FP16: the 24 moving populations as 16-bit deviations from a
                   rest equilibrium: of the site they stream into for g and h
                   (w_i phi, w_i Cp_ref T), of their source site's pressure
                   for f (scaled by 2^12). The three rest populations stay
                   FP32 and absorb the rounding errors of the site's moving
                   ones, so the phi, H and f sums a site sends out are kept
                   exactly. phi and T of each site are two more FP32 planes:
                   176 bytes per lattice update. Needs every lattice periodic
                   in x (strip layout). lbm_get_state / lbm_set_state convert
                   to and from the same double layouts as FP32.
   LBM_STORE_BF16: the FP16 arrangement with bfloat16 values (7-bit
                   mantissa, FP32 exponent range): 176 bytes per lattice
                   update; the row-staged strip layout with 4 warps per CTA
                   only (registers 128 or 168). */
#define LBM_STORE_FP32  0
#define LBM_STORE_FP16  1
#define LBM_STORE_BF16  2

/* Problem statement of one lattice (Sections 4.1-4.3). */
typedef struct lbm_params {
    int32_t nx, ny;                 /* lattice size, >= 3 each                */
    int32_t periodic_x, periodic_y; /* 1 periodic, 0 walls at both ends       */
    int32_t dirichlet_x_lo, dirichlet_x_hi;  /* per wall: 1 temperature held  */
    int32_t dirichlet_y_lo, dirichlet_y_hi;  /* at T_w, 0 adiabatic           */
    int32_t st_mask_liquid;         /* 1: surface tension times (1 - f_s)     */
    int32_t reserved;               /* set to 0                               */
    double W;            /* interface width (Eq. 3), > 0                      */
    double sigma;        /* surface tension (Eq. 13), >= 0                    */
    double mobility;     /* M (Eq. 2), > 0; tau_g = M / c_s^2 + 1/2           */
    double tau_f_liquid; /* flow relaxation time of the liquid, > 1/2         */
    double tau_h;        /* enthalpy relaxation time (Eq. 27), > 1/2          */
    double rho_l;        /* liquid density, > 0                               */
    double rho_ratio_lg; /* rho_l / rho_g, > 0                                */
    double rho_ratio_sl; /* rho_s / rho_l, > 0                                */
    double mu_ratio_lg;  /* mu_l / mu_g, > 0                                  */
    double Ste;          /* Stefan number (Eq. 42), > 0                       */
    double Cp, Cp_ref;   /* heat capacity, reference heat capacity (Eq. 28)   */
    double T_m, T_w;     /* melting and wall temperature, T_w < T_m           */
    double theta_deg;    /* wall contact angle (Eq. 39), in (0, 180)          */
    double pc_ramp;      /* width in phi of the window where phase change
                            switches on (solid forms only in liquid), > 0     */
    double normal_eps;   /* interface-normal regularisation, > 0:
                            n = grad phi / sqrt(|grad phi|^2 + eps^2)         */
    double gx, gy;       /* gravity of the Boussinesq force (Section 4.3)     */
    double beta_T;       /* volumetric expansion coefficient; with gx, gy it
                            adds F_g = -rho_0 g beta_T (T - T_ref) to the
                            force of every site (0 switches it off)          */
    double T_ref;        /* reference temperature of F_g                      */
    double rho_0;        /* reference density of F_g                          */
    double Cp_ratio_sl;  /* C_p,s / C_p,l (Cp is the liquid's), > 0; with the
                            next three, per-phase thermal properties mixed by
                            Eq. 1; all 1: uniform properties                  */
    double Cp_ratio_gl;  /* C_p,g / C_p,l, > 0                                */
    double k_ratio_sl;   /* k_s / k_l, > 0: tau_h - 1/2 scales with k, the
                            liquid's tau_h being tau_h                        */
    double k_ratio_gl;   /* k_g / k_l, > 0                                    */
} lbm_params;

/* Observables of the most recent step of an instance (index into the
   record filled by lbm_observables); sums in FP64 over all sites. */
#define LBM_OBS_VOLUME          0   /* sum phi (drop volume)               */
#define LBM_OBS_SOLID           1   /* sum f_s (solid volume)              */
#define LBM_OBS_ENTHALPY        2   /* sum H                               */
#define LBM_OBS_MASS            3   /* sum rho                             */
#define LBM_OBS_CONDENSED_MASS  4   /* sum f_s rho_s + (1 - f_s) phi rho_l  */
#define LBM_OBS_MDOT            5   /* sum mdot (mass source, Eq. 19)      */
#define LBM_OBS_PHI_MDOT        6   /* sum phi * mdot                      */
#define LBM_OBS_SOLID_COL       7   /* sum_y f_s on column x = nx / 2      */
#define LBM_OBS_SOLID_ROW       8   /* sum_x f_s on row y = ny / 2         */
#define LBM_OBS_UMAX            9   /* max |u|                             */
#define LBM_OBS_NONFINITE      10   /* sites with a non-finite field       */
#define LBM_OBS_COUNT          11

/* Freezing record of an instance (lbm_freezing): quantities that span the
   whole run since lbm_init_fields rather than one step.
   LBM_FRZ_STEP           step index of the last observable step (the last
                          step of the latest lbm_step call).
   LBM_FRZ_MDOT_INTEGRAL  the mass-source integral: sum over every step since
                          lbm_init_fields (or lbm_set_state) and every site of
                          mdot (Eq. 19), accumulated in FP64 on the device as
                          the steps run (each step's per-tile or per-strip sum
                          is FP32).
   LBM_FRZ_FREEZE_STEP    the first observable step at which the solidified
                          fraction X = sum f_s / sum phi reached
                          LBM_FREEZE_FRACTION (the freezing time of Sections
                          4.2-4.3, observed at the observable steps only, so
                          its resolution is the caller's lbm_step length);
                          -1 while not reached.
   LBM_FRZ_SOLID_FRACTION X at the last observable step. */
#define LBM_FRZ_STEP            0
#define LBM_FRZ_MDOT_INTEGRAL   1
#define LBM_FRZ_FREEZE_STEP     2
#define LBM_FRZ_SOLID_FRACTION  3
#define LBM_FRZ_COUNT           4
#define LBM_FREEZE_FRACTION     0.99

typedef struct lbm_handle lbm_handle;

/* Device workspace (bytes) that lbm_create needs for n_inst lattices with
   parameters p[0..n_inst-1] in the given storage format. Returns LBM_EINVAL
   for bad arguments. Host only; touches no device. */
int lbm_workspace_size(const lbm_params* p, int32_t n_inst, int32_t storage,
                       uint64_t* bytes);

/* Create a handle over n_inst independent lattices (the paper's problem
   statement per lattice, Section 4). d_workspace is caller-owned device
   memory of at least lbm_workspace_size bytes, 256-byte aligned; the library
   carves every device buffer from it and never allocates device memory (the
   handle's pinned observable mirror is host memory). cuda_stream is a
   cudaStream_t (NULL for the legacy default stream). Uploads the tile and
   instance tables (host-to-device copies on the stream). On success *out
   holds the handle; the fields still need lbm_init_fields. */
int lbm_create(const lbm_params* p, int32_t n_inst, int32_t storage,
               void* d_workspace, uint64_t workspace_bytes, void* cuda_stream,
               lbm_handle** out);

/* Start instance `inst` at rest (u = 0, p = 0) with every distribution at its
   equilibrium (Eqs. 24, 28, 31) for the host fields phi0 and T0 (nx*ny
   doubles each, read during the call). The material starts liquid-like:
   H = Cp T0 + L (Eq. 8). Runs an initialisation kernel on the stream. */
int lbm_init_fields(lbm_handle* h, int32_t inst, const double* phi0,
                    const double* T0);

/* Advance every instance by n >= 0 time steps (streaming, the three
   collisions of Eqs. 21, 27, 30 and the carried fields). Asynchronous on the
   stream; the last step of the call also reduces the observables. Launch
   errors return LBM_ECUDA; device-side faults surface at the next
   synchronising call. */
int lbm_step(lbm_handle* h, int64_t n);

/* Copy the observables record (LBM_OBS_COUNT doubles) of instance `inst`
   from the last step to out. Synchronises the stream. Returns LBM_EUNSTABLE
   (with the record filled) when any field was non-finite or the largest
   speed exceeded 0.5 lattice units (the scheme's low-Mach expansion of
   Eqs. 24, 28 and 31 has long broken down there). */
int lbm_observables(lbm_handle* h, int32_t inst, double* out);

/* Freezing record (LBM_FRZ_COUNT doubles, indices LBM_FRZ_*) of instance
   `inst` as of the last observable step. Synchronises the stream.
   LBM_ESTATE before the first lbm_step of a run. */
int lbm_freezing(lbm_handle* h, int32_t inst, double* out);

/* Solid height profile of instance `inst` at the last observable step:
   out[x] = sum over y of f_s at column x (nx doubles), the frozen shape of
   Section 4.2 seen from the cold wall below (with a wall in y). Each
   column's sum is FP32 over the rows of one tile or strip item, those sums
   added in FP64. Synchronises the stream. LBM_ESTATE before the first
   lbm_step of a run. */
int lbm_solid_profile(lbm_handle* h, int32_t inst, double* out);

/* Observables of every instance: out holds n_inst * LBM_OBS_COUNT doubles.
   Synchronises the stream. LBM_EUNSTABLE (records filled) as
   lbm_observables, for any instance. */
int lbm_observables_all(lbm_handle* h, double* out);

/* Read back instance `inst`: pops (27*nx*ny doubles) and aux (5*nx*ny
   doubles), either may be NULL. Values are the stored post-collision
   distributions converted to double. Synchronises the stream. Used for
   parity checks and checkpoints. */
int lbm_get_state(lbm_handle* h, int32_t inst, double* pops, double* aux);

/* Overwrite instance `inst` with host pops/aux (layouts as lbm_get_state;
   both required). A lbm_get_state / lbm_set_state round trip of FP32 storage
   restores every stored value exactly, except that h_0 (kept on the device
   shifted by -L f_l) can move by one float ulp where its shifted value is
   below ~1e-8, i.e. by at most ~2e-15. */
int lbm_set_state(lbm_handle* h, int32_t inst, const double* pops,
                  const double* aux);

/* Kernel layouts for lbm_step. All of them evaluate the same expressions in
   the same order, but the compiler contracts multiply-adds differently in
   each kernel, so their results agree to FP32 rounding (about 1e-6 after 60
   steps), not bit for bit.
   LBM_KERNEL_TILE:  one CTA per tile of a x b sites with a shared-memory
                     halo; handles every wall combination. (a, b) in
                     {(32,8), (32,4), (64,4), (32,16)}; c ignored.
   LBM_KERNEL_STRIP: one warp per strip of 30 columns x b rows (b >= 2) that
                     keeps its halo in registers and warp shuffles; needs every
                     lattice of the handle periodic in x. a = warps per CTA,
                     c = register budget per thread: (a, c) in {(4,128),
                     (4,168), (4,255), (8,128), (2,128)}.
   LBM_KERNEL_STAGED: the strip layout with every row a lane consumes
                     copied ahead (cp.async) into a per-warp ring of
                     shared-memory slots, so that several rows of loads are
                     in flight while a row is computed. FP32 and FP16
                     storage; the same (a, c) pairs as STRIP.
   For both strip layouts b = 0 picks the rows per strip that let one wave
   of resident warps take every strip of every lattice; lbm_get_kernel
   reports the rows in effect.
   LBM_KERNEL_BLOCK: one warp per 32-site column of the layout's row blocks
                     (b rows each): every row it needs arrives as four bulk
                     copies (cp.async.bulk on an mbarrier) of contiguous
                     chunks of the rows y - 1, y, y + 1, the two columns on
                     either side as small copies; offsets inside a staged
                     row are compile-time constants. All storage formats;
                     needs every lattice periodic in x. (a, c) in {(4,128),
                     (4,168), (8,128)}.
   For the strip and block layouts b = 0 picks the rows per item that let
   one wave of resident warps take every item of every lattice.
   lbm_create picks STAGED (4, 0, 168) when every lattice is periodic in x,
   else TILE (32, 8). */
#define LBM_KERNEL_TILE   0
#define LBM_KERNEL_STRIP  1
#define LBM_KERNEL_STAGED 2
#define LBM_KERNEL_BLOCK  3

/* Thermal type of the walls of lattice `inst` from now on (1 = held at T_w,
   0 = adiabatic; flags as in lbm_params). The paper relaxes a drop to its
   contact angle without cooling and then cools the substrate (Sections 4.2,
   4.3): step with the walls adiabatic, switch them here, keep stepping; the
   state, the latent heat (set by T_w and Ste) and every other parameter are
   untouched. Periodic directions have no walls (their flags must be 0).
   Synchronises the stream; drops captured graphs. LBM_EINVAL otherwise. */
int lbm_set_thermal_walls(lbm_handle* h, int32_t inst, int32_t x_lo, int32_t x_hi,
                          int32_t y_lo, int32_t y_hi);

/* Select the kernel layout (host tables are rebuilt and uploaded on the
   stream; synchronises it). LBM_EINVAL for an unsupported combination. */
int lbm_set_kernel(lbm_handle* h, int32_t kind, int32_t a, int32_t b, int32_t c);

/* Current layout: out[0] = kind, out[1..3] = a, b, c as for lbm_set_kernel. */
int lbm_get_kernel(const lbm_handle* h, int32_t* out);

/* Autotuner: time every supported layout for this handle twice over `steps`
   time steps each (after one warm-up step), measured with CUDA events on the
   stream, and keep the one with the shortest time. The lattices are advanced by every step it
   runs (lbm_step_count grows accordingly); the layouts compute the same
   update and agree to FP32 rounding, so the trajectory is the one lbm_step
   would have produced up to that rounding.
   times_ms (may be NULL) receives up to `cap` mean step times in the order
   the candidates were tried; *n_tried their number. Synchronises. */
int lbm_autotune(lbm_handle* h, int32_t steps, double* times_ms, int32_t cap, int32_t* n_tried);

/* Execution form of lbm_step (no counterpart in the paper, which specifies
   the update of Section 3, not how it is scheduled). Every form runs the
   same step arithmetic; the last step of each lbm_step call is always one
   ordinary launch that also writes the observable partials.
   LBM_EXEC_LAUNCH:     one kernel launch per step (the default).
   LBM_EXEC_GRAPH:      runs of `chunk` steps replay a CUDA graph of `chunk`
                        step launches, captured on first use (one graph per
                        starting buffer) on a private stream and launched on
                        the handle's stream.
   LBM_EXEC_PERSISTENT: runs of `chunk` steps replay a CUDA graph holding one
                        cooperative persistent launch: a co-resident grid
                        (lbm_get_exec out[2] CTAs) walks every strip item of
                        every lattice, with a device-wide barrier between
                        steps. Strip layout only. A barrier wait is bounded
                        (2 s); one that runs out makes the kernel return and
                        the next synchronising call (lbm_observables*) return
                        LBM_ETIMEOUT, after which lbm_step refuses with
                        LBM_ETIMEOUT until lbm_init_fields gives a new state.
   Step results of LAUNCH and GRAPH are bitwise identical; PERSISTENT agrees
   with them to FP32 rounding (a separately compiled kernel). */
#define LBM_EXEC_LAUNCH      0
#define LBM_EXEC_GRAPH       1
#define LBM_EXEC_PERSISTENT  2

/* Select the execution form; chunk in [1, 65536] steps. Captured graphs are
   dropped (also by lbm_set_kernel, whose tables they use). LBM_EINVAL for an
   unknown mode or chunk, or PERSISTENT with the tile layout (and
   lbm_set_kernel refuses the tile layout while PERSISTENT is selected). */
int lbm_set_exec(lbm_handle* h, int32_t mode, int32_t chunk);

/* out[0] = mode, out[1] = chunk, out[2] = CTAs of one persistent launch for
   the current layout (0 for the tile layout). */
int lbm_get_exec(const lbm_handle* h, int32_t* out);

/* Self-test of the bounded device-wide barrier: one CTA waits at a barrier
   that no other CTA joins, gives up after limit_ns (0 < limit_ns <= 2e9),
   raises its error word and returns. *err_flag receives that word (1 when
   the expiry was reported). The handle's own state is untouched.
   Synchronises. */
int lbm_barrier_selftest(lbm_handle* h, uint64_t limit_ns, int32_t* err_flag);

/* Number of time steps taken since the last lbm_init_fields of instance 0. */
int64_t lbm_step_count(const lbm_handle* h);

/* Number of kernel launches the library queued since the handle was created
   (every kernel, including initialisation and reductions). */
int64_t lbm_launch_count(const lbm_handle* h);

/* ---------------------------------------------------------------------------
   Allocation-free single step (the paper has no counterpart; this entry point
   exists for callers of the library, not for the method).

   Some callers cannot allocate device memory at all: code that runs while a
   CUDA graph is being captured, plugins inside a host application that owns
   every device allocation, or real-time loops that must never stall in the
   allocator. lbm_create needs a caller-owned workspace for its tables and
   scratch; this entry point needs none. It advances one lattice by one time
   step from the caller's state buffers (in) to the caller's state buffers
   (out) and writes the observables record of that step, and it calls no
   cudaMalloc, cudaFree or other allocating routine.

   Buffers (device, caller-owned, FP32, 16-byte aligned), in the library's
   blocked state layout: sites are numbered site = y * pitch + x with pitch a
   multiple of 32 and >= nx, i.e. site = 32 blk + l (blk = site / 32 the row
   block, l = x % 32), plane = pitch * ny. pops_in/pops_out hold 24 * plane
   floats, 768 per block in three chunks by the y component of the
   direction: P (directions 2, 5, 6) at 0, Z (1, 3) at 288, M (4, 7, 8) at
   480; inside a chunk of n directions the k-th (in that order) keeps its
   pairs (g_i, h_i) at 64 k + 2 l and f_i at 64 n + 32 k + l, all offsets
   from 768 blk;
   aux_in/aux_out hold 10 * plane floats, 320 per block: the group
   (g_0, h_0 - L f_l, f_0, f_l) at 320 blk + 4 l and ((phi u)_x, (phi u)_y,
   p, S) at 320 blk + 128 + 4 l (the last 64 floats of a block are not used;
   L = Cp (T_m - T_w) / Ste). This is exactly the layout of a handle's FP32
   state buffers. An output buffer may share no byte with any of the other
   three (LBM_EINVAL otherwise). d_obs receives LBM_OBS_COUNT doubles
   (device memory).

   Scratch: the per-tile partial sums of the observables live in one array of
   LBM_NOALLOC_MAX_TILES * LBM_OBS_COUNT doubles (720 KiB) that is part of the
   library's device image: every GPU that loads the library holds it until the
   process exits. A lattice may have at most LBM_NOALLOC_MAX_TILES tiles of
   32 x 8 sites, i.e. ceil(nx/32) * ceil(ny/8) <= 8192 (for example 1024 x 2048);
   larger lattices get LBM_ETOOLARGE. Every slot the reduction reads is
   written earlier in the same call, so nothing needs clearing, but all calls
   share the array: calls that overlap on the GPU (for example on two streams
   at once) race on it and their observables are undefined.

   Device: the current device of the calling thread. On the first call for a
   device the library looks up the array's device address (no allocation)
   and caches it for the life of the process; make that first call before
   any stream capture begins. The cached address does not survive the
   destruction of the device's context (cudaDeviceReset, or a primary
   context released and retained again): do not call this entry point after
   that. Works for every wall combination (tile kernel). Returns LBM_EINVAL
   for bad parameters, pointers, pitch or overlapping buffers, LBM_ECUDA for
   launch errors. */
#define LBM_NOALLOC_MAX_TILES 8192
int lbm_step_noalloc(const lbm_params* p, const float* pops_in, const float* aux_in,
                     float* pops_out, float* aux_out, int32_t pitch, double* d_obs,
                     void* cuda_stream);

/* Release the handle (host memory only; the workspace stays the caller's).
   Waits for queued work on the stream first. NULL is accepted. */
void lbm_destroy(lbm_handle* h);

/* Static description of a return code. */
const char* lbm_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
