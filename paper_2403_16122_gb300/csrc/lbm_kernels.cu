// lbm_kernels.cu -- sm_103a kernels of the freezing LB time step
// (arXiv 2403.16122, Section 3): one fused pull-stream + collide kernel over
// the three D2Q9 populations, the equilibrium initialisation, and the FP64
// observable reduction.
//
// Fused step, per CTA tile of TX x TY sites (one thread per site):
//   phase A  every thread pulls g, h, f of its own site (Section 3, streaming
//            with half-way bounce-back / anti-bounce-back at walls) and forms
//            H, f_s (Eqs. 8-9), mdot (Eq. 19), phi (Eq. 26) and rho (Eq. 1);
//            phi and rho go to shared memory.
//   phase B  the one-cell ring around the tile (and, next to a wall, the two
//            extra cells per wall row that the wetting ghost needs) is pulled
//            the same way by the first threads; the lagged p and S of the ring
//            are staged too.
//   phase C  ring cells behind a wall get their ghost values: the wetting
//            condition for phi (Eqs. 39-41), a copy of the adjacent lattice
//            value for rho, p and S.
//   phase D  every thread evaluates the isotropic stencils (Eq. 38) from shared
//            memory, the chemical potential and forces (Eqs. 11-12), the flow
//            macroscopics (Eqs. 33-36), the three BGK collisions with their
//            source terms (Eqs. 21, 25, 27, 30) and stores the post-collision
//            populations and carried fields to the other buffer.
// Time levels match the CPU reference: grad p and grad S use the previous
// step's p and S; d_t(phi u) is a backward difference (Eq. 37).
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"
#include "lbm_math.cuh"

// The build compiles this file once per part, each compilation whole (nvcc's
// own partitioning of a file for parallel compilation makes the code of a
// kernel depend on the rest of the file and on the run), and links the parts:
//   0  storage dispatch; tile, initialisation and reduction kernels
//   1  FP32 row-staged strips (plain, observable and persistent steps)
//   2  FP32 strips that load in place
//   3  FP16 row-staged strips
//   4  FP16 strips that load in place
//   5  BF16 row-staged strips
// Without LBM_PART the one compilation holds every part.
#ifndef LBM_PART
#define LBM_PART -1
#endif
#define LBM_HAS_PART(k) (LBM_PART < 0 || LBM_PART == (k))

namespace lbmk {
namespace {

// D2Q9 weights (Eq. 22) in single precision, chosen so that the float values
// sum to exactly 1: w0 and w1 are the nearest floats to 4/9 and 1/9, w2 is one
// ulp below the nearest float to 1/36 (relative error 6e-8). With the nearest
// floats the weights sum to 1 + 7.45e-9, and every BGK collision then creates
// omega * 7.45e-9 * phi of order parameter (and likewise enthalpy) per site
// and step, a drift that grows linearly with time.
constexpr float kW0 = 0x1.c71c72p-2f, kW1 = 0x1.c71c72p-4f, kW2 = 0x1.c71c70p-6f;
static_assert((double)kW0 + 4.0 * (double)kW1 + 4.0 * (double)kW2 == 1.0,
              "D2Q9 float weights must sum to one exactly");
__host__ __device__ constexpr int CX(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int CY(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int OPP(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
__host__ __device__ constexpr float WGT(int i) { return i == 0 ? kW0 : (i <= 4 ? kW1 : kW2); }
// c_i . (a, b) with the components of c_i (0, +1, -1) applied as selects, so
// that an unrolled loop folds them: no multiplication by zero is issued
// (IEEE arithmetic cannot drop 0 * x) and a diagonal costs one addition.
__host__ __device__ __forceinline__ float cdot(int i, float a, float b) {
    const int cx = CX(i), cy = CY(i);
    if (cx == 0 && cy == 0) return 0.f;
    if (cx == 0) return cy > 0 ? b : -b;
    if (cy == 0) return cx > 0 ? a : -a;
    return (cx > 0 ? a : -a) + (cy > 0 ? b : -b);
}

static_assert(OPP(1) == 3 && OPP(2) == 4 && OPP(3) == 1 && OPP(4) == 2, "opp axis");
static_assert(OPP(5) == 7 && OPP(6) == 8 && OPP(7) == 5 && OPP(8) == 6, "opp diag");

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

// Mixing rule, Eq. 1, with phi clamped to [0, 1].
__device__ __forceinline__ float mix3(float fs, float phi, float zs, float zl, float zg) {
    float ph = clamp01(phi);
    float liq = 1.0f - fs;
    return fs * zs + liq * (ph * zl + (1.0f - ph) * zg);
}

// ---------------------------------------------------------------------------
// Storage access (FP32)
// ---------------------------------------------------------------------------
// NC selects the load path: true for kernels that run one step per launch
// (the read-only, non-coherent path), false for the persistent kernel, where
// a buffer read in one step was written by other CTAs in the previous step of
// the same launch, so its loads bypass L1 and are served by the coherent L2.
template <bool NC>
struct LatT {
    const float* __restrict__ A;  // source populations (27 planes)
    const float* __restrict__ Aaux;
    int plane;                    // elements per plane (27 planes fit 32-bit offsets)
    int nx, ny, pitch, flags;
};
using Lat = LatT<true>;

template <bool NC>
__device__ __forceinline__ float ld_f32(const float* p) {
    if constexpr (NC) return __ldg(p); else return __ldcg(p);
}
template <bool NC>
__device__ __forceinline__ unsigned short ld_u16(const unsigned short* p) {
    if constexpr (NC) return __ldg(p); else return __ldcg(p);
}

// FP16 storage: population i of a set is stored as a 16-bit deviation from a
// rest-equilibrium reference. For g and h the reference is taken at the site
// the population is pulled into (the destination of its streaming link, or
// the site itself for links that bounce at a wall): w_i phi for g, w_i Cp_ref
// T for h_1..8 and the rest equilibrium of h_0 (kept in the shifted form of
// the FP32 layout); the destination decodes with its own phi_ref and T_ref,
// two FP32 planes written by the previous step. For f the reference is the
// rest equilibrium at the pressure of the source site, p w_i / c_s^2
// (p (w_0 - 1) / c_s^2 for i = 0), and the deviation is scaled by 2^12; the
// destination reads the source pressures from the carried p plane it loads
// for the pressure gradient anyway. The rest populations g_0, h_0 (shifted)
// and f_0 stay in FP32 (own-site region) and absorb the rounding
// errors of the site's eight 16-bit outgoing populations, so the zeroth
// moment a site sends out (phi, H, and the f sum) is exact: rounding only
// displaces a little of it along one link, which cancels between
// neighbouring sites in smooth fields instead of accumulating.
constexpr float kFScale = 4096.f, kInvFScale = 1.f / 4096.f;
struct Ref {
    float phi, T;
};

// Stored population (set, i) of site idx (grouped layout, see Inst); the rest
// populations are FP32 in the own-site region for both storages.
template <typename ST, bool NC>
__device__ __forceinline__ float ldPop(const LatT<NC>& l, int set, int i, int idx) {
    if (i == 0) return ld_f32<NC>(l.Aaux + own0_at(idx, set));
    if constexpr (sizeof(ST) == 4) {
        return ld_f32<NC>(l.A + pop_at(set, i, idx));
    } else {
        const unsigned short* A = reinterpret_cast<const unsigned short*>(l.A);
        return Bits16<ST>::to_f(Bits16<ST>::from_bits(ld_u16<NC>(A + pop_at(set, i, idx))));
    }
}

// Stored value -> population (h_0 in the shifted form) for site reference r.
template <typename ST, int SET>
__device__ __forceinline__ float decode(int i, float raw, const Ref& r, float Cpref) {
    if constexpr (sizeof(ST) == 4) {
        return raw;
    } else {
        if (i == 0) return raw;  // rest populations are stored in FP32
        if (SET == 0) return raw + WGT(i) * r.phi;
        if (SET == 1) return raw + WGT(i) * Cpref * r.T;
        return raw * kInvFScale;  // the caller adds the source-pressure reference
    }
}

// Rest equilibrium of f at pressure p (Eq. 31 with u = 0).
__device__ __forceinline__ float f_rest(int i, float p) {
    return (i == 0 ? (kW0 - 1.f) : WGT(i)) * 3.f * p;
}
template <bool NC>
__device__ __forceinline__ float ldAux(const LatT<NC>& l, int k, int idx) {
    return ld_f32<NC>(l.Aaux + aux_at(k, idx));
}

// Pull of set `set` (0 g, 1 h, 2 f) at lattice site (x, y): v[i] is the
// population arriving along c_i. Sources behind a wall are replaced by the
// half-way bounce-back of the site's own opposite population; for h at a
// Dirichlet wall by anti-bounce-back -h + 2 w_i Cp_ref T_w (Section 4.1).
// h_0 is returned as stored (shifted, see Inst).
template <int SET, typename ST = float, bool NC>
__device__ __forceinline__ void pull_set(const LatT<NC>& l, int x, int y, float abb, float v[9],
                                         const Ref& ref = Ref{0.f, 0.f}, float Cpref = 0.f,
                                         const float* pref = nullptr) {
    constexpr bool kFref = sizeof(ST) != 4 && SET == 2;  // f: source-pressure reference
    const int own = y * l.pitch + x;
    v[0] = decode<ST, SET>(0, ldPop<ST>(l, SET, 0, own), ref, Cpref);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int xs = x - CX(i), ys = y - CY(i);
        bool wall = false, dir = false;
        if (xs < 0) {
            if (l.flags & kPeriodicX) xs += l.nx;
            else { wall = true; dir |= (l.flags & kDirXlo) != 0; }
        } else if (xs >= l.nx) {
            if (l.flags & kPeriodicX) xs -= l.nx;
            else { wall = true; dir |= (l.flags & kDirXhi) != 0; }
        }
        if (ys < 0) {
            if (l.flags & kPeriodicY) ys += l.ny;
            else { wall = true; dir |= (l.flags & kDirYlo) != 0; }
        } else if (ys >= l.ny) {
            if (l.flags & kPeriodicY) ys -= l.ny;
            else { wall = true; dir |= (l.flags & kDirYhi) != 0; }
        }
        if (!wall) {
            v[i] = decode<ST, SET>(i, ldPop<ST>(l, SET, i, ys * l.pitch + xs), ref, Cpref);
            if constexpr (kFref) v[i] += f_rest(i, pref[i]);
        } else {
            float b = decode<ST, SET>(OPP(i), ldPop<ST>(l, SET, OPP(i), own), ref, Cpref);
            if constexpr (kFref) b += f_rest(OPP(i), pref[0]);  // bounced: the site itself
            if (SET == 1 && dir) b = -b + 2.0f * WGT(i) * abb;
            v[i] = b;
        }
    }
}

struct Phys {
    float L, Hs, Tm, Cp, Cpref, Tw, omega_g, omega_h, kappa, beta, lam_coef;
    float rho_s, rho_l, rho_g, mu_s, mu_l, mu_g, mdot_coef, tan_w, inv_ramp, eps2;
    float inv_L, inv_Cp;
    float buoy_x, buoy_y, T_ref;
    float Cp_s, Cp_g, k_s, k_g, dtau_h;
    bool phase_props;
};

__device__ __forceinline__ Phys load_phys(const Inst& I) {
    Phys P;
    P.L = I.L; P.Hs = I.Hs; P.Tm = I.Tm; P.Cp = I.Cp; P.Cpref = I.Cpref; P.Tw = I.Tw;
    P.omega_g = I.omega_g; P.omega_h = I.omega_h; P.kappa = I.kappa; P.beta = I.beta;
    P.lam_coef = I.lam_coef; P.rho_s = I.rho_s; P.rho_l = I.rho_l; P.rho_g = I.rho_g;
    P.mu_s = I.mu_s; P.mu_l = I.mu_l; P.mu_g = I.mu_g; P.mdot_coef = I.mdot_coef;
    P.tan_w = I.tan_w; P.inv_ramp = I.inv_ramp; P.eps2 = I.normal_eps2;
    P.inv_L = I.inv_L; P.inv_Cp = I.inv_Cp;
    P.buoy_x = I.buoy_x; P.buoy_y = I.buoy_y; P.T_ref = I.T_ref;
    P.Cp_s = I.Cp_s; P.Cp_g = I.Cp_g; P.k_s = I.k_s; P.k_g = I.k_g; P.dtau_h = I.dtau_h;
    P.phase_props = (I.flags & kPhaseProps) != 0;
    return P;
}

// Local macroscopic values at a site from its pulled g and h (phase A/B).
// H' = H - L f_l^{n-1} is what the stored h_0 sums to (see Inst).
struct Macro {
    float Hp;    // shifted total enthalpy H'
    float fl, flp, fs, mdot, phi, rho;
    float T;     // Eq. 9b; inside the mushy range exactly T_m
    bool mushy;  // H strictly between H_s and H_l
};

__device__ __forceinline__ Macro local_macro(const Phys& P, const float g[9], const float h[9],
                                             float flp) {
    Macro m;
    float phihat = 0.0f, Hp = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) { phihat += g[i]; Hp += h[i]; }
    // Eq. 9a on the shifted enthalpy: (H - H_s)/L = (H' - H_s)/L + f_l^{n-1}
    const float q = (Hp - P.Hs) * P.inv_L + flp;
    const float fl = clamp01(q);
    m.mushy = q > 0.0f && q < 1.0f;
    // solid only in the liquid content of the site
    const float chi = clamp01((phihat - 0.5f) * P.inv_ramp + 0.5f);
    const float fs = chi * (1.0f - fl);
    const float mdot = P.mdot_coef * chi * (flp - fl);   // Eq. 19, phase change only
    const float phi = div_normal(phihat, 1.0f - 0.5f * mdot);    // Eq. 26
    m.Hp = Hp; m.fl = fl; m.flp = flp; m.fs = fs; m.mdot = mdot; m.phi = phi;
    m.rho = mix3(fs, phi, P.rho_s, P.rho_l, P.rho_g);   // Eq. 1
    // Eq. 9b on the shifted enthalpy, H - H_s - L f_l = H' - H_s + L (f_l^{n-1}
    // - f_l); inside the mushy range the exact value is T_m (evaluating the sum
    // there would only add the rounding of f_l times L)
    if (P.phase_props) {  // sensible branches with the local C_p of Eq. 1
        const float cp = mix3(fs, phi, P.Cp_s, P.Cp, P.Cp_g);
        m.T = m.mushy ? P.Tm : P.Tm + (Hp - P.Hs + P.L * (flp - fl)) / cp;
    } else {
        m.T = m.mushy ? P.Tm : P.Tm + (Hp - P.Hs + P.L * (flp - fl)) * P.inv_Cp;
    }
    return m;
}

// ---------------------------------------------------------------------------
// Block reduction of the observables (FP64)
// ---------------------------------------------------------------------------
// out: this tile's slot in observable-major partials (observable j at
// out[j * stride]).
template <int NT>
__device__ void block_reduce_obs(double v[kObs], double* __restrict__ out, int stride) {
    __shared__ double red[NT / 32][kObs];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kObs; ++j) {
        double x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (j == 9) ? fmax(x, y) : x + y;
        }
        v[j] = x;
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kObs; ++j) red[warp][j] = v[j];
    }
    __syncthreads();
    if (threadIdx.x < kObs) {
        const int j = threadIdx.x;
        double acc = red[0][j];
        for (int w = 1; w < NT / 32; ++w) acc = (j == 9) ? fmax(acc, red[w][j]) : acc + red[w][j];
        out[(long long)j * stride] = acc;
    }
}

// ---------------------------------------------------------------------------
// Per-site update shared by the tile and strip kernels
// ---------------------------------------------------------------------------
// Isotropic stencils of Eq. 38 at one site: gradients of phi, rho, p^{n-1},
// S^{n-1} and the Laplacian of phi.
struct Stencil {
    float gphx, gphy, lph, grx, gry, gpx, gpy, gSx, gSy;
};

// Eq. 38 written with per-column combinations of rows y-1 (m), y (c) and
// y+1 (p): with A = w1 c + w2 (p + m) and D = p - m of the columns x-1 (L),
// x (C) and x+1 (R),
//   grad_x = 3 (A_R - A_L),  grad_y = 3 (w1 D_C + w2 (D_R + D_L)),
//   lap    = 6 (w1 ((c_R + c_L) + (p_C + m_C) - 4 c_C)
//               + w2 ((p_R + m_R) + (p_L + m_L) - 4 c_C)).
// Pairwise sums keep a uniform field exactly stencil-free in FP32. Both kernel
// layouts evaluate exactly these expressions.
struct ColSums {
    float A, D;
};
__device__ __forceinline__ ColSums col_sums(float m, float c, float p) {
    ColSums r;
    r.A = kW1 * c + kW2 * (p + m);
    r.D = p - m;
    return r;
}
__device__ __forceinline__ void grad_cols(const ColSums& L, const ColSums& C, const ColSums& R,
                                          float& gx, float& gy) {
    gx = 3.f * (R.A - L.A);
    gy = 3.f * (kW1 * C.D + kW2 * (R.D + L.D));
}
// The same for two fields at once (paired FP32 operations, each component
// evaluated exactly as above); S2 = p + m is returned for the Laplacian.
struct ColSums2 {
    float2 A, D, S2;
};
__device__ __forceinline__ ColSums2 col_sums2(float2 m, float2 c, float2 p) {
    ColSums2 r;
    r.S2 = __fadd2_rn(p, m);
    r.A = __ffma2_rn(make_float2(kW1, kW1), c, __fmul2_rn(make_float2(kW2, kW2), r.S2));
    r.D = __fadd2_rn(p, make_float2(-m.x, -m.y));
    return r;
}
__device__ __forceinline__ void grad_cols2(const ColSums2& L, const ColSums2& C, const ColSums2& R,
                                           float2& gx, float2& gy) {
    const float2 k3 = make_float2(3.f, 3.f);
    gx = __fmul2_rn(k3, __fadd2_rn(R.A, make_float2(-L.A.x, -L.A.y)));
    gy = __fmul2_rn(k3, __ffma2_rn(make_float2(kW1, kW1), C.D,
                                   __fmul2_rn(make_float2(kW2, kW2), __fadd2_rn(R.D, L.D))));
}
// cL, cR: row-y values of the side columns; sL, sC, sR: p + m of each column
__device__ __forceinline__ float lap_cols(float cL, float cC, float cR, float sL, float sC,
                                          float sR) {
    const float t1 = (cR + cL) + sC - 4.f * cC;
    const float t2 = (sR + sL) - 4.f * cC;
    return 6.f * (kW1 * t1 + kW2 * t2);
}

// Pulled populations of one site as site_update reads them: from arrays, or
// (row-staged FP32 strips) straight from the lane's ring slot at each use, so
// that they need not stay live in registers across the collision. The slot
// form applies the anti-bounce-back of h on the links in hmask.
struct ArrPops {
    const float *g, *h, *f;
    __device__ __forceinline__ float G(int i) const { return g[i]; }
    __device__ __forceinline__ float H(int i) const { return h[i]; }
    __device__ __forceinline__ float F(int i) const { return f[i]; }
};
struct SlotPops {
    const float* s;  // the slot (layout: see the row staging below)
    int lane;
    int hmask;       // bit i: h_i arrives through a Dirichlet wall
    float abb;       // Cp_ref T_w
    __device__ __forceinline__ float rd(int off) const {
        return *reinterpret_cast<const volatile float*>(s + off);
    }
    __device__ __forceinline__ float G(int i) const {
        return rd(i == 0 ? 4 * lane : 256 + 64 * (i - 1) + 2 * lane);
    }
    __device__ __forceinline__ float H(int i) const {
        const float v = rd(i == 0 ? 4 * lane + 1 : 256 + 64 * (i - 1) + 2 * lane + 1);
        return ((hmask >> i) & 1) ? -v + 2.0f * WGT(i) * abb : v;
    }
    __device__ __forceinline__ float F(int i) const {
        return rd(i == 0 ? 4 * lane + 2 : 768 + 32 * (i - 1) + lane);
    }
};

// Row-staged 16-bit strips: g and h decoded in the slot, f decoded into
// registers just before the collision.
struct SlotGHPops {
    const float* s;
    int lane;
    const float* f;
    __device__ __forceinline__ float rd(int off) const {
        return *reinterpret_cast<const volatile float*>(s + off);
    }
    __device__ __forceinline__ float G(int i) const {
        return rd(i == 0 ? 4 * lane : 256 + 64 * (i - 1) + 2 * lane);
    }
    __device__ __forceinline__ float H(int i) const {
        return rd(i == 0 ? 4 * lane + 1 : 256 + 64 * (i - 1) + 2 * lane + 1);
    }
    __device__ __forceinline__ float F(int i) const { return f[i]; }
};

// Per-thread observable sums of the sites it updates. The sums run in FP32
// with Neumaier's compensation (the running sum and the rounding error each
// addition dropped), and (s + c) is taken in FP64 before the warp, block and
// item reductions, which are FP64: the result matches an FP64 running sum of
// the same FP32 per-site values to well below their own rounding, without
// FP64 arithmetic per site (the FP64 rate of the GPU is a small fraction of
// its FP32 rate). Slot 9 is a maximum, not a sum.
struct ObsAcc {
    float s[kObs], c[kObs];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int j = 0; j < kObs; ++j) { s[j] = 0.f; c[j] = 0.f; }
    }
    __device__ __forceinline__ void add(int j, float x) {
        const float t = s[j] + x;
        c[j] += fabsf(s[j]) >= fabsf(x) ? (s[j] - t) + x : (x - t) + s[j];
        s[j] = t;
    }
    __device__ __forceinline__ void max(int j, float x) { s[j] = fmaxf(s[j], x); }
    __device__ __forceinline__ double total(int j) const { return (double)s[j] + (double)c[j]; }
};

// Observable sums of a warp strip, taken row by row: at the end of each row
// the values of its sites (at most 30) are summed across the warp in FP32,
// and one lane carries each observable's running sum over the rows with
// Neumaier's compensation, so a lane keeps two running values instead of
// 2 kObs (the row values are dead between rows). Slots 0-6 go through one
// reduce-scatter: at each of lane bits 4, 3 and 2 a lane keeps half of its
// vector and adds the partner's copy of that half, then two xor steps finish
// the sums, and lane L holds the warp total of slot (L >> 2) & 7 (7 is
// padding). Slot 9 (a maximum) takes its own xor tree; slots 7, 8 and 10 are
// zero on all but a few rows, and their tree runs only when a lane holds a
// nonzero value (skipping it adds nothing). Lanes that update no site
// contribute zeros. The order of every sum is fixed by the lane indices.
struct RowObs {
    static_assert(kObs == 11, "slot assignment below");
    float v[kObs];
    float s, c;
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int j = 0; j < kObs; ++j) v[j] = 0.f;
        s = 0.f;
        c = 0.f;
    }
    __device__ __forceinline__ void add(int j, float x) { v[j] += x; }
    __device__ __forceinline__ void max(int j, float x) { v[j] = fmaxf(v[j], x); }
    // the observable lane `lane` carries (-1: none)
    static __device__ __forceinline__ int carried(int lane) {
        if ((lane & 3) == 0) return lane < 28 ? lane >> 2 : -1;
        return lane == 1 ? 9 : (lane == 2 ? 7 : (lane == 3 ? 8 : (lane == 5 ? 10 : -1)));
    }
    static __device__ __forceinline__ float warp_sum(float t) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        return t;
    }
    // all 32 lanes, once per row
    __device__ __forceinline__ void flush(int lane) {
        constexpr unsigned kAll = 0xffffffffu;
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        float k4[4], k2[2];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float lo = v[q], hi = q + 4 < 7 ? v[q + 4] : 0.f;
            k4[q] = (b4 ? hi : lo) + __shfl_xor_sync(kAll, b4 ? lo : hi, 16);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
            k2[q] = (b3 ? k4[q + 2] : k4[q]) + __shfl_xor_sync(kAll, b3 ? k4[q] : k4[q + 2], 8);
        float t = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(kAll, b2 ? k2[0] : k2[1], 4);
        t += __shfl_xor_sync(kAll, t, 2);
        t += __shfl_xor_sync(kAll, t, 1);
        float mx = v[9];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kAll, mx, o));
        float x7 = 0.f, x8 = 0.f, x10 = 0.f;
        if (__any_sync(kAll, v[7] != 0.f)) x7 = warp_sum(v[7]);
        if (__any_sync(kAll, v[8] != 0.f)) x8 = warp_sum(v[8]);
        if (__any_sync(kAll, v[10] != 0.f)) x10 = warp_sum(v[10]);
        const float mine = (lane & 3) == 0 ? t
                           : (lane == 1 ? mx : (lane == 2 ? x7 : (lane == 3 ? x8 : (lane == 5 ? x10 : 0.f))));
#pragma unroll
        for (int j = 0; j < kObs; ++j) v[j] = 0.f;
        if (lane == 1) {
            s = fmaxf(s, mine);
        } else {
            const float u = s + mine;
            c += fabsf(s) >= fabsf(mine) ? (s - u) + mine : (mine - u) + s;
            s = u;
        }
    }
    __device__ __forceinline__ double total() const { return (double)s + (double)c; }
};

// Where site_update writes one site's post-collision values: by site index
// through the layout's index functions (every kernel but the block one), or
// at a lane of a row block whose base the caller holds (block kernel: the
// offsets inside the block are compile-time constants).
struct SiteStore {
    void* B;
    float* Baux;
    int own;
    __device__ __forceinline__ void gh32(int i, float g, float h) const {
        *reinterpret_cast<float2*>(static_cast<float*>(B) + gh_at(i, own, 0)) = make_float2(g, h);
    }
    __device__ __forceinline__ void f32(int i, float f) const { static_cast<float*>(B)[f_at(i, own)] = f; }
    __device__ __forceinline__ void gh16(int i, unsigned w) const {
        *reinterpret_cast<unsigned*>(static_cast<unsigned short*>(B) + gh_at(i, own, 0)) = w;
    }
    __device__ __forceinline__ void f16(int i, unsigned short v) const {
        static_cast<unsigned short*>(B)[f_at(i, own)] = v;
    }
    __device__ __forceinline__ void own0(float4 v) const {
        *reinterpret_cast<float4*>(Baux + own0_at(own, 0)) = v;
    }
    __device__ __forceinline__ void own1(float4 v) const {
        *reinterpret_cast<float4*>(Baux + own1_at(own, 0)) = v;
    }
    __device__ __forceinline__ void ref(float2 v) const {
        *reinterpret_cast<float2*>(Baux + ref_at(own, 0)) = v;
    }
};
struct BlockStore {
    void* B;      // population block of the site's row block (elements of the storage type)
    float* Baux;  // own-site block
    int l;        // the site's place in the block
    __device__ __forceinline__ void gh32(int i, float g, float h) const {
        *reinterpret_cast<float2*>(static_cast<float*>(B) + gh_off(i) + 2 * l) = make_float2(g, h);
    }
    __device__ __forceinline__ void f32(int i, float f) const { static_cast<float*>(B)[f_off(i) + l] = f; }
    __device__ __forceinline__ void gh16(int i, unsigned w) const {
        *reinterpret_cast<unsigned*>(static_cast<unsigned short*>(B) + gh_off(i) + 2 * l) = w;
    }
    __device__ __forceinline__ void f16(int i, unsigned short v) const {
        static_cast<unsigned short*>(B)[f_off(i) + l] = v;
    }
    __device__ __forceinline__ void own0(float4 v) const { *reinterpret_cast<float4*>(Baux + 4 * l) = v; }
    __device__ __forceinline__ void own1(float4 v) const {
        *reinterpret_cast<float4*>(Baux + 128 + 4 * l) = v;
    }
    __device__ __forceinline__ void ref(float2 v) const {
        *reinterpret_cast<float2*>(Baux + 256 + 2 * l) = v;
    }
};

// Eq. 38 stencils, forces (Eqs. 11-12), flow macroscopics (Eqs. 33-36), the
// three collisions (Eqs. 21, 25, 27-28, 30-33) and the store of the
// post-collision populations and carried fields of one site. The order of
// every floating-point operation is fixed here; kernels differ only in which
// multiply-adds the compiler contracts.
template <bool OBS, typename ST = float, typename Pops = ArrPops, typename Acc = ObsAcc,
          typename Store = SiteStore>
__device__ __forceinline__ void site_update_to(const Phys& P, int flags, const Macro& m,
                                               const Pops& pop, float phiux_p, float phiuy_p,
                                               const Stencil& st, const Store& out, bool on_col,
                                               bool on_row, Acc& ob, const Ref* dref = nullptr) {
    const float phi = m.phi, rho = m.rho, fs = m.fs, mdot = m.mdot;
    const float gphx = st.gphx, gphy = st.gphy, lph = st.lph, grx = st.grx, gry = st.gry;
    const float gpx = st.gpx, gpy = st.gpy, gSx = st.gSx, gSy = st.gSy;

    // Eqs. 11-12 (phi_l = 1, phi_g = 0)
    const float muphi = 4.f * P.beta * (phi - 1.f) * phi * (phi - 0.5f) - P.kappa * lph;
    float Fx = muphi * gphx, Fy = muphi * gphy;
    if (flags & kStMask) { Fx *= (1.f - fs); Fy *= (1.f - fs); }
    if (flags & kBuoy) {  // Boussinesq buoyancy of Section 4.3 at every site
        Fx += P.buoy_x * (m.T - P.T_ref);
        Fy += P.buoy_y * (m.T - P.T_ref);
    }

    // Eqs. 34-35: u* from the flow moments, solid forcing f = -f_s u*
    float mx = 0.f, my = 0.f, fne0 = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float fi = pop.F(i);
        if (CX(i) > 0) mx += fi; else if (CX(i) < 0) mx -= fi;
        if (CY(i) > 0) my += fi; else if (CY(i) < 0) my -= fi;
        if (i) fne0 += fi;
    }
    const float inv_rho = div_normal(1.f, rho);
    const float usx = (mx + 0.5f * Fx) * inv_rho, usy = (my + 0.5f * Fy) * inv_rho;
    const float ffx = -fs * usx, ffy = -fs * usy;
    const float ux = usx + 0.5f * ffx, uy = usy + 0.5f * ffy;
    const float uu = ux * ux + uy * uy;

    // Eq. 33 source terms (grad p, grad S lagged one step)
    const float S = rho * mdot + ux * grx + uy * gry;
    const float Ftx = Fx - gpx + (grx + gSx) * (1.f / 3.f);
    const float Fty = Fy - gpy + (gry + gSy) * (1.f / 3.f);
    const float uFt = ux * Ftx + uy * Fty;
    const float mu = mix3(fs, phi, P.mu_s, P.mu_l, P.mu_g);
    const float tau_f = 3.f * mu * inv_rho + 0.5f;
    const float omega_f = div_normal(1.f, tau_f);
    const float Fpx = Fx + rho * ffx, Fpy = Fy + rho * ffy;  // F + rho f
    const float F0 = kW0 * (S - 3.f * uFt);
    // Eq. 36 with s_0(u) = -w_0 u.u / (2 c_s^2); the F_0 correction is the
    // first-order non-equilibrium part of f_0 that Eq. 30 implies,
    // (tau_f - 1/2) F_0
    const float pn = (1.f / 3.f) / (1.f - kW0) *
                     (fne0 + 0.5f * S + (tau_f - 0.5f) * F0 + rho * (-kW0 * 1.5f * uu));

    // Phase field: n, lambda (Eq. 3), d_t(phi u) (Eq. 37), G_i (Eq. 25)
    // regularised normal n = grad phi / sqrt(|grad phi|^2 + eps^2)
    const float rn = rsqrtf(gphx * gphx + gphy * gphy + P.eps2);
    const float nx_ = gphx * rn, ny_ = gphy * rn;
    const float lam = P.lam_coef * phi * (1.f - phi);
    const float phiux = phi * ux, phiuy = phi * uy;
    const float ax = (phiux - phiux_p) + (1.f / 3.f) * lam * nx_;
    const float ay = (phiuy - phiuy_p) + (1.f / 3.f) * lam * ny_;
    const float gsrc = 1.f - 0.5f * P.omega_g;
    const float pmd = phi * mdot;

    // Enthalpy (T from the local macroscopic step)
    const float dL = P.L * (m.flp - m.fl);
    const float T = m.T;

    const float fsrc = 1.f - 0.5f * omega_f;
    // per-phase properties: local C_p in h^eq, tau_h - 1/2 scaled by k / k_l
    float Cp_loc = P.Cp, omega_h = P.omega_h;
    if (P.phase_props) {
        Cp_loc = mix3(fs, phi, P.Cp_s, P.Cp, P.Cp_g);
        omega_h = 1.f / (mix3(fs, phi, P.k_s, 1.f, P.k_g) * P.dtau_h + 0.5f);
    }
    const float TCp = T * Cp_loc, TCpref = T * P.Cpref;
    const float uu15 = 1.5f * uu;
    // rest populations (c_0 = 0)
    const float gi0 = pop.G(0), hi0 = pop.H(0), fi0 = pop.F(0);
    float g0n, h0n, f0n;
    {
        const float si = kW0 * -uu15;
        const float geq = kW0 * phi;
        g0n = gi0 - P.omega_g * (gi0 - geq) + gsrc * (kW0 * pmd);
        // h_0 carried shifted by -L f_l
        const float heq0 = m.Hp + dL - TCpref + kW0 * (TCpref - TCp * uu15);
        h0n = (1.f - omega_h) * (hi0 + dL) + omega_h * heq0;
        const float feq = (kW0 - 1.f) * 3.f * pn + rho * si;
        f0n = fi0 - omega_f * (fi0 - feq) + fsrc * (kW0 * (S - 3.f * uFt));
    }
    // 16-bit storage: what the stored values add to the site's outgoing
    // deviations (sum of q - d), taken back from the rest populations
    float eg = 0.f, eh = 0.f, ef = 0.f;
    // the moving populations in pairs of opposite directions i and j = OPP(i):
    // c_j = -c_i, so every term odd in c changes sign and every even term is
    // shared, and each update below is one paired FP32 operation (FFMA2 /
    // FADD2) for both directions
    const float2 sgn = make_float2(1.f, -1.f);
    auto bc = [](float v) { return make_float2(v, v); };
    auto sub2 = [](float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); };
    const float2 og = bc(-P.omega_g), oh = bc(-omega_h), of = bc(-omega_f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = q < 2 ? q + 1 : q + 3;  // 1, 2, 5, 6
        const int j = OPP(i);                  // 3, 4, 7, 8
        const float w = WGT(i);
        const float cu = cdot(i, ux, uy);
        const float w3cu = 3.f * w * cu;
        // s(u) of Eq. 32 (shared by the flow and enthalpy equilibria): its odd
        // part 3 w c.u and its even part w (4.5 (c.u)^2 - 1.5 u.u)
        const float sev = w * (4.5f * cu * cu - uu15);
        const float2 si = __ffma2_rn(bc(w3cu), sgn, bc(sev));
        // f (Eqs. 30-33): 9 (c.u)(c.Ft) is even, 3 c.(F + rho f) odd
        const float2 feq = __ffma2_rn(bc(rho), si, bc(w * 3.f * pn));
        const float Fev = w * (S + 9.f * cu * cdot(i, Ftx, Fty) - 3.f * uFt);
        const float2 Fi = __ffma2_rn(bc(3.f * w * cdot(i, Fpx, Fpy)), sgn, bc(Fev));
        const float2 f = make_float2(pop.F(i), pop.F(j));
        const float2 fn = __ffma2_rn(bc(fsrc), Fi, __ffma2_rn(of, sub2(f, feq), f));
        if constexpr (sizeof(ST) == 4) {  // f first: its registers are free for g and h
            out.f32(i, fn.x);
            out.f32(j, fn.y);
        }
        // g (Eqs. 21, 24, 25)
        const float2 geq = __ffma2_rn(bc(phi * w3cu), sgn, bc(w * phi));
        const float2 Gi = __ffma2_rn(bc(3.f * w * cdot(i, ax, ay)), sgn, bc(w * pmd));
        const float2 g = make_float2(pop.G(i), pop.G(j));
        const float2 gn = __ffma2_rn(bc(gsrc), Gi, __ffma2_rn(og, sub2(g, geq), g));
        // h (Eqs. 27-28)
        const float2 heq = __ffma2_rn(bc(TCp), si, bc(w * TCpref));
        const float2 h = make_float2(pop.H(i), pop.H(j));
        const float2 hn = __ffma2_rn(oh, sub2(h, heq), h);
        if constexpr (sizeof(ST) == 4) {
            out.gh32(i, gn.x, hn.x);
            out.gh32(j, gn.y, hn.y);
        } else {
            // deviations from the rest equilibria (g, h: destination's
            // references dref[i]; f: this site's pressure), and what their
            // rounding to 16 bits takes away from what the site sends
            using C16 = Bits16<ST>;
            const float2 dphi = make_float2(dref[i].phi, dref[j].phi);
            const float2 dT = make_float2(dref[i].T, dref[j].T);
            const float2 dg = __ffma2_rn(bc(-w), dphi, gn);
            const float2 dh = __ffma2_rn(bc(-w * P.Cpref), dT, hn);
            const float2 df = __fmul2_rn(__fadd2_rn(fn, bc(-f_rest(i, pn))), bc(kFScale));
            const unsigned qi = C16::pack2(dg.x, dh.x), qj = C16::pack2(dg.y, dh.y);
            const ST fi_ = C16::from_f(df.x), fj_ = C16::from_f(df.y);
            out.gh16(i, qi);
            out.gh16(j, qj);
            out.f16(i, C16::bits(fi_));
            out.f16(j, C16::bits(fj_));
            eg = C16::add_lo(qi, eg - dg.x);
            eh = C16::add_hi(qi, eh - dh.x);
            ef = C16::add_lo((unsigned)C16::bits(fi_), ef - df.x);
            eg = C16::add_lo(qj, eg - dg.y);
            eh = C16::add_hi(qj, eh - dh.y);
            ef = C16::add_lo((unsigned)C16::bits(fj_), ef - df.y);
        }
    }
    if constexpr (sizeof(ST) != 4) {  // the rest populations carry the rounding
        g0n -= eg;
        h0n -= eh;
        f0n -= ef * kInvFScale;
    }
    out.own0(make_float4(g0n, h0n, f0n, m.fl));
    out.own1(make_float4(phiux, phiuy, pn, S));
    if constexpr (sizeof(ST) != 4)  // references of this site for the next step
        out.ref(make_float2(phi, T));

    if (OBS) {
        ob.add(0, phi);
        ob.add(1, fs);
        // H = H' + L f_l^{n-1}: the product enters with its exact rounding error
        const float lf = P.L * m.flp;
        ob.add(2, m.Hp);
        ob.add(2, lf);
        ob.add(2, fmaf(P.L, m.flp, -lf));
        ob.add(3, rho);
        ob.add(4, fs * P.rho_s + (1.f - fs) * clamp01(phi) * P.rho_l);
        ob.add(5, mdot);
        ob.add(6, phi * mdot);
        if (on_col) ob.add(7, fs);
        if (on_row) ob.add(8, fs);
        ob.max(9, sqrtf(uu));
        const bool bad = !isfinite(phi) || !isfinite(m.Hp) || !isfinite(ux) || !isfinite(uy) ||
                         !isfinite(pn);
        if (bad) ob.add(10, 1.f);
    }
}

template <bool OBS, typename ST = float, typename Pops = ArrPops, typename Acc = ObsAcc>
__device__ __forceinline__ void site_update(const Phys& P, int flags, const Macro& m,
                                            const Pops& pop,
                                            float phiux_p, float phiuy_p, const Stencil& st,
                                            void* __restrict__ Bv, float* __restrict__ Baux,
                                            int /*plane*/, int own, bool on_col, bool on_row,
                                            Acc& ob, const Ref* dref = nullptr) {
    site_update_to<OBS, ST>(P, flags, m, pop, phiux_p, phiuy_p, st, SiteStore{Bv, Baux, own}, on_col,
                            on_row, ob, dref);
}

// ---------------------------------------------------------------------------
// The fused step kernel
// ---------------------------------------------------------------------------
// One CTA advances tile T of lattice I (the body of every tile kernel).
template <int TX, int TY, bool OBS>
__device__ __forceinline__ void tile_step(const Inst& I, const Tile& T, int parity,
                                          double* __restrict__ partials) {
    constexpr int NT = TX * TY;
    constexpr int SW = TX + 4;                  // shared row width (2-cell halo)
    constexpr int SH = TY + 4;
    __shared__ float s_phi[SH * SW], s_rho[SH * SW], s_p[SH * SW], s_S[SH * SW];

    const Phys P = load_phys(I);
    Lat l;
    l.A = static_cast<const float*>(I.pop[parity]);
    l.Aaux = I.aux[parity];
    l.plane = (int)I.plane; l.nx = I.nx; l.ny = I.ny; l.pitch = I.pitch; l.flags = I.flags;
    float* __restrict__ B = static_cast<float*>(I.pop[parity ^ 1]);
    float* __restrict__ Baux = I.aux[parity ^ 1];
    const float abb = P.Cpref * P.Tw;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int tw = T.tw, th = T.th, x0 = T.x0, y0 = T.y0;
    const bool active = tx < tw && ty < th;
    const int x = x0 + tx, y = y0 + ty;
    auto SI = [](int ox, int oy) { return (oy + 2) * SW + (ox + 2); };

    // ---- phase A: own site ----
    float g[9], h[9], f[9];
    Macro m;
    float phiux_p = 0.f, phiuy_p = 0.f;
    if (active) {
        const int own = y * l.pitch + x;
        pull_set<0>(l, x, y, abb, g);
        pull_set<1>(l, x, y, abb, h);
        pull_set<2>(l, x, y, abb, f);
        const float flp = ldAux(l, 0, own);
        phiux_p = ldAux(l, 1, own);
        phiuy_p = ldAux(l, 2, own);
        m = local_macro(P, g, h, flp);
        s_phi[SI(tx, ty)] = m.phi;
        s_rho[SI(tx, ty)] = m.rho;
        s_p[SI(tx, ty)] = ldAux(l, 3, own);
        s_S[SI(tx, ty)] = ldAux(l, 4, own);
    }

    // ---- phase B: ring cells and wall extras ----
    const bool wxlo = !(l.flags & kPeriodicX) && x0 == 0;
    const bool wxhi = !(l.flags & kPeriodicX) && x0 + tw == l.nx;
    const bool wylo = !(l.flags & kPeriodicY) && y0 == 0;
    const bool wyhi = !(l.flags & kPeriodicY) && y0 + th == l.ny;
    const int nring = 2 * (tw + 2) + 2 * th;
    const int nent = nring + 4 * ((int)wxlo + (int)wxhi + (int)wylo + (int)wyhi);

    // Entry k -> tile-relative cell (ox, oy).
    auto entry = [&](int k, int& ox, int& oy) {
        if (k < tw + 2) { ox = k - 1; oy = -1; return; }
        k -= tw + 2;
        if (k < tw + 2) { ox = k - 1; oy = th; return; }
        k -= tw + 2;
        if (k < th) { ox = -1; oy = k; return; }
        k -= th;
        if (k < th) { ox = tw; oy = k; return; }
        k -= th;
        // wall extras, 4 per touched wall, in the order y lo, y hi, x lo, x hi
        int w = k >> 2, j = k & 3;
        int side = 0;
        for (int t = 0, seen = 0; t < 4; ++t) {  // the w-th touched wall
            const bool touched = t == 0 ? wylo : (t == 1 ? wyhi : (t == 2 ? wxlo : wxhi));
            if (touched && seen++ == w) side = t;
        }
        int a = (j & 1), b = (j >> 1);   // a: layer (adjacent/next), b: which end
        if (side == 0) { ox = b ? tw + 1 : -2; oy = a; }
        else if (side == 1) { ox = b ? tw + 1 : -2; oy = th - 1 - a; }
        else if (side == 2) { oy = b ? th + 1 : -2; ox = a; }
        else { oy = b ? th + 1 : -2; ox = tw - 1 - a; }
    };
    // Resolve a tile-relative cell to lattice coordinates; false when behind a wall.
    auto resolve = [&](int ox, int oy, int& gx, int& gy, bool& outx, bool& outy) {
        gx = x0 + ox; gy = y0 + oy;
        outx = outy = false;
        if (gx < 0 || gx >= l.nx) {
            if (l.flags & kPeriodicX) gx = (gx + l.nx) % l.nx; else outx = true;
        }
        if (gy < 0 || gy >= l.ny) {
            if (l.flags & kPeriodicY) gy = (gy + l.ny) % l.ny; else outy = true;
        }
        return !(outx || outy);
    };

    for (int k = tid; k < nent; k += NT) {
        int ox, oy, gx, gy;
        bool outx, outy;
        entry(k, ox, oy);
        if (resolve(ox, oy, gx, gy, outx, outy)) {
            float gg[9], hh[9];
            pull_set<0>(l, gx, gy, abb, gg);
            pull_set<1>(l, gx, gy, abb, hh);
            const int idx = gy * l.pitch + gx;
            Macro mm = local_macro(P, gg, hh, ldAux(l, 0, idx));
            s_phi[SI(ox, oy)] = mm.phi;
            s_rho[SI(ox, oy)] = mm.rho;
            if (k < nring) {
                s_p[SI(ox, oy)] = ldAux(l, 3, idx);
                s_S[SI(ox, oy)] = ldAux(l, 4, idx);
            }
        } else if (k < nring) {
            // ghost: p and S copy the adjacent lattice value
            int cx = min(max(x0 + ox, 0), l.nx - 1), cy = min(max(y0 + oy, 0), l.ny - 1);
            if (!outx) cx = gx;
            if (!outy) cy = gy;
            const int idx = cy * l.pitch + cx;
            s_p[SI(ox, oy)] = ldAux(l, 3, idx);
            s_S[SI(ox, oy)] = ldAux(l, 4, idx);
        }
    }
    __syncthreads();

    // ---- phase C: ghosts of phi (wetting) and rho (copy) ----
    // Shared-memory slot of a lattice coordinate (periodic axes wrap into the
    // tile's 2-cell halo).
    auto lat_slot = [&](int xl, int yl) {
        int ox = xl - x0, oy = yl - y0;
        if (ox < -2) ox += l.nx; else if (ox > tw + 1) ox -= l.nx;
        if (oy < -2) oy += l.ny; else if (oy > th + 1) oy -= l.ny;
        return SI(ox, oy);
    };
    auto wrap_or_clamp = [](int v, int n, bool periodic) {
        if (v >= 0 && v < n) return v;
        if (periodic) return (v + n) % n;
        return v < 0 ? 0 : n - 1;
    };
    for (int k = tid; k < nring; k += NT) {
        int ox, oy, gx, gy;
        bool outx, outy;
        entry(k, ox, oy);
        if (resolve(ox, oy, gx, gy, outx, outy)) continue;
        const int cxl = outx ? (x0 + ox < 0 ? 0 : l.nx - 1) : gx;
        const int cyl = outy ? (y0 + oy < 0 ? 0 : l.ny - 1) : gy;
        s_rho[SI(ox, oy)] = s_rho[lat_slot(cxl, cyl)];
        float ghost;
        if (outy && !outx) {
            const int ya = cyl, yb = (y0 + oy < 0) ? 1 : l.ny - 2;
            const bool px = (l.flags & kPeriodicX) != 0;
            const int xm = wrap_or_clamp(gx - 1, l.nx, px), xp = wrap_or_clamp(gx + 1, l.nx, px);
            const float d0 = 0.5f * (s_phi[lat_slot(xp, ya)] - s_phi[lat_slot(xm, ya)]);
            const float d1 = 0.5f * (s_phi[lat_slot(xp, yb)] - s_phi[lat_slot(xm, yb)]);
            ghost = s_phi[lat_slot(gx, ya)] + P.tan_w * fabsf(1.5f * d0 - 0.5f * d1);
        } else if (outx && !outy) {
            const int xa = cxl, xb = (x0 + ox < 0) ? 1 : l.nx - 2;
            const bool py = (l.flags & kPeriodicY) != 0;
            const int ym = wrap_or_clamp(gy - 1, l.ny, py), yp = wrap_or_clamp(gy + 1, l.ny, py);
            const float d0 = 0.5f * (s_phi[lat_slot(xa, yp)] - s_phi[lat_slot(xa, ym)]);
            const float d1 = 0.5f * (s_phi[lat_slot(xb, yp)] - s_phi[lat_slot(xb, ym)]);
            ghost = s_phi[lat_slot(xa, gy)] + P.tan_w * fabsf(1.5f * d0 - 0.5f * d1);
        } else {
            ghost = s_phi[lat_slot(cxl, cyl)];
        }
        s_phi[SI(ox, oy)] = ghost;
    }
    __syncthreads();

    // ---- phase D: stencils, forces, collisions, store ----
    ObsAcc ob;
    if (OBS) ob.zero();
    if (active) {
        Stencil st;
        {
            // column sums of x-1, x, x+1 from shared memory (same expressions as
            // the strip kernel's shuffled column sums)
            auto col = [&](const float* a, int dx, float& m_, float& c_, float& p_) {
                m_ = a[SI(tx + dx, ty - 1)];
                c_ = a[SI(tx + dx, ty)];
                p_ = a[SI(tx + dx, ty + 1)];
            };
            float mL, cL, pL, mC, cC, pC, mR, cR, pR;
            col(s_phi, -1, mL, cL, pL); col(s_phi, 0, mC, cC, pC); col(s_phi, 1, mR, cR, pR);
            grad_cols(col_sums(mL, cL, pL), col_sums(mC, cC, pC), col_sums(mR, cR, pR),
                      st.gphx, st.gphy);
            st.lph = lap_cols(cL, cC, cR, pL + mL, pC + mC, pR + mR);
            col(s_rho, -1, mL, cL, pL); col(s_rho, 0, mC, cC, pC); col(s_rho, 1, mR, cR, pR);
            grad_cols(col_sums(mL, cL, pL), col_sums(mC, cC, pC), col_sums(mR, cR, pR),
                      st.grx, st.gry);
            col(s_p, -1, mL, cL, pL); col(s_p, 0, mC, cC, pC); col(s_p, 1, mR, cR, pR);
            grad_cols(col_sums(mL, cL, pL), col_sums(mC, cC, pC), col_sums(mR, cR, pR),
                      st.gpx, st.gpy);
            col(s_S, -1, mL, cL, pL); col(s_S, 0, mC, cC, pC); col(s_S, 1, mR, cR, pR);
            grad_cols(col_sums(mL, cL, pL), col_sums(mC, cC, pC), col_sums(mR, cR, pR),
                      st.gSx, st.gSy);
        }
        site_update<OBS>(P, l.flags, m, ArrPops{g, h, f}, phiux_p, phiuy_p, st, B, Baux, l.plane,
                         y * l.pitch + x, x == l.nx / 2, y == l.ny / 2, ob);
    }
    if (OBS) {
        double v[kObs];
#pragma unroll
        for (int j = 0; j < kObs; ++j) v[j] = ob.total(j);
        block_reduce_obs<NT>(v, partials + T.part, I.part_stride);
    }
    // the tile's mdot of this step joins its FP64 running sum (warp sums,
    // then the warps in order), and on observable steps each column's f_s
    // (rows in order) is added to the lattice's column profile
    __shared__ float s_md[NT / 32];
    __shared__ float s_col[TY][TX];
    if (I.macc || (OBS && I.prof)) {
        float md = active ? m.mdot : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md += __shfl_xor_sync(0xffffffffu, md, o);
        if ((tid & 31) == 0) s_md[tid >> 5] = md;
        if (OBS) s_col[ty][tx] = active ? m.fs : 0.f;
        __syncthreads();
        if (I.macc && tid == 0) {
            float sum = 0.f;
            for (int w = 0; w < NT / 32; ++w) sum += s_md[w];
            I.macc[T.part] += (double)sum;
        }
        if (OBS && I.prof && ty == 0 && tx < tw) {
            float sum = 0.f;
            for (int r = 0; r < th; ++r) sum += s_col[r][tx];
            atomicAdd(I.prof + x0 + tx, (double)sum);
        }
    }
}

template <int TX, int TY, bool OBS>
__global__ void __launch_bounds__(TX * TY)
step_fp32(const Inst* __restrict__ insts, const Tile* __restrict__ tiles, int parity,
          double* __restrict__ partials) {
    const Tile T = tiles[blockIdx.x];
    tile_step<TX, TY, OBS>(insts[T.inst], T, parity, partials);
}

// Handle-free variant for lbm_step_noalloc: the lattice record arrives by
// value, the 32 x 8 tile follows from the block index, and the per-tile
// observable partials go to the caller-supplied scratch array.
template <bool OBS>
__global__ void __launch_bounds__(256)
step_tile_noalloc(const Inst I, int tiles_x, double* __restrict__ partials) {
    Tile T;
    T.inst = 0;
    T.x0 = (int)(blockIdx.x % tiles_x) * 32;
    T.y0 = (int)(blockIdx.x / tiles_x) * 8;
    T.tw = min(32, I.nx - T.x0);
    T.th = min(8, I.ny - T.y0);
    T.part = (int)blockIdx.x;
    tile_step<32, 8, OBS>(I, T, 0, partials);
}


// ---------------------------------------------------------------------------
// Warp-strip kernel (lattices periodic in x)
// ---------------------------------------------------------------------------
// One warp advances a strip of 30 output columns over rows [y0, y1). Lane l
// holds column x0 - 1 + l, so lanes 0 and 31 are the halo of the strip and
// neighbours along x come from warp shuffles. Along y the warp keeps phi,
// rho, p^{n-1} and S^{n-1} of rows y-1, y and y+1 in registers and computes
// the macroscopic fields one row ahead of the row it collides. No shared
// memory and no block barrier are involved; the y halo costs two extra rows
// of local macroscopic fields per strip.

// Pull of set SET at (x, y) for a row whose sources do not cross a wall; the
// column offsets xm/xp and row offsets rm/rp are already wrapped.
template <int SET, typename ST, bool NC>
__device__ __forceinline__ void pull_rows(const LatT<NC>& l, int xc, int xm, int xp, int r0,
                                          int rm, int rp, float v[9], const Ref& ref,
                                          float Cpref, const float* pref) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int r = CY(i) > 0 ? rm : (CY(i) < 0 ? rp : r0);   // source row y - cy
        const int c = CX(i) > 0 ? xm : (CX(i) < 0 ? xp : xc);   // source column x - cx
        v[i] = decode<ST, SET>(i, ldPop<ST>(l, SET, i, r + c), ref, Cpref);
        if constexpr (sizeof(ST) != 4 && SET == 2) {
            if (i) v[i] += f_rest(i, pref[i]);
        }
    }
}

struct RowCtx {
    int xc, xm, xp;   // this lane's column and its periodic neighbours
    bool py;          // periodic y
};

// Pulls and local macroscopic fields of lattice row y at this lane's column.
template <int SET, typename ST = float, bool NC>
__device__ __forceinline__ void pull_row(const LatT<NC>& l, const RowCtx& c, int y, float abb,
                                         float v[9], const Ref& ref = Ref{0.f, 0.f},
                                         float Cpref = 0.f,
                                         const float* pref = nullptr) {
    if (c.py || (y >= 1 && y <= l.ny - 2)) {
        const int ym = y == 0 ? l.ny - 1 : y - 1;
        const int yp = y == l.ny - 1 ? 0 : y + 1;
        pull_rows<SET, ST>(l, c.xc, c.xm, c.xp, y * l.pitch, ym * l.pitch, yp * l.pitch, v, ref,
                           Cpref, pref);
    } else {
        pull_set<SET, ST>(l, c.xc, y, abb, v, ref, Cpref, pref);
    }
}

// Value of `v` at the lane c_x columns away (c_x in {-1, 0, 1}).
__device__ __forceinline__ float lane_shift(float v, int cx) {
    if (cx > 0) return __shfl_down_sync(0xffffffffu, v, 1);
    if (cx < 0) return __shfl_up_sync(0xffffffffu, v, 1);
    return v;
}

// Wetting ghost (Eqs. 39-41) for the row behind a wall: a is the adjacent
// lattice row, b the next one; outer_a/outer_b hold phi one column beyond
// the strip for the halo lanes.
__device__ __forceinline__ float strip_wet_ghost(float a, float b, float outer_a, float outer_b,
                                                 int lane, float tan_w) {
    float ap = __shfl_down_sync(0xffffffffu, a, 1), am = __shfl_up_sync(0xffffffffu, a, 1);
    float bp = __shfl_down_sync(0xffffffffu, b, 1), bm = __shfl_up_sync(0xffffffffu, b, 1);
    if (lane == 31) { ap = outer_a; bp = outer_b; }
    if (lane == 0) { am = outer_a; bm = outer_b; }
    const float d0 = 0.5f * (ap - am);
    const float d1 = 0.5f * (bp - bm);
    return a + tan_w * fabsf(1.5f * d0 - 0.5f * d1);
}

// ---------------------------------------------------------------------------
// Row staging: each lane copies, asynchronously and several rows ahead, every
// value it will consume from a lattice row into its own part of a per-warp
// ring of shared-memory slots: the populations pulled into its site (for a
// link that crosses a wall, the site's own opposite populations, i.e. the
// bounce-back sources) and the own-site group of its site. A lane reads back
// only what it copied itself, so no warp or block barrier is involved;
// cp.async.wait_group orders the copies before the reads. With the grouped
// layout one copy moves a (g_i, h_i) pair (8 bytes, FP16: 4) and one four
// own-site values (16 bytes), so a row takes 18 copies instead of 32.
// Slot layout in floats, lane l: 4l + c the own-site group (g_0, h_0, f_0,
// f_l), 128 + 4l + c ((phi u)_x, (phi u)_y, p, S), 256 + 64 (i - 1) + 2l + s
// the pair (g_i, h_i), 768 + 32 (i - 1) + l f_i, and for FP16 storage
// 1024 + 2l + c (phi_ref, T_ref). FP16 pairs and f_i arrive as the aligned
// 32-bit word holding them; decoded pairs go back over it, f_i to registers.
// ---------------------------------------------------------------------------
constexpr int kSlotO1 = 128, kSlotGH = 256, kSlotF = 768, kSlotR = 1024;
__device__ __forceinline__ int slot_gh(int i, int lane) { return kSlotGH + 64 * (i - 1) + 2 * lane; }
__device__ __forceinline__ int slot_f(int i, int lane) { return kSlotF + 32 * (i - 1) + lane; }
template <typename ST>
__host__ __device__ constexpr int stage_planes() { return sizeof(ST) == 4 ? 32 : 34; }
template <typename ST>
__host__ __device__ constexpr int slot_floats() { return stage_planes<ST>() * 32; }
// Dynamic shared memory of one warp of a staged kernel: STG ring slots, then
// one float per lane for the running mdot sum of the warp's item.
template <typename ST, int STG>
__host__ __device__ constexpr int warp_smem_floats() { return STG * slot_floats<ST>() + 32; }

__device__ __forceinline__ void cp_async4(float* dst_smem, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(float* dst_smem, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst_smem, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// The same copies with an L2 eviction priority (createpolicy below).
template <int N>
__device__ __forceinline__ void cp_async_p(float* dst_smem, const float* src,
                                           unsigned long long pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;" ::"r"(d),
                 "l"(src), "n"(N), "l"(pol)
                 : "memory");
}
// 16-byte copies that bypass L1 (data no other copy of the warp reads again).
__device__ __forceinline__ void cp_async_cg16(float* dst_smem, const float* src,
                                              unsigned long long pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "l"(pol)
                 : "memory");
}
// L2 priority of a staged row: 1 keep (evict last), 2 release (evict first),
// otherwise normal.
__device__ __forceinline__ unsigned long long l2_policy(int hint) {
    unsigned long long pol;
    if (hint == 1)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else if (hint == 2)
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    else
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the copies of lattice row r (possibly -1 or ny for periodic y) into
// this lane's part of the ring slot at `slot`. macro_only: only what the
// local macroscopic step needs (everything but f_i). hint: the rows an item
// shares with the item below it are read by this item first and by that one
// at the end of the step; they are kept in L2 (1) until then and released (2)
// by the second read.
// Offsets of the blocked layout split into a column part, fixed for a lane
// over a strip item, and a row part (pitch is a multiple of 32, so a site's
// block is row * (pitch / 32) + column / 32): element offset = row term +
// column term + the plane's offset inside the block.
struct ColTerms {
    int gh[3], f[3], aux, ref;  // columns x - 1, x, x + 1 (gh, f); the lane's own (aux, ref)
    __device__ __forceinline__ ColTerms(int xm, int xc, int xp) {
        const int c[3] = {xm, xc, xp};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gh[k] = (c[k] >> 5) * kPopBlock + 2 * (c[k] & 31);
            f[k] = (c[k] >> 5) * kPopBlock + (c[k] & 31);
        }
        aux = (xc >> 5) * kAuxBlock + 4 * (xc & 31);
        ref = (xc >> 5) * kAuxBlock + 256 + 2 * (xc & 31);
    }
};

template <typename ST, bool NC>
__device__ __forceinline__ void stage_row(const LatT<NC>& l, int lane, const ColTerms& ct, bool py,
                                          int r, bool macro_only, float* slot, int hint = 0) {
    constexpr bool kHalf = sizeof(ST) != 4;
    const int ny = l.ny, nxb = l.pitch >> 5;
    const bool wlo = !py && r == 0, whi = !py && r == ny - 1;
    const int rr = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    const int ym = rr == 0 ? ny - 1 : rr - 1, yp = rr == ny - 1 ? 0 : rr + 1;
    // row terms of the rows y, y - 1, y + 1
    const int t0 = rr * nxb * kPopBlock, tm = ym * nxb * kPopBlock, tp = yp * nxb * kPopBlock;
    const int ra = rr * nxb * kAuxBlock;
    const unsigned long long pol = l2_policy(hint);
    // the site's own values: read by this lane only, so past L1
    cp_async_cg16(slot + 4 * lane, l.Aaux + ra + ct.aux, pol);
    cp_async_cg16(slot + kSlotO1 + 4 * lane, l.Aaux + ra + ct.aux + 128, pol);
    if constexpr (kHalf) cp_async_p<8>(slot + kSlotR + 2 * lane, l.Aaux + ra + ct.ref, pol);
    const unsigned short* A16 = reinterpret_cast<const unsigned short*>(l.A);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int cy = CY(i), cx = CX(i);
        const bool wall = (cy > 0 && wlo) || (cy < 0 && whi);
        const int si = wall ? OPP(i) : i;
        // source: the site itself (bounce-back) or x - c_i in row y - c_iy
        // (the column index is a constant: no array indexed at run time)
        const int k = cx > 0 ? 0 : (cx < 0 ? 2 : 1);
        const int rt = wall ? t0 : (cy > 0 ? tm : (cy < 0 ? tp : t0));
        const int cg = wall ? ct.gh[1] : ct.gh[k], cf = wall ? ct.f[1] : ct.f[k];
        const int eg = rt + cg + gh_off(si), ef = rt + cf + f_off(si);
        if constexpr (kHalf) {
            // blocks and plane rows hold an even number of 16-bit values, so
            // every aligned word lies inside its plane row
            cp_async_p<4>(slot + slot_gh(i, lane), reinterpret_cast<const float*>(A16 + eg), pol);
            if (!macro_only)
                cp_async_p<4>(slot + slot_f(i, lane), reinterpret_cast<const float*>(A16 + (ef & ~1)),
                              pol);
        } else {
            cp_async_p<8>(slot + slot_gh(i, lane), l.A + eg, pol);
            if (!macro_only) cp_async_p<4>(slot + slot_f(i, lane), l.A + ef, pol);
        }
    }
}

// Which 16-bit half of each staged word a lane wants, as __byte_perm
// selectors for the source columns x, x - 1 and x + 1 (periodic): 0x3232 the
// upper half (odd column), 0x1010 the lower half.
struct ColPar {
    unsigned c, m, p;
};
__device__ __forceinline__ unsigned half_sel(int col) { return (col & 1) ? 0x3232u : 0x1010u; }

// Set `set` of a staged row, decoded as pull_set does: for FP16 storage with
// the site's own references (g, h) and the source pressures pref (f; the
// site's own pressure pref[0] on bounced links); for h at a Dirichlet wall
// row the bounced populations become anti-bounce-back, -h + 2 w_i Cp_ref T_w.
template <int SET, typename ST = float>
__device__ __forceinline__ void staged_set(const float* slot, int lane, int r, int ny, bool py,
                                           int flags, float abb, float v[9],
                                           const ColPar& par = ColPar{0, 0, 0},
                                           const Ref& ref = Ref{0.f, 0.f}, float Cpref = 0.f,
                                           const float* pref = nullptr) {
    const bool wlo = !py && r == 0, whi = !py && r == ny - 1;
    v[0] = slot[4 * lane + SET];  // FP32 rest population (h_0 shifted)
    if constexpr (sizeof(ST) == 4) {
#pragma unroll
        for (int i = 1; i < 9; ++i) v[i] = SET < 2 ? slot[slot_gh(i, lane) + SET] : slot[slot_f(i, lane)];
        if (SET == 1 && !py) {
            const bool lo = wlo && (flags & kDirYlo), hi = whi && (flags & kDirYhi);
#pragma unroll
            for (int i = 1; i < 9; ++i)
                if ((CY(i) > 0 && lo) || (CY(i) < 0 && hi)) v[i] = -v[i] + 2.0f * WGT(i) * abb;
        }
    } else {
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const bool wall = (CY(i) > 0 && wlo) || (CY(i) < 0 && whi);
        if (SET < 2) {
            const unsigned w = __float_as_uint(slot[slot_gh(i, lane)]);
            const float raw = Bits16<ST>::to_f(
                Bits16<ST>::from_bits((unsigned short)(SET == 0 ? (w & 0xffffu) : (w >> 16))));
            v[i] = SET == 0 ? raw + WGT(i) * ref.phi : raw + WGT(i) * Cpref * ref.T;
        } else {
            const unsigned w = __float_as_uint(slot[slot_f(i, lane)]);
            const unsigned sel = wall ? par.c : (CX(i) > 0 ? par.m : (CX(i) < 0 ? par.p : par.c));
            v[i] = Bits16<ST>::fma_lo_2m12(__byte_perm(w, 0u, sel), f_rest(i, wall ? pref[0] : pref[i]));
        }
        if (SET == 1 && wall) {
            const bool dir = (wlo && (flags & kDirYlo)) || (whi && (flags & kDirYhi));
            if (dir) v[i] = -v[i] + 2.0f * WGT(i) * abb;
        }
    }
    }
}

// Sets g and h of a staged row together (16-bit storage): each (g_i, h_i)
// word is loaded once and decoded by one paired conversion, then treated as
// staged_set treats it.
template <typename ST>
__device__ __forceinline__ void staged_gh(const float* slot, int lane, int r, int ny, bool py,
                                          int flags, float abb, float g[9], float h[9],
                                          const Ref& ref, float Cpref) {
    const bool wlo = !py && r == 0, whi = !py && r == ny - 1;
    const bool dir = (wlo && (flags & kDirYlo)) || (whi && (flags & kDirYhi));
    g[0] = slot[4 * lane];
    h[0] = slot[4 * lane + 1];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const unsigned wd = __float_as_uint(slot[slot_gh(i, lane)]);
        g[i] = Bits16<ST>::add_lo(wd, WGT(i) * ref.phi);
        h[i] = Bits16<ST>::add_hi(wd, WGT(i) * Cpref * ref.T);
        const bool wall = (CY(i) > 0 && wlo) || (CY(i) < 0 && whi);
        if (wall && dir) h[i] = -h[i] + 2.0f * WGT(i) * abb;
    }
}

// One warp advances strip item W by one step (the body of every strip kernel).
// STG = 0: populations are loaded where they are consumed; STG >= 3: rows are
// staged through `ring` (STG slots of this warp): while row y is computed,
// the copies of rows y + 2 .. y + STG - 1 are in flight.
template <bool OBS, typename ST, bool NC, int STG = 0>
__device__ __forceinline__ void strip_item(const Inst* __restrict__ insts, const Item& W,
                                           int parity, double* __restrict__ partials,
                                           float* ring = nullptr) {
    constexpr bool kHalf = sizeof(ST) != 4;
    static_assert(STG == 0 || STG >= 3, "staging needs at least three ring slots");
    // Staging: the collision reads its populations from the ring slot (FP16:
    // g, h decoded over the staged words; f decoded into registers)
    constexpr bool kSlotPops = STG > 0;
    const int lane = threadIdx.x & 31;
    const Inst& I = insts[W.inst];
    const Phys P = load_phys(I);
    LatT<NC> l;
    l.A = static_cast<const float*>(I.pop[parity]);
    l.Aaux = I.aux[parity];
    l.plane = (int)I.plane; l.nx = I.nx; l.ny = I.ny; l.pitch = I.pitch; l.flags = I.flags;
    void* __restrict__ B = I.pop[parity ^ 1];
    float* __restrict__ Baux = I.aux[parity ^ 1];
    const float abb = P.Cpref * P.Tw;
    const int nx = l.nx, ny = l.ny;

    RowCtx c;
    const int xl = W.x0 - 1 + lane;
    c.xc = ((xl % nx) + nx) % nx;
    c.xm = c.xc == 0 ? nx - 1 : c.xc - 1;
    c.xp = c.xc == nx - 1 ? 0 : c.xc + 1;
    c.py = (l.flags & kPeriodicY) != 0;
    const bool out_lane = lane >= 1 && lane <= kStripW && xl < nx;
    const bool halo_lane = lane == 0 || lane == 31;
    const ColTerms ct(c.xm, c.xc, c.xp);
    const int x_outer = lane == 0 ? c.xm : c.xp;   // one column beyond the strip

    // decoding references of a site (FP16 storage)
    auto site_ref = [&](int idx) {
        Ref r{0.f, 0.f};
        if constexpr (kHalf) { r.phi = ldAux(l, 5, idx); r.T = ldAux(l, 6, idx); }
        return r;
    };

    // phi one column beyond the strip at the wall-adjacent rows (halo lanes)
    float oB0 = 0.f, oB1 = 0.f, oT0 = 0.f, oT1 = 0.f;
    auto outer_phi = [&](int y) {
        float gg[9], hh[9];
        const int idx = y * l.pitch + x_outer;
        const Ref r = site_ref(idx);
        pull_set<0, ST>(l, x_outer, y, abb, gg, r, P.Cpref);
        pull_set<1, ST>(l, x_outer, y, abb, hh, r, P.Cpref);
        return local_macro(P, gg, hh, ldAux(l, 0, idx)).phi;
    };
    auto note_outer = [&](int y) {
        if (c.py || !halo_lane) return;
        if (y == 0) oB0 = outer_phi(y);
        if (y == 1) oB1 = outer_phi(y);
        if (y == ny - 1) oT0 = outer_phi(y);
        if (y == ny - 2) oT1 = outer_phi(y);
    };
    // local macroscopic fields of row y at this lane's column (the pulled g
    // and h are dropped; the collision of the row pulls them again, from L1)
    auto row_macro = [&](int y, Macro& m, float& p, float& S, Ref& r) {
        float gg[9], hh[9];
        const int idx = y * l.pitch + c.xc;
        r = site_ref(idx);
        pull_row<0, ST>(l, c, y, abb, gg, r, P.Cpref);
        pull_row<1, ST>(l, c, y, abb, hh, r, P.Cpref);
        m = local_macro(P, gg, hh, ldAux(l, 0, idx));
        p = ldAux(l, 3, idx);
        S = ldAux(l, 4, idx);
        note_outer(y);
    };

    // staged rows: ring index j <-> lattice row y0 - 1 + j, j = 0 .. R - 1
    const int y0 = W.y0;
    const int R = W.y1 - y0 + 2;
    const bool has_lo = y0 >= 1 || c.py, has_hi = W.y1 < ny || c.py;
    auto slot = [&](int j) { return ring + (j % (STG > 0 ? STG : 1)) * slot_floats<ST>(); };
    auto issue = [&](int j) {
        if constexpr (STG > 0) {
            if (j < R && (j > 0 || has_lo) && (j < R - 1 || has_hi))
                stage_row<ST>(l, lane, ct, c.py, y0 - 1 + j, j == 0 || j == R - 1,
                              slot(j), j <= 1 ? 1 : (j >= R - 2 ? 2 : 0));
            cp_async_commit();  // possibly empty: one group per ring index
        }
    };
    const ColPar par{half_sel(c.xc), half_sel(c.xm), half_sel(c.xp)};
    auto slot_ref = [&](const float* sl) {
        Ref r{0.f, 0.f};
        if constexpr (kHalf) { r.phi = sl[kSlotR + 2 * lane]; r.T = sl[kSlotR + 2 * lane + 1]; }
        return r;
    };
    auto row_macro_staged = [&](int j, int y, Macro& m, float& p, float& S, Ref& r) {
        float gg[9], hh[9];
        const float* sl = slot(j);
        r = slot_ref(sl);
        if constexpr (kHalf) {
            staged_gh<ST>(sl, lane, y, ny, c.py, l.flags, abb, gg, hh, r, P.Cpref);
            float* ws = const_cast<float*>(sl);  // the decoded values, for the collision
#pragma unroll
            for (int i = 1; i < 9; ++i)
                *reinterpret_cast<float2*>(ws + slot_gh(i, lane)) = make_float2(gg[i], hh[i]);
        } else {
            staged_set<0, ST>(sl, lane, y, ny, c.py, l.flags, abb, gg, par, r, P.Cpref);
            staged_set<1, ST>(sl, lane, y, ny, c.py, l.flags, abb, hh, par, r, P.Cpref);
        }
        m = local_macro(P, gg, hh, sl[4 * lane + 3]);
        p = sl[kSlotO1 + 4 * lane + 2];
        S = sl[kSlotO1 + 4 * lane + 3];
        note_outer(y);
    };

    RowObs ob;
    if (OBS) ob.zero();
    // mdot of this lane's sites over the item (every step; the staged kernels
    // keep it in shared memory after the ring, which spares a register), f_s
    // of its column over the item's rows (observable steps)
    float md_acc = 0.f, col_fs = 0.f;
    auto md_smem = [&]() -> float& { return ring[STG * slot_floats<ST>() + lane]; };
    if constexpr (STG > 0) md_smem() = 0.f;

    // rows y-1 (m), y (0) and y+1 (p) of phi, rho, p^{n-1}, S^{n-1} (and T)
    float phm = 0.f, ph0, php = 0.f, rhm = 0.f, rh0, rhp = 0.f;
    float pm = 0.f, p0, pp = 0.f, Sm = 0.f, S0, Sp = 0.f;
    float tm = 0.f, t0, tp = 0.f;
    Macro mO;
    Ref rO;
    if constexpr (STG > 0) {
#pragma unroll 1
        for (int j = 0; j < STG; ++j) issue(j);  // one copy of the row issue code
        cp_async_wait<STG - 2>();  // ring indices 0 and 1 have landed
        row_macro_staged(1, y0, mO, p0, S0, rO);
    } else {
        row_macro(y0, mO, p0, S0, rO);
    }
    ph0 = mO.phi; rh0 = mO.rho; t0 = mO.T;
    if (has_lo) {
        Macro mm;
        Ref rr;
        if constexpr (STG > 0) row_macro_staged(0, y0 == 0 ? ny - 1 : y0 - 1, mm, pm, Sm, rr);
        else row_macro(y0 == 0 ? ny - 1 : y0 - 1, mm, pm, Sm, rr);
        phm = mm.phi; rhm = mm.rho; tm = mm.T;
    }

    for (int y = y0; y < W.y1; ++y) {
        const int own = y * l.pitch + c.xc;
        const int jy = y - y0 + 1;  // ring index of row y
        if constexpr (STG > 0) {
            issue(jy + STG - 1);        // into the slot of row y - 1, no longer read
            cp_async_wait<STG - 2>();   // row y + 1 has landed
        }
        // Every load that goes to DRAM for this row is issued here, before any
        // of it is consumed: f and (phi u)^{n-1} of row y, then g, h and the
        // carried scalars of row y+1 (inside row_macro).
        float f[9];
        float pref[9];
        // FP16 storage: pressures of the sites the pulled f come from (rows
        // y-1..y+1 of the carried p, neighbouring lanes); links that bounce
        // at a wall use the site's own pressure (pref[0]). Valid once the
        // window holds row y+1, i.e. after the look-ahead below.
        auto pull_f = [&]() {
            if constexpr (kHalf) {
                pref[0] = p0;
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const int cy = CY(i);
                    const float v = cy > 0 ? pm : (cy < 0 ? pp : p0);  // source row y - cy
                    pref[i] = lane_shift(v, -CX(i));                     // source column x - cx
                }
            }
            if constexpr (STG > 0)
                staged_set<2, ST>(slot(jy), lane, y, ny, c.py, l.flags, abb, f, par, rO, P.Cpref,
                                  pref);
            else
                pull_row<2, ST>(l, c, y, abb, f, rO, P.Cpref, pref);
        };
        float phiux_p, phiuy_p;
        if constexpr (STG > 0) {
            const float* sl = slot(jy);
            if constexpr (!kHalf && !kSlotPops) pull_f();
            phiux_p = sl[kSlotO1 + 4 * lane];
            phiuy_p = sl[kSlotO1 + 4 * lane + 1];
        } else {
            if constexpr (!kHalf) pull_f();
            phiux_p = ldAux(l, 1, own);
            phiuy_p = ldAux(l, 2, own);
        }
        Macro mN;
        Ref rN{0.f, 0.f};
        const bool top_wall = !(y + 1 < ny || c.py);
        if (!top_wall) {
            if constexpr (STG > 0) row_macro_staged(jy + 1, y + 1 == ny ? 0 : y + 1, mN, pp, Sp, rN);
            else row_macro(y + 1 == ny ? 0 : y + 1, mN, pp, Sp, rN);
            php = mN.phi; rhp = mN.rho; tp = mN.T;
        } else {
            // row ny lies behind the top wall: ghost from rows ny-1 and ny-2
            php = strip_wet_ghost(ph0, phm, oT0, oT1, lane, P.tan_w);
            rhp = rh0; pp = p0; Sp = S0; tp = t0;
        }
        const bool bottom_wall = y == 0 && !c.py;
        if (bottom_wall) {
            // row -1 lies behind the bottom wall: ghost from rows 0 and 1
            phm = strip_wet_ghost(ph0, php, oB0, oB1, lane, P.tan_w);
            rhm = rh0; pm = p0; Sm = S0; tm = t0;
        }
        if constexpr (kHalf && STG == 0) pull_f();

        // Eq. 38 from column sums exchanged with the neighbouring lanes
        Stencil st;
        {
            // (phi, rho) and (p, S) in pairs
            const ColSums2 c1 = col_sums2(make_float2(phm, rhm), make_float2(ph0, rh0),
                                          make_float2(php, rhp));
            const ColSums2 c2 = col_sums2(make_float2(pm, Sm), make_float2(p0, S0),
                                          make_float2(pp, Sp));
            auto side = [](const ColSums2& v, int dx) {
                ColSums2 r;
                r.A = make_float2(lane_shift(v.A.x, dx), lane_shift(v.A.y, dx));
                r.D = make_float2(lane_shift(v.D.x, dx), lane_shift(v.D.y, dx));
                return r;
            };
            float2 gx, gy;
            grad_cols2(side(c1, -1), c1, side(c1, 1), gx, gy);
            st.gphx = gx.x; st.gphy = gy.x; st.grx = gx.y; st.gry = gy.y;
            const float sph = c1.S2.x;  // php + phm
            st.lph = lap_cols(lane_shift(ph0, -1), ph0, lane_shift(ph0, 1), lane_shift(sph, -1),
                              sph, lane_shift(sph, 1));
            grad_cols2(side(c2, -1), c2, side(c2, 1), gx, gy);
            st.gpx = gx.x; st.gpy = gy.x; st.gSx = gx.y; st.gSy = gy.y;
        }

        // FP16 storage: references of the sites each outgoing population
        // streams into (the site itself where the link bounces at a wall)
        Ref dref[9];
        if constexpr (kHalf) {
            dref[0] = Ref{ph0, t0};
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int cy = CY(i);
                const float vp = cy > 0 ? php : (cy < 0 ? phm : ph0);
                const float vt = cy > 0 ? tp : (cy < 0 ? tm : t0);
                const float sp = lane_shift(vp, CX(i)), stt = lane_shift(vt, CX(i));
                const bool wall = (cy > 0 && top_wall) || (cy < 0 && bottom_wall);
                dref[i] = wall ? Ref{ph0, t0} : Ref{sp, stt};
            }
        }

        if constexpr (kSlotPops && kHalf) {
            pull_f();  // all lanes (shuffles); f stays in registers for the collision
            if (out_lane)
                site_update<OBS, ST>(P, l.flags, mO, SlotGHPops{slot(jy), lane, f}, phiux_p,
                                     phiuy_p, st, B, Baux, l.plane, own, c.xc == nx / 2,
                                     y == ny / 2, ob, dref);
        } else if constexpr (kSlotPops) {
            if (out_lane) {
                int hmask = 0;
                if (!kHalf && !c.py) {
                    const bool lo = y == 0 && (l.flags & kDirYlo), hi = y == ny - 1 && (l.flags & kDirYhi);
#pragma unroll
                    for (int i = 1; i < 9; ++i)
                        if ((CY(i) > 0 && lo) || (CY(i) < 0 && hi)) hmask |= 1 << i;
                }
                site_update<OBS, ST>(P, l.flags, mO, SlotPops{slot(jy), lane, hmask, abb}, phiux_p,
                                     phiuy_p, st, B, Baux, l.plane, own, c.xc == nx / 2,
                                     y == ny / 2, ob, dref);
            }
        } else if (out_lane) {
            // g and h of row y were pulled one row earlier: these loads hit L1
            float g[9], h[9];
            if constexpr (STG > 0) {
                staged_set<0, ST>(slot(jy), lane, y, ny, c.py, l.flags, abb, g, par, rO, P.Cpref);
                staged_set<1, ST>(slot(jy), lane, y, ny, c.py, l.flags, abb, h, par, rO, P.Cpref);
            } else {
                pull_row<0, ST>(l, c, y, abb, g, rO, P.Cpref);
                pull_row<1, ST>(l, c, y, abb, h, rO, P.Cpref);
            }
            site_update<OBS, ST>(P, l.flags, mO, ArrPops{g, h, f}, phiux_p, phiuy_p, st, B, Baux,
                                 l.plane, own, c.xc == nx / 2, y == ny / 2, ob, dref);
        }

        if (OBS) ob.flush(lane);
        if (out_lane) {
            if constexpr (STG > 0) md_smem() += mO.mdot;
            else md_acc += mO.mdot;
            if (OBS) col_fs += mO.fs;
        }

        // advance the window
        phm = ph0; ph0 = php; rhm = rh0; rh0 = rhp;
        pm = p0; p0 = pp; Sm = S0; S0 = Sp;
        tm = t0; t0 = tp;
        mO = mN;
        rO = rN;
    }
    if constexpr (STG > 0) cp_async_wait<0>();  // the trailing groups are empty

    if (OBS && RowObs::carried(lane) >= 0)
        partials[(long long)RowObs::carried(lane) * I.part_stride + W.part] = ob.total();
    // the item's mdot of this step joins its FP64 running sum (one warp owns
    // the item, so the read-modify-write needs no atomic)
    double* const macc = insts[W.inst].macc;  // read here: no register held over the rows
    if (macc) {
        if constexpr (STG > 0) md_acc = md_smem();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md_acc += __shfl_xor_sync(0xffffffffu, md_acc, o);
        if (lane == 0) macc[W.part] += (double)md_acc;
    }
    if (OBS && I.prof && out_lane) atomicAdd(I.prof + c.xc, (double)col_fs);
}

template <int WARPS, int MINB, bool OBS, typename ST>
__global__ void __launch_bounds__(WARPS * 32, MINB)
step_strip(const Inst* __restrict__ insts, const Item* __restrict__ items, int n_items,
           int parity, double* __restrict__ partials) {
    const int it = blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (it >= n_items) return;  // whole warp leaves together; no block barrier in the body
    strip_item<OBS, ST, true>(insts, items[it], parity, partials);
}

// Staged form: STG ring slots of slot_floats<ST>() floats per warp in dynamic
// shared memory.
template <int WARPS, int MINB, int STG, bool OBS, typename ST>
__global__ void __launch_bounds__(WARPS * 32, MINB)
step_strip_staged(const Inst* __restrict__ insts, const Item* __restrict__ items, int n_items,
                  int parity, double* __restrict__ partials) {
    extern __shared__ __align__(16) float ring_smem[];
    // Programmatic dependent launch: let the next step's grid be scheduled as
    // soon as every CTA of this one has started, and touch no lattice data
    // before the previous step's grid has completed (a no-op when launched
    // without the attribute).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int warp = threadIdx.x >> 5;
    const int it = blockIdx.x * WARPS + warp;
    if (it >= n_items) return;  // whole warp leaves together; no block barrier in the body
    strip_item<OBS, ST, true, STG>(insts, items[it], parity, partials,
                                   ring_smem + warp * warp_smem_floats<ST, STG>());
}

// Device-wide barrier between the steps of the persistent kernel. Every CTA
// of the (cooperatively launched, hence co-resident) grid adds one to *bar
// and waits until it reaches `target`. The wait is bounded in time and in
// iterations: past either bound the CTA raises *err and returns false, as
// does every CTA that finds *err raised, so no CTA waits for a step that
// will not come.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* err,
                                             unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        unsigned long long t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (unsigned spin = 0;; ++spin) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if ((spin & 31u) == 31u) {
                int e;
                asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e) : "l"(err) : "memory");
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                if (e != 0) { ok = 0; break; }
                if (t - t0 > limit_ns || spin > (1u << 26)) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Persistent form: one cooperative launch advances every item of every
// lattice by `nsteps` steps (parity alternating from parity0), each warp
// taking items in grid-stride order, with a device-wide barrier between
// steps. *bar must be zero at launch. STG > 0: the row-staged body, with
// STG ring slots per warp in dynamic shared memory. The staged rows are
// copied through L1 (cp.async of 4 bytes has no L2-only form); they were
// written by other CTAs before the barrier, whose acquire orders these
// copies after those writes.
template <int WARPS, int MINB, int STG, typename ST>
__global__ void __launch_bounds__(WARPS * 32, MINB)
step_strip_persistent(const Inst* __restrict__ insts, const Item* __restrict__ items,
                      int n_items, int parity0, int nsteps, unsigned* bar, int* err,
                      unsigned long long limit_ns) {
    extern __shared__ __align__(16) float ring_smem[];
    float* ring = ring_smem + (threadIdx.x >> 5) * warp_smem_floats<ST, STG>();
    const int warp = blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int stride = gridDim.x * WARPS;
    for (int s = 0; s < nsteps; ++s) {
        const int parity = parity0 ^ (s & 1);
        for (int it = warp; it < n_items; it += stride)
            strip_item<false, ST, false, STG>(insts, items[it], parity, nullptr, ring);
        if (s + 1 < nsteps &&
            !grid_barrier(bar, (unsigned)(s + 1) * gridDim.x, err, limit_ns))
            return;
    }
}

#include "lbm_block.cuh"

// Block step: one warp per block item (a 32-site column of row blocks over a
// segment of rows), every offset inside a staged row a compile-time constant.
// Launched with programmatic dependent launch like the staged strips.
template <int WARPS, int MINB, bool OBS, typename ST>
__global__ void __launch_bounds__(WARPS * 32, MINB)
step_block(const Inst* __restrict__ insts, const Item* __restrict__ items, int n_items, int parity,
           double* __restrict__ partials, int* err) {
    extern __shared__ __align__(16) unsigned char block_smem[];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    using BW = BlockWarp<ST>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = block_smem + warp * BW::kBytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + BW::kMbar);
    if (lane == 0)
        for (int k = 0; k < kBlockStg; ++k) mbar_init(mbar + k, 33);  // expect_tx + 32 lanes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    const int it = blockIdx.x * WARPS + warp;
    if (it >= n_items) return;  // whole warp leaves together; no block barrier in the body
    unsigned phase = 0;
    block_item<OBS, ST, true>(insts, items[it], parity, partials, base, mbar, phase,
                              reinterpret_cast<float*>(base + BW::kHring),
                              reinterpret_cast<float*>(base + BW::kMd), err);
}

// Persistent form of the block step: every item of every lattice for nsteps
// steps in one cooperative launch, a device-wide barrier between steps. The
// staged rows are read by bulk copies (through L2, after a proxy fence that
// orders them behind the barrier's acquire); the few global loads of the
// side columns next to a wall bypass L1.
template <int WARPS, int MINB, typename ST>
__global__ void __launch_bounds__(WARPS * 32, MINB)
step_block_persistent(const Inst* __restrict__ insts, const Item* __restrict__ items, int n_items,
                      int parity0, int nsteps, unsigned* bar, int* err,
                      unsigned long long limit_ns) {
    extern __shared__ __align__(16) unsigned char block_smem[];
    using BW = BlockWarp<ST>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = block_smem + warp * BW::kBytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + BW::kMbar);
    if (lane == 0)
        for (int k = 0; k < kBlockStg; ++k) mbar_init(mbar + k, 33);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    unsigned phase = 0;
    const int gw = blockIdx.x * WARPS + warp;
    const int stride = gridDim.x * WARPS;
    bool ok = true;
    for (int s = 0; s < nsteps; ++s) {
        const int parity = parity0 ^ (s & 1);
        for (int it = gw; ok && it < n_items; it += stride)
            ok = block_item<false, ST, false>(insts, items[it], parity, nullptr, base, mbar, phase,
                                              reinterpret_cast<float*>(base + BW::kHring),
                                              reinterpret_cast<float*>(base + BW::kMd), err);
        if (s + 1 < nsteps) {
            if (!grid_barrier(bar, (unsigned)(s + 1) * gridDim.x, err, limit_ns)) return;
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
    }
}

// A barrier that no other CTA joins: the single CTA of this kernel waits for
// a count of two until the time limit, raises *err and returns. Used to check
// that an expired wait is reported to the host rather than hanging.
#if LBM_HAS_PART(0)
__global__ void barrier_timeout_probe(unsigned* bar, int* err, unsigned long long limit_ns) {
    grid_barrier(bar, 2u, err, limit_ns);
}

// ---------------------------------------------------------------------------
// Initialisation (double precision, then rounded to the storage format)
// ---------------------------------------------------------------------------
// Start of a site: liquid-like before freezing (f_l = 1), so H = H_l + C_p
// (T0 - T_m) with C_p the liquid/gas mixture of Eq. 1, then Eq. 9 back with
// the local C_p of the resulting state (uniform properties: C_p itself).
struct InitSite {
    double H, fl, T;
};
__device__ __forceinline__ InitSite init_site(const InitConst& c, double phi, double T0) {
    InitSite r;
    if (c.Cp_s == c.Cp && c.Cp_g == c.Cp) {
        r.H = c.Cp * T0 + c.L;
        double fl = (r.H - c.Hs) / c.L;                         // Eq. 9a
        r.fl = fl < 0 ? 0 : (fl > 1 ? 1 : fl);
        r.T = c.Tm + (r.H - c.Hs - c.L * r.fl) / c.Cp;          // Eq. 9b
        return r;
    }
    const double ph = phi < 0 ? 0 : (phi > 1 ? 1 : phi);
    r.H = c.Hl + (ph * c.Cp + (1.0 - ph) * c.Cp_g) * (T0 - c.Tm);
    double fl = (r.H - c.Hs) / c.L;
    r.fl = fl < 0 ? 0 : (fl > 1 ? 1 : fl);
    double chi = (phi - 0.5) * c.inv_ramp + 0.5;
    chi = chi < 0 ? 0 : (chi > 1 ? 1 : chi);
    const double fs = chi * (1.0 - r.fl);
    const double cp = fs * c.Cp_s + (1.0 - fs) * (ph * c.Cp + (1.0 - ph) * c.Cp_g);
    r.T = c.Tm + (r.H - c.Hs - c.L * r.fl) / cp;
    return r;
}

__global__ void init_fp32(const Inst* __restrict__ insts, int inst, InitConst c,
                          const double* __restrict__ phi0, const double* __restrict__ T0,
                          int parity) {
    const Inst& I = insts[inst];
    const int n = I.nx * I.ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int x = k % I.nx, y = k / I.nx;
        const long long idx = (long long)y * I.pitch + x;
        const double ph = phi0[k];
        const InitSite st = init_site(c, ph, T0[k]);
        const double H = st.H, fl = st.fl, T = st.T;
        float* P = static_cast<float*>(I.pop[parity]);
        float* A = I.aux[parity];
        const int plane = (int)I.plane, site = (int)idx;
        for (int i = 0; i < 9; ++i) {
            const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
            const float g = (float)(w * ph);                                       // Eq. 24, u = 0
            double hq = (i == 0) ? H - c.Cpref * T + w * c.Cp * T * (c.Cpref / c.Cp)
                                 : w * c.Cp * T * (c.Cpref / c.Cp);                // Eq. 28, u = 0
            if (i == 0) hq -= c.L * fl;                                            // shifted h_0
            if (i == 0) {  // Eq. 31 vanishes at p = 0, u = 0
                A[own0_at(site, 0)] = g;
                A[own0_at(site, 1)] = (float)hq;
                A[own0_at(site, 2)] = 0.f;
            } else {
                P[gh_at(i, site, 0)] = g;
                P[gh_at(i, site, 1)] = (float)hq;
                P[f_at(i, site)] = 0.f;
            }
        }
        A[own0_at(site, 3)] = (float)fl;
        for (int k = 0; k < 4; ++k) A[own1_at(site, k)] = 0.f;
    }
}

// FP16 storage: the same equilibrium start, each population stored as its
// deviation from the rest-equilibrium reference of the site it streams into.
__device__ __forceinline__ double init_T(const InitConst& c, double phi, double T0) {
    return init_site(c, phi, T0).T;
}

template <typename ST>
__global__ void init_16(const Inst* __restrict__ insts, int inst, InitConst c,
                          const double* __restrict__ phi0, const double* __restrict__ T0,
                          int parity) {
    const Inst& I = insts[inst];
    const int n = I.nx * I.ny;
    const int plane = (int)I.plane;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int x = k % I.nx, y = k / I.nx;
        const int idx = y * I.pitch + x;
        const double ph = phi0[k];
        const InitSite st = init_site(c, ph, T0[k]);
        const double H = st.H, fl = st.fl, T = st.T;
        ST* P = static_cast<ST*>(I.pop[parity]);
        float* A = I.aux[parity];
        const float phr = (float)ph, Tr = (float)T;
        for (int i = 0; i < 9; ++i) {
            const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
            const float wf = WGT(i);
            // destination of the link (the site itself behind a wall)
            int xd = x + CX(i), yd = y + CY(i);
            bool wall = false;
            if (xd < 0 || xd >= I.nx) {
                if (I.flags & kPeriodicX) xd = (xd + I.nx) % I.nx; else wall = true;
            }
            if (yd < 0 || yd >= I.ny) {
                if (I.flags & kPeriodicY) yd = (yd + I.ny) % I.ny; else wall = true;
            }
            const int kd = wall ? k : yd * I.nx + xd;
            const float phd = (float)phi0[kd];
            const float Td = (float)init_T(c, phi0[kd], T0[kd]);
            if (i == 0) {  // rest populations in FP32
                A[own0_at(idx, 0)] = (float)(w * ph);                                 // Eq. 24
                A[own0_at(idx, 1)] =
                    (float)(H - c.Cpref * T + w * c.Cp * T * (c.Cpref / c.Cp) - c.L * fl);  // shifted h_0
                A[own0_at(idx, 2)] = 0.f;
                continue;
            }
            P[gh_at(i, idx, 0)] = Bits16<ST>::from_d(w * ph - (double)(wf * phd));  // Eq. 24, u = 0
            P[gh_at(i, idx, 1)] =
                Bits16<ST>::from_d(w * c.Cp * T * (c.Cpref / c.Cp) - (double)(wf * I.Cpref * Td));  // Eq. 28
            P[f_at(i, idx)] = Bits16<ST>::from_f(0.f);  // Eq. 31 vanishes at p = 0, u = 0
        }
        A[own0_at(idx, 3)] = (float)fl;
        for (int k = 0; k < 4; ++k) A[own1_at(idx, k)] = 0.f;
        A[ref_at(idx, 0)] = phr;
        A[ref_at(idx, 1)] = Tr;
    }
}

// Reduction of the per-tile partials of the allocation-free step: thread t
// sums partials t, t + 256, ... in order, then a fixed shared-memory tree
// combines the 256 sums, so the result does not depend on scheduling. The
// partials are observable-major, so each observable's loads are coalesced.
constexpr int kRedThreads = 256;
__device__ __forceinline__ void reduce_range(int begin, int end,
                                             const double* __restrict__ partials, int stride,
                                             double* __restrict__ out) {
    __shared__ double red[kObs][kRedThreads];
    const int t = threadIdx.x;
    double acc[kObs];
#pragma unroll
    for (int j = 0; j < kObs; ++j) acc[j] = 0.0;
    for (int p = begin + t; p < end; p += kRedThreads) {
#pragma unroll
        for (int j = 0; j < kObs; ++j) {
            const double v = partials[(long long)j * stride + p];
            acc[j] = (j == 9) ? fmax(acc[j], v) : acc[j] + v;
        }
    }
#pragma unroll
    for (int j = 0; j < kObs; ++j) red[j][t] = acc[j];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
#pragma unroll
            for (int j = 0; j < kObs; ++j)
                red[j][t] = (j == 9) ? fmax(red[j][t], red[j][t + w]) : red[j][t] + red[j][t + w];
        }
        __syncthreads();
    }
    if (t < kObs) out[t] = red[t][0];
}

__global__ void __launch_bounds__(kRedThreads)
reduce_noalloc(int n_parts, const double* __restrict__ partials, double* __restrict__ out) {
    reduce_range(0, n_parts, partials, n_parts, out);
}

#endif  // LBM_HAS_PART(0)

template <int TX, int TY>
cudaError_t launch_tile(const Inst* d_inst, const Tile* d_tiles, int n_tiles, int parity,
                        int obs, double* d_partials, cudaStream_t s) {
    if (obs)
        step_fp32<TX, TY, true><<<n_tiles, TX * TY, 0, s>>>(d_inst, d_tiles, parity, d_partials);
    else
        step_fp32<TX, TY, false><<<n_tiles, TX * TY, 0, s>>>(d_inst, d_tiles, parity, d_partials);
    return cudaGetLastError();
}

template <int WARPS, int MINB, typename ST>
cudaError_t launch_strip_w(const Inst* d_inst, const Item* d_items, int n_items, int parity,
                           int obs, double* d_partials, cudaStream_t s) {
    const int blocks = (n_items + WARPS - 1) / WARPS;
    if (obs)
        step_strip<WARPS, MINB, true, ST><<<blocks, WARPS * 32, 0, s>>>(d_inst, d_items, n_items,
                                                                       parity, d_partials);
    else
        step_strip<WARPS, MINB, false, ST><<<blocks, WARPS * 32, 0, s>>>(d_inst, d_items, n_items,
                                                                        parity, d_partials);
    return cudaGetLastError();
}

// Staged launches: ring depth and dynamic shared memory of a variant.
template <int WARPS, int MINB, int STG, typename ST>
struct Staged {
    static constexpr int kSmem = WARPS * warp_smem_floats<ST, STG>() * (int)sizeof(float);
    static cudaError_t prepare() {
        cudaError_t e = cudaFuncSetAttribute(step_strip_staged<WARPS, MINB, STG, false, ST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_strip_staged<WARPS, MINB, STG, true, ST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        return e;
    }
    static int resident_warps() {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, step_strip_staged<WARPS, MINB, STG, false, ST>, WARPS * 32, kSmem) != cudaSuccess)
            return 0;
        return per_sm * sms * WARPS;
    }
    static cudaError_t launch(const Inst* d_inst, const Item* d_items, int n_items, int parity,
                              int obs, double* d_partials, cudaStream_t s) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((n_items + WARPS - 1) / WARPS);
        cfg.blockDim = dim3(WARPS * 32);
        cfg.dynamicSmemBytes = kSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (obs)
            return cudaLaunchKernelEx(&cfg, step_strip_staged<WARPS, MINB, STG, true, ST>, d_inst,
                                      d_items, n_items, parity, d_partials);
        return cudaLaunchKernelEx(&cfg, step_strip_staged<WARPS, MINB, STG, false, ST>, d_inst,
                                  d_items, n_items, parity, d_partials);
    }
};

// Dispatch over the supported staged variants (warps per CTA, register
// budget): the ring depth follows from what the register budget leaves
// resident per SM, keeping every variant's shared memory within ~210 KB/SM.
template <typename ST, typename F>
auto staged_dispatch(int warps, int regs, F&& f) -> decltype(f(Staged<4, 3, 3, ST>())) {
    if (warps == 4 && regs == 128) return f(Staged<4, 4, 3, ST>());
    if (warps == 4 && regs == 255) return f(Staged<4, 2, 5, ST>());
    if (warps == 8 && regs == 128) return f(Staged<8, 2, 3, ST>());
    if (warps == 2 && regs == 128) return f(Staged<2, 8, 3, ST>());
    return f(Staged<4, 3, 3, ST>());
}

// Warps resident at once for a plain strip variant.
template <int WARPS, int MINB, typename ST>
int plain_resident_warps() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_strip<WARPS, MINB, false, ST>,
                                                      WARPS * 32, 0) != cudaSuccess)
        return 0;
    return per_sm * sms * WARPS;
}

// Persistent launches: the kernel of a (warps, regs, storage) variant, and
// the co-resident grid for it.
template <int WARPS, int MINB, int STG, typename ST>
struct Persist {
    static constexpr int kSmem = WARPS * warp_smem_floats<ST, STG>() * (int)sizeof(float);
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(step_strip_persistent<WARPS, MINB, STG, ST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    }
    static int grid(int n_items) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (prepare() != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, step_strip_persistent<WARPS, MINB, STG, ST>, WARPS * 32, kSmem) != cudaSuccess)
            return 0;
        const int want = (n_items + WARPS - 1) / WARPS;
        return std::max(1, std::min(want, per_sm * sms));
    }
    static cudaError_t launch(int grid, const Inst* d_inst, const Item* d_items, int n_items,
                              int parity0, int nsteps, unsigned* bar, int* err,
                              unsigned long long limit_ns, cudaStream_t s) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(WARPS * 32);
        cfg.dynamicSmemBytes = kSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, step_strip_persistent<WARPS, MINB, STG, ST>, d_inst,
                                  d_items, n_items, parity0, nsteps, bar, err, limit_ns);
    }
};

// Dispatch of a persistent call F over the supported strip variants: the
// row-staged ones (ring depths of the staged kernels) and the plain ones.
template <typename ST, typename F>
auto persist_dispatch_staged(int warps, int regs, F&& f) -> decltype(f(Persist<4, 3, 3, ST>())) {
    if (warps == 4 && regs == 128) return f(Persist<4, 4, 3, ST>());
    if (warps == 4 && regs == 255) return f(Persist<4, 2, 5, ST>());
    if (warps == 8 && regs == 128) return f(Persist<8, 2, 3, ST>());
    if (warps == 2 && regs == 128) return f(Persist<2, 8, 3, ST>());
    return f(Persist<4, 3, 3, ST>());
}
template <typename ST, typename F>
auto persist_dispatch_plain(int warps, int regs, F&& f) -> decltype(f(Persist<4, 3, 0, ST>())) {
    if (warps == 4 && regs == 128) return f(Persist<4, 4, 0, ST>());
    if (warps == 4 && regs == 168) return f(Persist<4, 3, 0, ST>());
    if (warps == 4 && regs == 255) return f(Persist<4, 1, 0, ST>());
    if (warps == 8 && regs == 128) return f(Persist<8, 2, 0, ST>());
    return f(Persist<2, 8, 0, ST>());
}

template <typename ST>
cudaError_t launch_strip_st(int warps, int regs, const Inst* d_inst, const Item* d_items,
                            int n_items, int parity, int obs, double* d_partials, cudaStream_t s) {
    // regs: register budget per thread (128, 168 or 255) via the minimum
    // number of resident CTAs requested from the compiler
    if (warps == 4 && regs == 128) return launch_strip_w<4, 4, ST>(d_inst, d_items, n_items, parity, obs, d_partials, s);
    if (warps == 4 && regs == 168) return launch_strip_w<4, 3, ST>(d_inst, d_items, n_items, parity, obs, d_partials, s);
    if (warps == 4 && regs == 255) return launch_strip_w<4, 1, ST>(d_inst, d_items, n_items, parity, obs, d_partials, s);
    if (warps == 8 && regs == 128) return launch_strip_w<8, 2, ST>(d_inst, d_items, n_items, parity, obs, d_partials, s);
    if (warps == 2 && regs == 128) return launch_strip_w<2, 8, ST>(d_inst, d_items, n_items, parity, obs, d_partials, s);
    return cudaErrorInvalidValue;
}

// BF16 storage is built for the two four-warp staged variants only.
using bf16 = __nv_bfloat16;
template <typename F>
auto staged_dispatch_bf16(int regs, F&& f) -> decltype(f(Staged<4, 3, 3, bf16>())) {
    if (regs == 128) return f(Staged<4, 4, 3, bf16>());
    return f(Staged<4, 3, 3, bf16>());
}
template <typename F>
auto persist_dispatch_bf16(int regs, F&& f) -> decltype(f(Persist<4, 3, 3, bf16>())) {
    if (regs == 128) return f(Persist<4, 4, 3, bf16>());
    return f(Persist<4, 3, 3, bf16>());
}

// Block launches: the (warps, regs) variants.
template <int WARPS, int MINB, typename ST>
struct Block {
    static constexpr int kSmem = WARPS * BlockWarp<ST>::kBytes;
    static cudaError_t prepare() {
        cudaError_t e = cudaFuncSetAttribute(step_block<WARPS, MINB, false, ST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_block<WARPS, MINB, true, ST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_block_persistent<WARPS, MINB, ST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        return e;
    }
    static int resident_warps() {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (prepare() != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, step_block<WARPS, MINB, false, ST>, WARPS * 32, kSmem) != cudaSuccess)
            return 0;
        return per_sm * sms * WARPS;
    }
    static cudaError_t launch(const Inst* d_inst, const Item* d_items, int n_items, int parity,
                              int obs, double* d_partials, int* d_err, cudaStream_t s) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((n_items + WARPS - 1) / WARPS);
        cfg.blockDim = dim3(WARPS * 32);
        cfg.dynamicSmemBytes = kSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (obs)
            return cudaLaunchKernelEx(&cfg, step_block<WARPS, MINB, true, ST>, d_inst, d_items, n_items,
                                      parity, d_partials, d_err);
        return cudaLaunchKernelEx(&cfg, step_block<WARPS, MINB, false, ST>, d_inst, d_items, n_items,
                                  parity, d_partials, d_err);
    }
    static int grid(int n_items) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (prepare() != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, step_block_persistent<WARPS, MINB, ST>, WARPS * 32, kSmem) != cudaSuccess)
            return 0;
        const int want = (n_items + WARPS - 1) / WARPS;
        return std::max(1, std::min(want, per_sm * sms));
    }
    static cudaError_t persist(int grid, const Inst* d_inst, const Item* d_items, int n_items,
                               int parity0, int nsteps, unsigned* bar, int* err,
                               unsigned long long limit_ns, cudaStream_t s) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(WARPS * 32);
        cfg.dynamicSmemBytes = kSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, step_block_persistent<WARPS, MINB, ST>, d_inst, d_items,
                                  n_items, parity0, nsteps, bar, err, limit_ns);
    }
};
template <typename ST, typename F>
auto block_dispatch(int warps, int regs, F&& f) -> decltype(f(Block<4, 4, ST>())) {
    if (warps == 4 && regs == 168) return f(Block<4, 3, ST>());
    if (warps == 8 && regs == 128) return f(Block<8, 2, ST>());
    return f(Block<4, 4, ST>());
}

// The staged or plain strip variants of one storage type, each reached by
// (warps, regs); the calls check nothing (the dispatchers below do).
template <typename ST, bool STAGED>
struct StripKind;
template <typename ST>
struct StripKind<ST, true> {
    template <typename F>
    static auto on(int warps, int regs, F&& f) {
        if constexpr (std::is_same_v<ST, bf16>) return staged_dispatch_bf16(regs, f);
        else return staged_dispatch<ST>(warps, regs, f);
    }
    template <typename F>
    static auto on_persist(int warps, int regs, F&& f) {
        if constexpr (std::is_same_v<ST, bf16>) return persist_dispatch_bf16(regs, f);
        else return persist_dispatch_staged<ST>(warps, regs, f);
    }
};
template <typename ST>
struct StripKind<ST, false> {
    template <typename F>
    static auto on_persist(int warps, int regs, F&& f) {
        return persist_dispatch_plain<ST>(warps, regs, f);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// The strip kernels of one storage type and kind, as compiled in their part
// ---------------------------------------------------------------------------
#if LBM_PART != 0
template <typename ST, bool STAGED>
cudaError_t StripPart<ST, STAGED>::launch(int warps, int regs, const Inst* d_inst,
                                          const Item* d_items, int n_items, int parity, int obs,
                                          double* d_partials, cudaStream_t s) {
    if constexpr (STAGED) {
        auto go = [&](auto v) {
            return decltype(v)::launch(d_inst, d_items, n_items, parity, obs, d_partials, s);
        };
        return StripKind<ST, true>::on(warps, regs, go);
    } else {
        return launch_strip_st<ST>(warps, regs, d_inst, d_items, n_items, parity, obs, d_partials,
                                   s);
    }
}

template <typename ST, bool STAGED>
cudaError_t StripPart<ST, STAGED>::prepare(int warps, int regs) {
    if constexpr (STAGED) {
        auto go = [](auto v) { return decltype(v)::prepare(); };
        return StripKind<ST, true>::on(warps, regs, go);
    } else {
        return cudaSuccess;
    }
}

template <typename ST, bool STAGED>
int StripPart<ST, STAGED>::resident_warps(int warps, int regs) {
    if constexpr (STAGED) {
        auto go = [](auto v) { return decltype(v)::resident_warps(); };
        return StripKind<ST, true>::on(warps, regs, go);
    } else {
        if (warps == 4 && regs == 128) return plain_resident_warps<4, 4, ST>();
        if (warps == 4 && regs == 255) return plain_resident_warps<4, 1, ST>();
        if (warps == 8 && regs == 128) return plain_resident_warps<8, 2, ST>();
        if (warps == 2 && regs == 128) return plain_resident_warps<2, 8, ST>();
        return plain_resident_warps<4, 3, ST>();
    }
}

template <typename ST, bool STAGED>
int StripPart<ST, STAGED>::persist_grid(int warps, int regs, int n_items) {
    auto g = [&](auto v) { return decltype(v)::grid(n_items); };
    return StripKind<ST, STAGED>::on_persist(warps, regs, g);
}

template <typename ST, bool STAGED>
cudaError_t StripPart<ST, STAGED>::persist_launch(int warps, int regs, int grid,
                                                  const Inst* d_inst, const Item* d_items,
                                                  int n_items, int parity0, int nsteps,
                                                  unsigned* d_bar, int* d_err,
                                                  unsigned long long limit_ns, cudaStream_t s) {
    auto go = [&](auto v) {
        return decltype(v)::launch(grid, d_inst, d_items, n_items, parity0, nsteps, d_bar, d_err,
                                   limit_ns, s);
    };
    return StripKind<ST, STAGED>::on_persist(warps, regs, go);
}
#endif

#if LBM_PART == 1
template struct StripPart<float, true>;
#elif LBM_PART == 2
template struct StripPart<float, false>;
#elif LBM_PART == 3
template struct StripPart<__half, true>;
#elif LBM_PART == 4
template struct StripPart<__half, false>;
#elif LBM_PART == 5
template struct StripPart<__nv_bfloat16, true>;
#endif

// ---------------------------------------------------------------------------
// The block kernels of one storage type, as compiled in their part
// ---------------------------------------------------------------------------
#if LBM_PART < 0 || LBM_PART >= 6
template <typename ST>
cudaError_t BlockPart<ST>::launch(int warps, int regs, const Inst* d_inst, const Item* d_items,
                                  int n_items, int parity, int obs, double* d_partials, int* d_err,
                                  cudaStream_t s) {
    auto go = [&](auto v) {
        return decltype(v)::launch(d_inst, d_items, n_items, parity, obs, d_partials, d_err, s);
    };
    return block_dispatch<ST>(warps, regs, go);
}
template <typename ST>
cudaError_t BlockPart<ST>::prepare(int warps, int regs) {
    auto go = [](auto v) { return decltype(v)::prepare(); };
    return block_dispatch<ST>(warps, regs, go);
}
template <typename ST>
int BlockPart<ST>::resident_warps(int warps, int regs) {
    auto go = [](auto v) { return decltype(v)::resident_warps(); };
    return block_dispatch<ST>(warps, regs, go);
}
template <typename ST>
int BlockPart<ST>::persist_grid(int warps, int regs, int n_items) {
    auto go = [&](auto v) { return decltype(v)::grid(n_items); };
    return block_dispatch<ST>(warps, regs, go);
}
template <typename ST>
cudaError_t BlockPart<ST>::persist_launch(int warps, int regs, int grid, const Inst* d_inst,
                                          const Item* d_items, int n_items, int parity0, int nsteps,
                                          unsigned* d_bar, int* d_err, unsigned long long limit_ns,
                                          cudaStream_t s) {
    auto go = [&](auto v) {
        return decltype(v)::persist(grid, d_inst, d_items, n_items, parity0, nsteps, d_bar, d_err,
                                    limit_ns, s);
    };
    return block_dispatch<ST>(warps, regs, go);
}
#endif
#if LBM_PART == 6 || LBM_PART < 0
template struct BlockPart<float>;
#endif
#if LBM_PART == 7 || LBM_PART < 0
template struct BlockPart<__half>;
#endif
#if LBM_PART == 8 || LBM_PART < 0
template struct BlockPart<__nv_bfloat16>;
#endif

// ---------------------------------------------------------------------------
// Storage dispatch and the tile, initialisation and reduction kernels
// ---------------------------------------------------------------------------
#if LBM_HAS_PART(0)
namespace {
// F applied to the StripPart of `storage` (FP32, FP16 or BF16) and kind.
template <bool STAGED, typename F>
auto on_storage(int storage, F&& f) {
    if (storage == LBM_STORE_FP16) return f(StripPart<__half, STAGED>());
    if constexpr (STAGED)
        if (storage == LBM_STORE_BF16) return f(StripPart<__nv_bfloat16, true>());
    return f(StripPart<float, STAGED>());
}
}  // namespace

cudaError_t launch_step_strip(int warps, int regs, int storage, const Inst* d_inst,
                              const Item* d_items, int n_items, int parity, int obs,
                              double* d_partials, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (storage != LBM_STORE_FP32 && storage != LBM_STORE_FP16) return cudaErrorNotSupported;
    if (!strip_supported(warps, regs)) return cudaErrorInvalidValue;
    auto go = [&](auto part) {
        return decltype(part)::launch(warps, regs, d_inst, d_items, n_items, parity, obs,
                                      d_partials, s);
    };
    return on_storage<false>(storage, go);
}

bool staged_supported(int warps, int regs, int storage) {
    if (storage == LBM_STORE_BF16) return warps == 4 && (regs == 128 || regs == 168);
    return (storage == LBM_STORE_FP32 || storage == LBM_STORE_FP16) && strip_supported(warps, regs);
}

cudaError_t prepare_staged(int warps, int regs, int storage) {
    if (!staged_supported(warps, regs, storage)) return cudaErrorInvalidValue;
    auto go = [&](auto part) { return decltype(part)::prepare(warps, regs); };
    return on_storage<true>(storage, go);
}

cudaError_t launch_step_staged(int warps, int regs, int storage, const Inst* d_inst,
                               const Item* d_items, int n_items, int parity, int obs,
                               double* d_partials, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (!staged_supported(warps, regs, storage)) return cudaErrorInvalidValue;
    auto go = [&](auto part) {
        return decltype(part)::launch(warps, regs, d_inst, d_items, n_items, parity, obs,
                                      d_partials, s);
    };
    return on_storage<true>(storage, go);
}

int strip_resident_warps(int staged, int warps, int regs, int storage) {
    if (!strip_supported(warps, regs)) return 0;
    auto go = [&](auto part) { return decltype(part)::resident_warps(warps, regs); };
    if (staged) {
        if (!staged_supported(warps, regs, storage)) return 0;
        return on_storage<true>(storage, go);
    }
    if (storage != LBM_STORE_FP32 && storage != LBM_STORE_FP16) return 0;  // plain: FP32, FP16
    return on_storage<false>(storage, go);
}

int persistent_grid(int staged, int warps, int regs, int storage, int n_items) {
    if (!strip_supported(warps, regs) || n_items <= 0) return 0;
    auto go = [&](auto part) { return decltype(part)::persist_grid(warps, regs, n_items); };
    if (staged) {
        if (!staged_supported(warps, regs, storage)) return 0;
        return on_storage<true>(storage, go);
    }
    if (storage != LBM_STORE_FP32 && storage != LBM_STORE_FP16) return 0;
    return on_storage<false>(storage, go);
}

cudaError_t launch_step_strip_persistent(int staged, int warps, int regs, int storage, int grid,
                                         const Inst* d_inst, const Item* d_items, int n_items,
                                         int parity0, int nsteps, unsigned* d_bar, int* d_err,
                                         unsigned long long limit_ns, cudaStream_t s) {
    if (!strip_supported(warps, regs) || grid <= 0) return cudaErrorInvalidValue;
    if (n_items <= 0 || nsteps <= 0) return cudaSuccess;
    auto go = [&](auto part) {
        return decltype(part)::persist_launch(warps, regs, grid, d_inst, d_items, n_items,
                                              parity0, nsteps, d_bar, d_err, limit_ns, s);
    };
    if (staged) {
        if (!staged_supported(warps, regs, storage)) return cudaErrorInvalidValue;
        return on_storage<true>(storage, go);
    }
    if (storage == LBM_STORE_BF16) return cudaErrorInvalidValue;
    if (storage != LBM_STORE_FP32 && storage != LBM_STORE_FP16) return cudaErrorNotSupported;
    return on_storage<false>(storage, go);
}


namespace {
template <typename F>
auto on_block_storage(int storage, F&& f) {
    if (storage == LBM_STORE_FP16) return f(BlockPart<__half>());
    if (storage == LBM_STORE_BF16) return f(BlockPart<__nv_bfloat16>());
    return f(BlockPart<float>());
}
}  // namespace

bool block_supported(int warps, int regs) {
    return (warps == 4 && (regs == 128 || regs == 168)) || (warps == 8 && regs == 128);
}

cudaError_t prepare_block(int warps, int regs, int storage) {
    if (!block_supported(warps, regs)) return cudaErrorInvalidValue;
    auto go = [&](auto part) { return decltype(part)::prepare(warps, regs); };
    return on_block_storage(storage, go);
}

cudaError_t launch_step_block(int warps, int regs, int storage, const Inst* d_inst,
                              const Item* d_items, int n_items, int parity, int obs,
                              double* d_partials, int* d_err, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (!block_supported(warps, regs)) return cudaErrorInvalidValue;
    auto go = [&](auto part) {
        return decltype(part)::launch(warps, regs, d_inst, d_items, n_items, parity, obs, d_partials,
                                      d_err, s);
    };
    return on_block_storage(storage, go);
}

int block_resident_warps(int warps, int regs, int storage) {
    if (!block_supported(warps, regs)) return 0;
    auto go = [&](auto part) { return decltype(part)::resident_warps(warps, regs); };
    return on_block_storage(storage, go);
}

int block_persistent_grid(int warps, int regs, int storage, int n_items) {
    if (!block_supported(warps, regs) || n_items <= 0) return 0;
    auto go = [&](auto part) { return decltype(part)::persist_grid(warps, regs, n_items); };
    return on_block_storage(storage, go);
}

cudaError_t launch_step_block_persistent(int warps, int regs, int storage, int grid,
                                         const Inst* d_inst, const Item* d_items, int n_items,
                                         int parity0, int nsteps, unsigned* d_bar, int* d_err,
                                         unsigned long long limit_ns, cudaStream_t s) {
    if (!block_supported(warps, regs) || grid <= 0) return cudaErrorInvalidValue;
    if (n_items <= 0 || nsteps <= 0) return cudaSuccess;
    auto go = [&](auto part) {
        return decltype(part)::persist_launch(warps, regs, grid, d_inst, d_items, n_items, parity0,
                                              nsteps, d_bar, d_err, limit_ns, s);
    };
    return on_block_storage(storage, go);
}

cudaError_t launch_barrier_timeout_probe(unsigned* d_bar, int* d_err, unsigned long long limit_ns,
                                         cudaStream_t s) {
    barrier_timeout_probe<<<1, 32, 0, s>>>(d_bar, d_err, limit_ns);
    return cudaGetLastError();
}

bool strip_supported(int warps, int regs) {
    return (warps == 4 && (regs == 128 || regs == 168 || regs == 255)) ||
           (warps == 8 && regs == 128) || (warps == 2 && regs == 128);
}

bool tile_supported(int tx, int ty) {
    return (tx == 32 && ty == 8) || (tx == 32 && ty == 4) || (tx == 64 && ty == 4) ||
           (tx == 32 && ty == 16);
}

cudaError_t launch_step(int tx, int ty, int storage, const Inst* d_inst, const Tile* d_tiles,
                        int n_tiles, int parity, int obs, double* d_partials, cudaStream_t s) {
    if (storage != 0) return cudaErrorNotSupported;
    if (tx == 32 && ty == 8) return launch_tile<32, 8>(d_inst, d_tiles, n_tiles, parity, obs, d_partials, s);
    if (tx == 32 && ty == 4) return launch_tile<32, 4>(d_inst, d_tiles, n_tiles, parity, obs, d_partials, s);
    if (tx == 64 && ty == 4) return launch_tile<64, 4>(d_inst, d_tiles, n_tiles, parity, obs, d_partials, s);
    if (tx == 32 && ty == 16) return launch_tile<32, 16>(d_inst, d_tiles, n_tiles, parity, obs, d_partials, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_noalloc(const Inst& I, int tiles_x, int n_tiles, double* scratch,
                                double* d_obs, cudaStream_t s) {
    step_tile_noalloc<true><<<n_tiles, 256, 0, s>>>(I, tiles_x, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_noalloc<<<1, kRedThreads, 0, s>>>(n_tiles, scratch, d_obs);
    return cudaGetLastError();
}

cudaError_t launch_init(const Inst* d_inst, int inst, int n_sites, int storage, InitConst c,
                        const double* d_phi0, const double* d_T0, int parity, cudaStream_t s) {
    const int threads = 256;
    int blocks = (n_sites + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (storage == LBM_STORE_FP32)
        init_fp32<<<blocks, threads, 0, s>>>(d_inst, inst, c, d_phi0, d_T0, parity);
    else if (storage == LBM_STORE_FP16)
        init_16<__half><<<blocks, threads, 0, s>>>(d_inst, inst, c, d_phi0, d_T0, parity);
    else if (storage == LBM_STORE_BF16)
        init_16<__nv_bfloat16><<<blocks, threads, 0, s>>>(d_inst, inst, c, d_phi0, d_T0, parity);
    else
        return cudaErrorNotSupported;
    return cudaGetLastError();
}

#endif  // LBM_HAS_PART(0)

}  // namespace lbmk
