/*
 * lbm_oracle.c -- FP64 CPU oracle: one time step of the phase-field LB method
 * for freezing with volume change (arXiv 2403.16122, Sections 2-3), written
 * as plain nested loops over the lattice in the order the paper builds the
 * scheme. TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).
 *
 * Readings of passages the paper leaves open, garbles or states in two ways:
 *   R1  Eq. 26's mobility relation names tau_f; the phase-field LB relaxes
 *       with tau_g, so tau_g = M / c_s^2 + 1/2.
 *   R2  Local tau_f = mu / (rho c_s^2) + 1/2 with rho, mu from Eq. 1;
 *       mu_l = rho_l c_s^2 (tau_f_liquid - 1/2), mu_g = mu_l / (mu_l/mu_g),
 *       mu_s = mu_l rho_s / rho_l. phi is clamped to [0, 1] inside Eq. 1.
 *   R3  The thermal model of Section 2.2 carries no phase field: T and the
 *       liquid fraction f_l follow from H alone by Eqs. 8-9, everywhere. The
 *       gas starts liquid-like (f_l = 1, H = Cp T + L), so the latent heat is
 *       uniform as Section 2.2 assumes when it drops div(rho u Delta H).
 *       Solid forms only in the liquid (Section 2): the solid fraction that
 *       enters Eq. 1, Eq. 19 and the solid forcing is f_s = chi(phihat) (1 - f_l),
 *       chi a linear ramp from 0 to 1 over phihat in
 *       [1/2 - pc_ramp/2, 1/2 + pc_ramp/2], phihat = sum_i g_i.
 *   R4  Pure substance: T_s = T_l = T_m, H_s = Cp T_m, H_l = Cp T_m + L (the
 *       second "H_s" after Eq. 9b is read as H_l).
 *   R5  div u in Eqs. 25-26 is mdot (Eq. 19): phi = sum g / (1 - mdot/2),
 *       and the last term of G_i is w_i phi mdot.
 *   R6  df_s/dt in mdot (Eq. 19) is the change of f_s by phase change over one
 *       step, chi(phihat^n) (f_l^{n-1} - f_l^n): the solid does not move, so
 *       only freezing or melting of the liquid content changes it.
 *   R7  The pressure gradient and the gradient of S inside F~ (Eq. 33) use the
 *       previous step's p and S (carried planes), which breaks the p <-> grad p
 *       circularity of Eq. 36.
 *   R8  n = grad phi / |grad phi| is undefined where grad phi vanishes, which
 *       happens at extrema of phi in the bulk where lambda is not zero; there
 *       the unit normal flips with the sign of an arbitrarily small gradient.
 *       The normal is regularised as n = grad phi / sqrt(|grad phi|^2 + eps^2)
 *       (eps = normal_eps, 1e-3 by default: |n| > 0.99999 across the interface
 *       core where |grad phi| ~ 1/W, and lambda n stays Lipschitz in the bulk).
 *   R9  "c_s^2 div S" in F~ is read as c_s^2 grad S (S is a scalar, dt = 1);
 *       the tensor of Eq. 33 is (u F~ + F~ u).
 *   R10 With st_mask_liquid the surface tension is (1 - f_s) mu_phi grad phi
 *       (Section 4.3 writes f_s; the stated purpose, a force only at the
 *       bubble-liquid interface, needs the liquid fraction).
 *   R11 The F_0 term of Eq. 36 is the first-order non-equilibrium part of the
 *       rest population that Eq. 30 implies, (tau_f - 1/2) Delta t F_0, with
 *       the local tau_f. (Eq. 36 prints tau Delta t F_0; a Chapman-Enskog
 *       expansion of Eq. 30, whose source carries 1 - 1/(2 tau_f), gives
 *       f_0 - f_0^eq = -tau dt d_t f_0^eq + (tau - 1/2) dt F_0, and the printed
 *       coefficient makes bulk phi depart from 1 without bound near a
 *       freezing wall.)
 *   R12 The solid interaction force of Eq. 35 is f = f_s (0 - u*) (u_s = 0),
 *       u = u* + f/2, and rho f enters F_i (Eq. 33).
 *   R13 Wetting ghosts (Eqs. 39-41): for a wall below row 0 the ghost at
 *       (x, -1) is phi(x,0) + tan(pi/2 - theta) |1.5 d_x phi(x,0) -
 *       0.5 d_x phi(x,1)|, d_x a central difference; the other walls are the
 *       same rotated. rho, p and S ghosts copy the adjacent lattice value.
 *       Where a tangential neighbour falls behind a second wall the adjacent
 *       lattice value is used; a corner ghost copies the corner site.
 *   R14 Dirichlet walls use anti-bounce-back for h:
 *       h_i = -h_ibar^* + 2 w_i Cp_ref T_w ; no-flux (g) and no-slip (f) walls
 *       use half-way bounce-back (Section 4.1).
 *   R22 The Boussinesq force of Section 4.3, F_g = -rho_0 g beta (T - T_ref),
 *       joins F at every site with the step's T (zero unless g, beta given).
 *   R23 Per-phase C_p and k mix by Eq. 1; tau_h - 1/2 scales with k / k_l;
 *       Eq. 9 keeps the melting-state datum (H_s = C_p,l T_m, H_l = H_s + L)
 *       and divides the sensible enthalpy by the local C_p.
 *   Parity unpinned (no closed form separates the alternatives; the choice
 *   defines the scheme): R7, R9, R12, the ramp width of R3 and the eps of R8.
 *   The carried planes are f_l, (phi u)_x, (phi u)_y, p, S.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 velocities and weights, Eqs. 22-23: i = 1..4 point E, N, W, S and
   i = 5..8 point NE, NW, SW, SE. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2 / 3 */

enum { SET_G = 0, SET_H = 1, SET_F = 2 };
enum { AUX_FL = 0, AUX_PHIUX, AUX_PHIUY, AUX_P, AUX_S, AUX_COUNT };

struct oracle_state {
    oracle_params p;
    int64_t n;        /* sites */
    int64_t step;
    /* derived constants */
    double L, Hs, Hl, tau_g, kappa, beta, rho_g, rho_s, mu_l, mu_g, mu_s, tan_w;
    double *pop, *pop_new; /* 27 planes, post-collision */
    double *aux, *aux_new; /* 5 carried planes          */
    double *pre;           /* 27 planes, post-streaming (pre-collision) */
    double *fld;           /* 10 planes of the step's macroscopic fields */
    double *pre_fl;        /* liquid fraction of the step */
    double mdot_int;       /* sum over steps and sites of mdot (Eq. 19) */
};

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* ---------------------------------------------------------------------- */
/* Pointwise pieces                                                        */
/* ---------------------------------------------------------------------- */

void oracle_lattice(int32_t* cx, int32_t* cy, double* w, int32_t* opp) {
    for (int i = 0; i < 9; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = WT[i];
        opp[i] = OPP[i];
    }
}

/* Eq. 24: g_i^eq = w_i phi (1 + c_i.u / c_s^2). */
void oracle_geq(double phi, double ux, double uy, double* out) {
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        out[i] = WT[i] * phi * (1.0 + cu / CS2);
    }
}

/* Eq. 28: total-enthalpy equilibrium of the Huang et al. (2013) model. */
void oracle_heq(double H, double T, double Cp, double Cp_ref, double ux,
                double uy, double* out) {
    double uu = ux * ux + uy * uy;
    out[0] = H - Cp_ref * T + WT[0] * Cp * T * (Cp_ref / Cp - uu / (2.0 * CS2));
    for (int i = 1; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        out[i] = WT[i] * Cp * T *
                 (Cp_ref / Cp + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
    }
}

/* Eq. 32: s_i(u). */
static double s_i(int i, double ux, double uy) {
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WT[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 31: pressure-based flow equilibrium. */
void oracle_feq(double p, double rho, double ux, double uy, double* out) {
    out[0] = p / CS2 * (WT[0] - 1.0) + rho * s_i(0, ux, uy);
    for (int i = 1; i < 9; ++i) out[i] = p / CS2 * WT[i] + rho * s_i(i, ux, uy);
}

/* Eq. 33: F_i = w_i [S + c_i.(F + rho f)/c_s^2
                       + (u F~ + F~ u):(c_i c_i - c_s^2 I) / (2 c_s^4)],
   with (fx, fy) = F + rho f and (Ftx, Fty) = F~. */
void oracle_force_F(double S, double fx, double fy, double ux, double uy,
                    double Ftx, double Fty, double* out) {
    for (int i = 0; i < 9; ++i) {
        double c[2] = {(double)CX[i], (double)CY[i]};
        double u[2] = {ux, uy};
        double ft[2] = {Ftx, Fty};
        double tens = 0.0; /* (u F~ + F~ u):(c c - c_s^2 I) */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double A = u[a] * ft[b] + ft[a] * u[b];
                double Q = c[a] * c[b] - (a == b ? CS2 : 0.0);
                tens += A * Q;
            }
        out[i] = WT[i] * (S + (c[0] * fx + c[1] * fy) / CS2 + tens / (2.0 * CS2 * CS2));
    }
}

/* Eq. 25: G_i = w_i c_i.[d_t(phi u) + c_s^2 lambda n] / c_s^2 + w_i phi div u,
   with div u = mdot (reading R5). */
void oracle_source_G(double phi, double mdot, double dtx, double dty,
                     double lam, double nx_, double ny_, double* out) {
    double ax = dtx + CS2 * lam * nx_;
    double ay = dty + CS2 * lam * ny_;
    for (int i = 0; i < 9; ++i)
        out[i] = WT[i] * (CX[i] * ax + CY[i] * ay) / CS2 + WT[i] * phi * mdot;
}

/* Eqs. 8-9 with readings R3/R4: liquid fraction and temperature from H. */
/* Eq. 9 with the local heat capacity cp of the site (R23: the enthalpy datum
   is the melting state, H_s = C_p,l T_m and H_l = H_s + L, for every phase;
   the sensible branches divide by the mixture C_p of Eq. 1). */
static double liquid_fraction(const oracle_state* s, double H) {
    return clamp01((H - s->Hs) / s->L);                   /* Eq. 9a */
}
static double temperature(const oracle_state* s, double H, double fl, double cp) {
    return s->p.T_m + (H - s->Hs - s->L * fl) / cp;       /* Eq. 9b */
}

/* R3: solid only in the liquid content of a site. */
static double solid_fraction(const oracle_state* s, double fl, double phihat) {
    double chi = clamp01((phihat - 0.5) / s->p.pc_ramp + 0.5);
    return chi * (1.0 - fl);
}

/* Eq. 1 (reading R2: phi clamped to [0, 1]). */
static double mix(double fs, double phi, double zs, double zl, double zg) {
    double ph = clamp01(phi);
    return fs * zs + (1.0 - fs) * ph * zl + (1.0 - fs) * (1.0 - ph) * zg;
}

/* Local heat capacity and enthalpy relaxation time (Eq. 1 for C_p and k;
   R23: tau_h - 1/2 proportional to k, the liquid's given by tau_h). */
static double heat_capacity(const oracle_state* s, double fs, double phi) {
    const oracle_params* p = &s->p;
    return mix(fs, phi, p->Cp * p->Cp_ratio_sl, p->Cp, p->Cp * p->Cp_ratio_gl);
}
static double tau_enthalpy(const oracle_state* s, double fs, double phi) {
    const oracle_params* p = &s->p;
    return mix(fs, phi, p->k_ratio_sl, 1.0, p->k_ratio_gl) * (p->tau_h - 0.5) + 0.5;
}

/* Pointwise closure for tests: phihat stands in for phi in the mixture. */
void oracle_closure(const oracle_state* s, double H, double phihat, double* fs,
                    double* T) {
    double fl = liquid_fraction(s, H);
    *fs = solid_fraction(s, fl, phihat);
    *T = temperature(s, H, fl, heat_capacity(s, *fs, phihat));
}

/* ---------------------------------------------------------------------- */
/* Lattice access, boundary links, ghosts                                  */
/* ---------------------------------------------------------------------- */

static int64_t site(const oracle_state* s, int x, int y) {
    return (int64_t)y * s->p.nx + x;
}

/* Population arriving at (x, y) along c_i: the post-collision value leaving
   (x, y) - c_i, or the half-way wall rule when that source lies behind a wall
   (Section 4.1; R14 for Dirichlet walls in the enthalpy set). */
static double pull(const oracle_state* s, const double* post, int set, int i,
                   int x, int y) {
    const oracle_params* p = &s->p;
    int xs = x - CX[i], ys = y - CY[i];
    int wall = 0, dirichlet = 0;
    if (xs < 0 || xs >= p->nx) {
        if (p->periodic_x) xs = (xs + p->nx) % p->nx;
        else { wall = 1; dirichlet |= xs < 0 ? p->dirichlet_x_lo : p->dirichlet_x_hi; }
    }
    if (ys < 0 || ys >= p->ny) {
        if (p->periodic_y) ys = (ys + p->ny) % p->ny;
        else { wall = 1; dirichlet |= ys < 0 ? p->dirichlet_y_lo : p->dirichlet_y_hi; }
    }
    if (!wall) return post[(int64_t)(set * 9 + i) * s->n + site(s, xs, ys)];
    double back = post[(int64_t)(set * 9 + OPP[i]) * s->n + site(s, x, y)];
    if (set == SET_H && dirichlet) return -back + 2.0 * WT[i] * p->Cp_ref * p->T_w;
    return back;
}

/* Lattice value at a column/row index that may sit one cell behind a wall on
   the tangential axis: periodic axes wrap, walled axes use the adjacent
   lattice value (R13). */
static int wrap_or_clamp(int v, int n, int periodic) {
    if (v >= 0 && v < n) return v;
    if (periodic) return (v + n) % n;
    return v < 0 ? 0 : n - 1;
}

/* Value of a field at (x, y), which may lie one cell outside the lattice.
   kind 0: ghosts copy the adjacent lattice value; kind 1: wetting ghost. */
double oracle_ghost(const oracle_state* s, const double* Z, int32_t x, int32_t y,
                    int32_t kind) {
    const oracle_params* p = &s->p;
    int nx = p->nx, ny = p->ny;
    int outx = 0, outy = 0;
    if (x < 0 || x >= nx) {
        if (p->periodic_x) x = (x + nx) % nx; else outx = 1;
    }
    if (y < 0 || y >= ny) {
        if (p->periodic_y) y = (y + ny) % ny; else outy = 1;
    }
    if (!outx && !outy) return Z[site(s, x, y)];
    if (kind == 1 && outy && !outx) {
        /* wall normal to y: layers y0 (adjacent) and y1 (next) */
        int y0 = y < 0 ? 0 : ny - 1;
        int y1 = y < 0 ? 1 : ny - 2;
        int xm = wrap_or_clamp(x - 1, nx, p->periodic_x);
        int xp = wrap_or_clamp(x + 1, nx, p->periodic_x);
        double d0 = 0.5 * (Z[site(s, xp, y0)] - Z[site(s, xm, y0)]); /* Eq. 41 */
        double d1 = 0.5 * (Z[site(s, xp, y1)] - Z[site(s, xm, y1)]);
        double tang = 1.5 * d0 - 0.5 * d1;                            /* Eq. 40b */
        /* Eq. 39 with Eq. 40a: phi_adj - phi_ghost = -tan(pi/2-theta)|tang| */
        return Z[site(s, x, y0)] + s->tan_w * fabs(tang);
    }
    if (kind == 1 && outx && !outy) {
        int x0 = x < 0 ? 0 : nx - 1;
        int x1 = x < 0 ? 1 : nx - 2;
        int ym = wrap_or_clamp(y - 1, ny, p->periodic_y);
        int yp = wrap_or_clamp(y + 1, ny, p->periodic_y);
        double d0 = 0.5 * (Z[site(s, x0, yp)] - Z[site(s, x0, ym)]);
        double d1 = 0.5 * (Z[site(s, x1, yp)] - Z[site(s, x1, ym)]);
        double tang = 1.5 * d0 - 0.5 * d1;
        return Z[site(s, x0, y)] + s->tan_w * fabs(tang);
    }
    /* copy ghost (and corner ghosts for either kind) */
    int xc = outx ? (x < 0 ? 0 : nx - 1) : x;
    int yc = outy ? (y < 0 ? 0 : ny - 1) : y;
    return Z[site(s, xc, yc)];
}

/* Eq. 38: grad Z = sum_{i!=0} w_i c_i Z(x + c_i) / c_s^2,
           lap Z  = sum_{i!=0} 2 w_i [Z(x + c_i) - Z(x)] / c_s^2. */
void oracle_stencil(const oracle_state* s, const double* Z, int32_t x, int32_t y,
                    int32_t kind, double* gx, double* gy, double* lap) {
    double z0 = Z[site(s, x, y)];
    double sx = 0.0, sy = 0.0, sl = 0.0;
    for (int i = 1; i < 9; ++i) {
        double z = oracle_ghost(s, Z, x + CX[i], y + CY[i], kind);
        sx += WT[i] * CX[i] * z;
        sy += WT[i] * CY[i] * z;
        sl += 2.0 * WT[i] * (z - z0);
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
    *lap = sl / CS2;
}

/* ---------------------------------------------------------------------- */
/* Life cycle                                                              */
/* ---------------------------------------------------------------------- */

static int valid(const oracle_params* p) {
    if (p->nx < 3 || p->ny < 3) return 0;
    if (!(p->W > 0) || !(p->sigma >= 0) || !(p->mobility > 0)) return 0;
    if (!(p->tau_f_liquid > 0.5) || !(p->tau_h > 0.5)) return 0;
    if (!(p->rho_l > 0) || !(p->rho_ratio_lg > 0) || !(p->rho_ratio_sl > 0)) return 0;
    if (!(p->mu_ratio_lg > 0) || !(p->Ste > 0) || !(p->Cp > 0) || !(p->Cp_ref > 0)) return 0;
    if (!(p->T_w < p->T_m)) return 0;
    if (!(p->theta_deg > 0 && p->theta_deg < 180)) return 0;
    if (!(p->pc_ramp > 0)) return 0;
    if (!(p->normal_eps > 0)) return 0;
    if (!(p->Cp_ratio_sl > 0) || !(p->Cp_ratio_gl > 0)) return 0;
    if (!(p->k_ratio_sl > 0) || !(p->k_ratio_gl > 0)) return 0;
    return 1;
}

int oracle_create(const oracle_params* p, oracle_state** out) {
    *out = NULL;
    if (!p || !valid(p)) return -1;
    oracle_state* s = (oracle_state*)calloc(1, sizeof(oracle_state));
    if (!s) return -2;
    s->p = *p;
    s->n = (int64_t)p->nx * p->ny;
    s->L = p->Cp * (p->T_m - p->T_w) / p->Ste;   /* Eq. 42 */
    s->Hs = p->Cp * p->T_m;                     /* R4 */
    s->Hl = p->Cp * p->T_m + s->L;
    s->tau_g = p->mobility / CS2 + 0.5;         /* R1 */
    s->kappa = 1.5 * p->sigma * p->W;           /* Eq. 13 */
    s->beta = 12.0 * p->sigma / p->W;
    s->rho_g = p->rho_l / p->rho_ratio_lg;
    s->rho_s = p->rho_l * p->rho_ratio_sl;
    s->mu_l = p->rho_l * CS2 * (p->tau_f_liquid - 0.5); /* R2 */
    s->mu_g = s->mu_l / p->mu_ratio_lg;
    s->mu_s = s->mu_l * p->rho_ratio_sl;
    const double pi = acos(-1.0);
    s->tan_w = tan(pi / 2.0 - p->theta_deg * pi / 180.0);
    size_t np = (size_t)27 * s->n, na = (size_t)AUX_COUNT * s->n;
    s->pop = calloc(np, sizeof(double));
    s->pop_new = calloc(np, sizeof(double));
    s->pre = calloc(np, sizeof(double));
    s->aux = calloc(na, sizeof(double));
    s->aux_new = calloc(na, sizeof(double));
    s->fld = calloc((size_t)ORACLE_FLD_COUNT * s->n, sizeof(double));
    s->pre_fl = calloc((size_t)s->n, sizeof(double));
    if (!s->pop || !s->pop_new || !s->pre || !s->aux || !s->aux_new || !s->fld || !s->pre_fl) {
        oracle_destroy(s);
        return -2;
    }
    *out = s;
    return 0;
}

void oracle_destroy(oracle_state* s) {
    if (!s) return;
    free(s->pop); free(s->pop_new); free(s->pre);
    free(s->aux); free(s->aux_new); free(s->fld); free(s->pre_fl);
    free(s);
}

void oracle_derived(const oracle_state* s, double* o) {
    o[0] = s->L; o[1] = s->Hs; o[2] = s->Hl; o[3] = s->tau_g;
    o[4] = s->kappa; o[5] = s->beta; o[6] = s->rho_g; o[7] = s->rho_s;
    o[8] = s->mu_l; o[9] = s->mu_g; o[10] = s->mu_s; o[11] = s->tan_w;
}

/* Start at rest (u = 0, p = 0) with the distributions at equilibrium. The
   material is liquid-like before freezing starts (f_l = 1), so
   H = H_l + C_p (T0 - T_m) (Eq. 8) with C_p the mixture of liquid and gas. */
int oracle_init(oracle_state* s, const double* phi0, const double* T0) {
    const int64_t n = s->n;
    double eq[9];
    for (int64_t k = 0; k < n; ++k) {
        double cp0 = heat_capacity(s, 0.0, phi0[k]);
        double H = s->Hl + cp0 * (T0[k] - s->p.T_m);
        double fl = liquid_fraction(s, H);
        double fs = solid_fraction(s, fl, phi0[k]);
        double T = temperature(s, H, fl, heat_capacity(s, fs, phi0[k]));
        double rho = mix(fs, phi0[k], s->rho_s, s->p.rho_l, s->rho_g);
        oracle_geq(phi0[k], 0.0, 0.0, eq);
        for (int i = 0; i < 9; ++i) s->pop[(SET_G * 9 + i) * n + k] = eq[i];
        oracle_heq(H, T, heat_capacity(s, fs, phi0[k]), s->p.Cp_ref, 0.0, 0.0, eq);
        for (int i = 0; i < 9; ++i) s->pop[(SET_H * 9 + i) * n + k] = eq[i];
        oracle_feq(0.0, rho, 0.0, 0.0, eq);
        for (int i = 0; i < 9; ++i) s->pop[(SET_F * 9 + i) * n + k] = eq[i];
        s->aux[AUX_FL * n + k] = fl;
        s->aux[AUX_PHIUX * n + k] = 0.0;
        s->aux[AUX_PHIUY * n + k] = 0.0;
        s->aux[AUX_P * n + k] = 0.0;
        s->aux[AUX_S * n + k] = 0.0;
        double* F = s->fld;
        F[ORACLE_FLD_PHI * n + k] = phi0[k];
        F[ORACLE_FLD_H * n + k] = H;
        F[ORACLE_FLD_T * n + k] = T;
        F[ORACLE_FLD_FS * n + k] = fs;
        F[ORACLE_FLD_MDOT * n + k] = 0.0;
        F[ORACLE_FLD_RHO * n + k] = rho;
        F[ORACLE_FLD_UX * n + k] = 0.0;
        F[ORACLE_FLD_UY * n + k] = 0.0;
        F[ORACLE_FLD_P * n + k] = 0.0;
        F[ORACLE_FLD_S * n + k] = 0.0;
    }
    s->step = 0;
    s->mdot_int = 0.0;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* One time step                                                           */
/* ---------------------------------------------------------------------- */

static void step_once(oracle_state* s) {
    const oracle_params* p = &s->p;
    const int nx = p->nx, ny = p->ny;
    const int64_t n = s->n;
    double* F = s->fld;
    double* phi = F + ORACLE_FLD_PHI * n;
    double* Hf = F + ORACLE_FLD_H * n;
    double* Tf = F + ORACLE_FLD_T * n;
    double* fsf = F + ORACLE_FLD_FS * n;
    double* mdf = F + ORACLE_FLD_MDOT * n;
    double* rhof = F + ORACLE_FLD_RHO * n;
    double* flf = s->pre_fl;
    const double* fl_prev = s->aux + AUX_FL * n;
    const double* phiux_prev = s->aux + AUX_PHIUX * n;
    const double* phiuy_prev = s->aux + AUX_PHIUY * n;
    const double* p_prev = s->aux + AUX_P * n;
    const double* S_prev = s->aux + AUX_S * n;

    /* (1) Streaming: the left-hand sides of Eqs. 21, 27 and 30 move each
       post-collision population one link along c_i. */
    for (int set = 0; set < 3; ++set)
        for (int i = 0; i < 9; ++i)
#pragma omp parallel for
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x)
                    s->pre[(int64_t)(set * 9 + i) * n + site(s, x, y)] =
                        pull(s, s->pop, set, i, x, y);

    /* (2) Local macroscopic fields at the new time level. */
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t k = site(s, x, y);
            double H = 0.0, phihat = 0.0;
            for (int i = 0; i < 9; ++i) {
                H += s->pre[(SET_H * 9 + i) * n + k];      /* Eq. 29 */
                phihat += s->pre[(SET_G * 9 + i) * n + k];
            }
            double fl = liquid_fraction(s, H);             /* Eq. 9a, R3 */
            double chi = clamp01((phihat - 0.5) / p->pc_ramp + 0.5);
            double fs = chi * (1.0 - fl);
            double mdot = (1.0 - s->rho_s / p->rho_l) * chi * (fl_prev[k] - fl); /* Eq. 19, R6 */
            double ph = phihat / (1.0 - 0.5 * mdot);     /* Eq. 26, R5 */
            double T = temperature(s, H, fl, heat_capacity(s, fs, ph));  /* Eq. 9b, R23 */
            Hf[k] = H;
            Tf[k] = T;
            fsf[k] = fs;
            flf[k] = fl;
            mdf[k] = mdot;
            phi[k] = ph;
            rhof[k] = mix(fs, ph, s->rho_s, p->rho_l, s->rho_g); /* Eq. 1 */
        }

    /* (3) Gradients, forces, flow macroscopics and the three collisions. */
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t k = site(s, x, y);
            double ph = phi[k], fs = fsf[k], mdot = mdf[k], rho = rhof[k];
            double H = Hf[k], T = Tf[k];

            double gphx, gphy, lph, grx, gry, lr, gpx, gpy, lp, gSx, gSy, lS;
            oracle_stencil(s, phi, x, y, 1, &gphx, &gphy, &lph);    /* Eq. 38 */
            oracle_stencil(s, rhof, x, y, 0, &grx, &gry, &lr);
            oracle_stencil(s, p_prev, x, y, 0, &gpx, &gpy, &lp);    /* R7 */
            oracle_stencil(s, S_prev, x, y, 0, &gSx, &gSy, &lS);
            (void)lr; (void)lp; (void)lS;

            /* Eq. 12 with phi_l = 1, phi_g = 0; Eq. 11 (R10 for the mask). */
            double muphi = 4.0 * s->beta * (ph - 1.0) * ph * (ph - 0.5) - s->kappa * lph;
            double Fx = muphi * gphx, Fy = muphi * gphy;
            if (p->st_mask_liquid) { Fx *= (1.0 - fs); Fy *= (1.0 - fs); }
            /* F = F_s + F_g with the Boussinesq buoyancy of Section 4.3,
               F_g = -rho_0 g beta (T - T_ref), at every site (R22); zero
               unless gravity and beta are given. */
            Fx += -p->rho_0 * p->beta_T * (T - p->T_ref) * p->gx;
            Fy += -p->rho_0 * p->beta_T * (T - p->T_ref) * p->gy;

            const double* fpre = s->pre + (int64_t)(SET_F * 9) * n;
            double mx = 0.0, my = 0.0, fsum_ne0 = 0.0;
            for (int i = 0; i < 9; ++i) {
                double fi = fpre[i * n + k];
                mx += CX[i] * fi;
                my += CY[i] * fi;
                if (i) fsum_ne0 += fi;
            }
            double usx = (mx + 0.5 * Fx) / rho;              /* Eq. 34 */
            double usy = (my + 0.5 * Fy) / rho;
            double ffx = fs * (0.0 - usx), ffy = fs * (0.0 - usy); /* R12 */
            double ux = usx + 0.5 * ffx, uy = usy + 0.5 * ffy;     /* Eq. 35 */

            double S = rho * mdot + ux * grx + uy * gry;           /* Eq. 33 */
            double Ftx = Fx - gpx + CS2 * grx + CS2 * gSx;         /* R7, R9 */
            double Fty = Fy - gpy + CS2 * gry + CS2 * gSy;
            double mu = mix(fs, ph, s->mu_s, s->mu_l, s->mu_g);
            double tau_f = mu / (rho * CS2) + 0.5;                 /* R2 */
            double Fi[9];
            oracle_force_F(S, Fx + rho * ffx, Fy + rho * ffy, ux, uy, Ftx, Fty, Fi);
            double pnew = CS2 / (1.0 - WT[0]) *
                          (fsum_ne0 + 0.5 * S + (tau_f - 0.5) * Fi[0] +
                           rho * s_i(0, ux, uy)); /* Eq. 36, R11 */

            /* Phase field (Eqs. 21, 24, 25, 37). */
            double g2 = gphx * gphx + gphy * gphy;
            double gm = sqrt(g2 + p->normal_eps * p->normal_eps); /* R8 */
            double nnx = gphx / gm, nny = gphy / gm;
            double lam = 4.0 * ph * (1.0 - ph) / p->W;              /* Eq. 3 */
            double phiux = ph * ux, phiuy = ph * uy;
            double dtx = phiux - phiux_prev[k], dty = phiuy - phiuy_prev[k]; /* Eq. 37 */
            double Gi[9], geq[9];
            oracle_source_G(ph, mdot, dtx, dty, lam, nnx, nny, Gi);
            oracle_geq(ph, ux, uy, geq);
            const double* gpre = s->pre + (int64_t)(SET_G * 9) * n;
            for (int i = 0; i < 9; ++i) {
                double gi = gpre[i * n + k];
                s->pop_new[(int64_t)(SET_G * 9 + i) * n + k] =
                    gi - (gi - geq[i]) / s->tau_g + (1.0 - 0.5 / s->tau_g) * Gi[i];
            }

            /* Enthalpy (Eqs. 27-28). */
            double heq[9];
            oracle_heq(H, T, heat_capacity(s, fs, ph), p->Cp_ref, ux, uy, heq);
            const double tau_h = tau_enthalpy(s, fs, ph);
            const double* hpre = s->pre + (int64_t)(SET_H * 9) * n;
            for (int i = 0; i < 9; ++i) {
                double hi = hpre[i * n + k];
                s->pop_new[(int64_t)(SET_H * 9 + i) * n + k] = hi - (hi - heq[i]) / tau_h;
            }

            /* Flow (Eqs. 30-33). */
            double feq[9];
            oracle_feq(pnew, rho, ux, uy, feq);
            for (int i = 0; i < 9; ++i) {
                double fi = fpre[i * n + k];
                s->pop_new[(int64_t)(SET_F * 9 + i) * n + k] =
                    fi - (fi - feq[i]) / tau_f + (1.0 - 0.5 / tau_f) * Fi[i];
            }

            /* Carried planes for the next step. */
            s->aux_new[AUX_FL * n + k] = flf[k];
            s->aux_new[AUX_PHIUX * n + k] = phiux;
            s->aux_new[AUX_PHIUY * n + k] = phiuy;
            s->aux_new[AUX_P * n + k] = pnew;
            s->aux_new[AUX_S * n + k] = S;

            F[ORACLE_FLD_UX * n + k] = ux;
            F[ORACLE_FLD_UY * n + k] = uy;
            F[ORACLE_FLD_P * n + k] = pnew;
            F[ORACLE_FLD_S * n + k] = S;
        }

    /* The mass-source integral: this step's mdot of every site, in site
       order, added to the running FP64 sum. */
    for (int64_t k = 0; k < n; ++k) s->mdot_int += mdf[k];

    double* t = s->pop; s->pop = s->pop_new; s->pop_new = t;
    t = s->aux; s->aux = s->aux_new; s->aux_new = t;
    s->step += 1;
}

int oracle_step(oracle_state* s, int64_t n) {
    for (int64_t k = 0; k < n; ++k) step_once(s);
    return 0;
}

int64_t oracle_step_count(const oracle_state* s) { return s->step; }

/* Host threads of the site loops (OpenMP over lattice rows; each site's
   result depends only on the previous state, so the thread count does not
   change any value). Without OpenMP the oracle is single-threaded. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void oracle_get_state(const oracle_state* s, double* pops, double* aux) {
    if (pops) memcpy(pops, s->pop, sizeof(double) * 27 * (size_t)s->n);
    if (aux) memcpy(aux, s->aux, sizeof(double) * AUX_COUNT * (size_t)s->n);
}

double oracle_mdot_integral(const oracle_state* s) { return s->mdot_int; }

void oracle_set_state(oracle_state* s, const double* pops, const double* aux) {
    s->mdot_int = 0.0; /* a new run */
    if (pops) memcpy(s->pop, pops, sizeof(double) * 27 * (size_t)s->n);
    if (aux) memcpy(s->aux, aux, sizeof(double) * AUX_COUNT * (size_t)s->n);
}

void oracle_fields(const oracle_state* s, double* out) {
    memcpy(out, s->fld, sizeof(double) * ORACLE_FLD_COUNT * (size_t)s->n);
}

void oracle_observables(const oracle_state* s, double* o) {
    const int64_t n = s->n;
    const double* F = s->fld;
    for (int j = 0; j < ORACLE_OBS_COUNT; ++j) o[j] = 0.0;
    int xc = s->p.nx / 2, yc = s->p.ny / 2;
    for (int y = 0; y < s->p.ny; ++y)
        for (int x = 0; x < s->p.nx; ++x) {
            int64_t k = site(s, x, y);
            double ph = F[ORACLE_FLD_PHI * n + k], fs = F[ORACLE_FLD_FS * n + k];
            double md = F[ORACLE_FLD_MDOT * n + k];
            double ux = F[ORACLE_FLD_UX * n + k], uy = F[ORACLE_FLD_UY * n + k];
            double H = F[ORACLE_FLD_H * n + k], rho = F[ORACLE_FLD_RHO * n + k];
            double pr = F[ORACLE_FLD_P * n + k];
            o[ORACLE_OBS_VOLUME] += ph;
            o[ORACLE_OBS_SOLID] += fs;
            o[ORACLE_OBS_ENTHALPY] += H;
            o[ORACLE_OBS_MASS] += rho;
            o[ORACLE_OBS_CONDENSED_MASS] += fs * s->rho_s + (1.0 - fs) * clamp01(ph) * s->p.rho_l;
            o[ORACLE_OBS_MDOT] += md;
            o[ORACLE_OBS_PHI_MDOT] += ph * md;
            if (x == xc) o[ORACLE_OBS_SOLID_COL] += fs;
            if (y == yc) o[ORACLE_OBS_SOLID_ROW] += fs;
            double um = sqrt(ux * ux + uy * uy);
            if (um > o[ORACLE_OBS_UMAX]) o[ORACLE_OBS_UMAX] = um;
            if (!isfinite(ph) || !isfinite(H) || !isfinite(ux) || !isfinite(uy) ||
                !isfinite(pr))
                o[ORACLE_OBS_NONFINITE] += 1.0;
        }
}
