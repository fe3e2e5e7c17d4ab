/*
 * lbm_oracle.h -- FP64 CPU oracle for one time step of the phase-field lattice
 * Boltzmann (LB) method for freezing with volume change of Huang, Wang, Chai &
 * Shi, "Phase-field based lattice Boltzmann method for containerless freezing"
 * (arXiv 2403.16122), Sections 2 and 3.
 *
 * TEST INFRASTRUCTURE. This is the slow, plain, obviously-correct restatement
 * of the method that the CUDA library is checked against. Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never links or calls it. It shares no code, header or constant
 * table with the CUDA library.
 *
 * Conventions: lattice units (dx = dt = 1, Section 3.1), D2Q9 for all three
 * distribution sets (Eqs. 22-23). A site (x, y) has linear index y*nx + x.
 * Distribution planes are ordered g_0..g_8, h_0..h_8, f_0..f_8 (27 planes of
 * nx*ny doubles); the carried (lagged) scalar planes are ordered
 * f_l (liquid fraction), (phi u)_x, (phi u)_y, p, S (5 planes).
 *
 * Walls sit half-way between the last lattice row/column and a ghost layer
 * (Section 3.4). A non-periodic axis has a wall at both ends.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * except the parts listed as "parity unpinned" in the step routine's comment.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_params {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;     /* 1 periodic, 0 walls at both ends       */
    int32_t dirichlet_x_lo, dirichlet_x_hi;  /* thermal wall type: 1 = T held at */
    int32_t dirichlet_y_lo, dirichlet_y_hi;  /* T_w, 0 = adiabatic (Section 4.1)  */
    int32_t st_mask_liquid;             /* 1: F_s = (1 - f_s) mu_phi grad(phi)    */
    int32_t reserved;
    double W;              /* interface width (Eq. 3)                             */
    double sigma;          /* surface tension (Eq. 13)                            */
    double mobility;       /* M of Eq. 2; tau_g = M / c_s^2 + 1/2                 */
    double tau_f_liquid;   /* flow relaxation time in the liquid                  */
    double tau_h;          /* enthalpy relaxation time (Eq. 27)                   */
    double rho_l;          /* liquid density                                      */
    double rho_ratio_lg;   /* rho_l / rho_g                                       */
    double rho_ratio_sl;   /* rho_s / rho_l                                       */
    double mu_ratio_lg;    /* mu_l / mu_g                                         */
    double Ste;            /* Stefan number (Eq. 42), sets L = Cp (T_m - T_w)/Ste */
    double Cp, Cp_ref;     /* heat capacity and reference heat capacity (Eq. 28)  */
    double T_m, T_w;       /* melting temperature and cold-wall temperature       */
    double theta_deg;      /* contact angle of the wetting wall (Eq. 39)          */
    double pc_ramp;        /* width in phi of the window where phase change
                              switches on (solid forms only in the liquid)        */
    double normal_eps;     /* regularisation of the interface normal:
                              n = grad phi / sqrt(|grad phi|^2 + eps^2)           */
    double gx, gy;         /* gravity vector of the Boussinesq force (Section 4.3) */
    double beta_T;         /* volumetric expansion coefficient beta               */
    double T_ref;          /* reference temperature of the Boussinesq force       */
    double rho_0;          /* reference density rho_0 of the Boussinesq force     */
    double Cp_ratio_sl;    /* C_p,s / C_p,l (Section 4.2: 0.5); 1 = uniform       */
    double Cp_ratio_gl;    /* C_p,g / C_p,l                                       */
    double k_ratio_sl;     /* k_s / k_l (Section 4.2: 3.8); 1 = uniform           */
    double k_ratio_gl;     /* k_g / k_l                                           */
} oracle_params;

/* Observables of the most recent step (indices into the output array). */
enum {
    ORACLE_OBS_VOLUME = 0,     /* sum phi                                      */
    ORACLE_OBS_SOLID,          /* sum f_s                                      */
    ORACLE_OBS_ENTHALPY,       /* sum H                                        */
    ORACLE_OBS_MASS,           /* sum rho                                      */
    ORACLE_OBS_CONDENSED_MASS, /* sum f_s rho_s + (1 - f_s) phi rho_l          */
    ORACLE_OBS_MDOT,           /* sum mdot                                     */
    ORACLE_OBS_PHI_MDOT,       /* sum phi * mdot                               */
    ORACLE_OBS_SOLID_COL,      /* sum over y of f_s on column x = nx/2         */
    ORACLE_OBS_SOLID_ROW,      /* sum over x of f_s on row y = ny/2            */
    ORACLE_OBS_UMAX,           /* max |u|                                      */
    ORACLE_OBS_NONFINITE,      /* number of sites with a non-finite field      */
    ORACLE_OBS_COUNT
};

/* Macroscopic fields of the most recent step (plane order of oracle_fields). */
enum {
    ORACLE_FLD_PHI = 0, ORACLE_FLD_H, ORACLE_FLD_T, ORACLE_FLD_FS,
    ORACLE_FLD_MDOT, ORACLE_FLD_RHO, ORACLE_FLD_UX, ORACLE_FLD_UY,
    ORACLE_FLD_P, ORACLE_FLD_S, ORACLE_FLD_COUNT
};

typedef struct oracle_state oracle_state;

/* Returns 0, or -1 for invalid parameters, -2 when out of memory. */
int  oracle_create(const oracle_params* p, oracle_state** out);
void oracle_destroy(oracle_state* s);
/* Equilibrium start from phi0 and T0 (nx*ny each) at rest with p = 0. */
int  oracle_init(oracle_state* s, const double* phi0, const double* T0);
int  oracle_step(oracle_state* s, int64_t n);
int64_t oracle_step_count(const oracle_state* s);
/* Threads of the site loops: n > 0 sets them; returns the count in effect
   (1 without OpenMP). */
int oracle_set_threads(int n);
/* Sum over every step since oracle_init / oracle_set_state and every site of
   mdot (Eq. 19): the mass-source integral. */
double oracle_mdot_integral(const oracle_state* s);
/* pops: 27*nx*ny, aux: 5*nx*ny (layouts above). */
void oracle_get_state(const oracle_state* s, double* pops, double* aux);
void oracle_set_state(oracle_state* s, const double* pops, const double* aux);
void oracle_fields(const oracle_state* s, double* out);      /* 10*nx*ny */
void oracle_observables(const oracle_state* s, double* out); /* ORACLE_OBS_COUNT */
/* Derived constants: L, H_s, H_l, tau_g, kappa, beta, rho_g, rho_s, mu_l,
   mu_g, mu_s, tan(pi/2 - theta) (12 values). */
void oracle_derived(const oracle_state* s, double* out);

/* Pointwise pieces of the scheme, exposed for the pin tests. */
void oracle_lattice(int32_t* cx, int32_t* cy, double* w, int32_t* opp);
void oracle_geq(double phi, double ux, double uy, double* out9);
void oracle_heq(double H, double T, double Cp, double Cp_ref,
                double ux, double uy, double* out9);
void oracle_feq(double p, double rho, double ux, double uy, double* out9);
void oracle_force_F(double S, double fx, double fy, double ux, double uy,
                    double Ftx, double Fty, double* out9);
void oracle_source_G(double phi, double mdot, double dtx, double dty,
                     double lam, double nx_, double ny_, double* out9);
void oracle_closure(const oracle_state* s, double H, double phihat,
                    double* fs, double* T);
/* Isotropic gradient and Laplacian (Eq. 38) of a field at one site, with the
   oracle's ghost rules: kind 0 copies the adjacent lattice value across a
   wall, kind 1 applies the wetting condition (Eqs. 39-41). */
void oracle_stencil(const oracle_state* s, const double* field, int32_t x,
                    int32_t y, int32_t kind, double* gx, double* gy,
                    double* lap);
double oracle_ghost(const oracle_state* s, const double* field, int32_t x,
                    int32_t y, int32_t kind);

#ifdef __cplusplus
}
#endif
#endif
