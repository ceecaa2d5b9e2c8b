/*
 * lbfs_oracle.h -- plain, slow FP64 CPU oracle of the enthalpy-based lattice
 * Boltzmann flux solver (LBFS) time step for ferrofluid-droplet freezing.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or execute this code; only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark use it.  It shares no source with the CUDA
 * library.
 *
 * Every function follows the paper's equations directly, per D2Q9 direction,
 * in FP64, with no algebraic shortcuts:
 *   Eq. 8 (enthalpy inversion), Eq. 11 (mixture rule), Eq. 13/20/28/29
 *   (equilibria), Eq. 44 (reconstruction at x - e_a dt), Eq. 45 (compatibility),
 *   Eq. 16/22/32/33 (non-equilibrium and starred distributions), Eq. 43 (face
 *   fluxes), Eq. 41/42 (sources and finite-volume sum), Sec. 3.4 third-order
 *   Runge-Kutta, Table 1 (step order), and the steady magnetic potential
 *   equation Eq. 4.
 */
#ifndef LBFS_ORACLE_H
#define LBFS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Case description.  Lattice units: dx = 1, D2Q9 with c = 1, c_s^2 = 1/3. */
typedef struct oracle_case {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;   /* 1 = periodic axis                          */
    int32_t thermal_dirichlet[4];     /* walls 0 left, 1 right, 2 bottom, 3 top      */
    double  wall_T[4];                /* wall temperature where Dirichlet            */
    int32_t mag_bc;                   /* 0 Dirichlet on every wall; 1 Dirichlet
                                         bottom/top, insulating left/right          */
    int32_t init;                     /* 0 sessile drop centred (nx/2, 0); 1 free drop
                                         centred (drop_x, drop_y); 2 uniform C = 1  */
    double  radius, drop_x, drop_y;
    double  T_init;
    double  H0, field_angle_deg;      /* far-field |H| and direction from +x         */
    double  bo_m;                     /* > 0: H0 from the magnetic Bond number (Eq. 50)*/
    double  stefan;                   /* > 0: latent heat from the Stefan number     */
    double  latent;                   /* L, used when stefan <= 0                    */
    double  T_m;
    double  rho_l, rho_g, rho_s;
    double  mu_l, mu_g, mu_s;
    double  cp_l, cp_g, cp_s;
    double  lam_l, lam_g, lam_s;
    double  chi_l, chi_g, chi_s;
    double  sigma, xi, mobility, Q_g, gravity;
    double  dt, dts;                  /* finite-volume step and streaming step       */
    double  contact_angle_deg;        /* static contact angle at the walls (90: none)  */
    int32_t flags;                    /* oracle-only reading switches (ORACLE_FLAG_*) */
    int32_t pad_;
} oracle_case;

/* Oracle-only switches that replace a reading by the paper's literal print.
 * They exist so that tests can show that a pin catches the literal form. */
#define ORACLE_FLAG_LITERAL_FSTAR_SIGN  1  /* Eq. 32 with "-" instead of "+"    */
#define ORACLE_FLAG_LITERAL_MUC_SIGN    2  /* mu_c with "+kappa lap C"          */
/* Keep the potential that was set instead of solving it at the start of a step: lets
 * a test advance a window of a larger grid with that grid's solved potential. */
#define ORACLE_FLAG_KEEP_POTENTIAL      4
/* Planted mistakes: each flips or rescales one term of the step so that a test can
 * show that the pin on that term fails.  Never set outside those tests. */
#define ORACLE_FLAG_PLANT_VOLUME_SIGN   8   /* (rho_s/rho_l - 1) for (1 - rho_s/rho_l)   */
#define ORACLE_FLAG_PLANT_GRAVITY_SIGN  16  /* F_g = -rho g                               */
#define ORACLE_FLAG_PLANT_WALL_SIDE     32  /* wall shear du_t/dn taken towards the wall  */
#define ORACLE_FLAG_PLANT_WALL_FULL     64  /* the wall a full cell from the inner centre */
#define ORACLE_FLAG_PLANT_IBM_SIGN      128 /* F_IBM = +rho u dF_s/dt                      */

/* Field identifiers (same numbering as the library's field mask bits). */
enum { OF_PHI = 0, OF_HE, OF_T, OF_FL, OF_P, OF_U, OF_V, OF_C, OF_MUC, OF_RHO,
       OF_MX, OF_MY, OF_FSPREV, OF_COUNT };

typedef struct oracle_state oracle_state;

typedef struct oracle_stats {
    double sum_C, sum_He, sum_Fl_drop, n_drop, Q_L, t;
    double t_freeze;          /* < 0 until Q_L first reaches 0.99 */
    double pot_resid;         /* relative residual of the last potential solve */
    int32_t pot_iters, nonfinite;
} oracle_stats;

int  oracle_create(const oracle_case* cs, oracle_state** out);
void oracle_destroy(oracle_state* s);
int  oracle_step(oracle_state* s, int32_t nsteps);
int  oracle_get_field(oracle_state* s, int32_t field, double* out);   /* nx*ny, row-major, x fastest */
int  oracle_set_field(oracle_state* s, int32_t field, const double* in);
void oracle_get_stats(oracle_state* s, oracle_stats* out);
void oracle_set_threads(int32_t n);

/* Sec. 5 diagnostics of the current state (see oracle_diagnostics). */
typedef struct oracle_diag {
    double H_m;        /* droplet height above the bottom wall                      */
    double U_max;      /* largest speed over droplet cells (C >= 1/2)               */
    double Pe;         /* U_max D / alpha_l, D = 2 R_0                              */
    double Fo;         /* lambda_l t / (rho_l C_p,l R_0^2)                           */
    double Q_wall;     /* sum over the bottom-wall faces of the local heat flux Q dx */
} oracle_diag;
int oracle_diagnostics(oracle_state* s, oracle_diag* out, double* q_wall /* nx or NULL */);

/* Pieces exposed for pin tests. */
void   oracle_eq8(const oracle_case* cs, double He, double C, double* T, double* Fl);
double oracle_mix(double Fs, double C, double g_s, double g_l, double g_g);
void   oracle_equilibria(const oracle_case* cs, int32_t a, double p, double u, double v,
                         double C, double muc, double T, double He, double rho, double cp,
                         double* feq, double* geq, double* heq);
int    oracle_face_flux(oracle_state* s, int32_t axis, int32_t i, int32_t j, double* flux5);
double oracle_mag_lbfs_flux(oracle_state* s, int32_t axis, int32_t i, int32_t j, double mu_face);
int    oracle_solve_potential(oracle_state* s);
int    oracle_pseudo_time_potential(oracle_state* s, int32_t iters, double dtau);
int    oracle_rhs(oracle_state* s, double* rhs5);   /* R(W) of the current state, 5*nx*ny */

#ifdef __cplusplus
}
#endif
#endif
