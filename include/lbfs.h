/*
 * lbfs.h -- C ABI of the GB300 (sm_103a) enthalpy-based lattice Boltzmann flux
 * solver (LBFS) for ferrofluid-droplet freezing in a uniform magnetic field.
 *
 * One call of lbfs_step advances every case of a context by whole time steps of
 * the finite-volume update (paper Sec. 3.4, Table 1):
 *   - enthalpy -> temperature and liquid fraction (Eq. 8), solid held at rest
 *     (F_IBM of Eq. 9);
 *   - magnetic scalar potential, div(mu_m grad phi_m) = 0 (Eq. 4), whose
 *     steady magnetic LBFS (Eqs. 12-18) this solves directly;
 *   - per-face LBFS reconstruction (Eqs. 44, 45) of the mass, momentum,
 *     phase-field and enthalpy fluxes (Eqs. 20-37, 43);
 *   - Kelvin and surface-tension body forces (Eq. 6, F_surf = -C grad mu_c) and
 *     the sources of Eq. 41; finite-volume sum (Eq. 42); third-order
 *     Runge-Kutta in time (Sec. 3.4).
 *
 * Lattice units throughout: dx = 1, D2Q9 with c = 1 and c_s^2 = 1/3.
 * All pointers are plain host or device pointers; no C++ or framework types
 * cross this boundary.  No function throws; every failure is a status code with
 * a message available from lbfs_last_error.
 */
#ifndef LBFS_H
#define LBFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbfs_ctx lbfs_ctx; /* opaque; owns all device state of its cases */

typedef enum {
    LBFS_OK = 0,
    LBFS_EINVAL = 1,         /* bad argument or unsupported case; nothing was launched   */
    LBFS_ENOMEM = 2,         /* device allocation failed                                 */
    LBFS_ECUDA = 3,          /* a CUDA call failed; the message names it                 */
    LBFS_ETIMEOUT = 4,       /* a bounded device wait ran out                            */
    LBFS_EDIVERGED = 5,      /* a non-finite value appeared in a case's state            */
    LBFS_ENOTCONVERGED = 6   /* the potential solve missed its tolerance in max cycles   */
} lbfs_status;

typedef enum {
    LBFS_FP64 = 0,   /* every field and flux in FP64                                      */
    LBFS_MIXED = 1   /* fluxes, forces and state in FP32 except H_e, which is stored,
                        updated and inverted (Eq. 8 thresholds) as an FP32 pair of about
                        48 significant bits; potential by FP32 multigrid inside
                        FP64-accurate residual refinement; FP64-accurate global sums     */
} lbfs_precision;

/* Context configuration.  Zero-initialise and set what you need. */
typedef struct lbfs_config {
    int32_t device;          /* CUDA device ordinal                                        */
    int32_t precision;       /* lbfs_precision                                             */
    int32_t max_cases;       /* number of case slots (batched cases advance together)      */
    int32_t use_graph;       /* 1: record the step as a CUDA graph and replay it           */
    void*   cuda_stream;     /* borrowed cudaStream_t; NULL: the context creates its own   */
    void* (*dev_alloc)(size_t bytes, void* user);  /* optional device allocator, e.g. a   */
    void  (*dev_free)(void* ptr, void* user);      /* framework's caching allocator       */
    void*   alloc_user;
    int32_t mg_max_cycles;   /* refinement cycles of a potential solve after a state is set,
                                checked on the host (0: 40)                                */
    double  mg_tol;          /* relative residual ||b - A phi|| / ||b|| every solve must
                                reach (0: 1e-13 FP64, 1e-6 mixed)                          */
    int32_t tile;            /* stage-kernel tile shape id (see lbfs_autotune); 0: 32 x 8   */
    int32_t mg_warm_cycles;  /* refinement cycles available to the potential solve of each
                                later step (0: 12 FP64, 3 mixed).  Each cycle ends with the
                                residual of the corrected potential; once it meets mg_tol
                                the case's remaining kernels return at once, on the device,
                                so these steps need no host round trip and can be replayed
                                as a CUDA graph.  A residual still above mg_tol after the
                                last cycle makes lbfs_step return LBFS_ENOTCONVERGED     */
    int32_t mg_plain_cycles; /* 1: launch those cycles as mg_warm_cycles plain rounds of
                                kernels, each returning at once for a converged case,
                                instead of a conditional graph loop (kernel profilers
                                cannot follow conditional graph nodes); same results     */
    int32_t reserved[5];
} lbfs_config;

/* One case.  Walls are numbered 0 left (x = 0), 1 right (x = nx), 2 bottom (y = 0),
 * 3 top (y = ny).  Cell (i, j) has centre (i + 1/2, j + 1/2). */
typedef struct lbfs_case_desc {
    int32_t nx, ny;                 /* cells; both >= 4                                    */
    int32_t periodic_x, periodic_y; /* 1: periodic axis (no walls on it)                   */
    int32_t thermal_dirichlet[4];   /* 1: wall held at wall_T, 0: adiabatic                */
    double  wall_T[4];
    int32_t mag_bc;                 /* 0: uniform far field phi = -H0 (x cos a + y sin a) on
                                       every wall; 1: on bottom/top only, insulating sides */
    int32_t init;                   /* 0: sessile drop centred at (nx/2, 0); 1: free drop at
                                       (drop_x, drop_y); 2: uniform C = 1                  */
    double  radius, drop_x, drop_y;
    double  T_init;                 /* initial temperature (liquid everywhere)             */
    double  H0, field_angle_deg;    /* far-field |H| and its angle from +x                 */
    double  bo_m;                   /* > 0: H0 = sqrt(Bo_m sigma / (mu_0 2 radius)) (Eq. 50) */
    double  stefan;                 /* > 0: L = C_p,l (T_m - wall_T[2]) / Ste (Eq. 50)     */
    double  latent;                 /* L when stefan <= 0                                  */
    double  T_m;                    /* melting temperature (T_s = T_l = T_m)               */
    double  rho_l, rho_g, rho_s;    /* Eq. 11 phase properties                              */
    double  mu_l, mu_g, mu_s;
    double  cp_l, cp_g, cp_s;
    double  lam_l, lam_g, lam_s;
    double  chi_l, chi_g, chi_s;
    double  sigma, xi;              /* surface tension, interface width (beta, kappa of mu_c) */
    double  mobility, Q_g;          /* M_c and the phase-field diffusion parameter          */
    double  gravity;                /* g along y (F_g = rho g)                              */
    double  dt, dts;                /* finite-volume step and streaming step                */
    double  contact_angle_deg;      /* static contact angle theta_w at the walls, in (0, 180):
                                       the phase-field ghost takes
                                       C_in + (4/xi) cos(theta_w) C_in (1 - C_in) (the
                                       equilibrium-profile wetting condition); 90 is the
                                       no-flux (neutral) wall of Sec. 5                      */
    int32_t flags;                  /* must be 0                                            */
    int32_t pad_;
} lbfs_case_desc;

/* Per-case diagnostics after the last step (FP64 sums over the grid). */
typedef struct lbfs_case_stats {
    double  sum_C;        /* sum of C                                                     */
    double  sum_He;       /* sum of H_e                                                   */
    double  sum_Fl_drop;  /* sum of F_l over droplet cells (C >= 1/2)                     */
    double  n_drop;       /* number of droplet cells                                      */
    double  Q_L;          /* Eq. 51: mean solid fraction of the droplet cells             */
    double  t;            /* simulated time                                               */
    double  t_freeze;     /* first t with Q_L >= 0.99 (linear in time); < 0 if not yet    */
    double  pot_resid;    /* relative residual after the last potential solve             */
    int32_t pot_cycles;   /* refinement cycles of the last potential solve                */
    int32_t nonfinite;    /* 1 if a non-finite value appeared                             */
    double  pot_resid_max;   /* largest relative residual after a solve, over this call's steps */
    double  pot_cycles_mean; /* mean refinement cycles per step over this call's steps       */
} lbfs_case_stats;

/* Field identifiers; a field mask is a bit set of (1u << id).  lbfs_fields returns
 * FP64 row-major (x fastest) arrays of nx*ny values, one per set bit in increasing
 * id order. */
enum {
    LBFS_FIELD_PHI = 0,  /* magnetic potential                              */
    LBFS_FIELD_HE = 1,   /* total enthalpy H_e                              */
    LBFS_FIELD_T = 2,    /* temperature (Eq. 8)                             */
    LBFS_FIELD_FL = 3,   /* liquid fraction (Eq. 8)                         */
    LBFS_FIELD_P = 4,    /* pressure p                                      */
    LBFS_FIELD_U = 5,    /* velocity x                                      */
    LBFS_FIELD_V = 6,    /* velocity y                                      */
    LBFS_FIELD_C = 7,    /* order parameter C                               */
    LBFS_FIELD_MUC = 8,  /* chemical potential mu_c                         */
    LBFS_FIELD_RHO = 9,  /* density (Eq. 11)                                */
    LBFS_FIELD_MX = 10,  /* rho c_s^2 u                                     */
    LBFS_FIELD_MY = 11,  /* rho c_s^2 v                                     */
    LBFS_FIELD_FSPREV = 12 /* solid fraction of the previous step           */
};

/* Create a context on cfg->device (bookkeeping; no counterpart in the paper).  The
 * context owns its device memory and, unless cfg->cuda_stream is given (borrowed, not
 * destroyed), its stream.  Returns LBFS_EINVAL for a bad config, LBFS_ECUDA if the
 * device cannot be used, LBFS_ENOMEM if its tables cannot be allocated.  *out is NULL
 * on failure. */
lbfs_status lbfs_create(const lbfs_config* cfg, lbfs_ctx** out);

/* (Re)define case slot case_id (0 <= case_id < max_cases) and initialise its fields on
 * the host (Table 1 "Initialization": droplet C = 1/2 + 1/2 tanh(2 (R - r)/xi),
 * uniform T_init, liquid everywhere, p = 0, u = 0, phi the uniform far field), then
 * copy them to the device.  Checks the case (sizes: nx, ny >= 4 and the padded row
 * length, nx rounded up to 32, times ny below 2^31; positive properties; dt against the
 * explicit diffusion limit) before any allocation; LBFS_EINVAL on failure. */
lbfs_status lbfs_set_case(lbfs_ctx* ctx, int32_t case_id, const lbfs_case_desc* desc);

/* Overwrite stored fields of a case from host FP64 arrays: the evolved state of Eq. 39
 * (H_e, p, rho c_s^2 u, rho c_s^2 v, C), the potential phi and the previous step's F_s
 * (R13).  Layout as lbfs_fields: one nx*ny row-major array (x fastest) per set bit, in
 * increasing id order; host_in is caller-owned and only read.  Settable: PHI, HE, P,
 * C, MX, MY, FSPREV; other bits, an empty mask, a NULL buffer or an undefined case give
 * LBFS_EINVAL.  The statistics are recomputed from the imported state and the next
 * step re-converges the potential. */
lbfs_status lbfs_set_fields(lbfs_ctx* ctx, int32_t case_id, uint32_t mask, const double* host_in);

/* Advance every defined case by nsteps time steps (Table 1, Sec. 3.4): per step the
 * lagged solid-fraction rate, the magnetic potential of Eq. 4 (multigrid, to the
 * context's tolerance), then three SSP-RK3 stages of the LBFS finite-volume update
 * (reconstruction Eq. 44, interface values Eq. 45, equilibria Eqs. 20, 28, 29,
 * starred distributions Eqs. 16, 22, 32, 33, fluxes Eq. 43, sources Eqs. 6, 41,
 * finite-volume sum Eq. 42, Eq. 8 inversion), the solid held at rest, and the Eq. 51
 * statistics.  Runs on the context's stream and waits for completion.  out (nullable,
 * caller-owned, max_cases entries) receives each slot's statistics (undefined slots
 * zero).  nsteps < 0 gives LBFS_EINVAL before any launch; LBFS_EDIVERGED (a non-finite
 * value) and LBFS_ENOTCONVERGED (the potential missed its tolerance) are reported after
 * the steps ran, with the stats still filled. */
lbfs_status lbfs_step(lbfs_ctx* ctx, int32_t nsteps, lbfs_case_stats* out);

/* Copy fields of a case to caller-owned host memory: nx*ny FP64 values per set bit of
 * mask, row-major (x fastest), in increasing id order.  Derived fields are evaluated
 * from the stored state: T and F_l by Eq. 8, rho by Eq. 11, u and v from the momentum,
 * mu_c = 2 beta C (C-1)(2C-1) - kappa lap C (with the wall ghost rule).  An empty or
 * unknown mask, a NULL buffer or an undefined case give LBFS_EINVAL. */
lbfs_status lbfs_fields(lbfs_ctx* ctx, int32_t case_id, uint32_t mask, double* host_out);

/* Sec. 5 diagnostics of a case's current state (lattice units, FP64 arithmetic). */
typedef struct lbfs_case_diag {
    double H_m;      /* droplet height (Sec. 5.1): the highest point where C crosses 1/2 in
                        any column, linear in y between cell centres; 0 without droplet   */
    double U_max;    /* largest speed |u| over the droplet cells (C >= 1/2)               */
    double Pe;       /* Peclet number U_max D / alpha_l, D = 2 R_0, alpha_l = lambda_l /
                        (rho_l C_p,l) (Eq. 50, its garbled "D u^2/alpha" read as U D/alpha) */
    double Fo;       /* Fourier number lambda_l t / (rho_l C_p,l R_0^2) (Eq. 50)          */
    double Q_wall;   /* sum over the bottom-wall faces of the local heat flux Q dx        */
} lbfs_case_diag;

/* Diagnostics of case case_id (Sec. 5.1-5.2) computed on the device from the stored
 * state, on the context's stream, waiting for completion.  R_0 is the case's radius.
 * The local heat flux on the cold substrate is Q = -lambda dT/dy at y = 0, the slope
 * being the second-order one-sided difference (-8 T_w + 9 T_0 - T_1)/3 through the
 * wall temperature and the first two cell centres, lambda the first cell's Eq. 11
 * value; Q = 0 where the bottom wall is adiabatic or the y axis periodic.
 * out: caller-owned, one struct.  q_wall: caller-owned host array of nx doubles that
 * receives Q per column, or NULL.  LBFS_EINVAL for an undefined case or a NULL out. */
lbfs_status lbfs_diagnostics(lbfs_ctx* ctx, int32_t case_id, lbfs_case_diag* out, double* q_wall);

/* The paper's own magnetic solver (Sec. 3.2, Eqs. 12-18), offered beside the multigrid
 * solve that lbfs_step uses: `iters` explicit pseudo-time steps of Eq. 17,
 * phi <- phi - dtau div F, applied to case case_id's stored potential, with the
 * per-direction LBFS face flux of the magnetic distribution (equilibrium Eq. 13,
 * reconstruction Eq. 44 at x_f - e_a dts from the upwind cell, interface value Eq. 45,
 * tau = 1/2 + mu_f/(c_s^2 dts), starred distribution Eq. 16) and the coefficient
 * mu_m = 1 + chi(C, F_s) of the current state.  Its fixed point is the potential the
 * multigrid solve returns.  FP64 arithmetic in both precisions; the stable range is
 * about dtau < 1/(4 max mu_m).  iters >= 0, dtau > 0, else LBFS_EINVAL; waits for
 * completion. */
lbfs_status lbfs_potential_pseudo_time(lbfs_ctx* ctx, int32_t case_id, int32_t iters, double dtau);

/* Number of device kernel launches the last lbfs_step issued (graph nodes count);
 * bookkeeping, no counterpart in the paper. */
int64_t lbfs_last_launch_count(const lbfs_ctx* ctx);

/* Autotuner of the stage kernel's tile shape (no counterpart in the paper).  The tile
 * is a block's share of the grid; the halo is fixed at three cells by the stencil.
 * Times `reps` launches of each compiled tile shape on the context's current cases
 * (Runge-Kutta stage 2, which writes only a stage buffer, so the state is untouched),
 * keeps the fastest (a shape with a higher id must be more than 2 % faster than the
 * best before it) for later steps and writes its id to *chosen (nullable).  ms
 * (nullable, n entries) receives the milliseconds per launch of each shape id < n.
 * Shapes: 0 32x8, 1 32x16, 2 64x8, 3 16x16, 4 64x4, 5 16x16 and 6 32x8 with registers
 * cut for a third resident block per SM, 7 16x16 and 8 32x8 with registers cut for a
 * fourth, 9 16x16 and 10 32x8 with a fourth block of 256 threads instead of 288 (the
 * cuts apply in mixed precision).  LBFS_EINVAL without a defined case or for reps < 1. */
lbfs_status lbfs_autotune(lbfs_ctx* ctx, int32_t reps, int32_t* chosen, double* ms, int32_t n);

/* Kernel timing (no counterpart in the paper).  While enabled, lbfs_step brackets
 * every launch with CUDA events on the context's stream and accumulates the elapsed
 * device time per kernel class: LBFS_TIMING_STAGE (the fused Runge-Kutta stage
 * kernel), LBFS_TIMING_POTENTIAL (the whole potential solve of a step),
 * LBFS_TIMING_FINALIZE (step-end statistics).  Enabling clears the accumulators; while
 * enabled the step is never replayed from a graph.  lbfs_timing_read copies n (<= 3)
 * accumulated milliseconds and event-pair counts into caller-owned arrays (either may
 * be NULL). */
enum { LBFS_TIMING_STAGE = 0, LBFS_TIMING_POTENTIAL = 1, LBFS_TIMING_FINALIZE = 2 };
lbfs_status lbfs_timing(lbfs_ctx* ctx, int32_t enable);
lbfs_status lbfs_timing_read(lbfs_ctx* ctx, double* ms, int64_t* counts, int32_t n);

/* Diagnostics of a state that lives in the caller's device memory, computed without
 * allocating anything (the paper has no counterpart; it is a service for callers that
 * cannot allocate device memory, e.g. code running inside another component's fixed
 * memory pool or while that component records work, which must not call cudaMalloc).
 *   desc:  the case; only nx, ny, cp_l, cp_g, cp_s, T_m, stefan/latent and wall_T[2]
 *          are read (the enthalpy inversion the step uses).
 *   d_He, d_C: device arrays of nx*ny FP64 values, row-major with x fastest (caller-owned).
 *   d_out: device array of 5 FP64 values (caller-owned) receiving sum C, sum H_e,
 *          sum F_l over droplet cells (C >= 1/2), the number of droplet cells and Q_L.
 *   stream: cudaStream_t the two kernels run on (NULL: the legacy default stream); the
 *          call returns once they are enqueued.
 *   err, err_len: optional buffer for a message ("" on success).
 * Scratch: one row of partial sums per grid row in a fixed 16384 x 5 FP64 device array
 * (640 KiB) that every device using this library keeps until the process exits;
 * ny > 16384 returns LBFS_EINVAL before any launch.  No cudaMalloc, cudaFree or other
 * allocating call is made.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture.  A cudaDeviceReset
 * reloads the module, which leaves the kept address stale, so a process that resets a
 * device must not call this again afterwards.  All calls share the array and every call rewrites the rows it
 * uses, so nothing needs clearing, but calls whose kernels overlap on the GPU (other
 * streams, other host threads) race on it: order them on one stream. */
lbfs_status lbfs_state_stats_noalloc(const lbfs_case_desc* desc, const double* d_He, const double* d_C,
                                     double* d_out, void* stream, char* err, size_t err_len);

/* Release all device memory and the owned stream (if any); a borrowed stream is left
 * alone.  NULL is ignored.  Bookkeeping, no counterpart in the paper. */
void lbfs_destroy(lbfs_ctx* ctx);

/* Sticky message of the last failure on ctx ("" if none); valid until the next call
 * on ctx.  Bookkeeping, no counterpart in the paper. */
const char* lbfs_last_error(const lbfs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
