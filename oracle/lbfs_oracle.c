/*
 * lbfs_oracle.c -- plain FP64 CPU oracle of one LBFS time step.
 *
 * TEST INFRASTRUCTURE ONLY (see lbfs_oracle.h).  Slow on purpose: every
 * interface flux is built per D2Q9 direction exactly as the paper writes it,
 * with no reordering or fusion.  Readings of garbled or silent passages are
 * stated where they are used.
 */
#include "lbfs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- D2Q9 lattice: Eq. 14 and Fig. 1.  The printed weights (4/9 for all three
 * groups) are garbled; the D2Q9 model the paper cites has 4/9, 1/9, 1/36.  The
 * diagonal velocities are (+-1, +-1). ------------------------------------------ */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WA[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 with c = 1 */
#define ORACLE_PI 3.14159265358979323846

/* primitive set reconstructed by Eq. 44 */
enum { Q_P = 0, Q_U, Q_V, Q_C, Q_MUC, Q_T, Q_HE, Q_N };
/* conserved vector W of Eq. 39 without phi (phi is solved separately) */
enum { W_HE = 0, W_P, W_MX, W_MY, W_C, W_N };

struct oracle_state {
    oracle_case cs;
    int nx, ny;
    double H0, L, beta, kappa, cos_t, sin_t, cp_ref, vol_ratio;
    double wet;           /* 4 cos(theta_w)/xi of the wetting ghost rule (0 at 90 deg) */
    double* W[W_N];       /* evolved state, nx*ny */
    double* phi;          /* magnetic potential, nx*ny */
    double* Fs_prev;      /* F_s at the previous step */
    double* Sdot;         /* lagged dF_s/dt, held over the step */
    double* mu_m;         /* mu_0 (1 + chi), nx*ny */
    /* cell quantities with one ghost layer, (nx+2)*(ny+2) */
    double* q[Q_N];
    double* Fs;
    double* rho;
    double* H2;
    double* phig;         /* potential with its ghost layer (magnetic LBFS pin) */
    /* cell-centred gradients of the reconstructed set, nx*ny */
    double* gx[Q_N];
    double* gy[Q_N];
    double* Fx;           /* (nx+1)*ny*5 */
    double* Fy;           /* nx*(ny+1)*5 */
    double* rhs;          /* 5*nx*ny */
    double* w0;           /* 5*nx*ny copy of W^n */
    double t;
    long nstep;
    double QL_prev, t_freeze, pot_resid;
    int pot_iters;
};

static int g_threads = 1;
void oracle_set_threads(int32_t n) { g_threads = n > 0 ? n : 1; }

/* ---- Eq. 11: mixture rule for rho, mu, lambda, C_p and chi ------------------- */
double oracle_mix(double Fs, double C, double g_s, double g_l, double g_g)
{
    return Fs * g_s + (1.0 - Fs) * C * g_l + (1.0 - Fs) * (1.0 - C) * g_g;
}

/* ---- Eq. 8: total enthalpy -> (T, F_l).
 * Readings: T_s = T_l = T_m; H_es = C_p,s T_m; H_el = C_p,L T_m + L with C_p,L
 * the Eq. 11 mixture at F_s = 0 (the liquid state of the cell) and L the single
 * latent heat of Eq. 8.  Phase change happens only where C >= 1/2; elsewhere the
 * cell is treated as never solid (F_l = 1).  Ties: H_e == H_es gives F_l = 0 and
 * H_e == H_el gives F_l = 1, both branches agreeing there. ---------------------- */
void oracle_eq8(const oracle_case* cs, double He, double C, double* T, double* Fl)
{
    double L = cs->stefan > 0.0 ? cs->cp_l * (cs->T_m - cs->wall_T[2]) / cs->stefan : cs->latent;
    double cpL = C * cs->cp_l + (1.0 - C) * cs->cp_g;
    double Hes = cs->cp_s * cs->T_m;
    double Hel = cpL * cs->T_m + L;
    if (C < 0.5) {
        *Fl = 1.0;
        *T = cs->T_m + (He - Hel) / cpL;
        return;
    }
    if (He < Hes) {
        *Fl = 0.0;
        *T = He / cs->cp_s;
    } else if (He <= Hel) {
        *Fl = (He - Hes) / (Hel - Hes);
        *T = cs->T_m;
    } else {
        *Fl = 1.0;
        *T = cs->T_m + (He - Hel) / cpL;
    }
}

/* Gamma_a(u) = e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)  (Eq. 28) */
static double gamma_a(int a, double u, double v)
{
    double eu = EX[a] * u + EY[a] * v;
    return eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - (u * u + v * v) / (2.0 * CS2);
}

/* ---- Equilibria for direction a: f (Eq. 28), g (Eq. 29), h (Eq. 20) ---------- */
void oracle_equilibria(const oracle_case* cs, int32_t a, double p, double u, double v,
                       double C, double muc, double T, double He, double rho, double cp,
                       double* feq, double* geq, double* heq)
{
    double cp_ref = 0.5 * (cs->cp_s + cs->cp_l);
    double eu = EX[a] * u + EY[a] * v;
    double uu = u * u + v * v;
    *feq = WA[a] * (p + rho * CS2 * gamma_a(a, u, v));
    if (a == 0) {
        *geq = C - muc * cs->Q_g * (1.0 - WA[0]) / CS2;
        *heq = He - cp_ref * T + WA[0] * cp * T * (cp_ref / cp - uu / (2.0 * CS2));
    } else {
        *geq = WA[a] * (muc * cs->Q_g + C * eu) / CS2;
        *heq = WA[a] * cp * T *
               (cp_ref / cp + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* index helpers */
#define GI(s, i, j) ((size_t)((j) + 1) * (size_t)((s)->nx + 2) + (size_t)((i) + 1))
#define CI(s, i, j) ((size_t)(j) * (size_t)(s)->nx + (size_t)(i))

static double latent_of(const oracle_case* cs)
{
    return cs->stefan > 0.0 ? cs->cp_l * (cs->T_m - cs->wall_T[2]) / cs->stefan : cs->latent;
}

/* wall potential phi_w = -H0 (x cos + y sin) at a point (uniform far field) */
static double phi_far(const oracle_state* s, double x, double y)
{
    return -s->H0 * (x * s->cos_t + y * s->sin_t);
}

static int wall_is_dirichlet_phi(const oracle_state* s, int wall)
{
    if (wall < 2 && s->cs.periodic_x) return 0;
    if (wall >= 2 && s->cs.periodic_y) return 0;
    if (s->cs.mag_bc == 1 && wall < 2) return 0;
    return 1;
}

static int needs_potential_solve(const oracle_state* s)
{
    const oracle_case* c = &s->cs;
    if (c->chi_l == 0.0 && c->chi_s == 0.0 && c->chi_g == 0.0) return 0;
    for (int w = 0; w < 4; ++w)
        if (wall_is_dirichlet_phi(s, w)) return 1;
    return 0;
}

/* ---- cell quantities of a state W: Eq. 8, Eq. 11, u = (rho c_s^2 u)/(rho c_s^2),
 * and the chemical potential mu_c = 2 beta C (C-1)(2C-1) - kappa lap C.  The
 * printed "+kappa lap C" makes the Cahn-Hilliard equation anti-diffusive; the
 * standard "-" is used (the literal sign is ORACLE_FLAG_LITERAL_MUC_SIGN). ---- */
static void fill_ghosts(oracle_state* s, double* f, int kind);

enum { GH_EVEN = 0, GH_ODD, GH_T, GH_HE, GH_WET };

static void derive(oracle_state* s, double* const* W)
{
    const oracle_case* c = &s->cs;
    int nx = s->nx, ny = s->ny;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = CI(s, i, j), g = GI(s, i, j);
            double He = W[W_HE][k], C = W[W_C][k];
            double T, Fl;
            oracle_eq8(c, He, C, &T, &Fl);
            double Fs = 1.0 - Fl;
            double rho = oracle_mix(Fs, C, c->rho_s, c->rho_l, c->rho_g);
            s->q[Q_P][g] = W[W_P][k];
            s->q[Q_U][g] = W[W_MX][k] / (rho * CS2);
            s->q[Q_V][g] = W[W_MY][k] / (rho * CS2);
            s->q[Q_C][g] = C;
            s->q[Q_T][g] = T;
            s->q[Q_HE][g] = He;
            s->Fs[g] = Fs;
            s->rho[g] = rho;
        }
    fill_ghosts(s, s->q[Q_C], GH_WET);
    double ksign = (c->flags & ORACLE_FLAG_LITERAL_MUC_SIGN) ? 1.0 : -1.0;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double* Cq = s->q[Q_C];
            double C = Cq[GI(s, i, j)];
            double lap = Cq[GI(s, i + 1, j)] + Cq[GI(s, i - 1, j)] + Cq[GI(s, i, j + 1)] +
                         Cq[GI(s, i, j - 1)] - 4.0 * C;
            s->q[Q_MUC][GI(s, i, j)] =
                2.0 * s->beta * C * (C - 1.0) * (2.0 * C - 1.0) + ksign * s->kappa * lap;
        }
    fill_ghosts(s, s->Fs, GH_EVEN);
    fill_ghosts(s, s->rho, GH_EVEN);
    fill_ghosts(s, s->q[Q_P], GH_EVEN);
    fill_ghosts(s, s->q[Q_U], GH_ODD);
    fill_ghosts(s, s->q[Q_V], GH_ODD);
    fill_ghosts(s, s->q[Q_MUC], GH_EVEN);
    fill_ghosts(s, s->q[Q_T], GH_T);
    fill_ghosts(s, s->q[Q_HE], GH_HE);
    /* central gradients of the reconstructed set (second-order, dx = 1) */
    for (int n = 0; n < Q_N; ++n) {
        const double* f = s->q[n];
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                s->gx[n][CI(s, i, j)] = 0.5 * (f[GI(s, i + 1, j)] - f[GI(s, i - 1, j)]);
                s->gy[n][CI(s, i, j)] = 0.5 * (f[GI(s, i, j + 1)] - f[GI(s, i, j - 1)]);
            }
    }
}

/* ---- ghost layer.  Periodic axes wrap.  Walls: velocity no-slip (ghost = -inner),
 * p, mu_c, F_s, rho zero normal gradient (ghost = inner), C zero normal gradient at a
 * contact angle of 90 deg and the wetting rule below otherwise, T Dirichlet
 * 2 T_w - T_in or adiabatic T_in, H_e rebuilt from the ghost T with the inner C and
 * F_s through H_e = C_p T + L (1 - F_s). -------------------------------------------- */
static double ghost_value(oracle_state* s, const double* f, int kind, int wall, int ii, int jj)
{
    const oracle_case* c = &s->cs;
    size_t g = GI(s, ii, jj);
    switch (kind) {
    case GH_ODD: return -f[g];
    case GH_T:
        return c->thermal_dirichlet[wall] ? 2.0 * c->wall_T[wall] - f[g] : f[g];
    case GH_HE: {
        double T = s->q[Q_T][g];
        double Tg = c->thermal_dirichlet[wall] ? 2.0 * c->wall_T[wall] - T : T;
        double C = s->q[Q_C][g], Fs = s->Fs[g];
        double cp = oracle_mix(Fs, C, c->cp_s, c->cp_l, c->cp_g);
        return cp * Tg + s->L * (1.0 - Fs);
    }
    case GH_WET:
        /* wetting: the equilibrium profile C = (1 + tanh(2 d/xi))/2 meets the wall at the
         * contact angle theta_w when dC/dn = -(4/xi) cos(theta_w) C (1 - C) there (n into
         * the fluid); the ghost half a cell outside takes C_in - dC/dn, with C_in for C */
        return f[g] + s->wet * f[g] * (1.0 - f[g]);
    default: return f[g];
    }
}

static void fill_ghosts(oracle_state* s, double* f, int kind)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j) {
        if (s->cs.periodic_x) {
            f[GI(s, -1, j)] = f[GI(s, nx - 1, j)];
            f[GI(s, nx, j)] = f[GI(s, 0, j)];
        } else {
            f[GI(s, -1, j)] = ghost_value(s, f, kind, 0, 0, j);
            f[GI(s, nx, j)] = ghost_value(s, f, kind, 1, nx - 1, j);
        }
    }
    for (int i = 0; i < nx; ++i) {
        if (s->cs.periodic_y) {
            f[GI(s, i, -1)] = f[GI(s, i, ny - 1)];
            f[GI(s, i, ny)] = f[GI(s, i, 0)];
        } else {
            f[GI(s, i, -1)] = ghost_value(s, f, kind, 2, i, 0);
            f[GI(s, i, ny)] = ghost_value(s, f, kind, 3, i, ny - 1);
        }
    }
}

/* ---- Eq. 44: linear reconstruction of primitive n from cell (i, j) at the
 * offset (ox, oy) from its centre ------------------------------------------- */
static double recon(const oracle_state* s, int n, int i, int j, double ox, double oy)
{
    size_t k = CI(s, i, j);
    return s->q[n][GI(s, i, j)] + ox * s->gx[n][k] + oy * s->gy[n][k];
}

/* ---- one interior (or periodic) face: Eqs. 44, 45, 28/29/20, 32/33/22, 43.
 * axis 0: x-face between cells A = (i-1, j) and B = (i, j); axis 1: y-face
 * between A = (i, j-1) and B = (i, j).  Readings:
 *  - x - e_a dts lies in A when e_a.n > 0, in B when e_a.n < 0; when e_a.n = 0
 *    the point is reconstructed from both cells and the two results averaged
 *    (the paper's averaging rule for values on the interface).
 *  - rho and C_p at a surrounding point: Eq. 11 with the point's C and the F_s of
 *    the cell it comes from (mean of both cells for e_a.n = 0).
 *  - interface values follow Eq. 45 literally; F_s at the face is the mean of A
 *    and B; rho, C_p, lambda, mu at the face from Eq. 11 with (C_f, F_s,f); T_f
 *    from Eq. 8 with (H_e,f, C_f); mu_c,f is the averaged reconstruction at x_f.
 *  - f^{eq-m} at a surrounding point uses the interface density rho_f.
 *  - Eq. 32 is taken with "+" like Eqs. 16, 22, 33 (the printed "-" gives a
 *    negative viscosity; it is ORACLE_FLAG_LITERAL_FSTAR_SIGN).
 *  - relaxation times at the face: tau_f = 1/2 + mu/(rho c_s^2 dts),
 *    tau_h = 1/2 + lambda/(rho C_p,ref c_s^2 dts), tau_g = 1/2 + M_c/(Q_g dts). */
static void lbfs_face(oracle_state* s, int axis, int i, int j, double out[5])
{
    const oracle_case* c = &s->cs;
    const double dts = c->dts;
    int ia, ja, ib, jb;
    double ax0, ay0, bx0, by0; /* centre of A and B relative to the face centre */
    int nxn = axis == 0, nyn = axis == 1;
    if (axis == 0) {
        ia = i - 1; ja = j; ib = i; jb = j;
        if (ia < 0) ia += s->nx; /* periodic wrap; offsets stay geometric */
        if (ib >= s->nx) ib -= s->nx;
        ax0 = -0.5; ay0 = 0.0; bx0 = 0.5; by0 = 0.0;
    } else {
        ia = i; ja = j - 1; ib = i; jb = j;
        if (ja < 0) ja += s->ny;
        if (jb >= s->ny) jb -= s->ny;
        ax0 = 0.0; ay0 = -0.5; bx0 = 0.0; by0 = 0.5;
    }
    double FsA = s->Fs[GI(s, ia, ja)], FsB = s->Fs[GI(s, ib, jb)];

    double qp[9][Q_N], Fs_pt[9];
    double feq[9], geq[9], heq[9];
    for (int a = 0; a < 9; ++a) {
        int en = EX[a] * nxn + EY[a] * nyn;
        double px = -EX[a] * dts, py = -EY[a] * dts; /* x - e_a dts relative to x_f */
        for (int n = 0; n < Q_N; ++n) {
            double vA = recon(s, n, ia, ja, px - ax0, py - ay0);
            double vB = recon(s, n, ib, jb, px - bx0, py - by0);
            qp[a][n] = en > 0 ? vA : (en < 0 ? vB : 0.5 * (vA + vB));
        }
        Fs_pt[a] = en > 0 ? FsA : (en < 0 ? FsB : 0.5 * (FsA + FsB));
        double rho = oracle_mix(Fs_pt[a], qp[a][Q_C], c->rho_s, c->rho_l, c->rho_g);
        double cp = oracle_mix(Fs_pt[a], qp[a][Q_C], c->cp_s, c->cp_l, c->cp_g);
        oracle_equilibria(c, a, qp[a][Q_P], qp[a][Q_U], qp[a][Q_V], qp[a][Q_C], qp[a][Q_MUC],
                          qp[a][Q_T], qp[a][Q_HE], rho, cp, &feq[a], &geq[a], &heq[a]);
    }
    /* Eq. 45: interface values from the surrounding equilibria */
    double p_f = 0, jx = 0, jy = 0, C_f = 0, He_f = 0;
    for (int a = 0; a < 9; ++a) {
        p_f += feq[a];
        jx += EX[a] * feq[a];
        jy += EY[a] * feq[a];
        C_f += geq[a];
        He_f += heq[a];
    }
    double Fs_f = 0.5 * (FsA + FsB);
    double rho_f = oracle_mix(Fs_f, C_f, c->rho_s, c->rho_l, c->rho_g);
    double u_f = jx / (rho_f * CS2), v_f = jy / (rho_f * CS2);
    double cp_f = oracle_mix(Fs_f, C_f, c->cp_s, c->cp_l, c->cp_g);
    double lam_f = oracle_mix(Fs_f, C_f, c->lam_s, c->lam_l, c->lam_g);
    double mu_f = oracle_mix(Fs_f, C_f, c->mu_s, c->mu_l, c->mu_g);
    double T_f, Fl_f;
    oracle_eq8(c, He_f, C_f, &T_f, &Fl_f);
    double muc_f = 0.5 * (recon(s, Q_MUC, ia, ja, -ax0, -ay0) + recon(s, Q_MUC, ib, jb, -bx0, -by0));
    double tau_f = 0.5 + mu_f / (rho_f * CS2 * dts);
    double tau_h = 0.5 + lam_f / (rho_f * s->cp_ref * CS2 * dts);
    double tau_g = 0.5 + c->mobility / (c->Q_g * dts);
    double fsign = (c->flags & ORACLE_FLAG_LITERAL_FSTAR_SIGN) ? -1.0 : 1.0;

    for (int n = 0; n < 5; ++n) out[n] = 0.0;
    for (int a = 0; a < 9; ++a) {
        double feqF, geqF, heqF;
        oracle_equilibria(c, a, p_f, u_f, v_f, C_f, muc_f, T_f, He_f, rho_f, cp_f, &feqF, &geqF,
                          &heqF);
        double feqm = WA[a] * (qp[a][Q_P] + rho_f * CS2 * gamma_a(a, qp[a][Q_U], qp[a][Q_V]));
        double fneq = -tau_f * (feqF - feqm);
        double fstar = feqF + fsign * (1.0 - 1.0 / (2.0 * tau_f)) * fneq;
        double gneq = -tau_g * (geqF - geq[a]);
        double gstar = geqF + (1.0 - 1.0 / (2.0 * tau_g)) * gneq;
        double hneq = -tau_h * (heqF - heq[a]);
        double hstar = heqF + (1.0 - 1.0 / (2.0 * tau_h)) * hneq;
        double en = (double)(EX[a] * nxn + EY[a] * nyn);
        out[W_HE] += en * hstar;
        out[W_P] += en * feqF;
        out[W_MX] += en * EX[a] * fstar;
        out[W_MY] += en * EY[a] * fstar;
        out[W_C] += en * gstar;
    }
}

/* ---- wall face (the paper gives no boundary flux; reading): no mass or
 * phase-field flux through a no-slip, no-flux wall; momentum flux c_s^2 (p n -
 * mu du_t/dn) with the wall velocity zero half a cell from the inner centre; the
 * enthalpy flux is zero on adiabatic walls and -(lambda/rho) dT/dn with
 * dT/dn = (T_in - T_w)/(dx/2) on Dirichlet walls.  Properties are the inner
 * cell's.  wall: 0 left, 1 right, 2 bottom, 3 top. ------------------------------ */
static void wall_face(oracle_state* s, int wall, int i, int j, double out[5])
{
    const oracle_case* c = &s->cs;
    size_t g = GI(s, i, j);
    double Fs = s->Fs[g], C = s->q[Q_C][g];
    double rho = s->rho[g];
    double mu = oracle_mix(Fs, C, c->mu_s, c->mu_l, c->mu_g);
    double lam = oracle_mix(Fs, C, c->lam_s, c->lam_l, c->lam_g);
    double side = (wall == 0 || wall == 2) ? 1.0 : -1.0; /* +1: inner cell lies at +axis */
    double ut = (wall < 2) ? s->q[Q_V][g] : s->q[Q_U][g];
    double dn = (c->flags & ORACLE_FLAG_PLANT_WALL_FULL) ? 1.0 : 0.5; /* wall to inner centre */
    double sside = (c->flags & ORACLE_FLAG_PLANT_WALL_SIDE) ? -side : side;
    double dut = sside * ut / dn;
    double T = s->q[Q_T][g];
    double dT = side * (T - c->wall_T[wall]) / 0.5;
    for (int n = 0; n < 5; ++n) out[n] = 0.0;
    if (wall < 2) {
        out[W_MX] = CS2 * s->q[Q_P][g];
        out[W_MY] = CS2 * (-mu * dut);
    } else {
        out[W_MY] = CS2 * s->q[Q_P][g];
        out[W_MX] = CS2 * (-mu * dut);
    }
    out[W_HE] = c->thermal_dirichlet[wall] ? -(lam / rho) * dT : 0.0;
}

static void all_fluxes(oracle_state* s)
{
    int nx = s->nx, ny = s->ny;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            double* o = s->Fx + ((size_t)j * (nx + 1) + i) * 5;
            if (s->cs.periodic_x) {
                if (i == nx) continue;
                lbfs_face(s, 0, i, j, o);
            } else if (i == 0) {
                wall_face(s, 0, 0, j, o);
            } else if (i == nx) {
                wall_face(s, 1, nx - 1, j, o);
            } else {
                lbfs_face(s, 0, i, j, o);
            }
        }
    if (s->cs.periodic_x)
        for (int j = 0; j < ny; ++j)
            memcpy(s->Fx + ((size_t)j * (nx + 1) + nx) * 5, s->Fx + ((size_t)j * (nx + 1)) * 5,
                   5 * sizeof(double));
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double* o = s->Fy + ((size_t)j * nx + i) * 5;
            if (s->cs.periodic_y) {
                if (j == ny) continue;
                lbfs_face(s, 1, i, j, o);
            } else if (j == 0) {
                wall_face(s, 2, i, 0, o);
            } else if (j == ny) {
                wall_face(s, 3, i, ny - 1, o);
            } else {
                lbfs_face(s, 1, i, j, o);
            }
        }
    if (s->cs.periodic_y)
        memcpy(s->Fy + (size_t)ny * nx * 5, s->Fy, (size_t)nx * 5 * sizeof(double));
}

/* ---- R(W) of Eq. 46: minus the flux divergence of Eq. 42 (V = S = 1) plus the
 * sources of Eq. 41 at the cell centre:
 *   H_e : C_p T div u
 *   p   : u . grad(rho c_s^2) + rho c_s^2 (1 - rho_s/rho_l) dF_s/dt
 *   m   : c_s^2 (F_surf + F_mg + F_g + F_IBM), F_surf = -C grad mu_c,
 *         F_mg = (mu_0 chi / 2) grad |H|^2 (Eq. 6), F_g = rho g (y),
 *         F_IBM = -rho u dF_s/dt
 *   C   : C (1 - rho_s/rho_l) dF_s/dt
 * with central differences over the ghost layer. ------------------------------ */
static void compute_rhs(oracle_state* s, double* const* W, double* R)
{
    const oracle_case* c = &s->cs;
    int nx = s->nx, ny = s->ny;
    size_t N = (size_t)nx * ny;
    derive(s, W);
    all_fluxes(s);
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = CI(s, i, j), g = GI(s, i, j);
            const double* fl = s->Fx + ((size_t)j * (nx + 1) + i) * 5;
            const double* fr = s->Fx + ((size_t)j * (nx + 1) + i + 1) * 5;
            const double* fb = s->Fy + ((size_t)j * nx + i) * 5;
            const double* ft = s->Fy + ((size_t)(j + 1) * nx + i) * 5;
            double Fs = s->Fs[g], C = s->q[Q_C][g], T = s->q[Q_T][g];
            double u = s->q[Q_U][g], v = s->q[Q_V][g], rho = s->rho[g];
            double cp = oracle_mix(Fs, C, c->cp_s, c->cp_l, c->cp_g);
            double chi = oracle_mix(Fs, C, c->chi_s, c->chi_l, c->chi_g);
            double divu = s->gx[Q_U][k] + s->gy[Q_V][k];
            double drx = 0.5 * (s->rho[GI(s, i + 1, j)] - s->rho[GI(s, i - 1, j)]);
            double dry = 0.5 * (s->rho[GI(s, i, j + 1)] - s->rho[GI(s, i, j - 1)]);
            double dHx = 0.5 * (s->H2[GI(s, i + 1, j)] - s->H2[GI(s, i - 1, j)]);
            double dHy = 0.5 * (s->H2[GI(s, i, j + 1)] - s->H2[GI(s, i, j - 1)]);
            double dmx = s->gx[Q_MUC][k], dmy = s->gy[Q_MUC][k];
            double Sd = s->Sdot[k];
            double vr = (c->flags & ORACLE_FLAG_PLANT_VOLUME_SIGN) ? -s->vol_ratio : s->vol_ratio;
            double grav = (c->flags & ORACLE_FLAG_PLANT_GRAVITY_SIGN) ? -c->gravity : c->gravity;
            double ibm = (c->flags & ORACLE_FLAG_PLANT_IBM_SIGN) ? 1.0 : -1.0;
            double src[5];
            src[W_HE] = cp * T * divu;
            src[W_P] = u * CS2 * drx + v * CS2 * dry + rho * CS2 * vr * Sd;
            src[W_MX] = CS2 * (-C * dmx + 0.5 * chi * dHx + ibm * rho * u * Sd);
            src[W_MY] = CS2 * (-C * dmy + 0.5 * chi * dHy + rho * grav + ibm * rho * v * Sd);
            src[W_C] = C * vr * Sd;
            for (int n = 0; n < 5; ++n)
                R[n * N + k] = -(fr[n] - fl[n]) - (ft[n] - fb[n]) + src[n];
        }
}

/* ---- magnetic potential: steady Eq. 4, div(mu_m grad phi) = 0, on the cell-centred
 * five-point stencil with the arithmetic-mean face coefficient.  At dts = 1/2 this
 * is exactly the converged state of the magnetic LBFS of Eqs. 12-18 (see
 * oracle_mag_lbfs_flux).  Dirichlet walls hold the uniform far field
 * phi = -H0 (x cos + y sin) at the face centre (ghost 2 phi_w - phi_in); insulating
 * walls have zero normal gradient.  Solved by Jacobi-preconditioned conjugate
 * gradients on A phi = b, (A phi)_c = sum_nb mu_f (phi_c - phi_nb) + sum_Dirichlet
 * 2 mu_c phi_c, b_c = sum_Dirichlet 2 mu_c phi_w. ---------------------------- */
static void pot_apply(const oracle_state* s, const double* x, double* y)
{
    int nx = s->nx, ny = s->ny;
    const double* mu = s->mu_m;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = CI(s, i, j);
            double acc = 0.0;
            int nb_i[4] = {i - 1, i + 1, i, i};
            int nb_j[4] = {j, j, j - 1, j + 1};
            for (int w = 0; w < 4; ++w) {
                int ii = nb_i[w], jj = nb_j[w];
                int outside = ii < 0 || ii >= nx || jj < 0 || jj >= ny;
                if (outside) {
                    int periodic = (w < 2) ? s->cs.periodic_x : s->cs.periodic_y;
                    if (periodic) {
                        ii = (ii + nx) % nx;
                        jj = (jj + ny) % ny;
                    } else {
                        if (wall_is_dirichlet_phi(s, w)) acc += 2.0 * mu[k] * x[k];
                        continue;
                    }
                }
                size_t kn = CI(s, ii, jj);
                double mf = 0.5 * (mu[k] + mu[kn]);
                acc += mf * (x[k] - x[kn]);
            }
            y[k] = acc;
        }
}

static void pot_rhs_diag(const oracle_state* s, double* b, double* d)
{
    int nx = s->nx, ny = s->ny;
    const double* mu = s->mu_m;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = CI(s, i, j);
            double bb = 0.0, dd = 0.0;
            double wx[4] = {0.0, (double)nx, i + 0.5, i + 0.5};
            double wy[4] = {j + 0.5, j + 0.5, 0.0, (double)ny};
            int nb_i[4] = {i - 1, i + 1, i, i};
            int nb_j[4] = {j, j, j - 1, j + 1};
            for (int w = 0; w < 4; ++w) {
                int ii = nb_i[w], jj = nb_j[w];
                int outside = ii < 0 || ii >= nx || jj < 0 || jj >= ny;
                if (outside) {
                    int periodic = (w < 2) ? s->cs.periodic_x : s->cs.periodic_y;
                    if (periodic) {
                        ii = (ii + nx) % nx;
                        jj = (jj + ny) % ny;
                    } else {
                        if (wall_is_dirichlet_phi(s, w)) {
                            dd += 2.0 * mu[k];
                            bb += 2.0 * mu[k] * phi_far(s, wx[w], wy[w]);
                        }
                        continue;
                    }
                }
                dd += 0.5 * (mu[k] + mu[CI(s, ii, jj)]);
            }
            b[k] = bb;
            d[k] = dd;
        }
}

static double dot(const double* a, const double* b, size_t n)
{
    double acc = 0.0;
    for (size_t k = 0; k < n; ++k) acc += a[k] * b[k];
    return acc;
}

static void set_mu_m(oracle_state* s, double* const* W)
{
    const oracle_case* c = &s->cs;
    size_t N = (size_t)s->nx * s->ny;
    for (size_t k = 0; k < N; ++k) {
        double T, Fl;
        oracle_eq8(c, W[W_HE][k], W[W_C][k], &T, &Fl);
        s->mu_m[k] = 1.0 + oracle_mix(1.0 - Fl, W[W_C][k], c->chi_s, c->chi_l, c->chi_g);
    }
}

int oracle_solve_potential(oracle_state* s)
{
    size_t N = (size_t)s->nx * s->ny;
    if (!needs_potential_solve(s)) {
        /* chi = 0 everywhere (no Kelvin force) or no Dirichlet wall: the potential is
         * left as it is (the uniform far field unless imported) */
        s->pot_resid = 0.0;
        s->pot_iters = 0;
        return 0;
    }
    set_mu_m(s, s->W);
    double* b = (double*)malloc(N * sizeof(double));
    double* d = (double*)malloc(N * sizeof(double));
    double* r = (double*)malloc(N * sizeof(double));
    double* z = (double*)malloc(N * sizeof(double));
    double* p = (double*)malloc(N * sizeof(double));
    double* Ap = (double*)malloc(N * sizeof(double));
    pot_rhs_diag(s, b, d);
    double bn = sqrt(dot(b, b, N));
    if (bn == 0.0) bn = 1.0;
    pot_apply(s, s->phi, Ap);
    for (size_t k = 0; k < N; ++k) r[k] = b[k] - Ap[k];
    for (size_t k = 0; k < N; ++k) z[k] = r[k] / d[k];
    memcpy(p, z, N * sizeof(double));
    double rz = dot(r, z, N);
    int it = 0;
    const int max_it = 50000;
    while (sqrt(dot(r, r, N)) > 1e-14 * bn && it < max_it) {
        pot_apply(s, p, Ap);
        double alpha = rz / dot(p, Ap, N);
        for (size_t k = 0; k < N; ++k) {
            s->phi[k] += alpha * p[k];
            r[k] -= alpha * Ap[k];
        }
        for (size_t k = 0; k < N; ++k) z[k] = r[k] / d[k];
        double rz_new = dot(r, z, N);
        double beta = rz_new / rz;
        rz = rz_new;
        for (size_t k = 0; k < N; ++k) p[k] = z[k] + beta * p[k];
        ++it;
    }
    pot_apply(s, s->phi, Ap);
    for (size_t k = 0; k < N; ++k) r[k] = b[k] - Ap[k];
    s->pot_resid = sqrt(dot(r, r, N)) / bn;
    s->pot_iters = it;
    free(b); free(d); free(r); free(z); free(p); free(Ap);
    return s->pot_resid <= 1e-11 ? 0 : 3;
}

/* |H|^2 at cell centres, H = -grad phi (Eq. 3) by central differences; the ghost
 * potential follows the potential's wall condition; |H|^2 in the ghost layer
 * copies the inner value. */
static void compute_H2(oracle_state* s)
{
    int nx = s->nx, ny = s->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double ph[4];
            int nb_i[4] = {i - 1, i + 1, i, i};
            int nb_j[4] = {j, j, j - 1, j + 1};
            double wx[4] = {0.0, (double)nx, i + 0.5, i + 0.5};
            double wy[4] = {j + 0.5, j + 0.5, 0.0, (double)ny};
            double pc = s->phi[CI(s, i, j)];
            for (int w = 0; w < 4; ++w) {
                int ii = nb_i[w], jj = nb_j[w];
                if (ii >= 0 && ii < nx && jj >= 0 && jj < ny) {
                    ph[w] = s->phi[CI(s, ii, jj)];
                } else if ((w < 2) ? s->cs.periodic_x : s->cs.periodic_y) {
                    ph[w] = s->phi[CI(s, (ii + nx) % nx, (jj + ny) % ny)];
                } else if (wall_is_dirichlet_phi(s, w)) {
                    ph[w] = 2.0 * phi_far(s, wx[w], wy[w]) - pc;
                } else {
                    ph[w] = pc;
                }
            }
            double Hx = -0.5 * (ph[1] - ph[0]);
            double Hy = -0.5 * (ph[3] - ph[2]);
            s->H2[GI(s, i, j)] = Hx * Hx + Hy * Hy;
        }
    fill_ghosts(s, s->H2, GH_EVEN);
}

/* ---- one time step in the order of Table 1:
 *  1. F_s^n from Eq. 8; lagged dF_s/dt = (F_s^n - F_s^{n-1})/dt held over the step
 *  2. magnetic potential solved to convergence (the garbled "while magnetic field is
 *     convergent" is read as: converge the potential before the thermo-fluid update)
 *  3. three Runge-Kutta stages (Shu-Osher SSP-RK3, the third-order scheme cited)
 *  4. Eq. 8 of the new state; the solid is held at rest by F_IBM in the momentum
 *     source and, at the end of the step, (rho u) <- (1 - F_s)(rho u). ------- */
static void step_once(oracle_state* s, int* status)
{
    const oracle_case* c = &s->cs;
    size_t N = (size_t)s->nx * s->ny;
    double dt = c->dt;
    for (size_t k = 0; k < N; ++k) {
        double T, Fl;
        oracle_eq8(c, s->W[W_HE][k], s->W[W_C][k], &T, &Fl);
        double Fs = 1.0 - Fl;
        s->Sdot[k] = (Fs - s->Fs_prev[k]) / dt;
        s->Fs_prev[k] = Fs; /* becomes F_s^{n} for the next step */
    }
    if (!(c->flags & ORACLE_FLAG_KEEP_POTENTIAL)) {
        int st = oracle_solve_potential(s);
        if (st && !*status) *status = st;
    }
    compute_H2(s);
    for (int n = 0; n < W_N; ++n) memcpy(s->w0 + n * N, s->W[n], N * sizeof(double));
    double* W0[W_N];
    for (int n = 0; n < W_N; ++n) W0[n] = s->w0 + n * N;
    /* stage 1: W1 = W0 + dt R(W0) */
    compute_rhs(s, s->W, s->rhs);
    for (int n = 0; n < W_N; ++n)
        for (size_t k = 0; k < N; ++k) s->W[n][k] = W0[n][k] + dt * s->rhs[n * N + k];
    /* stage 2: W2 = 3/4 W0 + 1/4 (W1 + dt R(W1)) */
    compute_rhs(s, s->W, s->rhs);
    for (int n = 0; n < W_N; ++n)
        for (size_t k = 0; k < N; ++k)
            s->W[n][k] = 0.75 * W0[n][k] + 0.25 * (s->W[n][k] + dt * s->rhs[n * N + k]);
    /* stage 3: W^{n+1} = 1/3 W0 + 2/3 (W2 + dt R(W2)) */
    compute_rhs(s, s->W, s->rhs);
    for (int n = 0; n < W_N; ++n)
        for (size_t k = 0; k < N; ++k)
            s->W[n][k] = W0[n][k] / 3.0 + 2.0 / 3.0 * (s->W[n][k] + dt * s->rhs[n * N + k]);
    for (size_t k = 0; k < N; ++k) {
        double T, Fl;
        oracle_eq8(c, s->W[W_HE][k], s->W[W_C][k], &T, &Fl);
        s->W[W_MX][k] *= Fl;
        s->W[W_MY][k] *= Fl;
    }
    s->t += dt;
    s->nstep += 1;
    /* freezing time: first t with Q_L >= 0.99, interpolated between steps (Eq. 51
     * with A_0 the number of droplet cells C >= 1/2) */
    oracle_stats st2;
    oracle_get_stats(s, &st2);
    if (s->t_freeze < 0.0 && st2.Q_L >= 0.99) {
        double q0 = s->QL_prev;
        s->t_freeze = (s->t - dt) + dt * (0.99 - q0) / (st2.Q_L - q0);
    }
    s->QL_prev = st2.Q_L;
}

int oracle_step(oracle_state* s, int32_t nsteps)
{
    int status = 0;
    for (int n = 0; n < nsteps; ++n) step_once(s, &status);
    return status;
}

void oracle_get_stats(oracle_state* s, oracle_stats* out)
{
    const oracle_case* c = &s->cs;
    size_t N = (size_t)s->nx * s->ny;
    double sC = 0, sH = 0, nd = 0, sFs = 0, sFl = 0;
    int bad = 0;
    for (size_t k = 0; k < N; ++k) {
        double C = s->W[W_C][k], He = s->W[W_HE][k];
        for (int n = 0; n < W_N; ++n)
            if (!isfinite(s->W[n][k])) bad = 1;
        sC += C;
        sH += He;
        if (C >= 0.5) {
            double T, Fl;
            oracle_eq8(c, He, C, &T, &Fl);
            nd += 1.0;
            sFs += 1.0 - Fl;
            sFl += Fl;
        }
    }
    out->sum_C = sC;
    out->sum_He = sH;
    out->n_drop = nd;
    out->sum_Fl_drop = sFl;
    out->Q_L = nd > 0 ? sFs / nd : 0.0;
    out->t = s->t;
    out->t_freeze = s->t_freeze;
    out->pot_resid = s->pot_resid;
    out->pot_iters = s->pot_iters;
    out->nonfinite = bad;
}

/* ---- initial condition (Table 1 "Initialization"): droplet
 * C = 1/2 + 1/2 tanh(2 (R - r)/xi), the equilibrium profile of the mu_c free energy;
 * uniform T = T_init; liquid everywhere (F_s = 0) so H_e = C_p T + L; p = 0,
 * u = 0, phi = uniform far field. --------------------------------------------- */
static void init_fields(oracle_state* s)
{
    const oracle_case* c = &s->cs;
    for (int j = 0; j < s->ny; ++j)
        for (int i = 0; i < s->nx; ++i) {
            size_t k = CI(s, i, j);
            double x = i + 0.5, y = j + 0.5, C;
            if (c->init == 2) {
                C = 1.0;
            } else {
                double cx = c->init == 0 ? 0.5 * s->nx : c->drop_x;
                double cy = c->init == 0 ? 0.0 : c->drop_y;
                double r = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
                C = 0.5 + 0.5 * tanh(2.0 * (c->radius - r) / c->xi);
            }
            double cp = oracle_mix(0.0, C, c->cp_s, c->cp_l, c->cp_g);
            s->W[W_C][k] = C;
            s->W[W_HE][k] = cp * c->T_init + s->L;
            s->W[W_P][k] = 0.0;
            s->W[W_MX][k] = 0.0;
            s->W[W_MY][k] = 0.0;
            s->phi[k] = phi_far(s, x, y);
            double T, Fl;
            oracle_eq8(c, s->W[W_HE][k], C, &T, &Fl);
            s->Fs_prev[k] = 1.0 - Fl;
        }
}

int oracle_create(const oracle_case* cs, oracle_state** out)
{
    if (!cs || !out || cs->nx < 1 || cs->ny < 1) return 1;
    if (cs->dt <= 0.0 || cs->dts <= 0.0 || cs->Q_g <= 0.0) return 1;
    oracle_state* s = (oracle_state*)calloc(1, sizeof(oracle_state));
    if (!s) return 2;
    s->cs = *cs;
    s->nx = cs->nx;
    s->ny = cs->ny;
    /* magnetic Bond number on the droplet diameter (Eq. 50): H0 = sqrt(Bo_m sigma/(mu_0 2R)) */
    s->H0 = cs->bo_m > 0.0 ? sqrt(cs->bo_m * cs->sigma / (2.0 * cs->radius)) : cs->H0;
    s->L = latent_of(cs);
    s->beta = 12.0 * cs->sigma / cs->xi;
    s->kappa = 1.5 * cs->xi * cs->sigma;
    s->cos_t = cos(cs->field_angle_deg * ORACLE_PI / 180.0);
    s->sin_t = sin(cs->field_angle_deg * ORACLE_PI / 180.0);
    s->cp_ref = 0.5 * (cs->cp_s + cs->cp_l);
    s->vol_ratio = 1.0 - cs->rho_s / cs->rho_l;
    s->wet = cs->contact_angle_deg == 90.0 ? 0.0
                                           : 4.0 * cos(cs->contact_angle_deg * ORACLE_PI / 180.0) / cs->xi;
    size_t N = (size_t)s->nx * s->ny;
    size_t NG = (size_t)(s->nx + 2) * (s->ny + 2);
    for (int n = 0; n < W_N; ++n) s->W[n] = (double*)calloc(N, sizeof(double));
    s->phi = (double*)calloc(N, sizeof(double));
    s->Fs_prev = (double*)calloc(N, sizeof(double));
    s->Sdot = (double*)calloc(N, sizeof(double));
    s->mu_m = (double*)calloc(N, sizeof(double));
    for (int n = 0; n < Q_N; ++n) {
        s->q[n] = (double*)calloc(NG, sizeof(double));
        s->gx[n] = (double*)calloc(N, sizeof(double));
        s->gy[n] = (double*)calloc(N, sizeof(double));
    }
    s->Fs = (double*)calloc(NG, sizeof(double));
    s->rho = (double*)calloc(NG, sizeof(double));
    s->H2 = (double*)calloc(NG, sizeof(double));
    s->phig = (double*)calloc(NG, sizeof(double));
    s->Fx = (double*)calloc((size_t)(s->nx + 1) * s->ny * 5, sizeof(double));
    s->Fy = (double*)calloc((size_t)s->nx * (s->ny + 1) * 5, sizeof(double));
    s->rhs = (double*)calloc(5 * N, sizeof(double));
    s->w0 = (double*)calloc(5 * N, sizeof(double));
    s->t_freeze = -1.0;
    init_fields(s);
    oracle_stats st;
    oracle_get_stats(s, &st);
    s->QL_prev = st.Q_L;
    *out = s;
    return 0;
}

void oracle_destroy(oracle_state* s)
{
    if (!s) return;
    for (int n = 0; n < W_N; ++n) free(s->W[n]);
    free(s->phi); free(s->Fs_prev); free(s->Sdot); free(s->mu_m);
    for (int n = 0; n < Q_N; ++n) { free(s->q[n]); free(s->gx[n]); free(s->gy[n]); }
    free(s->Fs); free(s->rho); free(s->H2); free(s->phig); free(s->Fx); free(s->Fy); free(s->rhs); free(s->w0);
    free(s);
}

int oracle_get_field(oracle_state* s, int32_t field, double* out)
{
    size_t N = (size_t)s->nx * s->ny;
    const oracle_case* c = &s->cs;
    switch (field) {
    case OF_PHI: memcpy(out, s->phi, N * sizeof(double)); return 0;
    case OF_HE: memcpy(out, s->W[W_HE], N * sizeof(double)); return 0;
    case OF_P: memcpy(out, s->W[W_P], N * sizeof(double)); return 0;
    case OF_C: memcpy(out, s->W[W_C], N * sizeof(double)); return 0;
    case OF_MX: memcpy(out, s->W[W_MX], N * sizeof(double)); return 0;
    case OF_MY: memcpy(out, s->W[W_MY], N * sizeof(double)); return 0;
    case OF_FSPREV: memcpy(out, s->Fs_prev, N * sizeof(double)); return 0;
    case OF_MUC:
        derive(s, s->W);
        for (int j = 0; j < s->ny; ++j)
            for (int i = 0; i < s->nx; ++i) out[CI(s, i, j)] = s->q[Q_MUC][GI(s, i, j)];
        return 0;
    default: break;
    }
    for (size_t k = 0; k < N; ++k) {
        double He = s->W[W_HE][k], C = s->W[W_C][k], T, Fl;
        oracle_eq8(c, He, C, &T, &Fl);
        double rho = oracle_mix(1.0 - Fl, C, c->rho_s, c->rho_l, c->rho_g);
        switch (field) {
        case OF_T: out[k] = T; break;
        case OF_FL: out[k] = Fl; break;
        case OF_U: out[k] = s->W[W_MX][k] / (rho * CS2); break;
        case OF_V: out[k] = s->W[W_MY][k] / (rho * CS2); break;
        case OF_RHO: out[k] = rho; break;
        default: return 1;
        }
    }
    return 0;
}

int oracle_set_field(oracle_state* s, int32_t field, const double* in)
{
    size_t N = (size_t)s->nx * s->ny;
    double* dst = NULL;
    switch (field) {
    case OF_PHI: dst = s->phi; break;
    case OF_HE: dst = s->W[W_HE]; break;
    case OF_P: dst = s->W[W_P]; break;
    case OF_C: dst = s->W[W_C]; break;
    case OF_MX: dst = s->W[W_MX]; break;
    case OF_MY: dst = s->W[W_MY]; break;
    case OF_FSPREV: dst = s->Fs_prev; break;
    default: return 1;
    }
    memcpy(dst, in, N * sizeof(double));
    return 0;
}

/* ---- Sec. 5 diagnostics --------------------------------------------------------
 * Local heat flux on the cold substrate (Sec. 5.2): Q = -lambda dT/dy at y = 0, the
 * gradient by a second-order one-sided difference.  The quadratic through the wall
 * value T_w (y = 0) and the first two cell centres (y = 1/2, 3/2) has the slope
 * (-8 T_w + 9 T_0 - T_1)/3 at the wall; with a single row the two-point slope
 * (T_0 - T_w)/(1/2) is used.  lambda is the first cell's Eq. 11 value.  An adiabatic
 * bottom wall has Q = 0, and a periodic y axis has no wall (Q = 0).
 * Droplet height H_m (Sec. 5.1, Fig. 11): in each column the highest point where C
 * crosses 1/2, linear in y between the cell centres on either side (ny when the top
 * cell has C >= 1/2); H_m is the largest over the columns, 0 without droplet cells.
 * Peclet number (Eq. 50, printed garbled as D u^2/alpha): read as U D / alpha_l with
 * U the largest speed |u| over the droplet cells (C >= 1/2), D = 2 R_0 and
 * alpha_l = lambda_l/(rho_l C_p,l).  Fourier number (Eq. 50): lambda_l t/(rho_l C_p,l R_0^2).
 * ------------------------------------------------------------------------------ */
int oracle_diagnostics(oracle_state* s, oracle_diag* out, double* q_wall)
{
    const oracle_case* c = &s->cs;
    const int nx = s->nx, ny = s->ny;
    const int wall = !c->periodic_y && c->thermal_dirichlet[2];
    double Hm = 0.0, Umax = 0.0, Qsum = 0.0;
    for (int i = 0; i < nx; ++i) {
        /* height: scan down from the top for the first droplet cell */
        for (int j = ny - 1; j >= 0; --j) {
            double C = s->W[W_C][CI(s, i, j)];
            if (C >= 0.5) {
                double h;
                if (j == ny - 1) {
                    h = (double)ny;
                } else {
                    double Cu = s->W[W_C][CI(s, i, j + 1)];
                    h = (j + 0.5) + (C - 0.5) / (C - Cu);
                }
                if (h > Hm) Hm = h;
                break;
            }
        }
        /* largest speed over the column's droplet cells */
        for (int j = 0; j < ny; ++j) {
            size_t k = CI(s, i, j);
            double C = s->W[W_C][k];
            if (C < 0.5) continue;
            double T, Fl;
            oracle_eq8(c, s->W[W_HE][k], C, &T, &Fl);
            double rho = oracle_mix(1.0 - Fl, C, c->rho_s, c->rho_l, c->rho_g);
            double u = s->W[W_MX][k] / (rho * CS2), v = s->W[W_MY][k] / (rho * CS2);
            double sp = sqrt(u * u + v * v);
            if (sp > Umax) Umax = sp;
        }
        /* wall heat flux of this column */
        double Q = 0.0;
        if (wall) {
            double T0, Fl0;
            size_t k0 = CI(s, i, 0);
            oracle_eq8(c, s->W[W_HE][k0], s->W[W_C][k0], &T0, &Fl0);
            double lam = oracle_mix(1.0 - Fl0, s->W[W_C][k0], c->lam_s, c->lam_l, c->lam_g);
            double Tw = c->wall_T[2], dTdy;
            if (ny >= 2) {
                double T1, Fl1;
                size_t k1 = CI(s, i, 1);
                oracle_eq8(c, s->W[W_HE][k1], s->W[W_C][k1], &T1, &Fl1);
                dTdy = (-8.0 * Tw + 9.0 * T0 - T1) / 3.0;
            } else {
                dTdy = (T0 - Tw) / 0.5;
            }
            Q = -lam * dTdy;
        }
        if (q_wall) q_wall[i] = Q;
        Qsum += Q;
    }
    const double R0 = c->radius;
    const double alpha_l = c->lam_l / (c->rho_l * c->cp_l);
    out->H_m = Hm;
    out->U_max = Umax;
    out->Pe = Umax * 2.0 * R0 / alpha_l;
    out->Fo = c->lam_l * s->t / (c->rho_l * c->cp_l * R0 * R0);
    out->Q_wall = Qsum;
    return 0;
}

/* ---- pieces for pin tests ---------------------------------------------------- */

/* flux of one face of the current state; Sdot and |H|^2 are not used by fluxes */
int oracle_face_flux(oracle_state* s, int32_t axis, int32_t i, int32_t j, double* flux5)
{
    derive(s, s->W);
    int wall = -1;
    if (axis == 0 && !s->cs.periodic_x && (i == 0 || i == s->nx)) wall = i == 0 ? 0 : 1;
    if (axis == 1 && !s->cs.periodic_y && (j == 0 || j == s->ny)) wall = j == 0 ? 2 : 3;
    if (wall >= 0) {
        int ii = wall == 1 ? s->nx - 1 : (wall == 0 ? 0 : i);
        int jj = wall == 3 ? s->ny - 1 : (wall == 2 ? 0 : j);
        wall_face(s, wall, ii, jj, flux5);
    } else {
        lbfs_face(s, axis, i, j, flux5);
    }
    return 0;
}

/* Magnetic LBFS (Eqs. 13, 16, 17, 44, 45) at one interior face for the current
 * potential: m_eq = w_a phi at the surrounding points, phi_f by Eq. 45,
 * m_neq = -tau_m (m_eq(x_f) - m_eq(x - e_a dts)), m* by Eq. 16, flux
 * sum_a (e_a.n) m*_a, tau_m = 1/2 + mu_face D/(c_s^2 dts) with D = 1.
 * The potential's gradient uses the same ghost rule as |H|^2. */
double oracle_mag_lbfs_flux(oracle_state* s, int32_t axis, int32_t i, int32_t j, double mu_face)
{
    int nx = s->nx, ny = s->ny;
    const double dts = s->cs.dts;
    double* ph = s->phig;
    for (int jj = 0; jj < ny; ++jj)
        for (int ii = 0; ii < nx; ++ii) ph[GI(s, ii, jj)] = s->phi[CI(s, ii, jj)];
    for (int jj = 0; jj < ny; ++jj) {
        ph[GI(s, -1, jj)] = s->cs.periodic_x ? ph[GI(s, nx - 1, jj)]
                            : wall_is_dirichlet_phi(s, 0) ? 2.0 * phi_far(s, 0.0, jj + 0.5) - ph[GI(s, 0, jj)]
                                                          : ph[GI(s, 0, jj)];
        ph[GI(s, nx, jj)] = s->cs.periodic_x ? ph[GI(s, 0, jj)]
                            : wall_is_dirichlet_phi(s, 1) ? 2.0 * phi_far(s, nx, jj + 0.5) - ph[GI(s, nx - 1, jj)]
                                                          : ph[GI(s, nx - 1, jj)];
    }
    for (int ii = 0; ii < nx; ++ii) {
        ph[GI(s, ii, -1)] = s->cs.periodic_y ? ph[GI(s, ii, ny - 1)]
                            : wall_is_dirichlet_phi(s, 2) ? 2.0 * phi_far(s, ii + 0.5, 0.0) - ph[GI(s, ii, 0)]
                                                          : ph[GI(s, ii, 0)];
        ph[GI(s, ii, ny)] = s->cs.periodic_y ? ph[GI(s, ii, 0)]
                            : wall_is_dirichlet_phi(s, 3) ? 2.0 * phi_far(s, ii + 0.5, ny) - ph[GI(s, ii, ny - 1)]
                                                          : ph[GI(s, ii, ny - 1)];
    }
    int ia, ja, ib, jb;
    double ax0, ay0, bx0, by0;
    int nxn = axis == 0, nyn = axis == 1;
    if (axis == 0) {
        ia = (i - 1 + nx) % nx; ja = j; ib = i % nx; jb = j;
        ax0 = -0.5; ay0 = 0.0; bx0 = 0.5; by0 = 0.0;
    } else {
        ia = i; ja = (j - 1 + ny) % ny; ib = i; jb = j % ny;
        ax0 = 0.0; ay0 = -0.5; bx0 = 0.0; by0 = 0.5;
    }
    double gAx = 0.5 * (ph[GI(s, ia + 1, ja)] - ph[GI(s, ia - 1, ja)]);
    double gAy = 0.5 * (ph[GI(s, ia, ja + 1)] - ph[GI(s, ia, ja - 1)]);
    double gBx = 0.5 * (ph[GI(s, ib + 1, jb)] - ph[GI(s, ib - 1, jb)]);
    double gBy = 0.5 * (ph[GI(s, ib, jb + 1)] - ph[GI(s, ib, jb - 1)]);
    double meq[9], phi_f = 0.0;
    for (int a = 0; a < 9; ++a) {
        int en = EX[a] * nxn + EY[a] * nyn;
        double px = -EX[a] * dts, py = -EY[a] * dts;
        double vA = ph[GI(s, ia, ja)] + (px - ax0) * gAx + (py - ay0) * gAy;
        double vB = ph[GI(s, ib, jb)] + (px - bx0) * gBx + (py - by0) * gBy;
        double v = en > 0 ? vA : (en < 0 ? vB : 0.5 * (vA + vB));
        meq[a] = WA[a] * v; /* Eq. 13 */
        phi_f += meq[a];    /* Eq. 45 */
    }
    double tau = 0.5 + mu_face / (CS2 * dts);
    double F = 0.0;
    for (int a = 0; a < 9; ++a) {
        double meqF = WA[a] * phi_f;
        double mneq = -tau * (meqF - meq[a]);
        double mstar = meqF + (1.0 - 1.0 / (2.0 * tau)) * mneq; /* Eq. 16 */
        F += (EX[a] * nxn + EY[a] * nyn) * mstar;
    }
    return F;
}

/* The paper's own magnetic solver: integrate Eq. 17 in pseudo time with the
 * per-direction LBFS flux above (forward Euler in pseudo time), with the sign
 * chosen so that the iteration relaxes towards div(mu grad phi) = 0 and mu at a
 * face the arithmetic mean.  Used only to show that its steady state is the
 * potential the direct solver returns. */
int oracle_pseudo_time_potential(oracle_state* s, int32_t iters, double dtau)
{
    int nx = s->nx, ny = s->ny;
    size_t N = (size_t)nx * ny;
    set_mu_m(s, s->W);
    double* upd = (double*)malloc(N * sizeof(double));
    for (int it = 0; it < iters; ++it) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double div = 0.0;
                size_t k = CI(s, i, j);
                /* faces: left, right, bottom, top with outward sign */
                int fa[4] = {0, 0, 1, 1};
                int fi[4] = {i, i + 1, i, i};
                int fj[4] = {j, j, j, j + 1};
                double sg[4] = {-1.0, 1.0, -1.0, 1.0};
                for (int f = 0; f < 4; ++f) {
                    int wall = -1;
                    if (fa[f] == 0 && !s->cs.periodic_x && (fi[f] == 0 || fi[f] == nx))
                        wall = fi[f] == 0 ? 0 : 1;
                    if (fa[f] == 1 && !s->cs.periodic_y && (fj[f] == 0 || fj[f] == ny))
                        wall = fj[f] == 0 ? 2 : 3;
                    double Fl;
                    if (wall >= 0) {
                        if (!wall_is_dirichlet_phi(s, wall)) continue;
                        double wx = wall == 0 ? 0.0 : wall == 1 ? nx : i + 0.5;
                        double wy = wall == 2 ? 0.0 : wall == 3 ? ny : j + 0.5;
                        double side = (wall == 0 || wall == 2) ? 1.0 : -1.0;
                        /* compact flux -mu (phi_+ - phi_-) with the Dirichlet ghost */
                        Fl = -s->mu_m[k] * side * (s->phi[k] - phi_far(s, wx, wy)) * 2.0;
                    } else {
                        int ii = fa[f] == 0 ? fi[f] : i, jj = fa[f] == 1 ? fj[f] : j;
                        int ka_i = fa[f] == 0 ? (ii - 1 + nx) % nx : ii;
                        int ka_j = fa[f] == 1 ? (jj - 1 + ny) % ny : jj;
                        int kb_i = fa[f] == 0 ? ii % nx : ii;
                        int kb_j = fa[f] == 1 ? jj % ny : jj;
                        double muf = 0.5 * (s->mu_m[CI(s, ka_i, ka_j)] + s->mu_m[CI(s, kb_i, kb_j)]);
                        Fl = oracle_mag_lbfs_flux(s, fa[f], ii, jj, muf);
                    }
                    div += sg[f] * Fl;
                }
                upd[k] = -div;
            }
        for (size_t k = 0; k < N; ++k) s->phi[k] += dtau * upd[k];
    }
    free(upd);
    return 0;
}

int oracle_rhs(oracle_state* s, double* rhs5)
{
    const oracle_case* c = &s->cs;
    size_t N = (size_t)s->nx * s->ny;
    for (size_t k = 0; k < N; ++k) {
        double T, Fl;
        oracle_eq8(c, s->W[W_HE][k], s->W[W_C][k], &T, &Fl);
        s->Sdot[k] = ((1.0 - Fl) - s->Fs_prev[k]) / c->dt;
    }
    compute_H2(s);
    compute_rhs(s, s->W, rhs5);
    return 0;
}
