// lbfs_stage.cu -- one Runge-Kutta stage of the LBFS finite-volume update, fused per
// tile: load the stage state with a three-cell halo into shared memory, derive the
// cell quantities (Eq. 8 inversion, Eq. 11 mixture, velocity, mu_c, |H|^2), build
// every face flux of the tile by the LBFS reconstruction (Eqs. 44, 45, 20, 28, 29,
// 22, 32, 33, 43), add the sources (Eq. 41), form R(W) (Eq. 42) and the SSP-RK3
// combination, and write the next stage.  Stage 1 also forms the lagged dF_s/dt of
// the step; the last stage applies the step-end rest condition of the solid, writes
// the potential coefficient mu_m for the next solve, and reduces the diagnostics.
#include <cstdio>

#include "lbfs_internal.cuh"
#include "lbfs_kernels.h"

namespace lbfs {

enum { SP = 0, SU, SV, SC, ST, SHE, SFS, SRHO, SMU, SPHI, SH2, NSH };

template <int TX, int TY>
struct Geom {
    static constexpr int H = 3;
    static constexpr int RW = TX + 2 * H, RH = TY + 2 * H, RN = RW * RH;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NF = NFX + NFY;
};

// Per-face flux by the LBFS reconstruction, in the face frame (n normal, t
// tangential).  Cells A (lower/left) and B (upper/right) at region indices kA and
// kB = kA + sn; st is the region stride along t.  For X = h, g and the f^{eq-m} form
// of f the starred distribution is X*_a = (3/2 - tau) X_eq,a(x_f) + (tau - 1/2)
// X_eq,a(x - e_a dts) (Eqs. 16, 22, 32, 33 with X_neq = -tau (X_eq(x_f) -
// X_eq(x - e_a dts))); the x_f parts of the fluxes follow from the D2Q9 moments of
// the interface equilibria, so only the surrounding-point equilibria are summed per
// direction.  HALF: the streaming step is half a cell, so the points of the
// upwind cells sit on its centre line and the normal slopes drop out there.
// One side of a face: the three points with e_a.n = SG at c (e_a.t = 0), c - h (e_a.t = +1)
// and c + h (e_a.t = -1); weights 1/9 and 1/36 for SG = +-1, 4/9 and 1/9 for SG = 0, whose
// centre point is the rest direction a = 0.  Adds the side's equilibria (Eqs. 20, 28,
// 29) to the face sums: Sp = sum f_eq, Sjn/Sjt = sum e_n/e_t f_eq, SC_ = sum g_eq,
// SH = sum h_eq, Ah/Ag = sum e_n h_eq / g_eq, BGn/BGt = sum (e_n; e_n e_t) w Gamma_a.
// Each point's terms are formed unweighted and the weights applied once per side.
template <class R, int SG>
__device__ __forceinline__ void side_sums(const R c[7], const R h[7], R r0, R r1, R k0, R k1, R cpref, R Qg,
                                          R& Sp, R& Sjn, R& Sjt, R& SC_, R& SH, R& Ah, R& Ag, R& BGn, R& BGt) {
    constexpr bool REST = SG == 0;
    const R w0 = REST ? R(4.0 / 9.0) : R(1.0 / 9.0), w1 = REST ? R(1.0 / 9.0) : R(1.0 / 36.0);
    R F[3], Gm[3], Hh[3], Ga[3];
    R heq0 = 0, geq0 = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int et = e == 0 ? 0 : (e == 1 ? 1 : -1);
        R q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = et == 0 ? c[k] : (et > 0 ? c[k] - h[k] : c[k] + h[k]);
        const R p = q[0], un = q[1], ut = q[2], C = q[3], mu = q[4], T = q[5];
        const R rho = r0 + r1 * C, cp = k0 + k1 * C;
        const R eu = R(SG) * un + R(et) * ut;
        const R uu = un * un + ut * ut;
        const R G = eu * (R(3) + R(4.5) * eu) - R(1.5) * uu;   // Gamma_a(u)
        F[e] = p + rho * G * R(1.0 / 3.0);
        Gm[e] = G;
        Hh[e] = T * (cpref + cp * G);
        Ga[e] = mu * Qg + C * eu;
        if (REST && e == 0) {
            // a = 0: g_eq = C - (5/3) mu Q_g, h_eq = H_e - C_p,ref T + w0 T (C_p,ref + C_p Gamma)
            geq0 = C - R(5.0 / 3.0) * mu * Qg;
            heq0 = c[6] - cpref * T + w0 * Hh[0];
        }
    }
    const R Fs = w0 * F[0] + w1 * (F[1] + F[2]);
    Sp += Fs;
    Sjt += w1 * (F[1] - F[2]);
    if (REST) {
        SC_ += geq0 + R(3) * w1 * (Ga[1] + Ga[2]);
        SH += heq0 + w1 * (Hh[1] + Hh[2]);
    } else {
        const R gs = R(3) * (w0 * Ga[0] + w1 * (Ga[1] + Ga[2]));
        const R hs = w0 * Hh[0] + w1 * (Hh[1] + Hh[2]);
        SC_ += gs;
        SH += hs;
        Sjn += R(SG) * Fs;
        Ag += R(SG) * gs;
        Ah += R(SG) * hs;
        BGn += w0 * Gm[0] + w1 * (Gm[1] + Gm[2]);
        BGt += R(SG) * w1 * (Gm[1] - Gm[2]);
    }
}

// The cells one face reads, as offsets into a field's shared array: A (lower/left)
// and B (upper/right), the cells beyond them along the normal (Am = A - n, Bp = B + n)
// and their neighbours along the tangent (Atp/Atm = A +- t, Btp/Btm = B +- t).
struct FaceCells {
    int A, B, Am, Bp, Atp, Atm, Btp, Btm;
};

// One face.  The three sides are built one after the other, and only what a later
// side needs is kept (the cell values and tangential slopes of A and B), so that few
// values are live at once.
// ---- packed FP32: two lanes per instruction (Blackwell FADD2 / FMUL2 / FFMA2) ----
__device__ __forceinline__ float2 sp2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Sides A (e_a.n = +1, lane x) and B (e_a.n = -1, lane y) of a face together, as packed
// FP32: the same point equilibria as side_sums<float, +1> and <float, -1>, two sides per
// instruction.  c, h: the cell values and tangential half-slopes of A (x) and B (y);
// r0 + r1 C and k0 + k1 C: Eq. 11 for rho and C_p on each side.
__device__ __forceinline__ void side_sums_ab(const float2 c[6], const float2 h[6], float2 r0, float2 r1, float2 k0,
                                             float2 k1, float cpref, float Qg, float& Sp, float& Sjn, float& Sjt,
                                             float& SC_, float& SH, float& Ah, float& Ag, float& BGn, float& BGt) {
    const float2 sg = make_float2(1.f, -1.f);
    float2 F[3], Gm[3], Hh[3], Ga[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int et = e == 0 ? 0 : (e == 1 ? 1 : -1);
        float2 q[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = et == 0 ? c[k] : (et > 0 ? sub2(c[k], h[k]) : add2(c[k], h[k]));
        const float2 p = q[0], un = q[1], ut = q[2], C = q[3], mu = q[4], T = q[5];
        const float2 rho = fma2(r1, C, r0), cp = fma2(k1, C, k0);
        const float2 eu = et == 0 ? mul2(sg, un) : (et > 0 ? fma2(sg, un, ut) : fma2(sg, un, make_float2(-ut.x, -ut.y)));
        const float2 uu = fma2(un, un, mul2(ut, ut));
        const float2 G = fma2(sp2(-1.5f), uu, mul2(eu, fma2(sp2(4.5f), eu, sp2(3.f))));   // Gamma_a(u)
        F[e] = fma2(mul2(rho, G), sp2(1.f / 3.f), p);
        Gm[e] = G;
        Hh[e] = mul2(T, fma2(cp, G, sp2(cpref)));
        Ga[e] = fma2(C, eu, mul2(mu, sp2(Qg)));
    }
    const float w0 = 1.f / 9.f, w1 = 1.f / 36.f;
    const float2 F12 = add2(F[1], F[2]);
    const float2 Fs = fma2(sp2(w0), F[0], mul2(sp2(w1), F12));
    const float2 gs = mul2(sp2(3.f), fma2(sp2(w0), Ga[0], mul2(sp2(w1), add2(Ga[1], Ga[2]))));
    const float2 hs = fma2(sp2(w0), Hh[0], mul2(sp2(w1), add2(Hh[1], Hh[2])));
    const float2 bg = fma2(sp2(w0), Gm[0], mul2(sp2(w1), add2(Gm[1], Gm[2])));
    const float2 dF = mul2(sp2(w1), sub2(F[1], F[2]));
    const float2 dG = mul2(sp2(w1), sub2(Gm[1], Gm[2]));
    Sp += Fs.x + Fs.y;
    Sjn += Fs.x - Fs.y;
    Sjt += dF.x + dF.y;
    SC_ += gs.x + gs.y;
    Ag += gs.x - gs.y;
    SH += hs.x + hs.y;
    Ah += hs.x - hs.y;
    BGn += bg.x + bg.y;
    BGt += dG.x - dG.y;
}

// The rest side (e_a.n = 0) in packed FP32: its centre point (the rest direction) in
// scalar form, its two tangential points c - h (e_a.t = +1, lane x) and c + h
// (e_a.t = -1, lane y) as two lanes; the same equilibria as side_sums<float, 0>.
__device__ __forceinline__ void side_sums_rest2(const float c[7], const float h[7], float r0, float r1, float k0,
                                                float k1, float cpref, float Qg, float& Sp, float& Sjt, float& SC_,
                                                float& SH, float& BGn) {
    const float w0 = 4.f / 9.f, w1 = 1.f / 9.f;
    // centre: e_a = 0, so e.u = 0
    const float uu0 = c[1] * c[1] + c[2] * c[2];
    const float G0 = -1.5f * uu0;
    const float rho0 = r0 + r1 * c[3], cp0 = k0 + k1 * c[3];
    const float F0 = c[0] + rho0 * G0 * (1.f / 3.f);
    const float Hh0 = c[5] * (cpref + cp0 * G0);
    // the tangential pair
    float2 q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = make_float2(c[k] - h[k], c[k] + h[k]);
    const float2 un = q[1], ut = q[2], C = q[3];
    const float2 eu = make_float2(ut.x, -ut.y);
    const float2 rho = fma2(sp2(r1), C, sp2(r0)), cp = fma2(sp2(k1), C, sp2(k0));
    const float2 uu = fma2(un, un, mul2(ut, ut));
    const float2 G = fma2(sp2(-1.5f), uu, mul2(eu, fma2(sp2(4.5f), eu, sp2(3.f))));
    const float2 F = fma2(mul2(rho, G), sp2(1.f / 3.f), q[0]);
    const float2 Hh = mul2(q[5], fma2(cp, G, sp2(cpref)));
    const float2 Ga = fma2(C, eu, mul2(q[4], sp2(Qg)));
    // a = 0: g_eq = C - (5/3) mu Q_g, h_eq = H_e - C_p,ref T + w0 T (C_p,ref + C_p Gamma)
    const float geq0 = c[3] - (5.f / 3.f) * c[4] * Qg;
    const float heq0 = c[6] - cpref * c[5] + w0 * Hh0;
    Sp += w0 * F0 + w1 * (F.x + F.y);
    Sjt += w1 * (F.x - F.y);
    SC_ += geq0 + 3.f * w1 * (Ga.x + Ga.y);
    SH += heq0 + w1 * (Hh.x + Hh.y);
    (void)BGn;
}

template <class R, bool HALF>
__device__ __forceinline__ void face_flux(const PhysT<R>& Q, const R* __restrict__ s, int RN, const FaceCells& k,
                                          bool xface, R& Fh, R& Fp, R& Fmn, R& Fmt, R& Fc) {
    const int fun = xface ? SU : SV, fut = xface ? SV : SU;
    const int qf[7] = {SP, fun, fut, SC, SMU, ST, SHE};
    const R dts = Q.dts;
    const R FsA = s[SFS * RN + k.A], FsB = s[SFS * RN + k.B], Fsm = R(0.5) * (FsA + FsB);
    const R cpref = Q.cp_ref, Qg = Q.Q_g;
    const R rs = Q.rho_s, rl = Q.rho_l, rg = Q.rho_g, cs = Q.cp_s, cl = Q.cp_l, cg = Q.cp_g;
    R Sp = 0, Sjn = 0, Sjt = 0, SC_ = 0, SH = 0, Ah = 0, Ag = 0, BGn = 0, BGt = 0;
    R a[6], b[6], ta[6], tb[6];
    R pA, pB, hA0, hB0;
    if constexpr (sizeof(R) == 4) {
        // sides A (e_a.n = +1, from A) and B (e_a.n = -1, from B), two lanes of packed FP32
        float2 c[6], h[6];
        const float2 dt2 = sp2(dts);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const R* f = s + qf[q] * RN;
            a[q] = f[k.A];
            b[q] = f[k.B];
            const float2 t = mul2(sp2(0.5f), sub2(make_float2(f[k.Atp], f[k.Btp]), make_float2(f[k.Atm], f[k.Btm])));
            ta[q] = t.x;
            tb[q] = t.y;
            h[q] = mul2(dt2, t);
            c[q] = make_float2(a[q], b[q]);
            // the centre point moves along the normal by (1/2 - dts) cells unless dts = 1/2
            if (!HALF)
                c[q] = fma2(make_float2(R(0.5) - dts, R(-0.5) + dts),
                            mul2(sp2(0.5f), make_float2(f[k.B] - f[k.Am], f[k.Bp] - f[k.A])), c[q]);
        }
        const float2 Fs2 = make_float2(FsA, FsB);
        const float2 r0 = fma2(Fs2, sp2(rs - rg), sp2(rg)), r1 = mul2(sub2(sp2(1.f), Fs2), sp2(rl - rg));
        const float2 k0 = fma2(Fs2, sp2(cs - cg), sp2(cg)), k1 = mul2(sub2(sp2(1.f), Fs2), sp2(cl - cg));
        side_sums_ab(c, h, r0, r1, k0, k1, cpref, Qg, Sp, Sjn, Sjt, SC_, SH, Ah, Ag, BGn, BGt);
        pA = c[0].x;
        pB = c[0].y;
        hA0 = h[0].x;
        hB0 = h[0].y;
    } else {
    // side A: the three points with e_a.n = +1, reconstructed from A (Eq. 44)
    {
        R c[7], h[7];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const R* f = s + qf[q] * RN;
            a[q] = f[k.A];
            ta[q] = R(0.5) * (f[k.Atp] - f[k.Atm]);
            h[q] = dts * ta[q];
            c[q] = a[q];
            // the centre point moves along the normal by (1/2 - dts) cells unless dts = 1/2
            if (!HALF) c[q] += (R(0.5) - dts) * (R(0.5) * (f[k.B] - f[k.Am]));
        }
        c[6] = h[6] = R(0);
        // Eq. 11 at fixed F_s is affine in C: rho = r0 + r1 C, C_p = c0 + c1 C
        const R r0 = rg + FsA * (rs - rg), r1 = (R(1) - FsA) * (rl - rg);
        const R k0 = cg + FsA * (cs - cg), k1 = (R(1) - FsA) * (cl - cg);
        side_sums<R, 1>(c, h, r0, r1, k0, k1, cpref, Qg, Sp, Sjn, Sjt, SC_, SH, Ah, Ag, BGn, BGt);
        pA = c[0];
        hA0 = h[0];
    }
    // side B: e_a.n = -1, from B
    {
        R c[7], h[7];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const R* f = s + qf[q] * RN;
            b[q] = f[k.B];
            tb[q] = R(0.5) * (f[k.Btp] - f[k.Btm]);
            h[q] = dts * tb[q];
            c[q] = b[q];
            if (!HALF) c[q] += (R(-0.5) + dts) * (R(0.5) * (f[k.Bp] - f[k.A]));
        }
        c[6] = h[6] = R(0);
        const R r0 = rg + FsB * (rs - rg), r1 = (R(1) - FsB) * (rl - rg);
        const R k0 = cg + FsB * (cs - cg), k1 = (R(1) - FsB) * (cl - cg);
        side_sums<R, -1>(c, h, r0, r1, k0, k1, cpref, Qg, Sp, Sjn, Sjt, SC_, SH, Ah, Ag, BGn, BGt);
        pB = c[0];
        hB0 = h[0];
    }
    }
    // side M: e_a.n = 0, the mean of both cells' reconstructions at the face centre
    // (and half the mean tangential slope)
    const R rM0 = rg + Fsm * (rs - rg), rM1 = (R(1) - Fsm) * (rl - rg);
    const R cM0 = cg + Fsm * (cs - cg), cM1 = (R(1) - Fsm) * (cl - cg);
    {
        R m0[7], hs[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const R* f = s + qf[q] * RN;
            const R av = q < 6 ? a[q] : f[k.A], bv = q < 6 ? b[q] : f[k.B];
            // (a + b)/2 + ((b - a_m) - (b_p - a))/8: the mean of the two cells' linear
            // reconstructions at the face centre
            m0[q] = R(0.625) * (av + bv) - R(0.125) * (f[k.Am] + f[k.Bp]);
            hs[q] = q < 6 ? R(0.5) * dts * (ta[q] + tb[q]) : R(0);
        }
        if constexpr (sizeof(R) == 4)
            side_sums_rest2(m0, hs, rM0, rM1, cM0, cM1, cpref, Qg, Sp, Sjt, SC_, SH, BGn);
        else
            side_sums<R, 0>(m0, hs, rM0, rM1, cM0, cM1, cpref, Qg, Sp, Sjn, Sjt, SC_, SH, Ah, Ag, BGn, BGt);
    }
    // sum over e_a.n != 0 of w_a p and of (e_a.n)(e_a.t) w_a p: the three points of a side
    // carry the weights 1/9, 1/36, 1/36 and sit at c, c - h, c + h along t
    const R Bpn = R(1.0 / 6.0) * (pA + pB);
    const R Bpt = R(1.0 / 18.0) * (hB0 - hA0);
    // Eq. 45: interface values
    const R Cf = SC_, pf = Sp, Hef = SH;
    const R rhof = rM0 + rM1 * Cf;
    const R inv_rc = fdiv(R(3), rhof);                 // 1 / (rho_f c_s^2)
    const R ufn = Sjn * inv_rc, uft = Sjt * inv_rc;
    const R cpf = cM0 + cM1 * Cf;
    const R lamf = mix(Fsm, Cf, Q.lam_s, Q.lam_l, Q.lam_g);
    const R muf = mix(Fsm, Cf, Q.mu_s, Q.mu_l, Q.mu_g);
    R Tf, Flf;
    invert_h<R, R>(Q, cs * Q.T_m, Q.L, Hef, Cf, Tf, Flf);
    const R tau_f = R(0.5) + muf * inv_rc * Q.inv_dts;
    const R tau_h = R(0.5) + lamf * inv_rc * Q.inv_cpref_dts;
    const R tau_g = Q.tau_g;
    const R c3 = R(1.0 / 3.0);
    Fh = (R(1.5) - tau_h) * cpf * Tf * ufn + (tau_h - R(0.5)) * Ah;
    Fc = (R(1.5) - tau_g) * Cf * ufn + (tau_g - R(0.5)) * Ag;
    Fp = Sjn;
    Fmn = (R(1.5) - tau_f) * c3 * (pf + rhof * ufn * ufn) + (tau_f - R(0.5)) * (Bpn + rhof * c3 * BGn);
    Fmt = (R(1.5) - tau_f) * c3 * rhof * ufn * uft + (tau_f - R(0.5)) * (Bpt + rhof * c3 * BGt);
}

// the cells of an interior face in a region laid out with row stride st (x faces:
// normal stride 1; y faces: normal stride st, tangential stride 1)
__device__ __forceinline__ FaceCells region_face(int kA, int sn, int st) {
    FaceCells k;
    k.A = kA;
    k.B = kA + sn;
    k.Am = kA - sn;
    k.Bp = kA + 2 * sn;
    k.Atp = kA + st;
    k.Atm = kA - st;
    k.Btp = kA + sn + st;
    k.Btm = kA + sn - st;
    return k;
}

// Wall face (no-slip, no-flux): momentum flux c_s^2 (p n - mu du_t/dn) with the wall
// half a cell from the inner centre; enthalpy flux -(lambda/rho) dT/dn on Dirichlet
// walls, zero on adiabatic ones; no mass or phase-field flux.
template <class R>
__device__ __forceinline__ void wall_flux(const PhysT<R>& Q, int dirichlet, const R* __restrict__ s,
                                          int RN, int k, int wall, R F[5]) {
    const R Fs = s[SFS * RN + k], C = s[SC * RN + k];
    const R rho = s[SRHO * RN + k];
    const R mu = mix(Fs, C, Q.mu_s, Q.mu_l, Q.mu_g);
    const R lam = mix(Fs, C, Q.lam_s, Q.lam_l, Q.lam_g);
    const R side = (wall == 0 || wall == 2) ? R(1) : R(-1);
    const R ut = wall < 2 ? s[SV * RN + k] : s[SU * RN + k];
    const R dut = side * ut * R(2);
    const R dT = side * (s[ST * RN + k] - Q.wall_T[wall]) * R(2);
    const R c3 = R(1.0 / 3.0);
    F[1] = R(0);
    F[4] = R(0);
    if (wall < 2) {
        F[2] = c3 * s[SP * RN + k];
        F[3] = c3 * (-mu * dut);
    } else {
        F[3] = c3 * s[SP * RN + k];
        F[2] = c3 * (-mu * dut);
    }
    F[0] = dirichlet ? -fdiv(lam, rho) * dT : R(0);
}

// Asynchronous copy of one 4- or 8-byte element from global to shared memory
// (cp.async, cached in L1), and the wait for all of this thread's copies.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Eq. 8 on the stored enthalpy: FP64 differences in the FP64 mode, FP32-pair
// differences in mixed precision (the thresholds' lo parts are zero in FP64).
template <class R>
__device__ __forceinline__ void invert_state(const PhysT<R>& Q, typename HeStore<R>::T He, R C, R& T, R& Fl,
                                             R* He_r = nullptr) {
    if constexpr (sizeof(R) == 8)
        invert_h<double, double>(Q, Q.Hes_hi, Q.L_hi, He, C, T, Fl, He_r);
    else
        invert_hp(Q, He, C, T, Fl, He_r);
}

// H_e's Runge-Kutta update: stage 1 W + dt R(W); later stages W^n + b ((W + dt R) - W^n)
// (a W^n + b X with a + b = 1 exactly).  FP64 in the FP64 mode.  In mixed precision the
// stage increment is small next to H_e and is formed in FP32 from the pairs'
// difference (their high parts subtract exactly when close), then added to the pair.
__device__ __forceinline__ double he_rk(int stage, double Hek, double He0, double dt, double Rw, double b) {
    if (stage == 0) return Hek + dt * Rw;
    return He0 + b * ((Hek + dt * Rw) - He0);
}
__device__ __forceinline__ float2 he_rk(int stage, float2 Hek, float2 He0, float dt, float Rw, float b) {
    if (stage == 0) return pair_add_f(Hek, __fmul_rn(dt, Rw));
    const float d = __fadd_rn(__fsub_rn(Hek.x, He0.x), __fsub_rn(Hek.y, He0.y));
    return pair_add_f(He0, __fmul_rn(b, __fmaf_rn(dt, Rw, d)));
}
__device__ __forceinline__ bool he_finite(double h) { return isfinite(h); }
__device__ __forceinline__ bool he_finite(float2 h) { return isfinite(h.x) && isfinite(h.y); }

// byte offset of the prefetch area in the stage kernel's dynamic shared memory
template <class R>
__host__ __device__ constexpr size_t stage_pf_offset(int RN, int NF) {
    return ((size_t)(NSH * RN + 5 * NF) * sizeof(R) + RN + 15) / 16 * 16;
}

template <class R, class HR, int TX, int TY, int NT, int MINB, bool HALF>
__global__ void __launch_bounds__(NT, MINB) stage_kernel(const DevCase* __restrict__ cases,
                                                         const TileRef* __restrict__ tiles, int ntiles,
                                                         int stage) {
    using Gm = Geom<TX, TY>;
    constexpr int RW = Gm::RW, RH = Gm::RH, RN = Gm::RN, NFX = Gm::NFX, NF = Gm::NF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* s = reinterpret_cast<R*>(smem_raw);
    R* flux = s + NSH * RN;                                             // [5][NF]
    signed char* kind = reinterpret_cast<signed char*>(flux + 5 * NF);  // [RN]
    constexpr int TXY = TX * TY;
    HR* pf_h = reinterpret_cast<HR*>(smem_raw + stage_pf_offset<R>(RN, NF));  // [2][TXY]
    R* pf_r = reinterpret_cast<R*>(pf_h + 2 * TXY);                          // [9][TXY]
    __shared__ CaseParams P;
    __shared__ PhysT<R> Q;
    // step-end values of the tile's cells (last stage): C, F_l of droplet cells, H_e
    __shared__ R red_c[TX * TY], red_f[TX * TY];
    __shared__ HR red_h[TX * TY];
    __shared__ int red_n[NT / 32][2];
    static_assert(NT >= TX * TY, "phase 4 gives each thread at most one cell");

    // one tile per block
    const int tile_i = blockIdx.x;
    if (tile_i >= ntiles) return;
    const TileRef tr = tiles[tile_i];
    const DevCase* dc = cases + tr.case_id;
    {
        const int* src = reinterpret_cast<const int*>(&dc->P);
        int* dst = reinterpret_cast<int*>(&P);
        for (int i = threadIdx.x; i < (int)(sizeof(CaseParams) / sizeof(int)); i += NT) dst[i] = src[i];
        const int* srq = reinterpret_cast<const int*>(&phys_of<R>(dc));
        int* dsq = reinterpret_cast<int*>(&Q);
        for (int i = threadIdx.x; i < (int)(sizeof(PhysT<R>) / sizeof(int)); i += NT) dsq[i] = srq[i];
    }
    const int in = stage == 0 ? 0 : (stage == 1 ? 1 : 2);
    const int out = stage == 0 ? 1 : (stage == 1 ? 2 : 0);
    const HR* __restrict__ gHe = static_cast<const HR*>(dc->He[in]);
    const R* __restrict__ gP = static_cast<const R*>(dc->p[in]);
    const R* __restrict__ gMx = static_cast<const R*>(dc->mx[in]);
    const R* __restrict__ gMy = static_cast<const R*>(dc->my[in]);
    const R* __restrict__ gC = static_cast<const R*>(dc->C[in]);
    const R* __restrict__ gPhi = static_cast<const R*>(dc->phi);
    // the grid size and periodic flags in registers, read alongside the copy above, so
    // that the prefetch and the halo loads below are issued before the copy lands (the
    // barrier after the halo loads publishes P and Q)
    const int nx = dc->P.nx, ny = dc->P.ny, pitch = dc->P.pitch;
    const bool per_x = dc->P.periodic_x != 0, per_y = dc->P.periodic_y != 0;
    const int x0 = tr.x0, y0 = tr.y0;
    const HR* bHe = static_cast<const HR*>(dc->He[0]);
    const R* bP = static_cast<const R*>(dc->p[0]);
    const R* bMx = static_cast<const R*>(dc->mx[0]);
    const R* bMy = static_cast<const R*>(dc->my[0]);
    const R* bC = static_cast<const R*>(dc->C[0]);
    R* Fsp = static_cast<R*>(dc->Fs_prev);
    R* Sdp = static_cast<R*>(dc->Sdot);

    // ---- prefetch of the phase-4 operands of this thread's cell: asynchronous copies
    // into shared memory that land while phases 1-3 run.  pf_h: stage input H_e, W^n
    // H_e; pf_r: stage input p, m_x, m_y, C; F_s of the previous step (stage 1) or the
    // lagged dF_s/dt (stages 2, 3); W^n p, m_x, m_y, C.
    if (threadIdx.x < TXY) {
        const int pc = threadIdx.x;
        const int gx = x0 + pc % TX, gy = y0 + pc / TX;
        if (gx < nx && gy < ny) {
            const unsigned gi = (unsigned)gy * (unsigned)pitch + (unsigned)gx;
            cp_async_elem(&pf_h[pc], gHe + gi);
            cp_async_elem(&pf_r[0 * TXY + pc], gP + gi);
            cp_async_elem(&pf_r[1 * TXY + pc], gMx + gi);
            cp_async_elem(&pf_r[2 * TXY + pc], gMy + gi);
            cp_async_elem(&pf_r[3 * TXY + pc], gC + gi);
            if (stage == 0) {
                cp_async_elem(&pf_r[4 * TXY + pc], static_cast<const R*>(Fsp) + gi);
            } else {
                cp_async_elem(&pf_r[4 * TXY + pc], static_cast<const R*>(Sdp) + gi);
                cp_async_elem(&pf_h[TXY + pc], bHe + gi);
                cp_async_elem(&pf_r[5 * TXY + pc], bP + gi);
                cp_async_elem(&pf_r[6 * TXY + pc], bMx + gi);
                cp_async_elem(&pf_r[7 * TXY + pc], bMy + gi);
                cp_async_elem(&pf_r[8 * TXY + pc], bC + gi);
            }
        }
    }

    // ---- phase 1: load the stage state with halo, ghost rules at walls ----------
    // All of a thread's region loads are issued before any is used (one memory latency
    // per tile instead of one per region cell of the thread).
    // One region cell from its loaded stage state: T, F_l and the reconstruction H_e by
    // Eq. 8, rho by Eq. 11, u = m / (rho / 3); at a wall ghost the mirror rules.
    auto derive = [&](int k, HR He, R C, R pv, R mx, R my, R phi, int wall, unsigned gi) {
        R T, Fl;
        R Hes;   // H_e for the reconstruction (enters only the interface T_f)
        invert_state<R>(Q, He, C, T, Fl, &Hes);
        const R Fs = R(1) - Fl;
        const R rho = mix(Fs, C, Q.rho_s, Q.rho_l, Q.rho_g);
        const R rinv = fdiv(R(3), rho);
        R u = mx * rinv, v = my * rinv;
        if (wall >= 0) {
            u = -u;
            v = -v;
            if (P.thermal_dir[wall]) T = R(2) * Q.wall_T[wall] - T;
            const R cp = mix(Fs, C, Q.cp_s, Q.cp_l, Q.cp_g);
            Hes = cp * T + Q.L * (R(1) - Fs);
            if (P.mag_dir[wall]) {
                const int sx = (int)(gi % (unsigned)pitch), sy = (int)(gi / (unsigned)pitch);
                double wx = wall == 0 ? 0.0 : (wall == 1 ? (double)nx : sx + 0.5);
                double wy = wall == 2 ? 0.0 : (wall == 3 ? (double)ny : sy + 0.5);
                double pw = -P.H0 * (wx * P.cos_t + wy * P.sin_t);
                phi = R(2.0 * pw) - phi;
            }
        }
        s[SP * RN + k] = pv;
        s[SU * RN + k] = u;
        s[SV * RN + k] = v;
        // a wall ghost's C follows the wetting rule (unchanged at 90 degrees, wet = 0)
        s[SC * RN + k] = wall >= 0 ? C + Q.wet * C * (R(1) - C) : C;
        s[ST * RN + k] = T;
        s[SHE * RN + k] = Hes;
        s[SFS * RN + k] = Fs;
        s[SRHO * RN + k] = rho;
        s[SPHI * RN + k] = phi;
    };
    // An interior tile, whose region lies inside the grid, has no ghost and no wrap: its
    // region cell (lx, ly) is the grid cell (x0 - H + lx, y0 - H + ly).  The region's
    // border ring, three cells from the tile, enters only the Laplacian of C and the
    // gradient of phi in phase 2, so there an interior tile reads C and phi and derives
    // nothing.
    const bool interior = x0 >= Gm::H && x0 + TX + Gm::H <= nx && y0 >= Gm::H && y0 + TY + Gm::H <= ny;
    if (interior) {
        constexpr int IW = RW - 2, IN = IW * (RH - 2), IROUNDS = (IN + NT - 1) / NT;
        constexpr int NB = 2 * (RW + RH) - 4;
        static_assert(NB <= NT, "one border cell per thread");
        const R* __restrict__ cbase = gC + (size_t)(y0 - Gm::H) * pitch + (x0 - Gm::H);
        const R* __restrict__ pbase = gPhi + (size_t)(y0 - Gm::H) * pitch + (x0 - Gm::H);
        const HR* __restrict__ hbase = gHe + (size_t)(y0 - Gm::H) * pitch + (x0 - Gm::H);
        const R* __restrict__ qbase = gP + (size_t)(y0 - Gm::H) * pitch + (x0 - Gm::H);
        const R* __restrict__ xbase = gMx + (size_t)(y0 - Gm::H) * pitch + (x0 - Gm::H);
        const R* __restrict__ ybase = gMy + (size_t)(y0 - Gm::H) * pitch + (x0 - Gm::H);
        HR lHe[IROUNDS];
        R lC[IROUNDS], lP[IROUNDS], lMx[IROUNDS], lMy[IROUNDS], lPhi[IROUNDS];
#pragma unroll
        for (int i = 0; i < IROUNDS; ++i) {
            const int t = threadIdx.x + i * NT;
            if (t >= IN) break;
            const int lx = 1 + t % IW, ly = 1 + t / IW;
            const unsigned o = (unsigned)ly * (unsigned)pitch + (unsigned)lx;
            lHe[i] = hbase[o];
            lC[i] = cbase[o];
            lP[i] = qbase[o];
            lMx[i] = xbase[o];
            lMy[i] = ybase[o];
            lPhi[i] = pbase[o];
        }
        // the border ring: bottom row, top row, then the two side columns
        int kb = -1;
        R bC = 0, bPhi = 0;
        if (threadIdx.x < NB) {
            const int t = threadIdx.x;
            int lx, ly;
            if (t < RW) {
                lx = t;
                ly = 0;
            } else if (t < 2 * RW) {
                lx = t - RW;
                ly = RH - 1;
            } else {
                const int u = t - 2 * RW;
                lx = (u & 1) ? RW - 1 : 0;
                ly = 1 + (u >> 1);
            }
            kb = ly * RW + lx;
            const unsigned o = (unsigned)ly * (unsigned)pitch + (unsigned)lx;
            bC = cbase[o];
            bPhi = pbase[o];
        }
        __syncthreads();   // P and Q in shared memory
        if (kb >= 0) {
            s[SC * RN + kb] = bC;
            s[SPHI * RN + kb] = bPhi;
        }
#pragma unroll
        for (int i = 0; i < IROUNDS; ++i) {
            const int t = threadIdx.x + i * NT;
            if (t >= IN) break;
            const int k = (1 + t / IW) * RW + 1 + t % IW;
            derive(k, lHe[i], lC[i], lP[i], lMx[i], lMy[i], lPhi[i], -1, 0);
        }
    } else {
        constexpr int ROUNDS = (RN + NT - 1) / NT;
        HR lHe[ROUNDS];
        R lC[ROUNDS], lP[ROUNDS], lMx[ROUNDS], lMy[ROUNDS], lPhi[ROUNDS];
        unsigned lGi[ROUNDS];
        int lWall[ROUNDS];
#pragma unroll
        for (int i = 0; i < ROUNDS; ++i) {
            const int k = threadIdx.x + i * NT;
            if (k >= RN) break;
            const int lx = k % RW, ly = k / RW;
            const int gx = x0 - Gm::H + lx, gy = y0 - Gm::H + ly;
            int sx, sy, xs, ys;  // source cell and status: 0 inside, 1 ghost low, 2 ghost high, 3 far
            if (per_x) {
                sx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
                xs = 0;
            } else if (gx >= 0 && gx < nx) {
                sx = gx; xs = 0;
            } else if (gx == -1) {
                sx = 0; xs = 1;
            } else if (gx == nx) {
                sx = nx - 1; xs = 2;
            } else {
                sx = gx < 0 ? 0 : nx - 1; xs = 3;
            }
            if (per_y) {
                sy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
                ys = 0;
            } else if (gy >= 0 && gy < ny) {
                sy = gy; ys = 0;
            } else if (gy == -1) {
                sy = 0; ys = 1;
            } else if (gy == ny) {
                sy = ny - 1; ys = 2;
            } else {
                sy = gy < 0 ? 0 : ny - 1; ys = 3;
            }
            // a periodic halo can reach past one period only on grids narrower than the halo
            sx = sx < 0 ? 0 : (sx >= nx ? nx - 1 : sx);
            sy = sy < 0 ? 0 : (sy >= ny ? ny - 1 : sy);
            int wall = -1;
            signed char kd;
            if (xs == 0 && ys == 0) {
                kd = 0;
            } else if ((xs == 1 || xs == 2) && ys == 0) {
                wall = xs - 1;
                kd = (signed char)(1 + wall);
            } else if (xs == 0 && (ys == 1 || ys == 2)) {
                wall = 2 + ys - 1;
                kd = (signed char)(1 + wall);
            } else {
                kd = 5;
            }
            kind[k] = kd;
            const unsigned gi = (unsigned)sy * (unsigned)pitch + (unsigned)sx;
            lGi[i] = gi;
            lWall[i] = wall;
            lHe[i] = gHe[gi];
            lC[i] = gC[gi];
            lP[i] = gP[gi];
            lMx[i] = gMx[gi];
            lMy[i] = gMy[gi];
            lPhi[i] = gPhi[gi];
        }
        __syncthreads();   // P and Q in shared memory
#pragma unroll
        for (int i = 0; i < ROUNDS; ++i) {
            const int k = threadIdx.x + i * NT;
            if (k >= RN) break;
            derive(k, lHe[i], lC[i], lP[i], lMx[i], lMy[i], lPhi[i], lWall[i], lGi[i]);
        }
    }
    __syncthreads();
    // ---- phase 2: mu_c and |H|^2 at inner cells; a wall ghost takes the values of
    // the inner cell it mirrors (computed there again rather than copied, which saves
    // a barrier).  The faces and sources read mu_c and |H|^2 no further than two cells
    // from the tile, so an interior tile computes them on that (RW-2) x (RH-2) core
    // only, with no ghost to resolve. -------------------------------------------------
    if (interior) {
        constexpr int CW = RW - 2, CN = (RW - 2) * (RH - 2);
        for (int t = threadIdx.x; t < CN; t += NT) {
            const int k = (1 + t / CW) * RW + 1 + t % CW;
            const R* c = s + SC * RN;
            const R C = c[k];
            const R lap = (c[k + 1] + c[k - 1]) + (c[k + RW] + c[k - RW]) - R(4) * C;
            s[SMU * RN + k] = R(2) * Q.beta * C * (C - R(1)) * (R(2) * C - R(1)) - Q.kappa * lap;
            const R* ph = s + SPHI * RN;
            const R hx = R(-0.5) * (ph[k + 1] - ph[k - 1]);
            const R hy = R(-0.5) * (ph[k + RW] - ph[k - RW]);
            s[SH2 * RN + k] = hx * hx + hy * hy;
        }
    } else
    for (int k = threadIdx.x; k < RN; k += NT) {
        const int kd = kind[k];
        int kk = k;
        if (kd >= 1 && kd <= 4) {
            const int w = kd - 1;
            kk = k + (w == 0 ? 1 : w == 1 ? -1 : w == 2 ? RW : -RW);
        }
        const int lx = kk % RW, ly = kk / RW;
        R mu = 0, h2 = 0;
        if (kd <= 4 && kind[kk] == 0 && lx > 0 && lx < RW - 1 && ly > 0 && ly < RH - 1) {
            const R* c = s + SC * RN;
            const R C = c[kk];
            const R lap = (c[kk + 1] + c[kk - 1]) + (c[kk + RW] + c[kk - RW]) - R(4) * C;
            mu = R(2) * Q.beta * C * (C - R(1)) * (R(2) * C - R(1)) - Q.kappa * lap;
            const R* ph = s + SPHI * RN;
            const R hx = R(-0.5) * (ph[kk + 1] - ph[kk - 1]);
            const R hy = R(-0.5) * (ph[kk + RW] - ph[kk - RW]);
            h2 = hx * hx + hy * hy;
        }
        s[SMU * RN + k] = mu;
        s[SH2 * RN + k] = h2;
    }
    __syncthreads();
    // ---- phase 3: face fluxes ------------------------------------------------------
    // Face f is stored at flux index fs (x faces row by row, then y faces row by row).
    // With 16-row tiles the threads take the faces column by column instead: a warp
    // then reads two columns of 16 cells, whose shared-memory banks are all distinct
    // because the region pitch RW is twice an odd number; the last y row follows.
    constexpr bool COLS = TY == 16 && (RW % 4) == 2;
    for (int f = threadIdx.x; f < NF; f += NT) {
        R F[5] = {0, 0, 0, 0, 0};
        int fs;
        if (f < NFX) {
            const int fx = COLS ? f / TY : f % (TX + 1), ty = COLS ? f % TY : f / (TX + 1);
            fs = ty * (TX + 1) + fx;
            const int gxf = x0 + fx, gy = y0 + ty;
            if (gy < ny && gxf <= nx) {
                const int kB = (ty + Gm::H) * RW + fx + Gm::H, kA = kB - 1;
                if (!P.periodic_x && gxf == 0) {
                    wall_flux<R>(Q, P.thermal_dir[0], s, RN, kB, 0, F);
                } else if (!P.periodic_x && gxf == nx) {
                    wall_flux<R>(Q, P.thermal_dir[1], s, RN, kA, 1, F);
                } else {
                    face_flux<R, HALF>(Q, s, RN, region_face(kA, 1, RW), true, F[0], F[1], F[2], F[3], F[4]);
                }
            }
        } else {
            const int g = f - NFX;
            const int tx = (COLS && g < TX * TY) ? g / TY : g % TX;
            const int fy = (COLS && g < TX * TY) ? g % TY : g / TX;
            fs = NFX + fy * TX + tx;
            const int gx = x0 + tx, gyf = y0 + fy;
            if (gx < nx && gyf <= ny) {
                const int kB = (fy + Gm::H) * RW + tx + Gm::H, kA = kB - RW;
                if (!P.periodic_y && gyf == 0) {
                    wall_flux<R>(Q, P.thermal_dir[2], s, RN, kB, 2, F);
                } else if (!P.periodic_y && gyf == ny) {
                    wall_flux<R>(Q, P.thermal_dir[3], s, RN, kA, 3, F);
                } else {
                    face_flux<R, HALF>(Q, s, RN, region_face(kA, RW, 1), false, F[0], F[1], F[3], F[2], F[4]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) flux[c * NF + fs] = F[c];
    }
    __syncthreads();
    // ---- phase 4: R(W), sources, Runge-Kutta combination ------------------------
    const R c3 = R(1.0 / 3.0);
    const double b_rk = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
    const R b = R(b_rk);
    const R dt = Q.dt;
    // step-end sums of this thread's cells: C, H_e and F_l (FP64-accurate), counts
    int nDrop = 0, nBad = 0;
    HR* oHe = static_cast<HR*>(dc->He[out]);
    R* oP = static_cast<R*>(dc->p[out]);
    R* oMx = static_cast<R*>(dc->mx[out]);
    R* oMy = static_cast<R*>(dc->my[out]);
    R* oC = static_cast<R*>(dc->C[out]);
    cp_async_wait_all();   // this thread's prefetched operands (its own cell only)
    for (int c = threadIdx.x; c < TX * TY; c += NT) {
        const int tx = c % TX, ty = c / TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= nx || gy >= ny) {
            if (stage == 2) {
                red_c[c] = R(0);
                red_f[c] = R(0);
                red_h[c] = he_zero<HR>();
            }
            continue;
        }
        const int k = (ty + Gm::H) * RW + tx + Gm::H;
        const int fl = ty * (TX + 1) + tx, fb = NFX + ty * TX + tx;
        R Rw[5];
#pragma unroll
        for (int q = 0; q < 5; ++q)
            Rw[q] = -(flux[q * NF + fl + 1] - flux[q * NF + fl]) -
                    (flux[q * NF + fb + TX] - flux[q * NF + fb]);
        const R Fs = s[SFS * RN + k], C = s[SC * RN + k], T = s[ST * RN + k];
        const R u = s[SU * RN + k], v = s[SV * RN + k], rho = s[SRHO * RN + k];
        const R cp = mix(Fs, C, Q.cp_s, Q.cp_l, Q.cp_g);
        const R chi = mix(Fs, C, Q.chi_s, Q.chi_l, Q.chi_g);
        const R divu = R(0.5) * (s[SU * RN + k + 1] - s[SU * RN + k - 1]) +
                       R(0.5) * (s[SV * RN + k + RW] - s[SV * RN + k - RW]);
        const R drx = R(0.5) * (s[SRHO * RN + k + 1] - s[SRHO * RN + k - 1]);
        const R dry = R(0.5) * (s[SRHO * RN + k + RW] - s[SRHO * RN + k - RW]);
        const R dhx = R(0.5) * (s[SH2 * RN + k + 1] - s[SH2 * RN + k - 1]);
        const R dhy = R(0.5) * (s[SH2 * RN + k + RW] - s[SH2 * RN + k - RW]);
        const R dmx = R(0.5) * (s[SMU * RN + k + 1] - s[SMU * RN + k - 1]);
        const R dmy = R(0.5) * (s[SMU * RN + k + RW] - s[SMU * RN + k - RW]);
        const unsigned gi = (unsigned)gy * (unsigned)pitch + (unsigned)gx;
        // lagged dF_s/dt: formed by stage 1 from F_s^n (this stage's own input) and the
        // previous step's F_s, which is then replaced by F_s^n
        R Sd;
        if (stage == 0) {
            Sd = (Fs - pf_r[4 * TXY + c]) / dt;
            Fsp[gi] = Fs;
            Sdp[gi] = Sd;
        } else {
            Sd = pf_r[4 * TXY + c];
        }
        const R vr = Q.vol_ratio;
        Rw[0] += cp * T * divu;
        Rw[1] += c3 * (u * drx + v * dry) + rho * c3 * vr * Sd;
        Rw[2] += c3 * (-C * dmx + R(0.5) * chi * dhx - rho * u * Sd);
        Rw[3] += c3 * (-C * dmy + R(0.5) * chi * dhy + rho * Q.gravity - rho * v * Sd);
        Rw[4] += C * vr * Sd;
        // stage input at this cell
        const HR Hek = pf_h[c];
        const R pk = pf_r[0 * TXY + c], mxk = pf_r[1 * TXY + c], myk = pf_r[2 * TXY + c], Ck = pf_r[3 * TXY + c];
        const HR Hen = he_rk(stage, Hek, stage == 0 ? Hek : pf_h[TXY + c], dt, Rw[0], b);
        R pn, mxn, myn, Cn;
        if (stage == 0) {
            pn = pk + dt * Rw[1];
            mxn = mxk + dt * Rw[2];
            myn = myk + dt * Rw[3];
            Cn = Ck + dt * Rw[4];
        } else {
            // a W^n + b X written as W^n + b (X - W^n): a + b = 1 holds exactly, so a
            // steady state stays steady in FP32 (1/3 and 2/3 both round up in FP32)
            const R p0 = pf_r[5 * TXY + c], mx0 = pf_r[6 * TXY + c], my0 = pf_r[7 * TXY + c],
                    C0 = pf_r[8 * TXY + c];
            pn = p0 + b * ((pk + dt * Rw[1]) - p0);
            mxn = mx0 + b * ((mxk + dt * Rw[2]) - mx0);
            myn = my0 + b * ((myk + dt * Rw[3]) - my0);
            Cn = C0 + b * ((Ck + dt * Rw[4]) - C0);
        }
        if (stage == 2) {
            // step end: solid held at rest, (rho u) <- (1 - F_s)(rho u)
            R Tn, Fln;
            invert_state<R>(Q, Hen, Cn, Tn, Fln);
            mxn *= Fln;
            myn *= Fln;
            const R Fsn = R(1) - Fln;
            R* mu0 = static_cast<R*>(dc->lev[0].mu);
            mu0[(unsigned)gy * (unsigned)dc->lev[0].pitch + (unsigned)gx] = R(1) + mix(Fsn, Cn, Q.chi_s, Q.chi_l, Q.chi_g);
            red_c[c] = Cn;
            red_h[c] = Hen;
            red_f[c] = Cn >= R(0.5) ? Fln : R(0);
            nDrop += Cn >= R(0.5) ? 1 : 0;
            const bool fin = he_finite(Hen) && isfinite(pn) && isfinite(mxn) && isfinite(myn) && isfinite(Cn);
            if (!fin) nBad += 1;
        }
        oHe[gi] = Hen;
        oP[gi] = pn;
        oMx[gi] = mxn;
        oMy[gi] = myn;
        oC[gi] = Cn;
    }
    if (stage == 2) {
        // block reduction of the diagnostics in a fixed order: the cell counts by warp
        // (integers), then one warp per sum over the tile's cells (FP64, or FP32 pairs):
        // each lane adds every 32nd cell, then the lanes combine.  The droplet's solid
        // sum is its cell count minus its liquid sum.
        using Slot = typename DSum<R>::Slot;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        nDrop = __reduce_add_sync(0xffffffffu, nDrop);
        nBad = __reduce_add_sync(0xffffffffu, nBad);
        if (lane == 0) {
            red_n[wid][0] = nDrop;
            red_n[wid][1] = nBad;
        }
        __syncthreads();
        Slot* red = static_cast<Slot*>(dc->red) + (size_t)tr.slot * kRedN;
        if (wid == 0) {
            DSum<R> v = DSum<R>::zero();
            for (int c = lane; c < TX * TY; c += 32) v.add(red_c[c]);
            for (int o = 16; o > 0; o >>= 1) v.shfl_add(o);
            if (lane == 0) red[0] = v.slot();
        } else if (wid == 1) {
            DSum<R> v = DSum<R>::zero();
            for (int c = lane; c < TX * TY; c += 32) v.add(red_h[c]);
            for (int o = 16; o > 0; o >>= 1) v.shfl_add(o);
            if (lane == 0) red[1] = v.slot();
        } else if (wid == 2) {
            DSum<R> v = DSum<R>::zero();
            for (int c = lane; c < TX * TY; c += 32) v.add(red_f[c]);
            for (int o = 16; o > 0; o >>= 1) v.shfl_add(o);
            if (lane == 0) {
                int n = 0, nb = 0;
                for (int w = 0; w < NT / 32; ++w) {
                    n += red_n[w][0];
                    nb += red_n[w][1];
                }
                DSum<R> sol = DSum<R>::count(n);
                sol.sub(v);
                red[2] = v.slot();
                red[3] = DSum<R>::count(n).slot();
                red[4] = sol.slot();
                red[5] = DSum<R>::count(nb).slot();
            }
        }
    }
}

// ---- launch helpers ------------------------------------------------------------
template <int TX, int TY>
struct StageShape {
    static constexpr int NT = ((2 * TX * TY + TX + TY) / 2 + 31) / 32 * 32;
    // region fields, face fluxes and cell kinds, then (16-byte aligned) the prefetched
    // phase-4 operands: 2 enthalpies and 9 working-precision values per tile cell
    template <class R>
    static constexpr size_t smem() {
        using Gm = Geom<TX, TY>;
        return stage_pf_offset<R>(Gm::RN, Gm::NF) +
               (size_t)TX * TY * (2 * sizeof(typename HeStore<R>::T) + 9 * sizeof(R));
    }
};

// Tile shapes the autotuner chooses from (id -> TX x TY cells per block, and the
// number of blocks per SM the register budget is cut for in mixed precision: 1 for
// ids 0-2, 2 for 3-4, 3 for 5-6, 4 for 7-12).  Ids 9-12 run 256 threads instead of
// 288, which leaves 64 registers a thread at four blocks per SM.  Ids 11 (16 x 15) and
// 12 (32 x 7) are cut so that the halo load and the faces each split into two even
// rounds of 256 threads (the 16 x 16 and 32 x 8 tiles leave a small third round of
// faces or halo cells for one warp while the others wait at the barrier).
static constexpr int kShapes = 13;
static constexpr int kShapeW[kShapes] = {32, 32, 64, 16, 64, 16, 32, 16, 32, 16, 32, 16, 32};
static constexpr int kShapeH[kShapes] = {8, 16, 8, 16, 4, 16, 8, 16, 8, 16, 8, 15, 7};

int stage_tile_shapes() { return kShapes; }
int stage_tile_w(int prec, int tile) {
    (void)prec;
    return kShapeW[(tile >= 0 && tile < kShapes) ? tile : 0];
}
int stage_tile_h(int prec, int tile) {
    (void)prec;
    return kShapeH[(tile >= 0 && tile < kShapes) ? tile : 0];
}

// NT: threads per block (0: the shape's default, one thread per two faces)
template <class R, class HR, int TX, int TY, int MINB, bool HALF, int NTB = 0>
static cudaError_t launch_t(const DevCase* cases, const TileRef* tiles, int ntiles, int stage, cudaStream_t st) {
    using S = StageShape<TX, TY>;
    constexpr int NT = NTB > 0 ? NTB : S::NT;
    auto kern = stage_kernel<R, HR, TX, TY, NT, MINB, HALF>;
    static bool configured = false;
    const size_t sm = S::template smem<R>();
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kern<<<ntiles, NT, sm, st>>>(cases, tiles, ntiles, stage);
    return cudaGetLastError();
}

template <class R, int TX, int TY, int MINB, int NTB = 0>
static cudaError_t launch_h(int half, const DevCase* cases, const TileRef* tiles, int ntiles, int stage,
                            cudaStream_t st) {
    using HR = typename HeStore<R>::T;
    return half ? launch_t<R, HR, TX, TY, MINB, true, NTB>(cases, tiles, ntiles, stage, st)
                : launch_t<R, HR, TX, TY, MINB, false, NTB>(cases, tiles, ntiles, stage, st);
}

// MINB2/3/4: the blocks per SM of ids 3-4, 5-6 and 7-8 (all 1 in FP64, whose
// registers do not allow more)
template <class R, int MINB2, int MINB3, int MINB4>
static cudaError_t launch_prec(int tile, int half, const DevCase* cases, const TileRef* tiles, int ntiles,
                               int stage, cudaStream_t st) {
    switch (tile) {
    case 1: return launch_h<R, 32, 16, 1>(half, cases, tiles, ntiles, stage, st);
    case 2: return launch_h<R, 64, 8, 1>(half, cases, tiles, ntiles, stage, st);
    case 3: return launch_h<R, 16, 16, MINB2>(half, cases, tiles, ntiles, stage, st);
    case 4: return launch_h<R, 64, 4, MINB2>(half, cases, tiles, ntiles, stage, st);
    case 5: return launch_h<R, 16, 16, MINB3>(half, cases, tiles, ntiles, stage, st);
    case 6: return launch_h<R, 32, 8, MINB3>(half, cases, tiles, ntiles, stage, st);
    case 7: return launch_h<R, 16, 16, MINB4>(half, cases, tiles, ntiles, stage, st);
    case 8: return launch_h<R, 32, 8, MINB4>(half, cases, tiles, ntiles, stage, st);
    case 9: return launch_h<R, 16, 16, MINB4, 256>(half, cases, tiles, ntiles, stage, st);
    case 10: return launch_h<R, 32, 8, MINB4, 256>(half, cases, tiles, ntiles, stage, st);
    case 11: return launch_h<R, 16, 15, MINB4, 256>(half, cases, tiles, ntiles, stage, st);
    case 12: return launch_h<R, 32, 7, MINB4, 256>(half, cases, tiles, ntiles, stage, st);
    default: return launch_h<R, 32, 8, 1>(half, cases, tiles, ntiles, stage, st);
    }
}

cudaError_t launch_stage(int prec, int tile, int half, const DevCase* cases, const TileRef* tiles,
                         int ntiles, int stage, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    if (prec == 0) return launch_prec<double, 1, 1, 1>(tile, half, cases, tiles, ntiles, stage, st);
    return launch_prec<float, 2, 3, 4>(tile, half, cases, tiles, ntiles, stage, st);
}

}  // namespace lbfs
