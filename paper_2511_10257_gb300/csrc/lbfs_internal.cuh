// lbfs_internal.cuh -- device-side data layout and the per-point physics of the
// LBFS step shared by the stage, potential and reduction kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbfs {

constexpr int kMaxLevels = 16;
constexpr int kRedN = 6;        // per-tile partial sums of the step-end reduction
constexpr int kFinChunks = 32;  // blocks per case that reduce the tile partials
constexpr int kStatN = 20;      // per-case device statistics slots

// statistics slots (FP64, per case).  ST_POT_RESID_MAX, ST_POT_CYCLES_SUM and
// ST_STEPS_CALL accumulate over the steps of one lbfs_step call.
enum StatSlot {
    ST_SUM_C = 0, ST_SUM_HE, ST_SUM_FL_DROP, ST_N_DROP, ST_Q_L, ST_T, ST_T_FREEZE,
    ST_POT_RESID, ST_POT_CYCLES, ST_NONFINITE, ST_QL_PREV, ST_POT_DONE, ST_B2, ST_STEP,
    ST_POT_FAIL, ST_POT_RESID_MAX, ST_POT_CYCLES_SUM, ST_STEPS_CALL, ST_EXTRAP, ST_SPARE1
};

// Physical and numerical parameters of one case, resolved on the host in FP64.
struct CaseParams {
    int nx, ny, pitch;          // cells and row pitch (elements)
    int periodic_x, periodic_y;
    int thermal_dir[4];         // 1: Dirichlet temperature wall
    int mag_dir[4];             // 1: Dirichlet potential wall
    int solve_potential;        // 0: chi == 0 or no Dirichlet wall -> phi fixed
    double wall_T[4];
    double rho_l, rho_g, rho_s, mu_l, mu_g, mu_s, cp_l, cp_g, cp_s;
    double lam_l, lam_g, lam_s, chi_l, chi_g, chi_s;
    double beta, kappa, mobility, Q_g, gravity, T_m, L;
    double dt, dts, cp_ref, vol_ratio, H0, cos_t, sin_t;
    double wet;                 // 4 cos(theta_w)/xi of the wetting ghost rule (0 at 90 deg)
};

// The per-point coefficients in the working precision R, converted once on the host
// so that no kernel converts FP64 parameters inside its inner loops.
template <class R>
struct PhysT {
    R rho_s, rho_l, rho_g, mu_s, mu_l, mu_g, lam_s, lam_l, lam_g;
    R cp_s, cp_l, cp_g, chi_s, chi_l, chi_g;
    R beta, kappa, Q_g, cp_ref, dts, inv_dts, inv_cpref_dts, tau_g, dt, vol_ratio, gravity, T_m, L;
    R wall_T[4];
    R wet;
    // the thresholds H_es = C_p,s T_m and L of Eq. 8 as (hi, lo) pairs of R: the exact
    // FP64 value is hi + lo to FP32-pair accuracy (lo = 0 in FP64)
    R Hes_hi, Hes_lo, L_hi, L_lo;
};

struct MGLevel {
    int nx, ny, pitch;
    // Coarse levels halve the cell count with the size rounded up, so the last column
    // (row) of a level may cover fewer fine cells than the others: wlx (wly) is its
    // width (height) relative to the level's other cells, 1 when the level is regular.
    float wlx, wly;
    int ragged;  // wlx < 1 or wly < 1
    void* mu;   // cell coefficient mu_m (M precision)
    void* e;    // correction
    void* r;    // right-hand side / residual
};

// Everything the kernels need to know about one case.
struct DevCase {
    CaseParams P;
    // state sets: 0 = W^n (and W^{n+1}), 1 and 2 = Runge-Kutta stage buffers
    void* He[3];      // HR precision (FP64 in both modes)
    void* p[3];       // R precision
    void* mx[3];
    void* my[3];
    void* C[3];
    void* phi;        // potential read by the stage kernel (R); FP64 mode: the master
    double* phi64;    // FP64 mode: the master potential (== phi); mixed: unused
    double* phi_prev64;  // FP64 mode: the previous step's potential; mixed: unused
    float* phi_lo;    // mixed: low word of the master potential phi + phi_lo (FP32 pair)
    void* Fs_prev;    // R: F_s of the previous step, replaced by F_s^n in stage 1
    void* Sdot;       // R: lagged dF_s/dt of the current step, written by stage 1
    PhysT<float> qf;
    PhysT<double> qd;
    int nlev;
    MGLevel lev[kMaxLevels];
    void* red;        // stage-tile partial sums, kRedN 8-byte DSum slots per tile
    int red_tiles;    // number of stage tiles of this case
    void* mg_red;     // potential residual partial sums, 2 DSum slots per fine tile
    void* chunk;      // kFinChunks x (kRedN + 2) DSum slots: per-chunk sums of the partials
    unsigned* tickets;  // [0] step-end, [1] residual: chunks done (the last one finalises)
    int mg_tiles;
    double* stats;    // kStatN FP64 slots
};

// One block's work: the tile at (x0, y0) of a case; slot numbers the case's
// partial-sum entries.
struct TileRef {
    int case_id, x0, y0, slot;
};

// ---------------------------------------------------------------------------
// D2Q9 (Eq. 14, Fig. 1) with the textbook weights 4/9, 1/9, 1/36.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int d2q9_ex(int a) {
    return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr int d2q9_ey(int a) {
    return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
__host__ __device__ constexpr double d2q9_w(int a) {
    return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// Eq. 11 mixture: F_s g_s + (1 - F_s) C g_l + (1 - F_s)(1 - C) g_g
template <class R>
__device__ __forceinline__ R mixture(R Fs, R C, double gs, double gl, double gg) {
    R liq = R(gg) + C * (R(gl) - R(gg));
    return liq + Fs * (R(gs) - liq);
}

// Eq. 8 with T_s = T_l = T_m, H_es = C_p,s T_m, H_el = C_p,L(C) T_m + L, phase change
// only where C >= 1/2.  The differences against the thresholds are formed in the
// enthalpy's storage precision HR (FP64), the rest in R.
template <class R, class HR>
__device__ __forceinline__ void invert_enthalpy(const CaseParams& P, HR He, R C, R& T, R& Fl) {
    R cpL = R(P.cp_g) + C * (R(P.cp_l) - R(P.cp_g));
    HR Hes = HR(P.cp_s) * HR(P.T_m);
    HR Hel = HR(cpL) * HR(P.T_m) + HR(P.L);
    if (C < R(0.5)) {
        Fl = R(1);
        T = R(P.T_m) + R(He - Hel) / cpL;
    } else if (He < Hes) {
        Fl = R(0);
        T = R(He) / R(P.cp_s);
    } else if (He <= Hel) {
        Fl = R(He - Hes) / R(Hel - Hes);
        T = R(P.T_m);
    } else {
        Fl = R(1);
        T = R(P.T_m) + R(He - Hel) / cpL;
    }
}

// a / b: exact in FP64; in FP32 the fast reciprocal-multiply (within 2 ulp), which
// is below the rounding of the FP32 fluxes it feeds
template <class R>
__device__ __forceinline__ R fdiv(R a, R b) {
    return a / b;
}
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) {
    return __fdividef(a, b);
}

template <class R>
__device__ __forceinline__ R mix(R Fs, R C, R gs, R gl, R gg) {
    const R liq = gg + C * (gl - gg);
    return liq + Fs * (gs - liq);
}

// Eq. 8 as above with the two threshold differences H_e - H_es and H_e - H_el formed
// in precision H and everything after them in R.  Hes_h = C_p,s T_m and L_h = L are
// given in H.  Used with H = R (the interface enthalpy in the face fluxes) and with
// H = R = double (the stored enthalpy in FP64 mode); the mixed-precision stored
// enthalpy, an FP32 pair, goes through invert_hp.
template <class R, class H>
__device__ __forceinline__ void invert_h(const PhysT<R>& Q, H Hes_h, H L_h, H He, R C, R& T, R& Fl,
                                         R* He_r = nullptr) {
    const R cpL = Q.cp_g + C * (Q.cp_l - Q.cp_g);
    const bool tm0 = Q.T_m == R(0);   // then H_es = 0 and H_el = L
    const H Hel = tm0 ? L_h : L_h + H(cpL * Q.T_m);
    const R ds = tm0 ? R(He) : R(He - Hes_h), dl = R(He - Hel);
    if (He_r) *He_r = tm0 ? ds : ds + R(Hes_h);   // H_e in R for the reconstruction
    if (C < R(0.5)) {
        Fl = R(1);
        T = Q.T_m + fdiv(dl, cpL);
    } else if (ds < R(0)) {
        Fl = R(0);
        T = Q.T_m + fdiv(ds, Q.cp_s);
    } else if (dl <= R(0)) {
        Fl = fdiv(ds, ds - dl);
        T = Q.T_m;
    } else {
        Fl = R(1);
        T = Q.T_m + fdiv(dl, cpL);
    }
}

template <class R>
__device__ __forceinline__ const PhysT<R>& phys_of(const DevCase* dc);
template <>
__device__ __forceinline__ const PhysT<float>& phys_of<float>(const DevCase* dc) { return dc->qf; }
template <>
__device__ __forceinline__ const PhysT<double>& phys_of<double>(const DevCase* dc) { return dc->qd; }

// ---- FP64-accurate arithmetic on FP32 pairs (hi + lo, |lo| <= ulp(hi)/2) ---------
// Error-free transformations: two_sum (Knuth), two_prod (FMA).  Explicit round-to-
// nearest intrinsics keep the compiler from contracting or reordering them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// (sh, sl) += (ph, pl), renormalised
__device__ __forceinline__ void pair_add(float& sh, float& sl, float ph, float pl) {
    float s, e;
    two_sum(sh, ph, s, e);
    e = __fadd_rn(e, __fadd_rn(sl, pl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}
// split a double into the nearest FP32 pair
__device__ __forceinline__ void pair_from(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// (hi, lo) + x for an FP32 x, renormalised (|lo| <= ulp(hi)/2)
__device__ __forceinline__ float2 pair_add_f(float2 a, float x) {
    float s, e;
    two_sum(a.x, x, s, e);
    e = __fadd_rn(e, a.y);
    float2 r;
    r.x = __fadd_rn(s, e);
    r.y = __fsub_rn(e, __fsub_rn(r.x, s));
    return r;
}
// (hi, lo) + (hi, lo), renormalised
__device__ __forceinline__ float2 pair_add2(float2 a, float2 b) {
    float2 r = a;
    pair_add(r.x, r.y, b.x, b.y);
    return r;
}

// ---- FP64-accurate sums ------------------------------------------------------------
// FP64 in the FP64 mode.  In mixed precision an FP32 pair accumulated with error-free
// additions (about 48 bits), so that no per-cell or per-tile FP64 instruction is
// issued.  Slot is the 8-byte type of a partial sum kept in a global or shared buffer;
// counts below 2^24 are exact in either.
template <class R>
struct DSum;
template <>
struct DSum<double> {
    using Slot = double;
    double v;
    static __device__ __forceinline__ DSum zero() { DSum s; s.v = 0.0; return s; }
    static __device__ __forceinline__ DSum of(Slot x) { DSum s; s.v = x; return s; }
    static __device__ __forceinline__ DSum count(int n) { DSum s; s.v = (double)n; return s; }
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void add(DSum o) { v += o.v; }
    __device__ __forceinline__ void sub(DSum o) { v -= o.v; }
    __device__ __forceinline__ void shfl_add(int o) { v += __shfl_down_sync(0xffffffffu, v, o); }
    __device__ __forceinline__ Slot slot() const { return v; }
    __device__ __forceinline__ double value() const { return v; }
};
template <>
struct DSum<float> {
    using Slot = float2;
    float2 v;
    static __device__ __forceinline__ DSum zero() { DSum s; s.v.x = 0.0f; s.v.y = 0.0f; return s; }
    static __device__ __forceinline__ DSum of(Slot x) { DSum s; s.v = x; return s; }
    static __device__ __forceinline__ DSum count(int n) { DSum s; s.v.x = (float)n; s.v.y = 0.0f; return s; }
    __device__ __forceinline__ void add(float x) { v = pair_add_f(v, x); }
    __device__ __forceinline__ void add(float2 x) { v = pair_add2(v, x); }
    __device__ __forceinline__ void add(DSum o) { v = pair_add2(v, o.v); }
    __device__ __forceinline__ void sub(DSum o) {
        float2 m;
        m.x = -o.v.x;
        m.y = -o.v.y;
        v = pair_add2(v, m);
    }
    __device__ __forceinline__ void shfl_add(int o) {
        float2 w;
        w.x = __shfl_down_sync(0xffffffffu, v.x, o);
        w.y = __shfl_down_sync(0xffffffffu, v.y, o);
        v = pair_add2(v, w);
    }
    __device__ __forceinline__ Slot slot() const { return v; }
    __device__ __forceinline__ double value() const { return (double)v.x + (double)v.y; }
};

// Block sum in a fixed order (warp shuffles, then the warps in index order); the
// result is valid on thread 0 only.  sh: 32 slots of shared memory.
template <class R>
__device__ __forceinline__ DSum<R> block_sum0(DSum<R> v, typename DSum<R>::Slot* sh) {
    for (int o = 16; o > 0; o >>= 1) v.shfl_add(o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v.slot();
    __syncthreads();
    DSum<R> tot = DSum<R>::zero();
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)((blockDim.x + 31) >> 5); ++q) tot.add(DSum<R>::of(sh[q]));
    return tot;
}

// load that bypasses L1 (data written by other blocks of the same launch)
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }

// ---- enthalpy storage ------------------------------------------------------------
// H_e is FP64 in the FP64 mode.  In mixed precision it is an FP32 pair (hi, lo),
// hi = fl32(H_e) and lo = fl32(H_e - hi): about 48 significant bits, read, inverted
// and updated on the FP32 pipes only (GB300's FP64 rate is a small fraction of its
// FP32 rate).  Both take 8 bytes per cell.
template <class R>
struct HeStore;
template <>
struct HeStore<double> {
    using T = double;
};
template <>
struct HeStore<float> {
    using T = float2;
};
template <class S>
__device__ __forceinline__ S he_zero();
template <>
__device__ __forceinline__ double he_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ float2 he_zero<float2>() { return make_float2(0.0f, 0.0f); }
__device__ __forceinline__ double he_value(double h) { return h; }
__device__ __forceinline__ double he_value(float2 h) { return (double)h.x + (double)h.y; }
template <class R>
__device__ __forceinline__ double he_get(const void* base, size_t k) {
    return he_value(static_cast<const typename HeStore<R>::T*>(base)[k]);
}
template <class R>
__device__ __forceinline__ void he_set(void* base, size_t k, double v) {
    if constexpr (sizeof(R) == 8) {
        static_cast<double*>(base)[k] = v;
    } else {
        float2 h;
        pair_from(v, h.x, h.y);
        static_cast<float2*>(base)[k] = h;
    }
}

// Eq. 8 (as invert_h) on an FP32-pair enthalpy.  Each threshold difference is formed
// from the parts, (hi - t_hi) + (lo - t_lo): the high parts of two nearby values
// subtract exactly, so the difference is within an FP32 rounding of the FP64 one,
// and no FP64 instruction is needed.
__device__ __forceinline__ void invert_hp(const PhysT<float>& Q, float2 He, float C, float& T, float& Fl,
                                          float* He_r = nullptr) {
    const float cpL = Q.cp_g + C * (Q.cp_l - Q.cp_g);
    float ds, dl;
    if (Q.T_m == 0.0f) {   // H_es = 0 and H_el = L
        ds = __fadd_rn(He.x, He.y);
        dl = __fadd_rn(__fsub_rn(He.x, Q.L_hi), __fsub_rn(He.y, Q.L_lo));
        if (He_r) *He_r = ds;
    } else {
        float2 Hel;
        Hel.x = Q.L_hi;
        Hel.y = Q.L_lo;
        Hel = pair_add_f(Hel, cpL * Q.T_m);
        ds = __fadd_rn(__fsub_rn(He.x, Q.Hes_hi), __fsub_rn(He.y, Q.Hes_lo));
        dl = __fadd_rn(__fsub_rn(He.x, Hel.x), __fsub_rn(He.y, Hel.y));
        if (He_r) *He_r = ds + Q.Hes_hi;
    }
    if (C < 0.5f) {
        Fl = 1.0f;
        T = Q.T_m + fdiv(dl, cpL);
    } else if (ds < 0.0f) {
        Fl = 0.0f;
        T = Q.T_m + fdiv(ds, Q.cp_s);
    } else if (dl <= 0.0f) {
        Fl = fdiv(ds, ds - dl);
        T = Q.T_m;
    } else {
        Fl = 1.0f;
        T = Q.T_m + fdiv(dl, cpL);
    }
}

// master potential of cell k in FP64, whichever precision stores it
template <class R>
__device__ __forceinline__ double phi_get(const DevCase* dc, size_t k) {
    if (sizeof(R) == 8) return dc->phi64[k];
    return (double)static_cast<const float*>(dc->phi)[k] + (double)dc->phi_lo[k];
}
template <class R>
__device__ __forceinline__ void phi_set(const DevCase* dc, size_t k, double v) {
    if (sizeof(R) == 8) {
        dc->phi64[k] = v;
    } else {
        float h, l;
        pair_from(v, h, l);
        static_cast<float*>(dc->phi)[k] = h;
        dc->phi_lo[k] = l;
    }
}

template <class R>
__device__ __forceinline__ R load(const void* base, size_t idx) {
    return static_cast<const R*>(base)[idx];
}

}  // namespace lbfs
