// lbfs_fields.cu -- per-case utility kernels: initial condition, field export and
// import in FP64, the potential coefficient of a state, and the step-end statistics
// (Eq. 51 liquid fraction of the droplet, sums of C and H_e, freezing time).
#include "lbfs_kernels.h"

namespace lbfs {

namespace {


__device__ __forceinline__ bool cell_of(int nx, int ny, int& i, int& j) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y;
    return i < nx && j < ny;
}

// Table 1 "Initialization": droplet C = 1/2 + 1/2 tanh(2 (R - r)/xi) (the equilibrium
// profile of the Cahn-Hilliard free energy), uniform T_init, liquid everywhere so
// H_e = C_p T + L, p = 0, u = 0, uniform far-field potential.
template <class R>
__global__ void k_init(const DevCase* __restrict__ dc, InitArgs a) {
    int i, j;
    const CaseParams& P = dc->P;
    if (!cell_of(P.nx, P.ny, i, j)) return;
    const double x = i + 0.5, y = j + 0.5;
    double C = 1.0;
    if (a.kind != 2) {
        const double dx = x - a.cx, dy = y - a.cy;
        C = 0.5 + 0.5 * tanh(2.0 * (a.radius - sqrt(dx * dx + dy * dy)) / a.xi);
    }
    const double cp = mixture<double>(0.0, C, P.cp_s, P.cp_l, P.cp_g);
    const double He = cp * a.T_init + P.L;
    const size_t k = (size_t)j * P.pitch + i;
    he_set<R>(dc->He[0], k, He);
    static_cast<R*>(dc->p[0])[k] = R(0);
    static_cast<R*>(dc->mx[0])[k] = R(0);
    static_cast<R*>(dc->my[0])[k] = R(0);
    static_cast<R*>(dc->C[0])[k] = R(C);
    phi_set<R>(dc, k, -P.H0 * (x * P.cos_t + y * P.sin_t));
    R T, Fl;
    invert_enthalpy<R, double>(P, He, R(C), T, Fl);
    static_cast<R*>(dc->Fs_prev)[k] = R(1) - Fl;
}

template <class R>
__global__ void k_mu_from_state(const DevCase* __restrict__ dc) {
    int i, j;
    const CaseParams& P = dc->P;
    if (!cell_of(P.nx, P.ny, i, j)) return;
    const size_t k = (size_t)j * P.pitch + i;
    const R C = static_cast<const R*>(dc->C[0])[k];
    R T, Fl;
    invert_enthalpy<R, double>(P, he_get<R>(dc->He[0], k), C, T, Fl);
    static_cast<R*>(dc->lev[0].mu)[(size_t)j * dc->lev[0].pitch + i] =
        R(1) + mixture(R(1) - Fl, C, P.chi_s, P.chi_l, P.chi_g);
}

template <class R>
__device__ __forceinline__ R C_at(const CaseParams& P, const R* C, int i, int j) {
    // C with the wall ghost rule (wetting; zero gradient at 90 degrees) or periodic wrap
    bool wall = false;
    if (i < 0) { wall = !P.periodic_x; i = P.periodic_x ? i + P.nx : 0; }
    if (i >= P.nx) { wall = !P.periodic_x; i = P.periodic_x ? i - P.nx : P.nx - 1; }
    if (j < 0) { wall = wall || !P.periodic_y; j = P.periodic_y ? j + P.ny : 0; }
    if (j >= P.ny) { wall = wall || !P.periodic_y; j = P.periodic_y ? j - P.ny : P.ny - 1; }
    const R c = C[(size_t)j * P.pitch + i];
    return wall ? c + R(P.wet) * c * (R(1) - c) : c;
}

template <class R>
__global__ void k_derive(const DevCase* __restrict__ dc, uint32_t mask, double* __restrict__ out) {
    int i, j;
    const CaseParams& P = dc->P;
    if (!cell_of(P.nx, P.ny, i, j)) return;
    const size_t k = (size_t)j * P.pitch + i;
    const size_t N = (size_t)P.nx * P.ny, o = (size_t)j * P.nx + i;
    const double He = he_get<R>(dc->He[0], k);
    const R* Cg = static_cast<const R*>(dc->C[0]);
    const R C = Cg[k];
    R T, Fl;
    invert_enthalpy<R, double>(P, He, C, T, Fl);
    const R rho = mixture(R(1) - Fl, C, P.rho_s, P.rho_l, P.rho_g);
    const R mx = static_cast<const R*>(dc->mx[0])[k], my = static_cast<const R*>(dc->my[0])[k];
    int slot = 0;
    for (int f = 0; f < 13; ++f) {
        if (!(mask & (1u << f))) continue;
        double v = 0.0;
        switch (f) {
        case 0: v = phi_get<R>(dc, k); break;
        case 1: v = He; break;
        case 2: v = (double)T; break;
        case 3: v = (double)Fl; break;
        case 4: v = (double)static_cast<const R*>(dc->p[0])[k]; break;
        case 5: v = (double)(mx * R(3) / rho); break;
        case 6: v = (double)(my * R(3) / rho); break;
        case 7: v = (double)C; break;
        case 8: {
            const R lap = C_at<R>(P, Cg, i + 1, j) + C_at<R>(P, Cg, i - 1, j) + C_at<R>(P, Cg, i, j + 1) +
                          C_at<R>(P, Cg, i, j - 1) - R(4) * C;
            v = (double)(R(2) * R(P.beta) * C * (C - R(1)) * (R(2) * C - R(1)) - R(P.kappa) * lap);
            break;
        }
        case 9: v = (double)rho; break;
        case 10: v = (double)mx; break;
        case 11: v = (double)my; break;
        case 12: v = (double)static_cast<const R*>(dc->Fs_prev)[k]; break;
        }
        out[slot * N + o] = v;
        ++slot;
    }
}

// Sec. 5 diagnostics, one thread per column (rows are read coalesced across the
// threads of a block):
//  - the column's droplet height: the highest point where C crosses 1/2, linear in y
//    between the cell centres on either side, ny when the top cell has C >= 1/2;
//  - the largest speed |u| over the column's droplet cells (C >= 1/2);
//  - the local heat flux on a cold (Dirichlet) bottom wall, Q = -lambda dT/dy at y = 0
//    (Sec. 5.2).  The slope is that of the quadratic through the wall value at y = 0 and
//    the first two cell centres (y = 1/2, 3/2): (-8 T_w + 9 T_0 - T_1)/3; a single row
//    uses (T_0 - T_w)/(1/2).  lambda is the first cell's Eq. 11 conductivity.
// Everything is evaluated in FP64 from the stored state.  cols holds three rows of nx.
template <class R>
__global__ void k_diag_columns(const DevCase* __restrict__ dc, double* __restrict__ cols) {
    const CaseParams& P = dc->P;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nx) return;
    const R* Cg = static_cast<const R*>(dc->C[0]);
    const R* mxg = static_cast<const R*>(dc->mx[0]);
    const R* myg = static_cast<const R*>(dc->my[0]);
    const void* Heg = dc->He[0];
    double h = 0.0, umax = 0.0, C_above = 0.0;
    bool top_found = false;
    for (int j = P.ny - 1; j >= 0; --j) {
        const size_t k = (size_t)j * P.pitch + i;
        const double C = (double)Cg[k];
        if (C >= 0.5) {
            if (!top_found) {
                top_found = true;
                h = (j == P.ny - 1) ? (double)P.ny : (j + 0.5) + (C - 0.5) / (C - C_above);
            }
            double T, Fl;
            invert_enthalpy<double, double>(P, he_get<R>(Heg, k), C, T, Fl);
            const double rho = mixture<double>(1.0 - Fl, C, P.rho_s, P.rho_l, P.rho_g);
            const double u = (double)mxg[k] * 3.0 / rho, v = (double)myg[k] * 3.0 / rho;
            umax = fmax(umax, sqrt(u * u + v * v));
        }
        C_above = C;
    }
    double Q = 0.0;
    if (!P.periodic_y && P.thermal_dir[2]) {
        const double C0 = (double)Cg[i];
        double T0, Fl0;
        invert_enthalpy<double, double>(P, he_get<R>(Heg, i), C0, T0, Fl0);
        const double lam = mixture<double>(1.0 - Fl0, C0, P.lam_s, P.lam_l, P.lam_g);
        const double Tw = P.wall_T[2];
        double slope;
        if (P.ny >= 2) {
            const size_t k1 = (size_t)P.pitch + i;
            double T1, Fl1;
            invert_enthalpy<double, double>(P, he_get<R>(Heg, k1), (double)Cg[k1], T1, Fl1);
            slope = (-8.0 * Tw + 9.0 * T0 - T1) / 3.0;
        } else {
            slope = (T0 - Tw) / 0.5;
        }
        Q = -lam * slope;
    }
    cols[i] = h;
    cols[P.nx + i] = umax;
    cols[2 * (size_t)P.nx + i] = Q;
}

// Reduces the per-column diagnostics of one case with one block of kDiagThreads
// threads in a fixed order: H_m and U_max are maxima, Q_wall the sum of Q dx over the
// wall faces.  Pe = U_max D / alpha_l with D = 2 R_0 and alpha_l = lambda_l/(rho_l C_p,l)
// (Eq. 50, read with the largest droplet speed); Fo = lambda_l t/(rho_l C_p,l R_0^2).
constexpr int kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads) k_diag_finalize(const DevCase* __restrict__ dc,
                                                                 const double* __restrict__ cols,
                                                                 double R0, double* __restrict__ out) {
    __shared__ double sh[3][kDiagThreads];
    const int nx = dc->P.nx;
    double h = 0.0, u = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < nx; i += kDiagThreads) {
        h = fmax(h, cols[i]);
        u = fmax(u, cols[nx + i]);
        q += cols[2 * (size_t)nx + i];
    }
    sh[0][threadIdx.x] = h;
    sh[1][threadIdx.x] = u;
    sh[2][threadIdx.x] = q;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + w]);
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const CaseParams& P = dc->P;
        const double alpha_l = P.lam_l / (P.rho_l * P.cp_l);
        out[0] = sh[0][0];
        out[1] = sh[1][0];
        out[2] = sh[1][0] * 2.0 * R0 / alpha_l;
        out[3] = P.lam_l * dc->stats[ST_T] / (P.rho_l * P.cp_l * R0 * R0);
        out[4] = sh[2][0];
    }
}

template <class R>
__global__ void k_store(const DevCase* __restrict__ dc, uint32_t mask, const double* __restrict__ in) {
    int i, j;
    const CaseParams& P = dc->P;
    if (!cell_of(P.nx, P.ny, i, j)) return;
    const size_t k = (size_t)j * P.pitch + i;
    const size_t N = (size_t)P.nx * P.ny, o = (size_t)j * P.nx + i;
    int slot = 0;
    for (int f = 0; f < 13; ++f) {
        if (!(mask & (1u << f))) continue;
        const double v = in[slot * N + o];
        switch (f) {
        case 0: phi_set<R>(dc, k, v); break;
        case 1: he_set<R>(dc->He[0], k, v); break;
        case 4: static_cast<R*>(dc->p[0])[k] = R(v); break;
        case 7: static_cast<R*>(dc->C[0])[k] = R(v); break;
        case 10: static_cast<R*>(dc->mx[0])[k] = R(v); break;
        case 11: static_cast<R*>(dc->my[0])[k] = R(v); break;
        case 12: static_cast<R*>(dc->Fs_prev)[k] = R(v); break;
        default: break;
        }
        ++slot;
    }
}

// statistics of the stored state, after initialisation or import: kFinChunks blocks
// each sum a fixed range of rows (FP64, or FP32 pairs in mixed precision); the last
// block to finish (a ticket, no waiting) sums the chunks in order and writes sum C,
// sum H_e, the droplet sums and Q_L (Eq. 51), which also seeds the freezing-time
// interpolation
template <class R>
__global__ void k_stats_init(const DevCase* __restrict__ dc) {
    using Slot = typename DSum<R>::Slot;
    using HS = typename HeStore<R>::T;
    __shared__ Slot sh[32];
    __shared__ bool last;
    const CaseParams& P = dc->P;
    const int c = blockIdx.x;
    const int j0 = (int)((long long)P.ny * c / kFinChunks), j1 = (int)((long long)P.ny * (c + 1) / kFinChunks);
    DSum<R> acc[5];
    for (int q = 0; q < 5; ++q) acc[q] = DSum<R>::zero();
    const HS* He = static_cast<const HS*>(dc->He[0]);
    const R* Cg = static_cast<const R*>(dc->C[0]);
    for (int j = j0; j < j1; ++j)
        for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
            const size_t k = (size_t)j * P.pitch + i;
            const R C = Cg[k];
            R T, Fl;
            invert_enthalpy<R, double>(P, he_value(He[k]), C, T, Fl);
            acc[0].add(C);
            acc[1].add(He[k]);
            if (C >= R(0.5)) {
                acc[2].add(Fl);
                acc[3].add(R(1));
                acc[4].add(R(1) - Fl);
            }
        }
    for (int q = 0; q < 5; ++q) acc[q] = block_sum0<R>(acc[q], sh);
    Slot* ch = static_cast<Slot*>(dc->chunk);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 5; ++q) ch[c * kRedN + q] = acc[q].slot();
        __threadfence();
        last = atomicAdd(&dc->tickets[0], 1u) == (unsigned)(kFinChunks - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double a[5];
    for (int q = 0; q < 5; ++q) {
        DSum<R> v = DSum<R>::zero();
        for (int k = 0; k < kFinChunks; ++k) v.add(DSum<R>::of(ld_cg(&ch[k * kRedN + q])));
        a[q] = v.value();
    }
    dc->tickets[0] = 0u;
    double* st = dc->stats;
    st[ST_SUM_C] = a[0];
    st[ST_SUM_HE] = a[1];
    st[ST_SUM_FL_DROP] = a[2];
    st[ST_N_DROP] = a[3];
    st[ST_Q_L] = a[3] > 0 ? a[4] / a[3] : 0.0;
    st[ST_QL_PREV] = st[ST_Q_L];
}

// step end: fixed-order sum of the stage-tile partials (FP64, or FP32 pairs in mixed
// precision), Eq. 51 liquid-fraction measure, freezing time (first t with Q_L >= 0.99,
// linear between steps).  kFinChunks blocks per case each sum a fixed contiguous range
// of tiles; the block that finishes last (a ticket, no waiting) sums the chunk sums
// in chunk order and updates the statistics, so the result does not depend on which
// block is last.
template <class R>
__global__ void k_step_finalize(const DevCase* __restrict__ cases, const int* __restrict__ ids) {
    using Slot = typename DSum<R>::Slot;
    __shared__ Slot sh[32];
    __shared__ bool last;
    const DevCase* dc = cases + ids[blockIdx.y];
    const int T = dc->red_tiles, c = blockIdx.x;
    const int t0 = (int)((long long)T * c / kFinChunks), t1 = (int)((long long)T * (c + 1) / kFinChunks);
    const Slot* red = static_cast<const Slot*>(dc->red);
    DSum<R> acc[kRedN];
    for (int q = 0; q < kRedN; ++q) acc[q] = DSum<R>::zero();
    for (int t = t0 + (int)threadIdx.x; t < t1; t += blockDim.x)
        for (int q = 0; q < kRedN; ++q) acc[q].add(DSum<R>::of(red[(size_t)t * kRedN + q]));
    for (int q = 0; q < kRedN; ++q) acc[q] = block_sum0<R>(acc[q], sh);
    Slot* ch = static_cast<Slot*>(dc->chunk);
    if (threadIdx.x == 0) {
        for (int q = 0; q < kRedN; ++q) ch[c * kRedN + q] = acc[q].slot();
        __threadfence();
        last = atomicAdd(&dc->tickets[0], 1u) == (unsigned)(kFinChunks - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // the chunk sums, one per lane, combined by a fixed shuffle tree (the same order
    // whichever block is last)
    static_assert(kFinChunks <= 32, "one chunk per lane");
    const int lane = threadIdx.x;
    double a[kRedN];
    for (int q = 0; q < kRedN; ++q) {
        DSum<R> v = lane < kFinChunks ? DSum<R>::of(ld_cg(&ch[lane * kRedN + q])) : DSum<R>::zero();
        for (int o = 16; o > 0; o >>= 1) v.shfl_add(o);
        a[q] = v.value();
    }
    if (lane != 0) return;
    dc->tickets[0] = 0u;
    double* st = dc->stats;
    const double dt = dc->P.dt;
    st[ST_SUM_C] = a[0];
    st[ST_SUM_HE] = a[1];
    st[ST_SUM_FL_DROP] = a[2];
    st[ST_N_DROP] = a[3];
    const double QL = a[3] > 0.0 ? a[4] / a[3] : 0.0;
    st[ST_Q_L] = QL;
    if (a[5] > 0.0) st[ST_NONFINITE] = 1.0;
    st[ST_T] += dt;
    st[ST_STEP] += 1.0;
    if (st[ST_T_FREEZE] < 0.0 && QL >= 0.99) {
        const double q0 = st[ST_QL_PREV];
        st[ST_T_FREEZE] = (st[ST_T] - dt) + dt * (0.99 - q0) / (QL - q0);
    }
    st[ST_QL_PREV] = QL;
    if (dc->P.solve_potential) {
        st[ST_POT_RESID_MAX] = fmax(st[ST_POT_RESID_MAX], st[ST_POT_RESID]);
        st[ST_POT_CYCLES_SUM] += st[ST_POT_CYCLES];
    }
    st[ST_STEPS_CALL] += 1.0;
}

}  // namespace

static dim3 cell_grid(int nx, int ny) { return dim3((nx + 127) / 128, ny); }

cudaError_t launch_init(int prec, const DevCase* d, int nx, int ny, InitArgs a, cudaStream_t st) {
    if (prec == 0) k_init<double><<<cell_grid(nx, ny), 128, 0, st>>>(d, a);
    else k_init<float><<<cell_grid(nx, ny), 128, 0, st>>>(d, a);
    return cudaGetLastError();
}

cudaError_t launch_mu_from_state(int prec, const DevCase* d, int nx, int ny, cudaStream_t st) {
    if (prec == 0) k_mu_from_state<double><<<cell_grid(nx, ny), 128, 0, st>>>(d);
    else k_mu_from_state<float><<<cell_grid(nx, ny), 128, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_derive_fields(int prec, const DevCase* d, int nx, int ny, uint32_t mask, double* out,
                                 cudaStream_t st) {
    if (prec == 0) k_derive<double><<<cell_grid(nx, ny), 128, 0, st>>>(d, mask, out);
    else k_derive<float><<<cell_grid(nx, ny), 128, 0, st>>>(d, mask, out);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(int prec, const DevCase* d, int nx, double R0, double* cols, double* out5,
                               cudaStream_t st) {
    const int nb = (nx + 127) / 128;
    if (prec == 0) k_diag_columns<double><<<nb, 128, 0, st>>>(d, cols);
    else k_diag_columns<float><<<nb, 128, 0, st>>>(d, cols);
    k_diag_finalize<<<1, kDiagThreads, 0, st>>>(d, cols, R0, out5);
    return cudaGetLastError();
}

cudaError_t launch_store_fields(int prec, const DevCase* d, int nx, int ny, uint32_t mask,
                                const double* in, cudaStream_t st) {
    if (prec == 0) k_store<double><<<cell_grid(nx, ny), 128, 0, st>>>(d, mask, in);
    else k_store<float><<<cell_grid(nx, ny), 128, 0, st>>>(d, mask, in);
    return cudaGetLastError();
}

cudaError_t launch_stats_init(int prec, const DevCase* d, int nx, int ny, cudaStream_t st) {
    (void)nx;
    (void)ny;
    if (prec == 0) k_stats_init<double><<<kFinChunks, 512, 0, st>>>(d);
    else k_stats_init<float><<<kFinChunks, 512, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_step_finalize(int prec, const DevCase* cases, const int* ids, int ncases, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    const dim3 grid(kFinChunks, ncases);
    if (prec == 0) k_step_finalize<double><<<grid, 256, 0, st>>>(cases, ids);
    else k_step_finalize<float><<<grid, 256, 0, st>>>(cases, ids);
    return cudaGetLastError();
}

}  // namespace lbfs
