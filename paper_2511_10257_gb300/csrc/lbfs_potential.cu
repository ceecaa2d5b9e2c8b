// lbfs_potential.cu -- the magnetic scalar potential, div(mu_m grad phi) = 0 (Eq. 4),
// on the cell-centred five-point stencil with the arithmetic-mean face coefficient:
// the steady state of the paper's magnetic LBFS (Eqs. 12-18) at a half-cell streaming
// step.  Solved by residual refinement: the residual r = b - A phi is formed in FP64
// against the FP64 master potential, the correction A e = r by one multigrid V-cycle
// in the working precision M (FP32 in mixed mode), then phi += e.
//
// Operator (per level, homogeneous walls for the correction):
//   (A x)_c = sum_nb mu_f (x_c - x_nb) + sum_Dirichlet-walls 2 mu_c x_c,
//   mu_f = (mu_c + mu_nb)/2, b_c = sum_Dirichlet-walls 2 mu_c phi_wall.
// Coarse levels: 2 x 2 agglomeration, mu averaged, residual summed (the 2-D
// finite-volume operator is scale free), bilinear cell-centred prolongation,
// red-black Gauss-Seidel smoothing, conjugate gradients on the coarsest level.
#include "lbfs_kernels.h"

namespace lbfs {

namespace {

constexpr int kNT = kMgTX * kMgTY;  // 256 threads, one per cell of a 32 x 8 tile

__device__ __forceinline__ bool pot_done(const DevCase* dc) {
    return dc->stats[ST_POT_DONE] >= 1.0;
}

// Neighbour of (i, j) across side w (0 -x, 1 +x, 2 -y, 3 +y) on an nx x ny level.
// Returns 1 if it is a cell (wrapping periodic axes), 0 if the side is a wall.
__device__ __forceinline__ int neighbour(const CaseParams& P, int nx, int ny, int i, int j, int w,
                                         int& ii, int& jj) {
    ii = i + (w == 0 ? -1 : w == 1 ? 1 : 0);
    jj = j + (w == 2 ? -1 : w == 3 ? 1 : 0);
    if (ii < 0 || ii >= nx) {
        if (!P.periodic_x) return 0;
        ii = ii < 0 ? ii + nx : ii - nx;
    }
    if (jj < 0 || jj >= ny) {
        if (!P.periodic_y) return 0;
        jj = jj < 0 ? jj + ny : jj - ny;
    }
    return 1;
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T tot = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int q = 0; q < nw; ++q) tot += sh[q];
    return tot;
}

// (A x)_c with the level's coefficient, homogeneous Dirichlet walls
template <class M>
__device__ __forceinline__ M apply_A(const CaseParams& P, const M* mu, const M* x, int nx, int ny,
                                     int pitch, int i, int j) {
    const M mc = mu[(size_t)j * pitch + i];
    const M xc = x[(size_t)j * pitch + i];
    M acc = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        int ii, jj;
        if (neighbour(P, nx, ny, i, j, w, ii, jj)) {
            const size_t kn = (size_t)jj * pitch + ii;
            acc += M(0.5) * (mc + mu[kn]) * (xc - x[kn]);
        } else if (P.mag_dir[w]) {
            acc += M(2) * mc * xc;
        }
    }
    return acc;
}

template <class M>
__global__ void __launch_bounds__(kNT) k_restrict_mu(const DevCase* __restrict__ cases,
                                                     const TileRef* __restrict__ tiles, int L) {
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    const MGLevel c = dc->lev[L], f = dc->lev[L - 1];
    const int I = tr.x0 + threadIdx.x % kMgTX, J = tr.y0 + threadIdx.x / kMgTX;
    if (I >= c.nx || J >= c.ny) return;
    const M* mf = static_cast<const M*>(f.mu);
    const size_t k0 = (size_t)(2 * J) * f.pitch + 2 * I;
    static_cast<M*>(c.mu)[(size_t)J * c.pitch + I] =
        M(0.25) * ((mf[k0] + mf[k0 + 1]) + (mf[k0 + f.pitch] + mf[k0 + f.pitch + 1]));
}

// FP64 residual of the master potential on the fine level; zeroes the correction;
// per-tile partial sums of |r|^2 and |b|^2.
template <class M>
__global__ void __launch_bounds__(kNT) k_residual64(const DevCase* __restrict__ cases,
                                                    const TileRef* __restrict__ tiles) {
    __shared__ double sh[32];
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[0];
    const int i = tr.x0 + threadIdx.x % kMgTX, j = tr.y0 + threadIdx.x / kMgTX;
    double r2 = 0.0, b2 = 0.0;
    if (i < lv.nx && j < lv.ny) {
        const M* mu = static_cast<const M*>(lv.mu);
        const double* ph = dc->phi64;
        const size_t k = (size_t)j * lv.pitch + i;
        const M mcm = mu[k];
        const double pc = ph[k];
        // face coefficients in M (they are M-precision data), potentials and the
        // accumulation of the residual in FP64
        M diag = 0;
        double off = 0.0, b = 0.0;
        for (int w = 0; w < 4; ++w) {
            int ii, jj;
            if (neighbour(P, lv.nx, lv.ny, i, j, w, ii, jj)) {
                const size_t kn = (size_t)jj * lv.pitch + ii;
                const M mf = M(0.5) * (mcm + mu[kn]);
                diag += mf;
                off += (double)mf * ph[kn];
            } else if (P.mag_dir[w]) {
                const double wx = w == 0 ? 0.0 : (w == 1 ? (double)lv.nx : i + 0.5);
                const double wy = w == 2 ? 0.0 : (w == 3 ? (double)lv.ny : j + 0.5);
                const double pw = -P.H0 * (wx * P.cos_t + wy * P.sin_t);
                diag += M(2) * mcm;
                b += 2.0 * (double)mcm * pw;
            }
        }
        const double r = b - ((double)diag * pc - off);
        static_cast<M*>(lv.r)[k] = M(r);
        static_cast<M*>(lv.e)[k] = M(0);
        r2 = r * r;
        b2 = b * b;
    }
    r2 = block_sum(r2, sh);
    b2 = block_sum(b2, sh);
    if (threadIdx.x == 0) {
        dc->mg_red[2 * (size_t)tr.slot] = r2;
        dc->mg_red[2 * (size_t)tr.slot + 1] = b2;
    }
}

// one block per case: relative residual, convergence flag, cycle count
__global__ void k_mg_finalize(const DevCase* __restrict__ cases, const int* __restrict__ ids,
                              double tol, double fail_tol, int first, int* not_done) {
    __shared__ double sh[32];
    const DevCase* dc = cases + ids[blockIdx.x];
    double r2 = 0.0, b2 = 0.0;
    for (int t = threadIdx.x; t < dc->mg_tiles; t += blockDim.x) {
        r2 += dc->mg_red[2 * (size_t)t];
        b2 += dc->mg_red[2 * (size_t)t + 1];
    }
    r2 = block_sum(r2, sh);
    b2 = block_sum(b2, sh);
    if (threadIdx.x == 0) {
        const double rel = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
        double* st = dc->stats;
        st[ST_POT_RESID] = rel;
        const bool done = rel <= tol;
        st[ST_POT_DONE] = done ? 1.0 : 0.0;
        if (rel > fail_tol) st[ST_POT_FAIL] = 1.0;
        if (first) st[ST_POT_CYCLES] = 0.0;
        if (!done) {
            st[ST_POT_CYCLES] += 1.0;
            atomicAdd(not_done, 1);
        }
    }
}

template <class M>
__global__ void __launch_bounds__(kNT) k_smooth(const DevCase* __restrict__ cases,
                                                const TileRef* __restrict__ tiles, int L, int color) {
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (pot_done(dc) || L >= dc->nlev - 1) return;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[L];
    const int i = tr.x0 + threadIdx.x % kMgTX, j = tr.y0 + threadIdx.x / kMgTX;
    if (i >= lv.nx || j >= lv.ny || ((i + j) & 1) != color) return;
    const M* mu = static_cast<const M*>(lv.mu);
    M* e = static_cast<M*>(lv.e);
    const size_t k = (size_t)j * lv.pitch + i;
    const M mc = mu[k];
    M diag = 0, off = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        int ii, jj;
        if (neighbour(P, lv.nx, lv.ny, i, j, w, ii, jj)) {
            const size_t kn = (size_t)jj * lv.pitch + ii;
            const M mf = M(0.5) * (mc + mu[kn]);
            diag += mf;
            off += mf * e[kn];
        } else if (P.mag_dir[w]) {
            diag += M(2) * mc;
        }
    }
    e[k] = (static_cast<const M*>(lv.r)[k] + off) / diag;
}

// coarse residual r_L = sum over the four children of (r - A e) on level L-1; e_L = 0
template <class M>
__global__ void __launch_bounds__(kNT) k_restrict_resid(const DevCase* __restrict__ cases,
                                                        const TileRef* __restrict__ tiles, int L) {
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (pot_done(dc)) return;
    const CaseParams& P = dc->P;
    const MGLevel c = dc->lev[L], f = dc->lev[L - 1];
    const int I = tr.x0 + threadIdx.x % kMgTX, J = tr.y0 + threadIdx.x / kMgTX;
    if (I >= c.nx || J >= c.ny) return;
    const M* mu = static_cast<const M*>(f.mu);
    const M* e = static_cast<const M*>(f.e);
    const M* r = static_cast<const M*>(f.r);
    M acc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 2 * I + (q & 1), j = 2 * J + (q >> 1);
        acc += r[(size_t)j * f.pitch + i] - apply_A<M>(P, mu, e, f.nx, f.ny, f.pitch, i, j);
    }
    const size_t kc = (size_t)J * c.pitch + I;
    static_cast<M*>(c.r)[kc] = acc;
    static_cast<M*>(c.e)[kc] = M(0);
}

// coarse value at (I, J), possibly one cell outside: periodic wrap, Dirichlet wall
// (homogeneous) mirrors with a sign change, an insulating wall mirrors evenly
template <class M>
__device__ __forceinline__ M coarse_at(const CaseParams& P, const M* e, int nx, int ny, int pitch,
                                       int I, int J) {
    M sgn = M(1);
    if (I < 0 || I >= nx) {
        if (P.periodic_x) {
            I = I < 0 ? I + nx : I - nx;
        } else {
            const int w = I < 0 ? 0 : 1;
            I = I < 0 ? 0 : nx - 1;
            if (P.mag_dir[w]) sgn = -sgn;
        }
    }
    if (J < 0 || J >= ny) {
        if (P.periodic_y) {
            J = J < 0 ? J + ny : J - ny;
        } else {
            const int w = J < 0 ? 2 : 3;
            J = J < 0 ? 0 : ny - 1;
            if (P.mag_dir[w]) sgn = -sgn;
        }
    }
    return sgn * e[(size_t)J * pitch + I];
}

template <class M>
__global__ void __launch_bounds__(kNT) k_prolong(const DevCase* __restrict__ cases,
                                                 const TileRef* __restrict__ tiles, int L) {
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (pot_done(dc) || L >= dc->nlev - 1) return;
    const CaseParams& P = dc->P;
    const MGLevel f = dc->lev[L], c = dc->lev[L + 1];
    const int i = tr.x0 + threadIdx.x % kMgTX, j = tr.y0 + threadIdx.x / kMgTX;
    if (i >= f.nx || j >= f.ny) return;
    const int I = i >> 1, J = j >> 1;
    const int di = (i & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1;
    const M* ec = static_cast<const M*>(c.e);
    const M v = M(9.0 / 16.0) * coarse_at<M>(P, ec, c.nx, c.ny, c.pitch, I, J) +
                M(3.0 / 16.0) * coarse_at<M>(P, ec, c.nx, c.ny, c.pitch, I + di, J) +
                M(3.0 / 16.0) * coarse_at<M>(P, ec, c.nx, c.ny, c.pitch, I, J + dj) +
                M(1.0 / 16.0) * coarse_at<M>(P, ec, c.nx, c.ny, c.pitch, I + di, J + dj);
    static_cast<M*>(f.e)[(size_t)j * f.pitch + i] += v;
}

// conjugate gradients on the coarsest level, one block per case, in shared memory
template <class M>
__global__ void __launch_bounds__(256) k_coarsest(const DevCase* __restrict__ cases,
                                                  const int* __restrict__ ids) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ M red[32];
    const DevCase* dc = cases + ids[blockIdx.x];
    if (pot_done(dc)) return;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[dc->nlev - 1];
    const int nx = lv.nx, ny = lv.ny, n = nx * ny;
    M* x = reinterpret_cast<M*>(smem_raw);
    M* r = x + n;
    M* p = r + n;
    M* Ap = p + n;
    M* mu = Ap + n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int i = k % nx, j = k / nx;
        mu[k] = static_cast<const M*>(lv.mu)[(size_t)j * lv.pitch + i];
        r[k] = static_cast<const M*>(lv.r)[(size_t)j * lv.pitch + i];
        p[k] = r[k];
        x[k] = 0;
    }
    __syncthreads();
    M rr = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) rr += r[k] * r[k];
    rr = block_sum(rr, red);
    const M rr0 = rr;
    const M tol2 = sizeof(M) == 8 ? M(1e-28) : M(1e-12);
    const int maxit = 4 * (nx + ny) + 100;
    for (int it = 0; it < maxit && rr > tol2 * rr0 && rr > M(0); ++it) {
        M pAp = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const M a = apply_A<M>(P, mu, p, nx, ny, nx, k % nx, k / nx);
            Ap[k] = a;
            pAp += p[k] * a;
        }
        pAp = block_sum(pAp, red);
        const M alpha = rr / pAp;
        M rn = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            x[k] += alpha * p[k];
            r[k] -= alpha * Ap[k];
            rn += r[k] * r[k];
        }
        rn = block_sum(rn, red);
        const M beta = rn / rr;
        rr = rn;
        for (int k = threadIdx.x; k < n; k += blockDim.x) p[k] = r[k] + beta * p[k];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int i = k % nx, j = k / nx;
        static_cast<M*>(lv.e)[(size_t)j * lv.pitch + i] = x[k];
    }
}

template <class M>
__global__ void __launch_bounds__(kNT) k_correct(const DevCase* __restrict__ cases,
                                                 const TileRef* __restrict__ tiles) {
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (pot_done(dc)) return;
    const MGLevel lv = dc->lev[0];
    const int i = tr.x0 + threadIdx.x % kMgTX, j = tr.y0 + threadIdx.x / kMgTX;
    if (i >= lv.nx || j >= lv.ny) return;
    const size_t k = (size_t)j * lv.pitch + i;
    const double v = dc->phi64[k] + (double)static_cast<const M*>(lv.e)[k];
    dc->phi64[k] = v;
    static_cast<M*>(dc->phi)[k] = M(v);
}

}  // namespace

cudaError_t launch_mg_restrict_mu(int prec, const DevCase* cases, const TileRef* tiles, int n, int L,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_restrict_mu<double><<<n, kNT, 0, st>>>(cases, tiles, L);
    else k_restrict_mu<float><<<n, kNT, 0, st>>>(cases, tiles, L);
    return cudaGetLastError();
}

cudaError_t launch_mg_residual64(int prec, const DevCase* cases, const TileRef* tiles, int n,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_residual64<double><<<n, kNT, 0, st>>>(cases, tiles);
    else k_residual64<float><<<n, kNT, 0, st>>>(cases, tiles);
    return cudaGetLastError();
}

cudaError_t launch_mg_finalize(const DevCase* cases, const int* ids, int ncases, double tol,
                               double fail_tol, int first, int* not_done, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    k_mg_finalize<<<ncases, 256, 0, st>>>(cases, ids, tol, fail_tol, first, not_done);
    return cudaGetLastError();
}

cudaError_t launch_mg_smooth(int prec, const DevCase* cases, const TileRef* tiles, int n, int L,
                             int color, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_smooth<double><<<n, kNT, 0, st>>>(cases, tiles, L, color);
    else k_smooth<float><<<n, kNT, 0, st>>>(cases, tiles, L, color);
    return cudaGetLastError();
}

cudaError_t launch_mg_restrict_resid(int prec, const DevCase* cases, const TileRef* tiles, int n,
                                     int L, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_restrict_resid<double><<<n, kNT, 0, st>>>(cases, tiles, L);
    else k_restrict_resid<float><<<n, kNT, 0, st>>>(cases, tiles, L);
    return cudaGetLastError();
}

cudaError_t launch_mg_prolong(int prec, const DevCase* cases, const TileRef* tiles, int n, int L,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_prolong<double><<<n, kNT, 0, st>>>(cases, tiles, L);
    else k_prolong<float><<<n, kNT, 0, st>>>(cases, tiles, L);
    return cudaGetLastError();
}

size_t mg_coarsest_smem(int prec, int max_cells) {
    return (size_t)5 * max_cells * (prec == 0 ? sizeof(double) : sizeof(float));
}

cudaError_t launch_mg_coarsest(int prec, const DevCase* cases, const int* ids, int ncases,
                               int max_cells, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    const size_t sm = mg_coarsest_smem(prec, max_cells);
    cudaError_t e;
    if (prec == 0) {
        e = cudaFuncSetAttribute(k_coarsest<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_coarsest<double><<<ncases, 256, sm, st>>>(cases, ids);
    } else {
        e = cudaFuncSetAttribute(k_coarsest<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_coarsest<float><<<ncases, 256, sm, st>>>(cases, ids);
    }
    return cudaGetLastError();
}

cudaError_t launch_mg_correct(int prec, const DevCase* cases, const TileRef* tiles, int n,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_correct<double><<<n, kNT, 0, st>>>(cases, tiles);
    else k_correct<float><<<n, kNT, 0, st>>>(cases, tiles);
    return cudaGetLastError();
}

}  // namespace lbfs
