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
// Coarse levels: 2 x 2 agglomeration with the cell count rounded up, mu averaged over
// the children, residual summed (the 2-D finite-volume operator is scale free),
// bilinear cell-centred prolongation, red-black Gauss-Seidel smoothing, conjugate
// gradients on the coarsest level.  On a level of odd size the last column (row)
// agglomerates a single child and is narrower than the others; its face coefficients
// carry the true face length over centre distance, and the prolongation interpolates
// between the true centres, so every grid size keeps the contraction of the even
// ones.
#include "lbfs_kernels.h"

namespace lbfs {

namespace {

constexpr int kNT = 256;                 // threads of the fine-level cell kernels
constexpr int kRowsPT = kMgTY / (kNT / kMgTX);  // rows of a 32 x 32 tile per thread (4)
static_assert(kRowsPT * (kNT / kMgTX) == kMgTY, "a fine-level tile splits evenly over the threads");

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

// ---- geometry of a level whose last column or row may be narrower -------------
template <class M>
__device__ __forceinline__ M cell_wx(const MGLevel& lv, int i) {
    return i == lv.nx - 1 ? M(lv.wlx) : M(1);
}
template <class M>
__device__ __forceinline__ M cell_wy(const MGLevel& lv, int j) {
    return j == lv.ny - 1 ? M(lv.wly) : M(1);
}
// Face length over centre distance, in the level's cell units, for the face of cell
// (i, j) on side w (0 -x, 1 +x, 2 -y, 3 +y): to the neighbour cell, or to the wall half
// the cell's width away.  1 and 2 for regular cells.
template <class M>
__device__ __forceinline__ M face_factor(const MGLevel& lv, int i, int j, int w, bool wall) {
    const M wx = cell_wx<M>(lv, i), wy = cell_wy<M>(lv, j);
    if (w < 2) {
        const M d = wall ? M(0.5) * wx : M(0.5) * (wx + cell_wx<M>(lv, w == 0 ? i - 1 : i + 1));
        return wy / d;
    }
    const M d = wall ? M(0.5) * wy : M(0.5) * (wy + cell_wy<M>(lv, w == 2 ? j - 1 : j + 1));
    return wx / d;
}

// Prolongation along one axis: the fine cell i of a level with nf cells (last width
// wlf) takes 1 - w of its parent I = floor(i/2) on the coarse level (nc cells, last
// width wlc) and w of the coarse neighbour I + d, d in {-1, 0, 1}, by linear
// interpolation between the true centres (in fine-cell units).  Across a wall the
// neighbour is the parent's mirror image about the wall.  Regular cells give w = 1/4.
template <class M>
__device__ __forceinline__ void prolong_axis(int i, int nf, float wlf, int nc, float wlc, int& d, M& w) {
    const M xf = M(i) + (i == nf - 1 ? M(0.5f * wlf) : M(0.5));
    const int I = (i >= 0 ? i : i - 1) / 2;
    const M xp = M(2 * I) + (I == nc - 1 ? M(wlc) : M(1));
    if (xf == xp) {
        d = 0;
        w = M(0);
        return;
    }
    d = xf > xp ? 1 : -1;
    const int N = I + d;
    M xn;
    if (N < 0) xn = -xp;
    else if (N >= nc) xn = M(4 * (nc - 1)) + M(4) * M(wlc) - xp;
    else xn = M(2 * N) + (N == nc - 1 ? M(wlc) : M(1));
    w = (xf - xp) / (xn - xp);
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

// (A x)_c with the level's coefficient and geometry, homogeneous Dirichlet walls
template <class M>
__device__ __forceinline__ M apply_A(const CaseParams& P, const MGLevel& lv, const M* mu, const M* x, int nx,
                                     int ny, int pitch, int i, int j) {
    const M mc = mu[(size_t)j * pitch + i];
    const M xc = x[(size_t)j * pitch + i];
    M acc = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        int ii, jj;
        if (neighbour(P, nx, ny, i, j, w, ii, jj)) {
            const size_t kn = (size_t)jj * pitch + ii;
            if (lv.ragged) acc += face_factor<M>(lv, i, j, w, false) * M(0.5) * (mc + mu[kn]) * (xc - x[kn]);
            else acc += M(0.5) * (mc + mu[kn]) * (xc - x[kn]);
        } else if (P.mag_dir[w]) {
            acc += (lv.ragged ? face_factor<M>(lv, i, j, w, true) : M(2)) * mc * xc;
        }
    }
    return acc;
}

// FP64-accurate residual of the master potential on the fine level and per-tile
// partial sums of |r|^2 and |b|^2.
//   r = b - A phi = -[sum_nb mu_f (phi_c - phi_nb) + sum_Dirichlet 2 mu_c (phi_c - phi_w)]
// FP64 mode: in FP64.  Mixed mode: the master potential is the FP32 pair phi + phi_lo
// and the differences, products and sums are error-free pair operations on the FP32
// pipes (about 2^-48 relative), because FP64 issue is scarce on GB300; only the norms
// are accumulated in FP64.
template <class M>
__device__ __forceinline__ double residual_cell(const DevCase* dc, const CaseParams& P, const MGLevel& lv,
                                                int i, int j, double& b_out);

template <>
__device__ __forceinline__ double residual_cell<double>(const DevCase* dc, const CaseParams& P,
                                                        const MGLevel& lv, int i, int j, double& b_out) {
    const double* mu = static_cast<const double*>(lv.mu);
    const double* ph = dc->phi64;
    const size_t k = (size_t)j * lv.pitch + i;
    const double mc = mu[k], pc = ph[k];
    double diag = 0.0, off = 0.0, b = 0.0;
    for (int w = 0; w < 4; ++w) {
        int ii, jj;
        if (neighbour(P, lv.nx, lv.ny, i, j, w, ii, jj)) {
            const size_t kn = (size_t)jj * lv.pitch + ii;
            const double mf = 0.5 * (mc + mu[kn]);
            diag += mf;
            off += mf * ph[kn];
        } else if (P.mag_dir[w]) {
            const double wx = w == 0 ? 0.0 : (w == 1 ? (double)lv.nx : i + 0.5);
            const double wy = w == 2 ? 0.0 : (w == 3 ? (double)lv.ny : j + 0.5);
            const double pw = -P.H0 * (wx * P.cos_t + wy * P.sin_t);
            diag += 2.0 * mc;
            b += 2.0 * mc * pw;
        }
    }
    b_out = b;
    return b - (diag * pc - off);
}

// mixed precision: r rounded to FP32 (it feeds the FP32 correction solve); b and its
// FP64 wall terms only at cells next to a Dirichlet wall (has_b)
__device__ __forceinline__ float residual_cell_f(const DevCase* dc, const CaseParams& P, const MGLevel& lv,
                                                 int i, int j, double& b_out, bool& has_b) {
    const float* mu = static_cast<const float*>(lv.mu);
    const float* hi = static_cast<const float*>(dc->phi);
    const float* lo = dc->phi_lo;
    // 32-bit cell indices: a level holds fewer than 2^31 cells (checked at set-up)
    const unsigned pitch = (unsigned)lv.pitch;
    const unsigned k = (unsigned)j * pitch + (unsigned)i;
    const float mc = mu[k], hc = hi[k], lc = lo[k];
    float ah = 0.f, al = 0.f;   // A phi as a pair
    double b = 0.0;
    has_b = false;
    // (phi_c - phi_n) c added to A phi, error-free in pairs
    auto term = [&](float c, float nh, float nl) {
        float dh, de, p, pe;
        two_sum(hc, -nh, dh, de);
        const float dl = __fadd_rn(de, __fsub_rn(lc, nl));
        two_prod(c, dh, p, pe);
        pe = __fmaf_rn(c, dl, pe);
        pair_add(ah, al, p, pe);
    };
    if (i > 0 && i < lv.nx - 1 && j > 0 && j < lv.ny - 1) {
        // interior cell: four neighbour cells, no wall term (no FP64 instruction)
        const unsigned kw[4] = {k - 1, k + 1, k - pitch, k + pitch};
#pragma unroll
        for (int w = 0; w < 4; ++w) term(0.5f * (mc + mu[kw[w]]), hi[kw[w]], lo[kw[w]]);
        b_out = 0.0;
        return -__fadd_rn(ah, al);
    }
    for (int w = 0; w < 4; ++w) {
        int ii, jj;
        float c, nh, nl;
        if (neighbour(P, lv.nx, lv.ny, i, j, w, ii, jj)) {
            const unsigned kn = (unsigned)jj * pitch + (unsigned)ii;
            c = 0.5f * (mc + mu[kn]);
            nh = hi[kn];
            nl = lo[kn];
        } else if (P.mag_dir[w]) {
            const double wx = w == 0 ? 0.0 : (w == 1 ? (double)lv.nx : i + 0.5);
            const double wy = w == 2 ? 0.0 : (w == 3 ? (double)lv.ny : j + 0.5);
            const double pw = -P.H0 * (wx * P.cos_t + wy * P.sin_t);
            c = 2.f * mc;
            pair_from(pw, nh, nl);
            b += (double)c * pw;
            has_b = true;
        } else {
            continue;
        }
        term(c, nh, nl);
    }
    b_out = b;
    return -__fadd_rn(ah, al);
}

// One block per 32 x 32 tile of the fine level, each thread four rows of a column
// (rows interleaved so that a warp covers one row); the tile's partial norms are
// reduced once.  first: the step's first residual, which every case computes; later
// residuals skip the cases whose solve has converged.
template <class M>
__global__ void __launch_bounds__(kNT) k_residual64(const DevCase* __restrict__ cases,
                                                    const TileRef* __restrict__ tiles, int first) {
    using Slot = typename DSum<M>::Slot;
    __shared__ Slot sh[32];
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (!first && pot_done(dc)) return;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[0];
    DSum<M> r2 = DSum<M>::zero(), b2 = DSum<M>::zero();
    const int i = tr.x0 + threadIdx.x % kMgTX;
#pragma unroll
    for (int q = 0; q < kRowsPT; ++q) {
        const int j = tr.y0 + threadIdx.x / kMgTX + q * (kNT / kMgTX);
        if (i < lv.nx && j < lv.ny) {
            const unsigned k = (unsigned)j * (unsigned)lv.pitch + (unsigned)i;
            double b;
            if constexpr (sizeof(M) == 8) {
                const double r = residual_cell<double>(dc, P, lv, i, j, b);
                static_cast<double*>(lv.r)[k] = r;
                r2.add(r * r);
                b2.add(b * b);
            } else {
                bool has_b;
                const float r = residual_cell_f(dc, P, lv, i, j, b, has_b);
                static_cast<float*>(lv.r)[k] = r;
                r2.add(r * r);
                if (has_b) {
                    float2 bb;
                    pair_from(b * b, bb.x, bb.y);
                    b2.add(bb);
                }
            }
        }
    }
    r2 = block_sum0<M>(r2, sh);
    b2 = block_sum0<M>(b2, sh);
    if (threadIdx.x == 0) {
        Slot* red = static_cast<Slot*>(dc->mg_red);
        red[2 * (size_t)tr.slot] = r2.slot();
        red[2 * (size_t)tr.slot + 1] = b2.slot();
    }
}

// The one call of cudaGraphSetConditional of a check: every case adds one to the ticket
// after it has added its vote to not_done; the last one sets the loop condition (run
// another cycle while a case still needs one) and clears both counters.
__device__ __forceinline__ void decide_next_cycle(int* not_done, unsigned* ticket, int ncases,
                                                  cudaGraphConditionalHandle cond) {
    __threadfence();
    if (atomicAdd(ticket, 1u) == (unsigned)(ncases - 1)) {
        __threadfence();
        const int nd = atomicExch(not_done, 0);
        *ticket = 0u;
        cudaGraphSetConditional(cond, nd > 0 ? 1u : 0u);
    }
}

// relative residual, convergence flag, cycle count: kFinChunks blocks per case sum
// fixed contiguous ranges of the tile partials; the last block to finish (a ticket,
// no waiting) sums the chunk sums in chunk order and decides.  first: the step's
// first check (resets the cycle count); later checks skip converged cases.  A case
// that has not converged gets another cycle unless it has had kmax, in which case it
// is marked as failed and left alone.  set_cond: inside a conditional graph, the last
// case to decide sets whether the loop runs another cycle.
template <class M>
__global__ void k_mg_finalize(const DevCase* __restrict__ cases, const int* __restrict__ ids, double tol,
                              int first, int kmax, int* not_done, unsigned* ticket, int ncases,
                              cudaGraphConditionalHandle cond, int set_cond) {
    using Slot = typename DSum<M>::Slot;
    __shared__ Slot sh[32];
    __shared__ bool last;
    const DevCase* dc = cases + ids[blockIdx.y];
    if (!first && pot_done(dc)) {
        if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) decide_next_cycle(not_done, ticket, ncases, cond);
        return;
    }
    const int T = dc->mg_tiles, c = blockIdx.x;
    const int t0 = (int)((long long)T * c / kFinChunks), t1 = (int)((long long)T * (c + 1) / kFinChunks);
    const Slot* red = static_cast<const Slot*>(dc->mg_red);
    DSum<M> r2 = DSum<M>::zero(), b2 = DSum<M>::zero();
    for (int t = t0 + (int)threadIdx.x; t < t1; t += blockDim.x) {
        r2.add(DSum<M>::of(red[2 * (size_t)t]));
        b2.add(DSum<M>::of(red[2 * (size_t)t + 1]));
    }
    r2 = block_sum0<M>(r2, sh);
    b2 = block_sum0<M>(b2, sh);
    Slot* ch = static_cast<Slot*>(dc->chunk) + kFinChunks * kRedN;
    if (threadIdx.x == 0) {
        ch[2 * c] = r2.slot();
        ch[2 * c + 1] = b2.slot();
        __threadfence();
        last = atomicAdd(&dc->tickets[1], 1u) == (unsigned)(kFinChunks - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    // the chunk sums, one per lane, combined by a fixed shuffle tree (the same order
    // whichever block is last)
    static_assert(kFinChunks <= 32, "one chunk per lane");
    const int lane = threadIdx.x;
    DSum<M> R2 = lane < kFinChunks ? DSum<M>::of(ld_cg(&ch[2 * lane])) : DSum<M>::zero();
    DSum<M> B2 = lane < kFinChunks ? DSum<M>::of(ld_cg(&ch[2 * lane + 1])) : DSum<M>::zero();
    for (int o = 16; o > 0; o >>= 1) {
        R2.shfl_add(o);
        B2.shfl_add(o);
    }
    if (lane != 0) return;
    dc->tickets[1] = 0u;
    const double rr = R2.value(), bb = B2.value();
    const double rel = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    double* st = dc->stats;
    st[ST_POT_RESID] = rel;
    const bool done = rel <= tol;
    if (first) st[ST_POT_CYCLES] = 0.0;
    if (done) {
        st[ST_POT_DONE] = 1.0;
    } else if (st[ST_POT_CYCLES] >= (double)kmax) {
        st[ST_POT_FAIL] = 1.0;
        st[ST_POT_DONE] = 1.0;   // no further kernel of this step touches the case
    } else {
        st[ST_POT_DONE] = 0.0;
        st[ST_POT_CYCLES] += 1.0;
        atomicAdd(not_done, 1);
    }
    if (set_cond) decide_next_cycle(not_done, ticket, ncases, cond);
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
    return sgn * e[(unsigned)J * (unsigned)pitch + (unsigned)I];
}

// ---- fused V-cycle legs ------------------------------------------------------
// A block owns a TX x TY tile of one level (32 x 16, or 16 x 8 on levels with too few
// tiles to fill the GPU) and keeps it with a halo in shared memory.  Red-black Gauss-Seidel half-sweeps shrink the valid region by one cell
// each, so after kFNu full sweeps the tile (plus one cell) holds exactly the values the
// sweeps over the whole level would give.  Down leg: pre-smooth from e = 0, store e,
// restrict r - A e to the next level.  Up leg: add the bilinear prolongation of the
// coarse correction, post-smooth, store e.
constexpr int kFNu = 2;
constexpr int kHD = 2 * kFNu + 1, kHU = 2 * kFNu;

template <int TX, int TY, int H>
struct FRegion {
    static constexpr int W = TX + 2 * H, Hh = TY + 2 * H, N = W * Hh;
};

// global position of region cell k of a tile at (x0, y0) with halo H; returns 0 if it
// lies beyond a non-periodic wall, else 1 with (sx, sy) the (wrapped) source cell
__device__ __forceinline__ int region_source(const CaseParams& P, int nx, int ny, int x0, int y0, int H,
                                             int W, int k, int& gx, int& gy, int& sx, int& sy) {
    gx = x0 - H + k % W;
    gy = y0 - H + k / W;
    sx = gx;
    sy = gy;
    if (sx < 0 || sx >= nx) {
        if (!P.periodic_x) return 0;
        sx = ((sx % nx) + nx) % nx;
    }
    if (sy < 0 || sy >= ny) {
        if (!P.periodic_y) return 0;
        sy = ((sy % ny) + ny) % ny;
    }
    return 1;
}

// one red-black half-sweep of colour c over the region cells at least h from its edge.
// Threads take only the cells of colour c (every other cell of a row), and a
// neighbour is a cell exactly when its region entry lies inside the domain (in[]),
// which is how the level's walls and periodic wraps were resolved at load time.
// (A x) at region cell k of a tile at (x0, y0), split into its diagonal and the
// neighbour sum: A x = diag x_k - off.  Regular levels take the plain five-point
// coefficients; a ragged level the geometric factors of its narrower last cells.
template <class M, int TX, int TY, int H>
__device__ __forceinline__ void region_stencil(const CaseParams& P, const MGLevel& lv, int x0, int y0,
                                               const M* mu, const M* x, const unsigned char* in, int k,
                                               M& diag, M& off) {
    using G = FRegion<TX, TY, H>;
    const M mc = mu[k];
    diag = 0;
    off = 0;
    if (!lv.ragged) {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int kn = k + (w == 0 ? -1 : w == 1 ? 1 : w == 2 ? -G::W : G::W);
            if (in[kn]) {
                const M mf = M(0.5) * (mc + mu[kn]);
                diag += mf;
                off += mf * x[kn];
            } else if (P.mag_dir[w]) {
                diag += M(2) * mc;
            }
        }
        return;
    }
    const int gx = x0 - H + k % G::W, gy = y0 - H + k / G::W;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int kn = k + (w == 0 ? -1 : w == 1 ? 1 : w == 2 ? -G::W : G::W);
        if (in[kn]) {
            const M mf = face_factor<M>(lv, gx, gy, w, false) * M(0.5) * (mc + mu[kn]);
            diag += mf;
            off += mf * x[kn];
        } else if (P.mag_dir[w]) {
            diag += face_factor<M>(lv, gx, gy, w, true) * mc;
        }
    }
}

// (A x) at region cell k in difference form, sum_f g mu_f (x_k - x_nb) + walls
template <class M, int TX, int TY, int H>
__device__ __forceinline__ M region_apply(const CaseParams& P, const MGLevel& lv, int x0, int y0, const M* mu,
                                          const M* x, const unsigned char* in, int k) {
    using G = FRegion<TX, TY, H>;
    const M mc = mu[k], xc = x[k];
    M ax = 0;
    const int gx = x0 - H + k % G::W, gy = y0 - H + k / G::W;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int kn = k + (w == 0 ? -1 : w == 1 ? 1 : w == 2 ? -G::W : G::W);
        if (in[kn]) {
            if (lv.ragged) ax += face_factor<M>(lv, gx, gy, w, false) * M(0.5) * (mc + mu[kn]) * (xc - x[kn]);
            else ax += M(0.5) * (mc + mu[kn]) * (xc - x[kn]);
        } else if (P.mag_dir[w]) {
            ax += (lv.ragged ? face_factor<M>(lv, gx, gy, w, true) : M(2)) * mc * xc;
        }
    }
    return ax;
}

template <class M, int TX, int TY, int H>
__device__ __forceinline__ void region_half_sweep(const CaseParams& P, const MGLevel& lv, int x0, int y0,
                                                  const M* mu, const M* r, M* e, const unsigned char* in, int c,
                                                  int h) {
    using G = FRegion<TX, TY, H>;
    const int VW = G::W - 2 * h, VH = G::Hh - 2 * h, HW = (VW + 1) / 2;
    const int base = (x0 - H) + (y0 - H);
    for (int t = threadIdx.x; t < HW * VH; t += blockDim.x) {
        const int ly = h + t / HW;
        const int lx = h + ((c - base - ly - h) & 1) + 2 * (t % HW);
        if (lx >= G::W - h) continue;
        const int k = ly * G::W + lx;
        if (!in[k]) continue;
        M diag, off;
        region_stencil<M, TX, TY, H>(P, lv, x0, y0, mu, e, in, k, diag, off);
        e[k] = fdiv(r[k] + off, diag);
    }
}

template <class M, int TX, int TY, int H>
__device__ __forceinline__ void region_load(const CaseParams& P, const MGLevel& lv, int x0, int y0, M* smu,
                                            M* sr, M* se, unsigned char* in, bool load_e) {
    using G = FRegion<TX, TY, H>;
    const M* mu = static_cast<const M*>(lv.mu);
    const M* r = static_cast<const M*>(lv.r);
    const M* e = static_cast<const M*>(lv.e);
    for (int k = threadIdx.x; k < G::N; k += blockDim.x) {
        int gx, gy, sx, sy;
        const int ok = region_source(P, lv.nx, lv.ny, x0, y0, H, G::W, k, gx, gy, sx, sy);
        const unsigned g = (unsigned)sy * (unsigned)lv.pitch + (unsigned)sx;
        in[k] = (unsigned char)ok;
        smu[k] = ok ? mu[g] : M(0);
        sr[k] = ok ? r[g] : M(0);
        se[k] = (ok && load_e) ? e[g] : M(0);
    }
}

template <class M, int TX, int TY>
__global__ void __launch_bounds__(256) k_vdown(const DevCase* __restrict__ cases,
                                               const TileRef* __restrict__ tiles, int L) {
    using G = FRegion<TX, TY, kHD>;
    __shared__ M smu[G::N], sr[G::N], se[G::N];
    __shared__ unsigned char in[G::N];
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (pot_done(dc) || L >= dc->nlev - 1) return;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[L], cv = dc->lev[L + 1];
    region_load<M, TX, TY, kHD>(P, lv, tr.x0, tr.y0, smu, sr, se, in, false);
    __syncthreads();
    for (int h = 1; h <= 2 * kFNu; ++h) {
        region_half_sweep<M, TX, TY, kHD>(P, lv, tr.x0, tr.y0, smu, sr, se, in, (h - 1) & 1, h);
        __syncthreads();
    }
    // pre-smoothed correction of the tile
    M* e = static_cast<M*>(lv.e);
    for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
        const int gx = tr.x0 + t % TX, gy = tr.y0 + t / TX;
        if (gx < lv.nx && gy < lv.ny)
            e[(unsigned)gy * (unsigned)lv.pitch + (unsigned)gx] = se[(t / TX + kHD) * G::W + t % TX + kHD];
    }
    // restricted residual r - A e over the children of each coarse cell (four, or
    // fewer where the coarse cell is the narrower last one of its row or column), and
    // the coarse coefficient as the mean of the children's
    M* rc = static_cast<M*>(cv.r);
    M* muc = static_cast<M*>(cv.mu);
    for (int t = threadIdx.x; t < (TX / 2) * (TY / 2); t += blockDim.x) {
        const int ci = t % (TX / 2), cj = t / (TX / 2);
        const int I = tr.x0 / 2 + ci, J = tr.y0 / 2 + cj;
        if (I >= cv.nx || J >= cv.ny) continue;
        M acc = 0;
        {
            const int k0 = (kHD + 2 * cj) * G::W + kHD + 2 * ci;
            if (in[k0 + 1] && in[k0 + G::W]) {
                muc[(unsigned)J * (unsigned)cv.pitch + (unsigned)I] =
                    M(0.25) * ((smu[k0] + smu[k0 + 1]) + (smu[k0 + G::W] + smu[k0 + G::W + 1]));
            } else {
                M m = smu[k0];
                int n = 1;
                if (in[k0 + 1]) { m += smu[k0 + 1]; ++n; }
                if (in[k0 + G::W]) { m += smu[k0 + G::W]; ++n; }
                muc[(unsigned)J * (unsigned)cv.pitch + (unsigned)I] = m / M(n);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int lx = kHD + 2 * ci + (q & 1), ly = kHD + 2 * cj + (q >> 1);
            const int k = ly * G::W + lx;
            if (!in[k]) continue;
            acc += sr[k] - region_apply<M, TX, TY, kHD>(P, lv, tr.x0, tr.y0, smu, se, in, k);
        }
        rc[(unsigned)J * (unsigned)cv.pitch + (unsigned)I] = acc;
    }
}

template <class M, int TX, int TY>
__global__ void __launch_bounds__(256) k_vup(const DevCase* __restrict__ cases,
                                             const TileRef* __restrict__ tiles, int L) {
    using G = FRegion<TX, TY, kHU>;
    constexpr int CW = (TX + 2 * kHU) / 2 + 3, CH = (TY + 2 * kHU) / 2 + 3;
    __shared__ M smu[G::N], sr[G::N], se[G::N];
    __shared__ M sc[CW * CH];
    __shared__ unsigned char in[G::N];
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    if (pot_done(dc) || L >= dc->nlev - 1) return;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[L], cv = dc->lev[L + 1];
    region_load<M, TX, TY, kHU>(P, lv, tr.x0, tr.y0, smu, sr, se, in, true);
    // coarse corrections around the region (one cell beyond its parents)
    const int cx0 = (tr.x0 - kHU) / 2 - 1 - ((tr.x0 - kHU) < 0 ? 1 : 0);
    const int cy0 = (tr.y0 - kHU) / 2 - 1 - ((tr.y0 - kHU) < 0 ? 1 : 0);
    const M* ec = static_cast<const M*>(cv.e);
    for (int k = threadIdx.x; k < CW * CH; k += blockDim.x) {
        int I = cx0 + k % CW, J = cy0 + k / CW;
        // periodic axes wrap; across a wall only the one-cell ghost is ever used by a
        // cell inside the domain, so the rest is clamped onto it
        if (P.periodic_x) I = ((I % cv.nx) + cv.nx) % cv.nx;
        else I = I < -1 ? -1 : (I > cv.nx ? cv.nx : I);
        if (P.periodic_y) J = ((J % cv.ny) + cv.ny) % cv.ny;
        else J = J < -1 ? -1 : (J > cv.ny ? cv.ny : J);
        sc[k] = coarse_at<M>(P, ec, cv.nx, cv.ny, cv.pitch, I, J);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < G::N; k += blockDim.x) {
        if (!in[k]) continue;
        const int gx = tr.x0 - kHU + k % G::W, gy = tr.y0 - kHU + k / G::W;
        // parent of the region cell in unwrapped level coordinates
        const int I = (gx >= 0 ? gx : gx - 1) / 2, J = (gy >= 0 ? gy : gy - 1) / 2;
        const int a = (J - cy0) * CW + (I - cx0);
        M v;
        if (!lv.ragged && !cv.ragged) {
            const int di = (gx & 1) ? 1 : -1, dj = (gy & 1) ? 1 : -1;
            v = M(9.0 / 16.0) * sc[a] + M(3.0 / 16.0) * sc[a + di] + M(3.0 / 16.0) * sc[a + dj * CW] +
                M(1.0 / 16.0) * sc[a + di + dj * CW];
        } else {
            int di, dj;
            M wx, wy;
            prolong_axis<M>(gx, lv.nx, lv.wlx, cv.nx, cv.wlx, di, wx);
            prolong_axis<M>(gy, lv.ny, lv.wly, cv.ny, cv.wly, dj, wy);
            v = ((M(1) - wx) * (M(1) - wy)) * sc[a] + (wx * (M(1) - wy)) * sc[a + di] +
                ((M(1) - wx) * wy) * sc[a + dj * CW] + (wx * wy) * sc[a + di + dj * CW];
        }
        se[k] += v;
    }
    __syncthreads();
    for (int h = 1; h <= 2 * kFNu; ++h) {
        region_half_sweep<M, TX, TY, kHU>(P, lv, tr.x0, tr.y0, smu, sr, se, in, (h - 1) & 1, h);
        __syncthreads();
    }
    M* e = static_cast<M*>(lv.e);
    for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
        const int gx = tr.x0 + t % TX, gy = tr.y0 + t / TX;
        if (gx < lv.nx && gy < lv.ny)
            e[(unsigned)gy * (unsigned)lv.pitch + (unsigned)gx] = se[(t / TX + kHU) * G::W + t % TX + kHU];
    }
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
    // the coarse correction of a V-cycle needs only a few digits: FP32 stops at 1e-3
    // relative, FP64 at 1e-6 (either way the cycle contracts as with an exact coarse
    // solve; the fine-level residual test alone decides when the potential is converged)
    const M tol2 = sizeof(M) == 8 ? M(1e-12) : M(1e-6);
    const int maxit = 4 * (nx + ny) + 100;
    for (int it = 0; it < maxit && rr > tol2 * rr0 && rr > M(0); ++it) {
        M pAp = 0;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const M a = apply_A<M>(P, lv, mu, p, nx, ny, nx, k % nx, k / nx);
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

// The same solve by one warp per case, for coarsest levels of up to kCoarsestWarp
// cells: the operator's coefficients are formed once, and an iteration's two sums are
// warp shuffles, with no block-wide barrier.  Each iteration is a few hundred cycles
// instead of the block version's six barriers.
constexpr int kCoarsestWarp = 1024;

template <class M>
__device__ __forceinline__ M warp_allsum(M v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class M>
__global__ void __launch_bounds__(32) k_coarsest_warp(const DevCase* __restrict__ cases,
                                                      const int* __restrict__ ids) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevCase* dc = cases + ids[blockIdx.x];
    if (pot_done(dc)) return;
    const CaseParams& P = dc->P;
    const MGLevel lv = dc->lev[dc->nlev - 1];
    const int nx = lv.nx, ny = lv.ny, n = nx * ny;
    const int lane = threadIdx.x;
    // x, r, p, A p, the diagonal and the four off-diagonal coefficients per cell, then
    // the four neighbour indices (a wall side points at the cell itself with a zero
    // coefficient)
    M* x = reinterpret_cast<M*>(smem_raw);
    M* r = x + n;
    M* p = r + n;
    M* Ap = p + n;
    M* dg = Ap + n;
    M* cw = dg + n;                                        // [4][n]
    short* nb = reinterpret_cast<short*>(cw + 4 * n);       // [4][n]
    const M* gmu = static_cast<const M*>(lv.mu);
    M rr = 0;
    for (int k = lane; k < n; k += 32) {
        const int i = k % nx, j = k / nx;
        const M mc = gmu[(size_t)j * lv.pitch + i];
        M d = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            int ii, jj;
            M c = 0;
            int kn = k;
            if (neighbour(P, nx, ny, i, j, w, ii, jj)) {
                kn = jj * nx + ii;
                c = M(0.5) * (mc + gmu[(size_t)jj * lv.pitch + ii]);
                if (lv.ragged) c *= face_factor<M>(lv, i, j, w, false);
                d += c;
            } else if (P.mag_dir[w]) {
                d += (lv.ragged ? face_factor<M>(lv, i, j, w, true) : M(2)) * mc;
            }
            cw[w * n + k] = c;
            nb[w * n + k] = (short)kn;
        }
        dg[k] = d;
        const M rk = static_cast<const M*>(lv.r)[(size_t)j * lv.pitch + i];
        r[k] = rk;
        p[k] = rk;
        x[k] = 0;
        rr += rk * rk;
    }
    rr = warp_allsum(rr);
    __syncwarp();
    const M rr0 = rr;
    // the same stopping rule as the block version
    const M tol2 = sizeof(M) == 8 ? M(1e-12) : M(1e-6);
    const int maxit = 4 * (nx + ny) + 100;
    for (int it = 0; it < maxit && rr > tol2 * rr0 && rr > M(0); ++it) {
        M pAp = 0;
        for (int k = lane; k < n; k += 32) {
            M a = dg[k] * p[k];
#pragma unroll
            for (int w = 0; w < 4; ++w) a -= cw[w * n + k] * p[nb[w * n + k]];
            Ap[k] = a;
            pAp += p[k] * a;
        }
        pAp = warp_allsum(pAp);
        const M alpha = rr / pAp;
        M rn = 0;
        for (int k = lane; k < n; k += 32) {
            x[k] += alpha * p[k];
            const M rk = r[k] - alpha * Ap[k];
            r[k] = rk;
            rn += rk * rk;
        }
        rn = warp_allsum(rn);
        const M beta = rn / rr;
        rr = rn;
        __syncwarp();   // every lane's reads of p for A p are done
        for (int k = lane; k < n; k += 32) p[k] = r[k] + beta * p[k];
        __syncwarp();
    }
    for (int k = lane; k < n; k += 32) {
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
    const int i = tr.x0 + threadIdx.x % kMgTX;
    if (i >= lv.nx) return;
#pragma unroll
    for (int q = 0; q < kRowsPT; ++q) {
        const int j = tr.y0 + threadIdx.x / kMgTX + q * (kNT / kMgTX);
        if (j >= lv.ny) break;
        const unsigned k = (unsigned)j * (unsigned)lv.pitch + (unsigned)i;
        if (sizeof(M) == 8) {
            const double v = dc->phi64[k] + (double)static_cast<const M*>(lv.e)[k];
            dc->phi64[k] = v;
        } else {
            // (phi, phi_lo) += e as a renormalised FP32 pair
            float* hi = static_cast<float*>(dc->phi);
            float h = hi[k], l = dc->phi_lo[k];
            pair_add(h, l, (float)static_cast<const M*>(lv.e)[k], 0.f);
            hi[k] = h;
            dc->phi_lo[k] = l;
        }
    }
}

// The FP64 warm start, extrapolated linearly in time: phi <- 2 phi - phi_prev and
// phi_prev <- phi, cell by cell, once phi_prev holds the previous step's potential
// (ST_EXTRAP set); before that phi_prev <- phi only.  A start closer to the step's
// potential needs fewer refinement cycles to reach the FP64 tolerance; the converged
// potential is the same.  (The mixed path gains nothing from it: its potential moves
// only on steps that run a cycle.)
__global__ void __launch_bounds__(kNT) k_extrapolate(const DevCase* __restrict__ cases,
                                                     const TileRef* __restrict__ tiles) {
    const TileRef tr = tiles[blockIdx.x];
    const DevCase* dc = cases + tr.case_id;
    const MGLevel lv = dc->lev[0];
    const int i = tr.x0 + threadIdx.x % kMgTX;
    if (i >= lv.nx) return;
    const bool valid = dc->stats[ST_EXTRAP] > 0.0;
#pragma unroll
    for (int q = 0; q < kRowsPT; ++q) {
        const int j = tr.y0 + threadIdx.x / kMgTX + q * (kNT / kMgTX);
        if (j >= lv.ny) break;
        const unsigned k = (unsigned)j * (unsigned)lv.pitch + (unsigned)i;
        const double v = dc->phi64[k];
        if (valid) dc->phi64[k] = 2.0 * v - dc->phi_prev64[k];
        dc->phi_prev64[k] = v;
    }
}

// after k_extrapolate: phi_prev of every solving case now holds this step's start
__global__ void k_extrapolate_commit(const DevCase* __restrict__ cases, const int* __restrict__ ids, int n) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) cases[ids[c]].stats[ST_EXTRAP] = 1.0;
}

// ---- the paper's own magnetic solver (Sec. 3.2, Eqs. 12-18) ----------------------
// Explicit pseudo-time relaxation of Eq. 17, phi <- phi - dtau div F, with the LBFS
// face flux of the magnetic distribution.  Per face (cell A below/left, B above/right,
// normal n): the equilibrium w_a phi (Eq. 13) at the points x_f - e_a dts, each
// reconstructed from its upwind cell with central gradients (Eq. 44); interface value
// Eq. 45; tau = 1/2 + mu_f/(c_s^2 dts) (Eq. 12 with the arithmetic-mean face mu); the
// starred distribution of Eq. 16.  Summed over the D2Q9 directions, the flux
//   F = sum_a e_a.n phi*_a = (tau - 1/2) sum_a e_a.n w_a phi(x_f - e_a dts)
// (the interface part carries sum_a e_a.n w_a = 0), and the three points on each side
// average their tangential slopes out, leaving
//   F = mu_f/(2 dts) [phi_A - phi_B + (1/2 - dts)(g_A + g_B)],  g = normal central slope,
// the compact -mu_f (phi_B - phi_A) at dts = 1/2.  Walls: a Dirichlet face carries the
// compact flux to the wall value half a cell away, an insulating face none; the ghost
// layer for the slopes is 2 phi_w - phi (Dirichlet) or phi (insulating).  FP64
// arithmetic in both precisions; out receives the new potential.
template <class M>
__device__ __forceinline__ double phi_cell(const DevCase* dc, const CaseParams& P, int nx, int ny, int i, int j) {
    // phi at (i, j), which may be one cell outside the grid (ghost rules above)
    int w = -1;
    if (i < 0 || i >= nx) {
        if (P.periodic_x) i = i < 0 ? i + nx : i - nx;
        else w = i < 0 ? 0 : 1;
    }
    if (j < 0 || j >= ny) {
        if (P.periodic_y) j = j < 0 ? j + ny : j - ny;
        else w = j < 0 ? 2 : 3;
    }
    if (w < 0) return phi_get<M>(dc, (size_t)j * P.pitch + i);
    const int ii = i < 0 ? 0 : (i >= nx ? nx - 1 : i), jj = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
    const double pin = phi_get<M>(dc, (size_t)jj * P.pitch + ii);
    if (!P.mag_dir[w]) return pin;
    const double wx = w == 0 ? 0.0 : (w == 1 ? (double)nx : ii + 0.5);
    const double wy = w == 2 ? 0.0 : (w == 3 ? (double)ny : jj + 0.5);
    return 2.0 * (-P.H0 * (wx * P.cos_t + wy * P.sin_t)) - pin;
}

template <class M>
__global__ void k_pseudo_step(const DevCase* __restrict__ dc, double dtau, double* __restrict__ out) {
    const CaseParams& P = dc->P;
    const int nx = P.nx, ny = P.ny;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const M* mu = static_cast<const M*>(dc->lev[0].mu);
    const int mp = dc->lev[0].pitch;
    const double dts = P.dts, c1 = 0.5 - dts;
    const double pc = phi_cell<M>(dc, P, nx, ny, i, j);
    const double mc = (double)mu[(size_t)j * mp + i];
    double div = 0.0;
    // faces 0 left, 1 right, 2 bottom, 3 top; F is the flux along +x / +y
    for (int f = 0; f < 4; ++f) {
        const bool xf = f < 2, hi = (f & 1) != 0;
        const int ni = i + (xf ? (hi ? 1 : -1) : 0), nj = j + (xf ? 0 : (hi ? 1 : -1));
        const bool wall = xf ? (!P.periodic_x && (ni < 0 || ni >= nx)) : (!P.periodic_y && (nj < 0 || nj >= ny));
        double F;
        if (wall) {
            if (!P.mag_dir[f]) continue;
            const double wx = f == 0 ? 0.0 : (f == 1 ? (double)nx : i + 0.5);
            const double wy = f == 2 ? 0.0 : (f == 3 ? (double)ny : j + 0.5);
            const double pw = -P.H0 * (wx * P.cos_t + wy * P.sin_t);
            // compact flux to the wall half a cell away, along +x / +y
            F = hi ? 2.0 * mc * (pc - pw) : -2.0 * mc * (pc - pw);
        } else {
            const int wi = ni < 0 ? ni + nx : (ni >= nx ? ni - nx : ni);
            const int wj = nj < 0 ? nj + ny : (nj >= ny ? nj - ny : nj);
            const double mn = (double)mu[(size_t)wj * mp + wi];
            const double muf = 0.5 * (mc + mn);
            // A is the lower/left cell of the face, B the upper/right one
            const int ai = hi ? i : ni, aj = hi ? j : nj, bi = hi ? ni : i, bj = hi ? nj : j;
            const int dx = xf ? 1 : 0, dy = xf ? 0 : 1;
            const double pA = hi ? pc : phi_cell<M>(dc, P, nx, ny, ai, aj);
            const double pB = hi ? phi_cell<M>(dc, P, nx, ny, bi, bj) : pc;
            double gsum = 0.0;
            if (c1 != 0.0) {
                const double gA = 0.5 * (phi_cell<M>(dc, P, nx, ny, ai + dx, aj + dy) -
                                         phi_cell<M>(dc, P, nx, ny, ai - dx, aj - dy));
                const double gB = 0.5 * (phi_cell<M>(dc, P, nx, ny, bi + dx, bj + dy) -
                                         phi_cell<M>(dc, P, nx, ny, bi - dx, bj - dy));
                gsum = gA + gB;
            }
            F = muf / (2.0 * dts) * ((pA - pB) + c1 * gsum);
        }
        div += hi ? F : -F;
    }
    out[(size_t)j * nx + i] = pc - dtau * div;
}

template <class M>
__global__ void k_pseudo_store(const DevCase* __restrict__ dc, const double* __restrict__ in) {
    const CaseParams& P = dc->P;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= P.nx) return;
    phi_set<M>(dc, (size_t)j * P.pitch + i, in[(size_t)j * P.nx + i]);
}

}  // namespace

cudaError_t launch_pseudo_time(int prec, const DevCase* d, int nx, int ny, int iters, double dtau, double* tmp,
                               cudaStream_t st) {
    const dim3 grid((nx + 127) / 128, ny);
    for (int it = 0; it < iters; ++it) {
        if (prec == 0) {
            k_pseudo_step<double><<<grid, 128, 0, st>>>(d, dtau, tmp);
            k_pseudo_store<double><<<grid, 128, 0, st>>>(d, tmp);
        } else {
            k_pseudo_step<float><<<grid, 128, 0, st>>>(d, dtau, tmp);
            k_pseudo_store<float><<<grid, 128, 0, st>>>(d, tmp);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_mg_residual64(int prec, const DevCase* cases, const TileRef* tiles, int n, int first,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (prec == 0) k_residual64<double><<<n, kNT, 0, st>>>(cases, tiles, first);
    else k_residual64<float><<<n, kNT, 0, st>>>(cases, tiles, first);
    return cudaGetLastError();
}

cudaError_t launch_mg_finalize(int prec, const DevCase* cases, const int* ids, int ncases, double tol, int first,
                               int kmax, int* not_done, unsigned* ticket, cudaGraphConditionalHandle cond,
                               int set_cond, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    const dim3 grid(kFinChunks, ncases);
    if (prec == 0)
        k_mg_finalize<double><<<grid, 256, 0, st>>>(cases, ids, tol, first, kmax, not_done, ticket, ncases, cond,
                                                    set_cond);
    else
        k_mg_finalize<float><<<grid, 256, 0, st>>>(cases, ids, tol, first, kmax, not_done, ticket, ncases, cond,
                                                   set_cond);
    return cudaGetLastError();
}

cudaError_t launch_mg_vdown(int prec, const DevCase* cases, const TileRef* tiles, int n, int L, int small,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (small) {
        if (prec == 0) k_vdown<double, kFusedSmallTX, kFusedSmallTY><<<n, 128, 0, st>>>(cases, tiles, L);
        else k_vdown<float, kFusedSmallTX, kFusedSmallTY><<<n, 128, 0, st>>>(cases, tiles, L);
    } else {
        if (prec == 0) k_vdown<double, kFusedTX, kFusedTY><<<n, 256, 0, st>>>(cases, tiles, L);
        else k_vdown<float, kFusedTX, kFusedTY><<<n, 256, 0, st>>>(cases, tiles, L);
    }
    return cudaGetLastError();
}

cudaError_t launch_mg_vup(int prec, const DevCase* cases, const TileRef* tiles, int n, int L, int small,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (small) {
        if (prec == 0) k_vup<double, kFusedSmallTX, kFusedSmallTY><<<n, 128, 0, st>>>(cases, tiles, L);
        else k_vup<float, kFusedSmallTX, kFusedSmallTY><<<n, 128, 0, st>>>(cases, tiles, L);
    } else {
        if (prec == 0) k_vup<double, kFusedTX, kFusedTY><<<n, 256, 0, st>>>(cases, tiles, L);
        else k_vup<float, kFusedTX, kFusedTY><<<n, 256, 0, st>>>(cases, tiles, L);
    }
    return cudaGetLastError();
}

size_t mg_coarsest_smem(int prec, int max_cells) {
    const size_t m = prec == 0 ? sizeof(double) : sizeof(float);
    if (max_cells <= kCoarsestWarp) return (size_t)9 * max_cells * m + (size_t)4 * max_cells * sizeof(short);
    return (size_t)5 * max_cells * m;
}

cudaError_t launch_mg_coarsest(int prec, const DevCase* cases, const int* ids, int ncases,
                               int max_cells, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    const size_t sm = mg_coarsest_smem(prec, max_cells);
    const bool warp = max_cells <= kCoarsestWarp;
    cudaError_t e;
    if (prec == 0) {
        if (warp) {
            e = cudaFuncSetAttribute(k_coarsest_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_coarsest_warp<double><<<ncases, 32, sm, st>>>(cases, ids);
        } else {
            e = cudaFuncSetAttribute(k_coarsest<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_coarsest<double><<<ncases, 256, sm, st>>>(cases, ids);
        }
    } else {
        if (warp) {
            e = cudaFuncSetAttribute(k_coarsest_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_coarsest_warp<float><<<ncases, 32, sm, st>>>(cases, ids);
        } else {
            e = cudaFuncSetAttribute(k_coarsest<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
            k_coarsest<float><<<ncases, 256, sm, st>>>(cases, ids);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_mg_extrapolate(const DevCase* cases, const TileRef* tiles, int n, const int* ids, int ncases,
                                  cudaStream_t st) {
    if (n <= 0 || ncases <= 0) return cudaSuccess;
    k_extrapolate<<<n, kNT, 0, st>>>(cases, tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_extrapolate_commit<<<1, 128, 0, st>>>(cases, ids, ncases);
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
