// lbfs_kernels.h -- launch entry points of the device kernels (host-side declarations).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbfs_internal.cuh"

namespace lbfs {

// stage kernel (lbfs_stage.cu); prec 0 = FP64, 1 = mixed
int stage_tile_shapes();
int stage_tile_w(int prec, int tile);
int stage_tile_h(int prec, int tile);
// half: every case streams half a cell (dts = 1/2), which selects the reconstruction
// without normal slopes at the upwind points
cudaError_t launch_stage(int prec, int tile, int half, const DevCase* cases, const TileRef* tiles,
                         int ntiles, int stage, cudaStream_t st);

// potential multigrid (lbfs_potential.cu).  The fine-level cell kernels (residual,
// correction) take 32 x 32 tiles.  first: the step's first residual (every case);
// later ones skip converged cases.
constexpr int kMgTX = 32, kMgTY = 32;
cudaError_t launch_mg_residual64(int prec, const DevCase* cases, const TileRef* tiles, int n, int first,
                                 cudaStream_t st);
// tol: the convergence test.  first: the step's first check.  A case still above tol
// gets another cycle (one more vote in not_done) unless it has had kmax, when it is
// marked as failed.  set_cond: the call runs inside a conditional graph node; the
// last case to decide (ticket) sets cond to 1 while a case needs another cycle.
// `iters` explicit pseudo-time steps of the paper's magnetic LBFS (Eqs. 12-18) on one
// case, FP64 arithmetic; tmp holds nx*ny doubles.  2 launches per step.
cudaError_t launch_pseudo_time(int prec, const DevCase* dcase, int nx, int ny, int iters, double dtau,
                               double* tmp, cudaStream_t st);
cudaError_t launch_mg_finalize(int prec, const DevCase* cases, const int* case_ids, int ncases, double tol, int first,
                               int kmax, int* not_done, unsigned* ticket, cudaGraphConditionalHandle cond,
                               int set_cond, cudaStream_t st);
cudaError_t launch_mg_coarsest(int prec, const DevCase* cases, const int* case_ids, int ncases,
                               int max_cells, cudaStream_t st);
// FP64 only: the linearly extrapolated warm start of the potential (two launches)
cudaError_t launch_mg_extrapolate(const DevCase* cases, const TileRef* tiles, int n, const int* ids, int ncases,
                                  cudaStream_t st);
cudaError_t launch_mg_correct(int prec, const DevCase* cases, const TileRef* tiles, int n,
                              cudaStream_t st);
size_t mg_coarsest_smem(int prec, int max_cells);
// fused V-cycle legs over 32 x 16 tiles of one level (kFusedTX x kFusedTY), or over
// 16 x 8 tiles (small != 0) on a level whose 32 x 16 tiles would not fill the GPU
constexpr int kFusedTX = 32, kFusedTY = 16;
constexpr int kFusedSmallTX = 16, kFusedSmallTY = 8;
cudaError_t launch_mg_vdown(int prec, const DevCase* cases, const TileRef* tiles, int n, int level, int small,
                            cudaStream_t st);
cudaError_t launch_mg_vup(int prec, const DevCase* cases, const TileRef* tiles, int n, int level, int small,
                          cudaStream_t st);

// per-case utility kernels (lbfs_fields.cu)
struct InitArgs {
    int kind;
    double radius, cx, cy, T_init, xi;
};
cudaError_t launch_init(int prec, const DevCase* dcase, int nx, int ny, InitArgs a, cudaStream_t st);
cudaError_t launch_mu_from_state(int prec, const DevCase* dcase, int nx, int ny, cudaStream_t st);
cudaError_t launch_derive_fields(int prec, const DevCase* dcase, int nx, int ny, uint32_t mask,
                                 double* out, cudaStream_t st);
cudaError_t launch_store_fields(int prec, const DevCase* dcase, int nx, int ny, uint32_t mask,
                                const double* in, cudaStream_t st);
cudaError_t launch_stats_init(int prec, const DevCase* dcase, int nx, int ny, cudaStream_t st);
// Sec. 5 diagnostics of one case: per-column scratch cols (3 nx doubles) and out5 =
// {H_m, U_max, Pe, Fo, Q_wall}; two launches.
cudaError_t launch_diagnostics(int prec, const DevCase* dcase, int nx, double R0, double* cols,
                               double* out5, cudaStream_t st);
cudaError_t launch_step_finalize(int prec, const DevCase* cases, const int* case_ids, int ncases,
                                 cudaStream_t st);

}  // namespace lbfs
