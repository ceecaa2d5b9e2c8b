// lbfs_noalloc.cu -- statistics of a state held in caller device memory, computed
// without allocating anything.
//
// Some callers cannot allocate device memory: code running under an allocator that
// another component owns (a memory pool sized once at start-up, a framework that
// forbids cudaMalloc while it records work), or a host process that only lends
// buffers it already has.  For them, lbfs_state_stats_noalloc keeps its scratch --
// one row of partial sums per grid row -- in a fixed file-scope device array instead
// of memory it would have to allocate.  Every device that loads this library holds
// that array (kNoallocRows x kNoallocSums doubles, 640 KiB) until the process exits.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lbfs.h"
#include "lbfs_internal.cuh"

namespace {

constexpr int kNoallocRows = 16384;   // largest ny accepted
constexpr int kNoallocSums = 5;       // sum C, sum H_e, sum F_l (drop), drop cells, sum F_s (drop)
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a stand-in for the symbol, never a
// device address: the address comes from cudaGetSymbolAddress (see scratch_on).
static __device__ __align__(256) double g_row_sums[kNoallocRows * kNoallocSums];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

void set_msg(char* buf, size_t len, const char* msg) {
    if (buf && len) {
        std::strncpy(buf, msg, len - 1);
        buf[len - 1] = '\0';
    }
}

// Device address of the scratch on the current device, looked up once per device and
// kept for the life of the process (a cudaDeviceReset would make it stale).
cudaError_t scratch_on(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_row_sums);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// one block per grid row: the row's sums, written to its scratch row (every row of
// this call is rewritten, so nothing has to be cleared first)
__global__ void __launch_bounds__(256) k_row_sums(lbfs::CaseParams P, const double* __restrict__ He,
                                                  const double* __restrict__ C, double* __restrict__ rows) {
    __shared__ double sh[8][kNoallocSums];
    const int j = blockIdx.x;
    double acc[kNoallocSums] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < P.nx; i += blockDim.x) {
        const size_t k = (size_t)j * P.nx + i;
        const double h = He[k], c = C[k];
        double T, Fl;
        lbfs::invert_enthalpy<double, double>(P, h, c, T, Fl);
        acc[0] += c;
        acc[1] += h;
        if (c >= 0.5) {
            acc[2] += Fl;
            acc[3] += 1.0;
            acc[4] += 1.0 - Fl;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < kNoallocSums; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNoallocSums) {
        double v = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += sh[q][threadIdx.x];
        rows[(size_t)j * kNoallocSums + threadIdx.x] = v;
    }
}

// one block: rows in a fixed order, then sum_C, sum_He, sum_Fl_drop, n_drop, Q_L
__global__ void __launch_bounds__(256) k_rows_total(int ny, const double* __restrict__ rows,
                                                    double* __restrict__ out) {
    __shared__ double sh[8][kNoallocSums];
    double acc[kNoallocSums] = {0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < ny; j += blockDim.x)
        for (int q = 0; q < kNoallocSums; ++q) acc[q] += rows[(size_t)j * kNoallocSums + q];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < kNoallocSums; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[kNoallocSums];
        for (int q = 0; q < kNoallocSums; ++q) {
            t[q] = 0.0;
            for (int r = 0; r < (int)(blockDim.x >> 5); ++r) t[q] += sh[r][q];
        }
        out[0] = t[0];
        out[1] = t[1];
        out[2] = t[2];
        out[3] = t[3];
        out[4] = t[3] > 0.0 ? t[4] / t[3] : 0.0;
    }
}

}  // namespace

extern "C" lbfs_status lbfs_state_stats_noalloc(const lbfs_case_desc* desc, const double* d_He,
                                                const double* d_C, double* d_out, void* stream,
                                                char* err, size_t err_len) {
    if (!desc || !d_He || !d_C || !d_out) {
        set_msg(err, err_len, "lbfs_state_stats_noalloc: NULL argument");
        return LBFS_EINVAL;
    }
    if (desc->nx < 1 || desc->ny < 1) {
        set_msg(err, err_len, "lbfs_state_stats_noalloc: nx and ny must be >= 1");
        return LBFS_EINVAL;
    }
    if (desc->ny > kNoallocRows) {
        char m[160];
        std::snprintf(m, sizeof(m),
                      "lbfs_state_stats_noalloc: ny = %d exceeds the fixed scratch of %d rows", desc->ny,
                      kNoallocRows);
        set_msg(err, err_len, m);
        return LBFS_EINVAL;
    }
    lbfs::CaseParams P;
    std::memset(&P, 0, sizeof(P));
    P.nx = desc->nx;
    P.ny = desc->ny;
    P.cp_l = desc->cp_l;
    P.cp_g = desc->cp_g;
    P.cp_s = desc->cp_s;
    P.T_m = desc->T_m;
    // latent heat from the Stefan number with the cold bottom wall, as for a case
    P.L = desc->stefan > 0.0 ? desc->cp_l * (desc->T_m - desc->wall_T[2]) / desc->stefan : desc->latent;
    if (!(P.L > 0)) {
        set_msg(err, err_len, "lbfs_state_stats_noalloc: latent heat must be > 0");
        return LBFS_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_msg(err, err_len, "lbfs_state_stats_noalloc: no usable current device");
        return LBFS_ECUDA;
    }
    double* rows = nullptr;
    e = scratch_on(dev, &rows);
    if (e != cudaSuccess) {
        set_msg(err, err_len, cudaGetErrorString(e));
        return LBFS_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_row_sums<<<desc->ny, 256, 0, st>>>(P, d_He, d_C, rows);
    k_rows_total<<<1, 256, 0, st>>>(desc->ny, rows, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_msg(err, err_len, cudaGetErrorString(e));
        return LBFS_ECUDA;
    }
    set_msg(err, err_len, "");
    return LBFS_OK;
}
