// CFL time step of a caller-held state without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while its process's device memory is wholly
// reserved by another allocator, code on a latency-critical path where cudaMalloc's implicit
// synchronisation is not acceptable, or plugins whose host forbids allocation.  For them this file
// offers a variant of the CFL-rate reduction (rate_kernel + host division in gks_compute_dt) whose
// scratch (one partial maximum per block and the result) lives in a file-scope static device
// array.  Every GPU that loads the library holds that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "gks.h"
#include "gks_step.cuh"

namespace {

constexpr int kThreadsNA = 256;
constexpr long kCellsPerBlock = 16384;  // a block folds this many cells into one partial maximum
constexpr int kMaxBlocks = 1024;        // partial maxima held by the static scratch
constexpr long kMaxCells = kCellsPerBlock * kMaxBlocks;
static_assert(kMaxCells == GKS_NOALLOC_MAX_CELLS, "header and implementation disagree");

// [0, kMaxBlocks): partial maxima of sum_d (|U_d| + c)/h_d; [kMaxBlocks]: the resulting time step.
static __device__ __align__(256) double g_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of g_scratch on the current device.  Host code cannot use the symbol itself (in
// host code it names a host-side stand-in), so the address is looked up once per device.
gks_status scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
      cudaGetLastError();
      return GKS_ECUDA;
    }
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return GKS_OK;
}

template <int D>
__global__ void __launch_bounds__(kThreadsNA) rate_partials(const double* W, long ncell, double gamma, double h0,
                                                            double h1, double h2, double* scratch) {
  __shared__ double red[gks::kMaxWarps];
  const double h[3] = {h0, h1, h2};
  const long begin = (long)blockIdx.x * kCellsPerBlock;
  const long end = begin + kCellsPerBlock < ncell ? begin + kCellsPerBlock : ncell;
  double rmax = 0.0;
  for (long c = begin + threadIdx.x; c < end; c += kThreadsNA) {
    double w[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; ++v) w[v] = W[(long)v * ncell + c];
    rmax = fmax(rmax, gks::cell_rate<D, double>(w, gamma, h));
  }
  const double m = gks::block_max<double>(rmax, red);
  if (threadIdx.x == 0) scratch[blockIdx.x] = m;
}

// One block folds the partials written by this call (blocks [0, nblocks)) and stores cfl / max.
__global__ void __launch_bounds__(kThreadsNA) finish_dt(double* scratch, int nblocks, double cfl) {
  __shared__ double red[gks::kMaxWarps];
  double m = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreadsNA) m = fmax(m, scratch[b]);
  m = gks::block_max<double>(m, red);
  if (threadIdx.x == 0) scratch[kMaxBlocks] = cfl / m;
}

}  // namespace

extern "C" gks_status gks_cfl_dt_noalloc(int dim, const int* n, const double* h, double gamma, const double* W,
                                         double cfl, double* dt_out, void* cuda_stream) {
  if (dim < 1 || dim > 3 || !n || !h || !W || !dt_out || !(cfl > 0.0) || !(gamma > 1.0)) return GKS_EINVAL;
  long ncell = 1;
  double hh[3] = {1.0, 1.0, 1.0};
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 1 || !(h[d] > 0.0)) return GKS_EINVAL;
    ncell *= n[d];
    if (ncell > kMaxCells) return GKS_EINVAL;  // more cells than the static scratch has partials for
    hh[d] = h[d];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GKS_ECUDA;
  }
  double* scratch = nullptr;
  gks_status st = scratch_address(dev, &scratch);
  if (st != GKS_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nblocks = (int)((ncell + kCellsPerBlock - 1) / kCellsPerBlock);
  if (dim == 1)
    rate_partials<1><<<nblocks, kThreadsNA, 0, s>>>(W, ncell, gamma, hh[0], hh[1], hh[2], scratch);
  else if (dim == 2)
    rate_partials<2><<<nblocks, kThreadsNA, 0, s>>>(W, ncell, gamma, hh[0], hh[1], hh[2], scratch);
  else
    rate_partials<3><<<nblocks, kThreadsNA, 0, s>>>(W, ncell, gamma, hh[0], hh[1], hh[2], scratch);
  finish_dt<<<1, kThreadsNA, 0, s>>>(scratch, nblocks, cfl);
  if (cudaGetLastError() != cudaSuccess) return GKS_ECUDA;
  if (cudaMemcpyAsync(dt_out, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GKS_ECUDA;
  }
  return GKS_OK;
}
