// CFL time step of a caller-held state without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while its process's device memory is wholly
// reserved by another allocator, code on a latency-critical path where cudaMalloc's implicit
// synchronisation is not acceptable, or plugins whose host forbids allocation.  For them this file
// offers a variant of the CFL-rate reduction (rate_kernel + host division in gks_compute_dt) whose
// scratch (one partial maximum per block and the result) lives in a file-scope static device
// array.  Every GPU that loads the library holds that array until the process exits.  Like
// gks_compute_dt, it reports a state with a cell of rho <= 0 or p <= 0 as non-physical.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gks.h"
#include "gks_step.cuh"

namespace {

constexpr int kThreadsNA = 256;
constexpr int kMaxBlocks = 1024;  // partial maxima held by the static scratch
constexpr long kMaxCells = GKS_NOALLOC_MAX_CELLS;

// [0, kMaxBlocks): partial maxima of sum_d (|U_d| + c)/h_d, or -1 for a block that met a cell with
// rho <= 0, p <= 0 or NaN; [kMaxBlocks]: the resulting time step, or -1 for a non-physical state.
static __device__ __align__(256) double g_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};
std::mutex g_scratch_mutex;

// Device address of g_scratch on the current device (and its SM count).  Host code cannot use the
// symbol itself (in host code it names a host-side stand-in), so the address is looked up once per
// device, with that device current.
gks_status scratch_address(int dev, double** out, int* sms) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    int n = 0;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return GKS_ECUDA;
    }
    g_scratch_addr[dev] = (double*)p;
    g_sm_count[dev] = n > 0 ? n : 1;
  }
  *out = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return GKS_OK;
}

// Grid-stride partial maxima: block b folds cells b T + t, (b + gridDim) T + t, ...
template <int D>
__global__ void __launch_bounds__(kThreadsNA) rate_partials(const double* W, long ncell, double gamma, double h0,
                                                            double h1, double h2, double* scratch) {
  __shared__ double red[gks::kMaxWarps];
  const double h[3] = {h0, h1, h2};
  double rmax = 0.0;
  int bad = 0;
  for (long c = (long)blockIdx.x * kThreadsNA + threadIdx.x; c < ncell; c += (long)gridDim.x * kThreadsNA) {
    double w[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; ++v) w[v] = W[(long)v * ncell + c];
    if (!(w[0] > 0.0) || !(gks::pressure_of<double>(D, gamma, w) > 0.0)) {
      bad = 1;
      continue;
    }
    rmax = fmax(rmax, gks::cell_rate<D, double>(w, gamma, h));
  }
  const double m = gks::block_max<double>(rmax, red);
  const int any_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) scratch[blockIdx.x] = any_bad ? -1.0 : m;
}

// One block folds the partials written by this call (blocks [0, nblocks)) and stores cfl / max, or -1
// if a block met a non-physical cell.
__global__ void __launch_bounds__(kThreadsNA) finish_dt(double* scratch, int nblocks, double cfl) {
  __shared__ double red[gks::kMaxWarps];
  double m = 0.0;
  int bad = 0;
  for (int b = threadIdx.x; b < nblocks; b += kThreadsNA) {
    const double v = scratch[b];
    if (v < 0.0) bad = 1;
    m = fmax(m, v);
  }
  m = gks::block_max<double>(m, red);
  const int any_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) scratch[kMaxBlocks] = any_bad ? -1.0 : cfl / m;
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
    if (ncell > kMaxCells) return GKS_EINVAL;  // beyond the documented maximum of this entry point
    hh[d] = h[d];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the call copies to the host and synchronises: never on a stream that is being captured
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return GKS_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GKS_ECUDA;
  }
  double* scratch = nullptr;
  int sms = 1;
  gks_status st = scratch_address(dev, &scratch, &sms);
  if (st != GKS_OK) return st;
  // two blocks per SM, fewer for small states, at most the partials the scratch holds
  const long want = (ncell + kThreadsNA - 1) / kThreadsNA;
  const int nblocks = (int)std::min<long>(kMaxBlocks, std::min<long>(want, 2L * sms));
  if (dim == 1)
    rate_partials<1><<<nblocks, kThreadsNA, 0, s>>>(W, ncell, gamma, hh[0], hh[1], hh[2], scratch);
  else if (dim == 2)
    rate_partials<2><<<nblocks, kThreadsNA, 0, s>>>(W, ncell, gamma, hh[0], hh[1], hh[2], scratch);
  else
    rate_partials<3><<<nblocks, kThreadsNA, 0, s>>>(W, ncell, gamma, hh[0], hh[1], hh[2], scratch);
  finish_dt<<<1, kThreadsNA, 0, s>>>(scratch, nblocks, cfl);
  if (cudaGetLastError() != cudaSuccess) return GKS_ECUDA;
  double dt = 0.0;
  if (cudaMemcpyAsync(&dt, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return GKS_ECUDA;
  }
  if (dt < 0.0) return GKS_ENONPHYS;
  *dt_out = dt;
  return GKS_OK;
}
