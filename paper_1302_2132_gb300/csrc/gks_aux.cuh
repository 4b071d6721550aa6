// Kernels shared by the single-solve C ABI and the serving layer: state conversion between caller
// layouts and the stored form, the CFL rate of a stored state, and control-block parameters.
#pragma once
#include <cuda_runtime.h>

#include "gks.h"
#include "gks_step.cuh"

namespace gks {
namespace aux {

template <class Tin>
__global__ void state_in_kernel(const Tin* src, int layout, int D, long ncell, double gamma, int prec,
                                void* W, float* Wlo) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int nv = D + 2;
  double w[5];
  for (int v = 0; v < nv; ++v) w[v] = (double)(layout == GKS_LAYOUT_AOS_CONS ? src[c * nv + v] : src[v * ncell + c]);
  if (layout == GKS_LAYOUT_SOA_PRIM) {
    const double rho = w[0], p = w[D + 1];
    double q = 0.0;
    for (int i = 0; i < D; ++i) {
      q += w[1 + i] * w[1 + i];
      w[1 + i] = rho * w[1 + i];
    }
    w[D + 1] = p / (gamma - 1.0) + 0.5 * rho * q;
  }
  for (int v = 0; v < nv; ++v) {
    if (prec == PREC_F32) {
      const float hi = (float)w[v];
      ((float*)W)[v * ncell + c] = hi;
      Wlo[v * ncell + c] = (float)(w[v] - (double)hi);
    } else {
      ((double*)W)[v * ncell + c] = w[v];
    }
  }
}

template <class Tout>
__global__ void state_out_kernel(Tout* dst, int layout, int D, long ncell, double gamma, int prec, const void* W,
                                 const float* Wlo) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int nv = D + 2;
  double w[5];
  for (int v = 0; v < nv; ++v)
    w[v] = prec == PREC_F32 ? (double)((const float*)W)[v * ncell + c] + (double)Wlo[v * ncell + c]
                            : ((const double*)W)[v * ncell + c];
  if (layout == GKS_LAYOUT_SOA_PRIM) {
    double q = 0.0;
    for (int i = 0; i < D; ++i) q += w[1 + i] * w[1 + i];
    const double p = (gamma - 1.0) * (w[D + 1] - 0.5 * q / w[0]);
    for (int i = 0; i < D; ++i) w[1 + i] = w[1 + i] / w[0];
    w[D + 1] = p;
  }
  for (int v = 0; v < nv; ++v) {
    if (layout == GKS_LAYOUT_AOS_CONS)
      dst[c * nv + v] = (Tout)w[v];
    else
      dst[v * ncell + c] = (Tout)w[v];
  }
}

template <class Tin, class Tout>
__global__ void field_kernel(const Tin* src, Tout* dst, long n) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) dst[c] = (Tout)src[c];
}

// f *= rho (scale = 1) or out = f / rho (scale = 0) with rho the density of a stored state; the
// conversions between k, omega and the transported rho k, rho omega
template <class R, class S>
__global__ void density_scale_kernel(R* f, const S* W, long n) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) f[c] = f[c] * (R)W[c];
}
template <class R, class S, class O>
__global__ void density_unscale_kernel(const R* f, const S* W, O* out, long n) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) out[c] = (O)(f[c] / (R)W[c]);
}

template <class T>
__global__ void copy_kernel(const T* src, T* dst, long n) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) dst[c] = src[c];
}

// CFL rate of the stored state into ctrl->rate[slot] (a step computes it for its successor); a cell
// with rho <= 0 or p <= 0 sets the non-physical status bit, as the step's update does.
template <int D, int PREC>
__global__ void __launch_bounds__(kThreads) rate_kernel(const __grid_constant__ StepArgs A) {
  using R = typename PrecT<PREC>::R;
  __shared__ double red[kMaxWarps];
  const DevGrid& g = A.g;
  const Consts<R> kc = make_consts<R>(g);
  R rmax = R(0);
  int bad = 0;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += (long)gridDim.x * blockDim.x) {
    R w[D + 2];
    load_stored<D, PREC>(A.g, A.Win, c, w);
    int pos[3];
    pos[0] = (int)(c % g.n[0]);
    pos[1] = (int)((c / g.n[0]) % g.n[1]);
    pos[2] = (int)(c / ((long)g.n[0] * g.n[1]));
    R h[D];
    for (int d = 0; d < D; ++d) h[d] = (R)g.w[d][pos[d] + kWG];
    if (!(w[0] > R(0)) || !(pressure_of<R>(D, kc.gamma, w) > R(0))) bad = 1;
    rmax = fmax(rmax, cell_rate<D, R>(w, kc.gamma, h));
  }
  const double m = block_max<double>((double)rmax, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&A.ctrl->rate[A.slot], m);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&A.ctrl->status, 1u);
}

template <int unused = 0>
__global__ void set_params_kernel(Ctrl* c, double dt_fixed, double cfl, double t_end) {
  c->dt_fixed = dt_fixed;
  c->cfl = cfl;
  c->t_end = t_end;
  for (int v = 0; v < 5; ++v) {
    c->l2[v] = 0.0;
    c->total[v] = 0.0;
    c->linf[v] = 0ull;
  }
}

}  // namespace aux
}  // namespace gks
