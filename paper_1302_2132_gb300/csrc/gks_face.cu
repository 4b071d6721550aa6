// Stateless per-face flux evaluation (gks_face_flux).
#include "gks_dispatch.h"
#include "gks_flux.cuh"

namespace gks {

template <int D, class R, bool MULTID, bool RAR>
__global__ void __launch_bounds__(128) face_kernel(int abar_t0, double gamma, double mu, double C_a, double dt,
                                                   const double* faces, long nfaces, double* Fout, double* tout) {
  constexpr int nv = D + 2;
  constexpr int len = 6 * nv + 2 * (D - 1) * nv + 3;
  const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfaces) return;
  const double* r = faces + f * len;
  R wl[nv], wr[nv], cl[nv], cr[nv], sl[nv], sr[nv], tl[Dims<D>::nt][nv], tr[Dims<D>::nt][nv];
#pragma unroll
  for (int v = 0; v < nv; ++v) {
    wl[v] = (R)r[v];
    wr[v] = (R)r[nv + v];
    cl[v] = (R)r[2 * nv + v];
    cr[v] = (R)r[3 * nv + v];
    sl[v] = (R)r[4 * nv + v];
    sr[v] = (R)r[5 * nv + v];
  }
#pragma unroll
  for (int s = 0; s < D - 1; ++s)
#pragma unroll
    for (int v = 0; v < nv; ++v) {
      tl[s][v] = (R)r[6 * nv + s * nv + v];
      tr[s][v] = (R)r[6 * nv + (D - 1) * nv + s * nv + v];
    }
  const R dxl = (R)r[len - 3], dxr = (R)r[len - 2], tau_t = (R)r[len - 1];
  Gas<R> gas;
  gas.bK = (R)(2.0 / (gamma - 1.0));
  gas.ibK = (R)((gamma - 1.0) / 2.0);
  gas.K = (R)(2.0 / (gamma - 1.0) - D);
  gas.mu = (R)mu;
  gas.C_a = (R)C_a;
  R F[nv], tau;
  // the same flux code as the step kernels: in single precision below three dimensions the two sides
  // of the face on the paired FP32 instructions
  if constexpr (std::is_same<R, float>::value && D <= 2)
    face_flux_ps<D, MULTID, RAR>(wl, wr, cl, cr, sl, sr, tl, tr, dxl, dxr, tau_t, (R)dt, gas, abar_t0, F, &tau);
  else
    face_flux<D, R, MULTID, RAR>(wl, wr, cl, cr, sl, sr, tl, tr, dxl, dxr, tau_t, (R)dt, gas, abar_t0, F, &tau);
#pragma unroll
  for (int v = 0; v < nv; ++v) Fout[f * nv + v] = (double)F[v];
  if (tout) tout[f] = (double)tau;
}

template <int D, class R, bool M>
static void go(bool rar, int abar_t0, double gamma, double mu, double C_a, double dt, const double* faces, long n,
               double* F, double* tau, cudaStream_t s) {
  const int threads = 128;
  const long blocks = (n + threads - 1) / threads;
  if (rar)
    face_kernel<D, R, M, true><<<(unsigned)blocks, threads, 0, s>>>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
  else
    face_kernel<D, R, M, false><<<(unsigned)blocks, threads, 0, s>>>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
}

void launch_face_flux(int D, int prec, bool multid, int abar_t0, int rar, double gamma, double mu, double C_a,
                      double dt, const double* faces, long n, double* F, double* tau, cudaStream_t s) {
  const bool f64 = prec == 0, r = rar != 0;
  if (D == 1) {
    if (f64) go<1, double, false>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
    else go<1, float, false>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
  } else if (D == 2) {
    if (f64) {
      if (multid) go<2, double, true>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
      else go<2, double, false>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
    } else {
      if (multid) go<2, float, true>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
      else go<2, float, false>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
    }
  } else {
    if (f64) {
      if (multid) go<3, double, true>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
      else go<3, double, false>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
    } else {
      if (multid) go<3, float, true>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
      else go<3, float, false>(r, abar_t0, gamma, mu, C_a, dt, faces, n, F, tau, s);
    }
  }
}

}  // namespace gks
