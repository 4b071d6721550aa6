// Test harness: compiles the CUDA library's interface-flux source (gks_flux.cuh) for the host so
// that its algebra can be checked against the oracle without a GPU.  Not part of the library.
// The single-precision entry runs the scalar form and the form that pairs the two sides of a face
// (the FP32 flux of the 1D and 2D kernels), with the paired instructions emulated per lane.
#define GKS_HOST_COUNT 1
#define GKS_FN inline
#include "gks_flux.cuh"

template <int D, bool M>
static void run(int abar_t0, double gamma, double mu, double C_a, double dt, const double* faces, long n, double* F,
                double* tau) {
  constexpr int nv = D + 2;
  constexpr int len = 6 * nv + 2 * (D - 1) * nv + 3;
  gks::Gas<double> gas;
  gas.bK = 2.0 / (gamma - 1.0);
  gas.ibK = (gamma - 1.0) / 2.0;
  gas.K = gas.bK - D;
  gas.mu = mu;
  gas.C_a = C_a;
  for (long f = 0; f < n; ++f) {
    const double* r = faces + f * len;
    double tl[gks::Dims<D>::nt][nv] = {}, tr[gks::Dims<D>::nt][nv] = {};
    for (int s = 0; s < D - 1; ++s)
      for (int v = 0; v < nv; ++v) {
        tl[s][v] = r[6 * nv + s * nv + v];
        tr[s][v] = r[6 * nv + (D - 1) * nv + s * nv + v];
      }
    gks::face_flux<D, double, M>(r, r + nv, r + 2 * nv, r + 3 * nv, r + 4 * nv, r + 5 * nv, tl, tr, r[len - 3],
                                 r[len - 2], r[len - 1], dt, gas, abar_t0, F + f * nv, tau + f);
  }
}

extern "C" int flux_host(int D, int multid, int abar_t0, double gamma, double mu, double C_a, double dt,
                         const double* faces, long n, double* F, double* tau) {
  if (D == 1) run<1, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
  else if (D == 2 && multid) run<2, true>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
  else if (D == 2) run<2, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
  else if (D == 3 && multid) run<3, true>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
  else if (D == 3) run<3, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
  else return 1;
  return 0;
}

// Single precision, from the same double records rounded to float: the scalar form (face_flux with
// T = float) or, with PAIRED, face_flux_ps.
template <int D, bool M, bool PAIRED>
static void run_f32(int abar_t0, double gamma, double mu, double C_a, double dt, const double* faces, long n,
                    double* F, double* tau) {
  constexpr int nv = D + 2;
  constexpr int len = 6 * nv + 2 * (D - 1) * nv + 3;
  gks::Gas<float> gas;
  gas.bK = (float)(2.0 / (gamma - 1.0));
  gas.ibK = (float)((gamma - 1.0) / 2.0);
  gas.K = (float)(2.0 / (gamma - 1.0) - D);
  gas.mu = (float)mu;
  gas.C_a = (float)C_a;
  for (long f = 0; f < n; ++f) {
    const double* r = faces + f * len;
    float x[len];
    for (int i = 0; i < len; ++i) x[i] = (float)r[i];
    float tl[gks::Dims<D>::nt][nv] = {}, tr[gks::Dims<D>::nt][nv] = {};
    for (int s = 0; s < D - 1; ++s)
      for (int v = 0; v < nv; ++v) {
        tl[s][v] = x[6 * nv + s * nv + v];
        tr[s][v] = x[6 * nv + (D - 1) * nv + s * nv + v];
      }
    float Ff[nv], t = 0.0f;
    if constexpr (PAIRED)
      gks::face_flux_ps<D, M>(x, x + nv, x + 2 * nv, x + 3 * nv, x + 4 * nv, x + 5 * nv, tl, tr, x[len - 3],
                              x[len - 2], x[len - 1], (float)dt, gas, abar_t0, Ff, &t);
    else
      gks::face_flux<D, float, M>(x, x + nv, x + 2 * nv, x + 3 * nv, x + 4 * nv, x + 5 * nv, tl, tr, x[len - 3],
                                  x[len - 2], x[len - 1], (float)dt, gas, abar_t0, Ff, &t);
    for (int v = 0; v < nv; ++v) F[f * nv + v] = Ff[v];
    tau[f] = t;
  }
}

extern "C" int flux_host_f32(int D, int multid, int paired, int abar_t0, double gamma, double mu, double C_a,
                             double dt, const double* faces, long n, double* F, double* tau) {
  if (paired) {
    if (D == 1) run_f32<1, false, true>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else if (D == 2 && multid) run_f32<2, true, true>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else if (D == 2) run_f32<2, false, true>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else return 1;
  } else {
    if (D == 1) run_f32<1, false, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else if (D == 2 && multid) run_f32<2, true, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else if (D == 2) run_f32<2, false, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else if (D == 3 && multid) run_f32<3, true, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else if (D == 3) run_f32<3, false, false>(abar_t0, gamma, mu, C_a, dt, faces, n, F, tau);
    else return 1;
  }
  return 0;
}
