// Test harness: compiles the CUDA library's interface-flux source (gks_flux.cuh) for the host so
// that its algebra can be checked against the oracle without a GPU.  Not part of the library.
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
