// k-omega transport solved together with the flow: after each flow step, rho k and rho omega are
// advanced with the same dt by Wilcox's 2006 k-omega model (the paper's Section 4 evolves k and
// omega with the model it cites, without printing the equations):
//   d(rho k)/dt + div(rho U k) = P - beta* rho k omega + div((mu + sigma* rho k/omega) grad k)
//   d(rho w)/dt + div(rho U w) = alpha (omega/k) P - beta rho omega^2 + sigma_d (rho/omega) grad k . grad omega
//                                + div((mu + sigma rho k/omega) grad omega)
//   P = mu_T (2 S:S - 2/3 (div U)^2) - 2/3 rho k div U, mu_T = rho k / omega~,
//   omega~ = max(omega, C_lim sqrt(2 Sbar:Sbar / beta*)), Sbar = S - (div U)/3 I,
//   beta = beta0 (1 + 85 chi)/(1 + 100 chi), chi = |Omega_ij Omega_jk Shat_ki| / (beta* omega)^3, Shat = S - (div U)/2 I,
//   sigma_d = sigma_do where grad k . grad omega > 0, else 0.
// Discretisation: convection by the flow step's time-integrated mass flux F_rho of each face with
// the upwind cell's value plus half its limited slope times (width - F_rho / rho) (the face value at
// the half time); diffusion by the normal difference of the two cells with the mean coefficient;
// gradients in the sources by central differences; destruction point-implicit; then rho k >= 0 and
// omega >= omega_floor.  Ghost values of k and omega: periodic axes wrap, other axes repeat the
// nearest interior cell; ghost flow states follow the flow's boundary rules.
//
// One thread per cell; the inputs (state, k, omega, mass fluxes) of a 1024^2 grid stay in L2.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

namespace {

template <int D, int PREC>
__global__ void __launch_bounds__(256) komega_kernel(const __grid_constant__ KOmegaArgs K) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  constexpr int nv = D + 2;
  const DevGrid& g = K.g;
  const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= g.ncell) return;
  const int c[3] = {(int)(cell % g.n[0]), (int)((cell / g.n[0]) % g.n[1]), (int)(cell / ((long)g.n[0] * g.n[1]))};
  const Consts<R> kc = make_consts<R>(g);
  const R dt = (R)K.ctrl->last_dt;
  const R mu = kc.mu;
  const R* RK = (const R*)K.RKin;
  const R* RW = (const R*)K.RWin;
  const S* W = (const S*)K.Win;

  // cell index of the cell shifted by s along axis a: periodic wrap, otherwise the nearest cell
  auto mapped = [&](int a, int s) -> long {
    int cc[3] = {c[0], c[1], c[2]};
    const int n = g.n[a];
    cc[a] += s;
    if (cc[a] < 0 || cc[a] >= n) cc[a] = g.bc[a][0] == BC_PERIODIC ? (cc[a] + 2 * n) % n : min(max(cc[a], 0), n - 1);
    return cell_index(g, cc[0], cc[1], cc[2]);
  };

  R wc[nv];
  load_stored<D, PREC>(g, K.Win, cell, wc);
  const R rho = wc[0];
  const R kk = g_div(RK[cell], rho), om = g_div(RW[cell], rho);
  R ak = RK[cell], aw = RW[cell];
  R grad[3][3];  // grad[a][b] = dU_b / dx_a
  R gk[3], gw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gk[a] = gw[a] = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) grad[a][b] = R(0);
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const double* wd = g.w[a];
    // k, omega at the cells -2 .. +2 along a; flow states (boundary rules) at -1 and +1
    R phi[2][5], wid[5];
#pragma unroll
    for (int t = -2; t <= 2; ++t) {
      const long m = mapped(a, t);
      const R r = (R)W[m];
      phi[0][t + 2] = g_div(RK[m], r);
      phi[1][t + 2] = g_div(RW[m], r);
      wid[t + 2] = (R)wd[c[a] + t + 2];
    }
    R wm[nv], wp[nv];
    {
      int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
      cm[a] -= 1;
      cp[a] += 1;
      load_cell<D, PREC>(g, K.Win, kc, cm[0], cm[1], cm[2], wm);
      load_cell<D, PREC>(g, K.Win, kc, cp[0], cp[1], cp[2], wp);
    }
    const R rfl[3] = {wm[0], rho, wp[0]};  // flow densities of the cells -1, 0, +1
    const R dist = R(0.5) * wid[1] + wid[2] + R(0.5) * wid[3];
#pragma unroll
    for (int b = 0; b < D; ++b) grad[a][b] = g_div(g_div(wp[1 + b], wp[0]) - g_div(wm[1 + b], wm[0]), dist);
    gk[a] = g_div(phi[0][3] - phi[0][1], dist);
    gw[a] = g_div(phi[1][3] - phi[1][1], dist);
    // mass fluxes of the faces c - 1/2 and c + 1/2
    int nf[3] = {g.n[0], g.n[1], g.n[2]};
    nf[a] += 1;
    int fc[3] = {c[0], c[1], c[2]};
    const long f0 = ((long)fc[2] * nf[1] + fc[1]) * nf[0] + fc[0];
    fc[a] += 1;
    const long f1 = ((long)fc[2] * nf[1] + fc[1]) * nf[0] + fc[0];
    const R Fm[2] = {((const R*)K.mflux[a])[f0], ((const R*)K.mflux[a])[f1]};
    // diffusion coefficient part rho k / omega of the cells -1, 0, +1
    const R md[3] = {g_div(rfl[0] * phi[0][1], phi[1][1]), g_div(rfl[1] * phi[0][2], phi[1][2]),
                     g_div(rfl[2] * phi[0][3], phi[1][3])};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const R* v = phi[q];
      // limited slopes of the cells -1, 0, +1
      R sl[3];
#pragma unroll
      for (int t = 1; t <= 3; ++t) {
        const R hm = R(0.5) * (wid[t - 1] + wid[t]);
        const R hp = R(0.5) * (wid[t] + wid[t + 1]);
        sl[t - 1] = limiter<R>(g.limiter, g_div(v[t] - v[t - 1], hm), g_div(v[t + 1] - v[t], hp));
      }
      const R sig = q == 0 ? (R)K.sigma_star : (R)K.sigma;
      R G[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {  // face between cells e - 1 and e (relative positions)
        const int tl = e, tr = e + 1;  // indices into sl / rfl / md (cells -1, 0, +1)
        const R fr = Fm[e];
        const R hl = wid[tl + 1], hr = wid[tr + 1];
        const R phiL = v[tl + 1] + R(0.5) * sl[tl] * (hl - g_div(fr, rfl[tl]));
        const R phiR = v[tr + 1] - R(0.5) * sl[tr] * (hr + g_div(fr, rfl[tr]));
        R gf = fr * (fr >= R(0) ? phiL : phiR);
        if (K.diffusion) {
          const R coef = mu + sig * R(0.5) * (md[tl] + md[tr]);
          gf -= dt * coef * g_div(v[tr + 1] - v[tl + 1], R(0.5) * hl + R(0.5) * hr);
        }
        G[e] = gf;
      }
      const R dG = g_div(G[1] - G[0], wid[2]);
      if (q == 0)
        ak -= dG;
      else
        aw -= dG;
    }
  }
  R rate_k = R(0), rate_w = R(0);
  if (K.sources) {
    R div = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) div += grad[a][a];
    R Sm[3][3], Om[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Sm[a][b] = R(0.5) * (grad[a][b] + grad[b][a]);
        Om[a][b] = R(0.5) * (grad[b][a] - grad[a][b]);
      }
    R SS = R(0), SbSb = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        SS += Sm[a][b] * Sm[a][b];
        const R sb = Sm[a][b] - (a == b ? g_div(div, R(3)) : R(0));
        SbSb += sb * sb;
      }
    const R X = R(2) * SS - g_div(R(2), R(3)) * div * div;
    const R bstar = (R)K.beta_star;
    const R lim = (R)K.C_lim * g_sqrt(g_div(R(2) * SbSb, bstar));
    const R wt = om > lim ? om : lim;
    const R muT = g_div(rho * kk, wt);
    const R Pk = muT * X - g_div(R(2), R(3)) * rho * kk * div;
    R chi = R(0);
    if (D == 3) {
      R t = R(0);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int e = 0; e < 3; ++e) t += Om[a][b] * Om[b][e] * (Sm[e][a] - (e == a ? R(0.5) * div : R(0)));
      const R bo = bstar * om;
      chi = g_abs(g_div(t, bo * bo * bo));
    }
    const R fbeta = g_div(R(1) + R(85) * chi, R(1) + R(100) * chi);
    const R beta = (R)K.beta0 * fbeta;
    R dkdw = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) dkdw += gk[a] * gw[a];
    const R sd = dkdw > R(0) ? (R)K.sigma_do : R(0);
    const R CD = g_div(sd * rho, om) * dkdw;
    const R alpha = (R)K.alpha;
    ak += dt * Pk;
    aw += dt * (alpha * rho * g_div(om, wt) * X - g_div(R(2), R(3)) * alpha * rho * om * div + CD);
    rate_k = bstar * om;
    rate_w = beta * om;
  }
  ak = g_div(ak, R(1) + dt * rate_k);
  aw = g_div(aw, R(1) + dt * rate_w);
  const R rho_new = (R)((const S*)K.Wnew)[cell];
  const R wfloor = rho_new * (R)K.omega_floor;
  ((R*)K.RKout)[cell] = ak > R(0) ? ak : R(0);
  ((R*)K.RWout)[cell] = aw > wfloor ? aw : wfloor;
}

template <int D, int PREC>
void launch_d(const KOmegaArgs& K, cudaStream_t s) {
  const unsigned blocks = (unsigned)((K.g.ncell + 255) / 256);
  komega_kernel<D, PREC><<<blocks, 256, 0, s>>>(K);
}

}  // namespace

void launch_komega(int D, int prec, const KOmegaArgs& K, cudaStream_t s) {
  if (D == 1) {
    if (prec == PREC_F64) launch_d<1, PREC_F64>(K, s);
    else if (prec == PREC_F32) launch_d<1, PREC_F32>(K, s);
    else launch_d<1, PREC_F32D>(K, s);
  } else if (D == 2) {
    if (prec == PREC_F64) launch_d<2, PREC_F64>(K, s);
    else if (prec == PREC_F32) launch_d<2, PREC_F32>(K, s);
    else launch_d<2, PREC_F32D>(K, s);
  } else {
    if (prec == PREC_F64) launch_d<3, PREC_F64>(K, s);
    else if (prec == PREC_F32) launch_d<3, PREC_F32>(K, s);
    else launch_d<3, PREC_F32D>(K, s);
  }
}

}  // namespace gks
