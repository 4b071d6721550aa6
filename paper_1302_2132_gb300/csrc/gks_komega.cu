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
// Tiles of cells per block with a shared-memory halo (ghost cells resolved once per tile), one
// thread per cell; the inputs (state, k, omega, mass fluxes) of a 1024^2 grid stay in L2.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

namespace {

// Tile of cells per 256-thread block; k, omega, density and velocity of the tile and two halo
// layers are staged in shared memory once (ghost cells resolved there), then one thread per cell.
template <int D> struct KTile;
template <> struct KTile<1> { static constexpr int X = 256, Y = 1, Z = 1; };
template <> struct KTile<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct KTile<3> { static constexpr int X = 8, Y = 8, Z = 4; };

template <int D, int PREC>
__global__ void __launch_bounds__(256) komega_kernel(const __grid_constant__ KOmegaArgs K) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  using T = KTile<D>;
  constexpr int nv = D + 2;
  constexpr int HX = T::X + 4, HY = D >= 2 ? T::Y + 4 : 1, HZ = D >= 3 ? T::Z + 4 : 1, NH = HX * HY * HZ;
  __shared__ R sk[NH], sw[NH], sr[NH], su[D][NH];
  __shared__ R swid[HX + HY + HZ];  // widths of the halo cells along each axis (arithmetic type)
  __shared__ R s_dt;
  const DevGrid& g = K.g;
  const int tiles_x = (g.n[0] + T::X - 1) / T::X;
  const int tiles_y = D >= 2 ? (g.n[1] + T::Y - 1) / T::Y : 1;
  const int b = blockIdx.x;
  const int ox = (b % tiles_x) * T::X;
  const int oy = D >= 2 ? ((b / tiles_x) % tiles_y) * T::Y : 0;
  const int oz = D >= 3 ? (b / (tiles_x * tiles_y)) * T::Z : 0;
  const int tid = threadIdx.x;
  const Consts<R> kc = make_consts<R>(g);
  const R* RK = (const R*)K.RKin;
  const R* RW = (const R*)K.RWin;
  const S* W = (const S*)K.Win;

  // ---- stage: flow state with the boundary rules, k and omega of the source cell ------------
  for (int l = tid; l < NH; l += 256) {
    const int hi = l % HX, hj = (l / HX) % HY, hk = l / (HX * HY);
    const int gi = ox + hi - 2, gj = D >= 2 ? oy + hj - 2 : 0, gk = D >= 3 ? oz + hk - 2 : 0;
    R w[nv];
    load_cell<D, PREC>(g, K.Win, kc, gi, gj, gk, w);
    sr[l] = w[0];
#pragma unroll
    for (int a = 0; a < D; ++a) su[a][l] = g_div(w[1 + a], w[0]);
    const long m = field_cell(g, D, gi, gj, gk);
    const R rm = (R)W[m];
    sk[l] = g_div(RK[m], rm);
    sw[l] = g_div(RW[m], rm);
  }
  // widths (converted once per block: double-to-float conversions run on the FP64 pipe) and dt
  for (int l = tid; l < HX + HY + HZ; l += 256) {
    const int a = l < HX ? 0 : (l < HX + HY ? 1 : 2);
    const int p = a == 0 ? l : (a == 1 ? l - HX : l - HX - HY);
    const int o = a == 0 ? ox : (a == 1 ? oy : oz);
    swid[l] = a < D ? (R)g.w[a][min(o + p, g.n[a] + 3)] : R(1);
  }
  if (tid == 0) s_dt = (R)K.ctrl->last_dt;
  __syncthreads();

  const int li = tid % T::X, lj = (tid / T::X) % T::Y, lk = tid / (T::X * T::Y);
  const int c[3] = {ox + li, oy + lj, oz + lk};
  if (c[0] >= g.n[0] || (D >= 2 && c[1] >= g.n[1]) || (D >= 3 && c[2] >= g.n[2])) return;
  const long cell = cell_index(g, c[0], c[1], c[2]);
  const int h0 = ((lk + (D >= 3 ? 2 : 0)) * HY + (lj + (D >= 2 ? 2 : 0))) * HX + (li + 2);
  const int hs[3] = {1, HX, HX * HY};
  const R dt = s_dt;
  const R mu = kc.mu;
  constexpr bool F = sizeof(R) == sizeof(float);
  const R c_alpha = F ? (R)K.falpha : (R)K.alpha, c_beta0 = F ? (R)K.fbeta0 : (R)K.beta0;
  const R c_bstar = F ? (R)K.fbeta_star : (R)K.beta_star, c_sigma = F ? (R)K.fsigma : (R)K.sigma;
  const R c_sstar = F ? (R)K.fsigma_star : (R)K.sigma_star, c_sdo = F ? (R)K.fsigma_do : (R)K.sigma_do;
  const R c_clim = F ? (R)K.fC_lim : (R)K.C_lim, c_wfloor = F ? (R)K.fomega_floor : (R)K.omega_floor;
  const R rho = sr[h0];
  const R kk = sk[h0], om = sw[h0];
  R ak = RK[cell], aw = RW[cell];
  R grad[3][3];  // grad[a][b] = dU_b / dx_a
  R gk[3], gw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gk[a] = gw[a] = R(0);
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) grad[a][bb] = R(0);
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const R* wd = swid + (a == 0 ? 0 : (a == 1 ? HX : HX + HY));  // halo position p = cell + 2 - tile origin
    const int st = hs[a];
    const int pa = (a == 0 ? li : (a == 1 ? lj : lk)) + 2;
    // k, omega and widths at the cells -2 .. +2 along a
    R phi[2][5], wid[5];
#pragma unroll
    for (int t = -2; t <= 2; ++t) {
      phi[0][t + 2] = sk[h0 + t * st];
      phi[1][t + 2] = sw[h0 + t * st];
      wid[t + 2] = wd[pa + t];
    }
    const R rfl[3] = {sr[h0 - st], rho, sr[h0 + st]};  // flow densities of the cells -1, 0, +1
    const R dist = R(0.5) * wid[1] + wid[2] + R(0.5) * wid[3];
#pragma unroll
    for (int bb = 0; bb < D; ++bb) grad[a][bb] = g_div(su[bb][h0 + st] - su[bb][h0 - st], dist);
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
      const R sig = q == 0 ? c_sstar : c_sigma;
      R G[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {  // face between the cells e - 1 and e (relative positions)
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
    const R bstar = c_bstar;
    const R lim = c_clim * g_sqrt(g_div(R(2) * SbSb, bstar));
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
    const R beta = c_beta0 * fbeta;
    R dkdw = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) dkdw += gk[a] * gw[a];
    const R sd = dkdw > R(0) ? c_sdo : R(0);
    const R CD = g_div(sd * rho, om) * dkdw;
    const R alpha = c_alpha;
    ak += dt * Pk;
    aw += dt * (alpha * rho * g_div(om, wt) * X - g_div(R(2), R(3)) * alpha * rho * om * div + CD);
    rate_k = bstar * om;
    rate_w = beta * om;
  }
  ak = g_div(ak, R(1) + dt * rate_k);
  aw = g_div(aw, R(1) + dt * rate_w);
  const R rho_new = (R)((const S*)K.Wnew)[cell];
  const R wfloor = rho_new * c_wfloor;
  ((R*)K.RKout)[cell] = ak > R(0) ? ak : R(0);
  ((R*)K.RWout)[cell] = aw > wfloor ? aw : wfloor;
}

template <int D, int PREC>
void launch_d(const KOmegaArgs& K, cudaStream_t s) {
  using T = KTile<D>;
  unsigned blocks = 1;
  const int tt[3] = {T::X, T::Y, T::Z};
  for (int a = 0; a < 3; ++a) blocks *= (unsigned)((K.g.n[a] + tt[a] - 1) / tt[a]);
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
