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
// Tiles of cells per block with a shared-memory halo (ghost cells resolved once per tile); slopes
// once per cell, fluxes once per face.
#include "gks_dispatch.h"
#include "gks_step.cuh"

namespace gks {

namespace {

// Tile of cells per 256-thread block.  Phases, separated by barriers: (1) stage k, omega, density
// and velocity of the tile and two halo layers (ghost cells resolved once), widths and inverse
// distances; (2) limited slopes of k and omega and rho k / omega of the tile and its first halo
// ring, once per cell; (3) convective + diffusive flux of k and omega through every face of the
// tile, once per face; (4) per cell: flux divergence, sources, implicit destruction, floors.
template <int D> struct KTile;
template <> struct KTile<1> { static constexpr int X = 256, Y = 1, Z = 1; };
template <> struct KTile<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct KTile<3> { static constexpr int X = 8, Y = 8, Z = 4; };

template <int D> struct KGeom {
  using T = KTile<D>;
  static constexpr int X = T::X, Y = T::Y, Z = T::Z;
  static constexpr int HX = X + 4, HY = D >= 2 ? Y + 4 : 1, HZ = D >= 3 ? Z + 4 : 1, NH = HX * HY * HZ;
  static constexpr int RX = X + 2, RY = D >= 2 ? Y + 2 : 1, RZ = D >= 3 ? Z + 2 : 1, NR = RX * RY * RZ;
  static constexpr int NFX = (X + 1) * Y * Z, NFY = D >= 2 ? X * (Y + 1) * Z : 0, NFZ = D >= 3 ? X * Y * (Z + 1) : 0;
  static constexpr int NF = NFX + NFY + NFZ;
  static constexpr int NW = HX + HY + HZ;
  // stage: k, omega, rho, velocity (D); widths, inverse centre distances, inverse gradient distances;
  // ring: slopes of k and omega along each axis, rho k / omega; faces: flux of k and of omega
  static constexpr int NVAL = (3 + D) * NH + 3 * NW + (2 * D + 1) * NR + 2 * NF;
  template <class R> static constexpr size_t smem_bytes() { return sizeof(R) * (size_t)NVAL; }
};

template <int D, int PREC>
__global__ void __launch_bounds__(256) komega_kernel(const __grid_constant__ KOmegaArgs K) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  using G = KGeom<D>;
  constexpr int nv = D + 2, X = G::X, Y = G::Y, HX = G::HX, HY = G::HY;
  extern __shared__ __align__(16) unsigned char kom_smem[];
  R* sk = (R*)kom_smem;            // [NH] k
  R* sw = sk + G::NH;              // [NH] omega
  R* sr = sw + G::NH;              // [NH] density (boundary rules)
  R* su = sr + G::NH;              // [D][NH] velocity
  R* swid = su + D * G::NH;        // [NW] widths of the halo positions along each axis
  R* sic = swid + G::NW;           // [NW] 1 / centre distance between positions p - 1 and p
  R* sig_ = sic + G::NW;           // [NW] 1 / centre distance between positions p - 1 and p + 1
  R* ssl = sig_ + G::NW;           // [2][D][NR] limited slopes of k and omega
  R* smd = ssl + 2 * D * G::NR;    // [NR] rho k / omega
  R* sgk = smd + G::NR;            // [NF] flux of k
  R* sgw = sgk + G::NF;            // [NF] flux of omega
  __shared__ R s_dt;

  const DevGrid& g = K.g;
  const int tiles_x = (g.n[0] + X - 1) / X;
  const int tiles_y = D >= 2 ? (g.n[1] + Y - 1) / Y : 1;
  const int b = blockIdx.x;
  const int ox = (b % tiles_x) * X;
  const int oy = D >= 2 ? ((b / tiles_x) % tiles_y) * Y : 0;
  const int oz = D >= 3 ? (b / (tiles_x * tiles_y)) * G::Z : 0;
  const int org[3] = {ox, oy, oz};
  const int tid = threadIdx.x;
  const Consts<R> kc = make_consts<R>(g);
  const R* RK = (const R*)K.RKin;
  const R* RW = (const R*)K.RWin;
  const S* W = (const S*)K.Win;
  constexpr bool F = sizeof(R) == sizeof(float);
  const R c_alpha = F ? (R)K.falpha : (R)K.alpha, c_beta0 = F ? (R)K.fbeta0 : (R)K.beta0;
  const R c_bstar = F ? (R)K.fbeta_star : (R)K.beta_star, c_sigma = F ? (R)K.fsigma : (R)K.sigma;
  const R c_sstar = F ? (R)K.fsigma_star : (R)K.sigma_star, c_sdo = F ? (R)K.fsigma_do : (R)K.sigma_do;
  const R c_clim = F ? (R)K.fC_lim : (R)K.C_lim, c_wfloor = F ? (R)K.fomega_floor : (R)K.omega_floor;
  const R mu = kc.mu;
  const int hs[3] = {1, HX, HX * HY};
  const int woff[3] = {0, HX, HX + HY};

  // ---- (1) stage --------------------------------------------------------------------------
  for (int l = tid; l < G::NH; l += 256) {
    const int hi = l % HX, hj = (l / HX) % HY, hk = l / (HX * HY);
    const int gi = ox + hi - 2, gj = D >= 2 ? oy + hj - 2 : 0, gk = D >= 3 ? oz + hk - 2 : 0;
    R w[nv];
    load_cell<D, PREC>(g, K.Win, kc, gi, gj, gk, w);
    sr[l] = w[0];
    const R ir = g_rcp(w[0]);
#pragma unroll
    for (int a = 0; a < D; ++a) su[a * G::NH + l] = w[1 + a] * ir;
    const long m = field_cell(g, D, gi, gj, gk);
    const R irm = g_rcp((R)W[m]);
    sk[l] = RK[m] * irm;
    sw[l] = RW[m] * irm;
  }
  for (int l = tid; l < G::NW; l += 256) {
    // halo position p of axis a is the cell origin + p - 2 (width index that cell + kWG)
    const int a = l < HX ? 0 : (l < HX + HY ? 1 : 2);
    const int p = l - woff[a];
    if (a < D) {
      const int top = g.n[a] + 2 * kWG - 1, iw = org[a] + p - 2 + kWG;
      const R wm = (R)g.w[a][min(max(iw - 1, 0), top)];
      const R w0 = (R)g.w[a][min(max(iw, 0), top)];
      const R wp = (R)g.w[a][min(max(iw + 1, 0), top)];
      swid[l] = w0;
      sic[l] = g_rcp(R(0.5) * (wm + w0));
      sig_[l] = g_rcp(R(0.5) * wm + w0 + R(0.5) * wp);
    } else {
      swid[l] = sic[l] = sig_[l] = R(1);
    }
  }
  if (tid == 0) s_dt = (R)K.ctrl->last_dt;
  __syncthreads();
  const R dt = s_dt;

  // ---- (2) ring: slopes of k and omega, rho k / omega --------------------------------------
  for (int r = tid; r < G::NR; r += 256) {
    const int ri = r % G::RX, rj = (r / G::RX) % G::RY, rk = r / (G::RX * G::RY);
    const int hpos[3] = {ri + 1, D >= 2 ? rj + 1 : 0, D >= 3 ? rk + 1 : 0};
    const int h = (hpos[2] * HY + hpos[1]) * HX + hpos[0];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int st = hs[a];
      const R im = sic[woff[a] + hpos[a]], ip = sic[woff[a] + hpos[a] + 1];
      ssl[(0 * D + a) * G::NR + r] = limiter<R>(g.limiter, (sk[h] - sk[h - st]) * im, (sk[h + st] - sk[h]) * ip);
      ssl[(1 * D + a) * G::NR + r] = limiter<R>(g.limiter, (sw[h] - sw[h - st]) * im, (sw[h + st] - sw[h]) * ip);
    }
    smd[r] = g_div(sr[h] * sk[h], sw[h]);
  }
  __syncthreads();

  // ---- (3) faces: convection by the flow step's mass flux, diffusion -----------------------
  for (int f = tid; f < G::NF; f += 256) {
    int a, ci, cj, ck;  // face between tile cells c - e_a and c
    if (f < G::NFX) {
      a = 0;
      ci = f % (X + 1);
      cj = (f / (X + 1)) % Y;
      ck = f / ((X + 1) * Y);
    } else if (D >= 2 && f < G::NFX + G::NFY) {
      const int q = f - G::NFX;
      a = 1;
      ci = q % X;
      cj = (q / X) % (Y + 1);
      ck = q / (X * (Y + 1));
    } else {
      const int q = f - G::NFX - G::NFY;
      a = 2;
      ci = q % X;
      cj = (q / X) % Y;
      ck = q / (X * Y);
    }
    const int gc[3] = {ox + ci, oy + cj, oz + ck};
    int nf[3] = {g.n[0], g.n[1], g.n[2]};
    nf[a] += 1;
    if (gc[0] >= nf[0] || gc[1] >= nf[1] || gc[2] >= nf[2]) continue;  // outside the grid
    const R fr = ((const R*)K.mflux[a])[((long)gc[2] * nf[1] + gc[1]) * nf[0] + gc[0]];
    const int rst[3] = {1, G::RX, G::RX * G::RY};
    const int rR = ((ck + (D >= 3 ? 1 : 0)) * G::RY + (cj + (D >= 2 ? 1 : 0))) * G::RX + (ci + 1);
    const int rL = rR - rst[a];
    const int hR = ((ck + (D >= 3 ? 2 : 0)) * HY + (cj + (D >= 2 ? 2 : 0))) * HX + (ci + 2);
    const int hL = hR - hs[a];
    const int pR = (a == 0 ? ci : (a == 1 ? cj : ck)) + 2;
    const R hl = swid[woff[a] + pR - 1], hr = swid[woff[a] + pR];
    const R il = g_rcp(R(0.5) * hl + R(0.5) * hr);
    const R frl = g_div(fr, sr[hL]), frr = g_div(fr, sr[hR]);
    const R md = R(0.5) * (smd[rL] + smd[rR]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const R* v = q == 0 ? sk : sw;
      const R sL = ssl[(q * D + a) * G::NR + rL], sR = ssl[(q * D + a) * G::NR + rR];
      const R phiL = v[hL] + R(0.5) * sL * (hl - frl);
      const R phiR = v[hR] - R(0.5) * sR * (hr + frr);
      R gf = fr * (fr >= R(0) ? phiL : phiR);
      if (K.diffusion) {
        const R coef = mu + (q == 0 ? c_sstar : c_sigma) * md;
        gf -= dt * coef * (v[hR] - v[hL]) * il;
      }
      (q == 0 ? sgk : sgw)[f] = gf;
    }
  }
  __syncthreads();

  // ---- (4) cells ---------------------------------------------------------------------------
  const int li = tid % X, lj = (tid / X) % Y, lk = tid / (X * Y);
  const int c[3] = {ox + li, oy + lj, oz + lk};
  if (c[0] >= g.n[0] || (D >= 2 && c[1] >= g.n[1]) || (D >= 3 && c[2] >= g.n[2])) return;
  const long cell = cell_index(g, c[0], c[1], c[2]);
  const int h0 = ((lk + (D >= 3 ? 2 : 0)) * HY + (lj + (D >= 2 ? 2 : 0))) * HX + (li + 2);
  const int lc[3] = {li, lj, lk};
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
    const int st = hs[a];
    const int p = lc[a] + 2;
    const R id = sig_[woff[a] + p];
#pragma unroll
    for (int bb = 0; bb < D; ++bb) grad[a][bb] = (su[bb * G::NH + h0 + st] - su[bb * G::NH + h0 - st]) * id;
    gk[a] = (sk[h0 + st] - sk[h0 - st]) * id;
    gw[a] = (sw[h0 + st] - sw[h0 - st]) * id;
    // faces c - 1/2 and c + 1/2 along a in the tile's face numbering
    int fm, fp;
    if (a == 0) {
      fm = (lk * Y + lj) * (X + 1) + li;
      fp = fm + 1;
    } else if (a == 1) {
      fm = G::NFX + (lk * (Y + 1) + lj) * X + li;
      fp = fm + X;
    } else {
      fm = G::NFX + G::NFY + (lk * Y + lj) * X + li;
      fp = fm + X * Y;
    }
    const R ih = g_rcp(swid[woff[a] + p]);
    ak -= (sgk[fp] - sgk[fm]) * ih;
    aw -= (sgw[fp] - sgw[fm]) * ih;
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
  using R = typename PrecT<PREC>::R;
  unsigned blocks = 1;
  const int tt[3] = {T::X, T::Y, T::Z};
  for (int a = 0; a < 3; ++a) blocks *= (unsigned)((K.g.n[a] + tt[a] - 1) / tt[a]);
  komega_kernel<D, PREC><<<blocks, 256, KGeom<D>::template smem_bytes<R>(), s>>>(K);
}

template <int D, int PREC>
cudaError_t prepare_d() {
  using R = typename PrecT<PREC>::R;
  return cudaFuncSetAttribute(komega_kernel<D, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)KGeom<D>::template smem_bytes<R>());
}

}  // namespace

cudaError_t prepare_komega() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_d<1, PREC_F64>()) != cudaSuccess) e = r;
  if ((r = prepare_d<1, PREC_F32>()) != cudaSuccess) e = r;
  if ((r = prepare_d<1, PREC_F32D>()) != cudaSuccess) e = r;
  if ((r = prepare_d<2, PREC_F64>()) != cudaSuccess) e = r;
  if ((r = prepare_d<2, PREC_F32>()) != cudaSuccess) e = r;
  if ((r = prepare_d<2, PREC_F32D>()) != cudaSuccess) e = r;
  if ((r = prepare_d<3, PREC_F64>()) != cudaSuccess) e = r;
  if ((r = prepare_d<3, PREC_F32>()) != cudaSuccess) e = r;
  if ((r = prepare_d<3, PREC_F32D>()) != cudaSuccess) e = r;
  return e;
}

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
