// The fused tile step of body-fitted 2D grids (time step and steady residual), shared by the
// translation units that instantiate it (gks_curv.cu: MUSCL-2; gks_curv_recon.cu: MUSCL-3 and
// WENO-5).  Each unit gets its own internal copy of these templates.
#pragma once

#include "gks_curv.h"
#include "gks_flux.cuh"
#include "gks_step.cuh"

namespace gks {
namespace {

template <class R>
struct FaceView {
  const R* p;
  long nf;
  __device__ __forceinline__ R operator()(int q, long f) const { return p[(long)q * nf + f]; }
};

// Turbulent relaxation time of interior cell (gi, gj) from Green-Gauss gradients; st(q, v) gives
// the state of the cell (q = 4) and of its neighbours i-1, i+1, j-1, j+1 (q = 0..3).
// CONS = false: a caller whose fields are never rho k, rho omega (g.turb_cons unset) skips that test.
template <class R, bool CONS = true, class StateOf>
__device__ __forceinline__ R tau_gg(const DevGrid& g, const Consts<R>& kc, const CurvGeom& G, const void* f1p,
                                    const void* f2p, int gi, int gj, StateOf st) {
  const int n0 = g.n[0];
  const long c = (long)gj * n0 + gi;
  R w[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) w[v] = st(4, v);
  const R p = pressure_of<R>(2, kc.gamma, w);
  R f1 = ((const R*)f1p)[c];
  if (CONS && g.turb_cons) f1 = g_div(f1, w[0]);  // rho k -> k (k-omega transport)
  if (g.turb_model == TURB_MUT) return g_div(f1, p);
  R f2 = ((const R*)f2p)[c];
  if (CONS && g.turb_cons) f2 = g_div(f2, w[0]);
  const FaceView<R> fi{(const R*)G.face[0], G.nf[0]}, fj{(const R*)G.face[1], G.nf[1]};
  const long fa = (long)gj * (n0 + 1) + gi, fc = (long)gj * n0 + gi;
  const long fid[4] = {fa, fa + 1, fc, fc + n0};
  const R ir = g_rcp(w[0]);
  const R U[2] = {w[1] * ir, w[2] * ir};
  R gr[2][2] = {{R(0), R(0)}, {R(0), R(0)}};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const FaceView<R>& fv = q < 2 ? fi : fj;
    const R nx = fv(0, fid[q]), ny = fv(1, fid[q]), L = fv(2, fid[q]);
    const R sgn = (q & 1) ? R(1) : R(-1);
    const R irn = g_rcp(st(q, 0));
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const R uf = R(0.5) * (U[b] + st(q, 1 + b) * irn);
      gr[0][b] += sgn * uf * nx * L;
      gr[1][b] += sgn * uf * ny * L;
    }
  }
  const R ia = ((const R*)G.iarea)[c];
  R s2 = R(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const R sab = R(0.5) * (gr[a][b] + gr[b][a]) * ia;
      s2 += sab * sab;
    }
  const R S = g_sqrt(R(2) * s2);
  R nu, eta;
  if (g.turb_model == TURB_KEPS) {
    nu = g_div(kc.C_mu * f1 * f1, f2);
    eta = g_div(S * f1, f2);
  } else {
    nu = g_div(f1, f2);
    eta = g_div(S, kc.beta_star * f2);
  }
  return (f1 > R(0) && f2 > R(0)) ? g_div(w[0] * nu, p * g_sqrt(R(1) + eta * eta)) : R(0);
}

// ---- k-omega transport pieces (the transport kernels and the fused step) ----------------------
// Fluxes (rho k, rho omega) through one face, towards increasing index: v*[0..3] the four cells
// along the grid line, rl, rr the densities of the two cells beside the face, fv the face's mass flux
// followed by L, 1/d01, 1/d12, 1/d23, d_l, d_r of its record.
template <class R>
__device__ __forceinline__ void kw_face(const R* vk, const R* vw, R rl, R rr, const R* fv, R dt, R mu, R sigk, R sigw,
                                        int limiter_kind, bool diffusion, R* out) {
  const R fr = fv[0], L = fv[1], i01 = fv[2], i12 = fv[3], i23 = fv[4], dl = fv[5], dr = fv[6];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const R* v = q == 0 ? vk : vw;
    const R s0 = limiter<R>(limiter_kind, (v[1] - v[0]) * i01, (v[2] - v[1]) * i12);
    const R s1 = limiter<R>(limiter_kind, (v[2] - v[1]) * i12, (v[3] - v[2]) * i23);
    const R phiL = v[1] + s0 * (dl - R(0.5) * g_div(fr, rl * L));
    const R phiR = v[2] - s1 * (dr + R(0.5) * g_div(fr, rr * L));
    R gq = fr * (fr >= R(0) ? phiL : phiR);
    if (diffusion) {
      const R mdl = g_div(rl * vk[1], vw[1]), mdr = g_div(rr * vk[2], vw[2]);
      const R coef = mu + (q == 0 ? sigk : sigw) * R(0.5) * (mdl + mdr);
      gq -= dt * coef * (v[2] - v[1]) * i12 * L;
    }
    out[q] = gq;
  }
}

// Wilcox's production terms of the cell at staged index sc (destruction left to the caller):
// Sk = P_k, Sw = alpha rho (omega / omega~) X - 2/3 alpha rho omega div U + the cross diffusion, with
// Green-Gauss gradients from the staged neighbours (face values the means of the two cells);
// gsx, gsy: the outward n_x L, n_y L of the faces i-1/2, i+1/2, j-1/2, j+1/2.
template <class R, int SX>
__device__ __forceinline__ void kw_sources(const R* sk, const R* sw, const R* sr, const R* su, const R* sv, int sc,
                                           const R* gsx, const R* gsy, R A, R alpha, R beta_star, R sigma_do, R C_lim,
                                           R& Sk, R& Sw) {
  const R rho = sr[sc], k0 = sk[sc], w0 = sw[sc];
  const int nb[4] = {sc - 1, sc + 1, sc - SX, sc + SX};
  const R uc[2] = {su[sc], sv[sc]};
  R gu[2][2] = {{R(0), R(0)}, {R(0), R(0)}}, gk[2] = {R(0), R(0)}, gw[2] = {R(0), R(0)};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R sx = gsx[q], sy = gsy[q];
    const R un[2] = {su[nb[q]], sv[nb[q]]};
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const R uf = R(0.5) * (uc[b] + un[b]);
      gu[0][b] += uf * sx;
      gu[1][b] += uf * sy;
    }
    const R kff = R(0.5) * (k0 + sk[nb[q]]), wff = R(0.5) * (w0 + sw[nb[q]]);
    gk[0] += kff * sx;
    gk[1] += kff * sy;
    gw[0] += wff * sx;
    gw[1] += wff * sy;
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    gk[a] /= A;
    gw[a] /= A;
#pragma unroll
    for (int b = 0; b < 2; ++b) gu[a][b] /= A;
  }
  const R div = gu[0][0] + gu[1][1];
  R SS = R(0), SbSb = R(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const R sab = R(0.5) * (gu[a][b] + gu[b][a]);
      SS += sab * sab;
      const R sb = sab - (a == b ? div / R(3) : R(0));
      SbSb += sb * sb;
    }
  const R X = R(2) * SS - R(2) / R(3) * div * div;
  const R wt = fmax(w0, C_lim * g_sqrt(R(2) * SbSb / beta_star));
  const R muT = rho * k0 / wt;
  Sk = muT * X - R(2) / R(3) * rho * k0 * div;
  const R dkdw = gk[0] * gw[0] + gk[1] * gw[1];
  const R sd = dkdw > R(0) ? sigma_do : R(0);
  const R CD = sd * rho / w0 * dkdw;
  Sw = alpha * rho * (w0 / wt) * X - R(2) / R(3) * alpha * rho * w0 * div + CD;
}

// ---- fused tile step ---------------------------------------------------------------------------
// One CTA advances an X x Y tile of cells: the state of the tile and two halo layers (boundary rules
// applied) and the geometry records of the tile's faces are staged in shared memory, then the
// turbulent relaxation time of the tile and its first ring, the fluxes of the tile's faces (a face
// on the tile edge is evaluated by both tiles that share it), and the update of the tile's cells.
template <int V> struct CurvTile;
template <> struct CurvTile<0> { static constexpr int X = 32, Y = 15, T = 256; };
template <> struct CurvTile<1> { static constexpr int X = 16, Y = 7, T = 128; };
// 16 x 11: 379 faces fill three rounds of 128 threads; one wave of 4 CTAs per SM covers the paper's
// fine aerofoil grid (608 x 160: 570 tiles)
template <> struct CurvTile<2> { static constexpr int X = 16, Y = 11, T = 128; };

// H: halo layers (two for the four-cell MUSCL stencils, three for WENO-5's six cells)
template <int V, int H_ = 2>
struct CurvTileGeom {
  static constexpr int X = CurvTile<V>::X, Y = CurvTile<V>::Y, T = CurvTile<V>::T, H = H_;
  static constexpr int HX = X + 2 * H, HY = Y + 2 * H, NH = HX * HY;
  static constexpr int NFX = (X + 1) * Y, NFY = X * (Y + 1), NF = NFX + NFY;
  static constexpr int TX = X + 2, TY = Y + 2, NT = TX * TY;  // tile and first ring (tau)
  template <class R, bool TR = false> static constexpr size_t smem_bytes() {
    return sizeof(R) * (4 * (size_t)NH + 8 * (size_t)NF + 4 * (size_t)NF + NT + (TR ? 4 * (size_t)NH + 2 * (size_t)NF : 0)) +
           sizeof(float) * 4 * X * Y;
  }
};

// MODE 0: one time step (A.Win -> A.Wout, control block as the rectilinear step).  MODE 1: the
// steady residual of A.Win (SteadyArgs): face windows cfl_flux min(s_l, s_r) from the local steps s,
// flux rates times L summed per cell (plus the forcing) into R, tau_t of the tile cells stored.
// MD: the multi-dimensional expansion (tangential slopes of the two cells in the face frame).
// RC: the face reconstruction along the grid line (0 MUSCL-2 with limited slopes over the centroid
// distances; 1 MUSCL-3 and 2 WENO-5 in index space on the rotated states, normal slopes the
// one-sided differences to the face values over the centroid-to-face distances).
__host__ __device__ constexpr int halo_for(int rc) { return rc == 2 ? 3 : 2; }

// TR (MODE 0): k-omega transport fused into the step: f1, f2 are rho k, rho omega; k, omega, u, v of
// the tile and its halo are staged, each face also evaluates the transport fluxes of rho k and
// rho omega with its mass flux, and each cell's update advances them (the transport kernel's
// arithmetic) into A.RKout, A.RWout.
// RAR: the rarefaction option (eps = tau/tauhat in the faces' time coefficients).
template <int PREC, int V, int MODE, bool MD, int RC = 0, bool TR = false, bool RAR = false>
__global__ void __launch_bounds__(CurvTile<V>::T, PREC == PREC_F64 ? 1 : 512 / CurvTile<V>::T)
    curv_step_kernel(const __grid_constant__ StepArgs A, const __grid_constant__ CurvGeom G,
                     const __grid_constant__ SteadyArgs SA) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  using TG = CurvTileGeom<V, halo_for(RC)>;
  constexpr int X = TG::X, Y = TG::Y, T = TG::T, H = TG::H, HX = TG::HX, NH = TG::NH;
  // k-omega transport runs through this instantiation's fields and mass fluxes unless it is fused
  // (TR): the MUSCL-2 time step in FP64 or the FP32 float pair carries it fused, or has none
  constexpr bool SEPARATE_KW = MODE == 1 || RC != 0 || PREC == PREC_F32D;
  constexpr bool CONS = TR || SEPARATE_KW;
  constexpr int NFX = TG::NFX, NF = TG::NF, TX = TG::TX, NT = TG::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* Ws = (R*)smem_raw;    // [4][NH] state of the tile and its halo
  R* Gs = Ws + 4 * NH;     // [8][NF] face records: i-faces (X + 1) x Y, then j-faces X x (Y + 1)
  R* Fs = Gs + 8 * NF;     // [4][NF] face fluxes times length
  R* Ts = Fs + 4 * NF;     // [TY][TX] tau_t of the tile and its first ring
  float* Lo = (float*)(Ts + NT);  // [4][X * Y] low words of the tile's state (float pair form)
  // fused transport: k, omega, u, v of the tile and its halo, face fluxes of rho k and rho omega
  R* Ks = (R*)(Lo + 4 * X * Y);
  R* Os = Ks + (TR ? NH : 0);
  R* Us = Os + (TR ? NH : 0);
  R* Vs = Us + (TR ? NH : 0);
  R* Gk = Vs + (TR ? NH : 0);
  R* Gw = Gk + (TR ? NF : 0);
  __shared__ double red[kMaxWarps];
  __shared__ double s_dt;
  const DevGrid& g = A.g;
  const int tid = threadIdx.x;
  const int n0 = g.n[0], n1 = g.n[1];
  const int ntx = (n0 + X - 1) / X;
  const int ox = (blockIdx.x % ntx) * X, oy = (blockIdx.x / ntx) * Y;
  const Consts<R> kc = make_consts<R>(g);

  // ---- face records (asynchronous copies) and the time step ----------------------------------
  for (int l = tid; l < NF; l += T) {
    long gf;
    long nf;
    int a;
    if (l < NFX) {
      const int li = l % (X + 1), lj = l / (X + 1);
      const int fi = ox + li, j = oy + lj;
      if (fi > n0 || j >= n1) continue;
      a = 0;
      nf = G.nf[0];
      gf = (long)j * (n0 + 1) + fi;
    } else {
      const int m = l - NFX, li = m % X, lj = m / X;
      const int i = ox + li, fj = oy + lj;
      if (i >= n0 || fj > n1) continue;
      a = 1;
      nf = G.nf[1];
      gf = (long)fj * n0 + i;
    }
    const R* src = (const R*)G.face[a];
#pragma unroll
    for (int q = 0; q < 8; ++q) cp_async<sizeof(R)>(&Gs[q * NF + l], &src[(long)q * nf + gf]);
  }
  // everything below may read what the previous kernel in the stream wrote: with a programmatic
  // (early) launch of this kernel, wait here for that kernel's completion; the face records
  // above are the grid's static geometry
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the control words of the time step (thread 0), loaded before the state copies are issued so that
  // their latency overlaps them; the time step itself is formed once the copies are in flight
  double c_dtf = 0.0, c_cfl = 0.0, c_tend = 0.0, c_t = 0.0;
  unsigned long long c_rate = 0ull;
  if (MODE != 1 && tid == 0) {
    const Ctrl* c = A.ctrl;
    c_dtf = c->dt_fixed;
    c_cfl = c->cfl;
    c_tend = c->t_end;
    c_t = c->t[A.tslot];
    c_rate = c->rate[A.slot];
  }
  // ---- state of the tile and two halo layers, boundary rules applied -------------------------
  // (cells inside the grid by asynchronous copies where the stored type is the arithmetic one;
  // ghost cells through the boundary rules)
  for (int l = tid; l < NH; l += T) {
    const int hi = l % HX, hj = l / HX;
    const int gi = ox + hi - H, gj = oy + hj - H;
    R w[4];
    if (PREC != PREC_F32D && gi >= 0 && gi < n0 && gj >= 0 && gj < n1) {
      const S* src = (const S*)A.Win + (long)gj * n0 + gi;
#pragma unroll
      for (int v = 0; v < 4; ++v) cp_async<sizeof(R)>(&Ws[v * NH + l], src + (long)v * g.ncell);
      continue;
    }
    if (gi >= -H && gi < n0 + H && gj >= -H && gj < n1 + H) {
      load_cell<2, PREC>(g, A.Win, kc, gi, gj, 0, w);
    } else {
      w[0] = R(1);
      w[1] = w[2] = R(0);
      w[3] = R(1);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) Ws[v * NH + l] = w[v];
  }
  if (PREC == PREC_F32 && MODE == 0)
    for (int l = tid; l < X * Y; l += T) {
      const int gi = ox + l % X, gj = oy + l / X;
      if (gi >= n0 || gj >= n1) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v) cp_async<4>(&Lo[v * X * Y + l], &A.Win_lo[(long)v * g.ncell + (long)gj * n0 + gi]);
    }
  if (MODE == 1) {
    if (tid == 0) s_dt = 1.0;
  } else if (tid == 0) {
    double dtv = c_dtf > 0.0 ? c_dtf : c_cfl / __longlong_as_double((long long)c_rate);
    if (c_tend > 0.0) dtv = (c_t >= c_tend) ? 0.0 : fmin(dtv, c_tend - c_t);
    s_dt = dtv;
    if (blockIdx.x == 0) {
      Ctrl* c = A.ctrl;
      c->t[A.tslot ^ 1] = c_t + dtv;
      c->rate[(A.slot + 2) % 3] = 0ull;
      c->last_dt = dtv;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const double dt_d = s_dt;
  if (dt_d == 0.0) {  // t_end reached: carry the state over
    for (int l = tid; l < X * Y; l += T) {
      const int gi = ox + l % X, gj = oy + l / X;
      if (gi >= n0 || gj >= n1) continue;
      const long c = (long)gj * n0 + gi;
      for (int v = 0; v < 4; ++v) {
        ((S*)A.Wout)[(long)v * g.ncell + c] = ((const S*)A.Win)[(long)v * g.ncell + c];
        if (PREC == PREC_F32) A.Wout_lo[(long)v * g.ncell + c] = A.Win_lo[(long)v * g.ncell + c];
      }
      if (TR) {
        ((R*)A.RKout)[c] = ((const R*)A.f1)[c];
        ((R*)A.RWout)[c] = ((const R*)A.f2)[c];
      }
    }
    return;
  }
  const R dt = (R)dt_d;

  if (TR) {  // k, omega of each cell's source cell (rho k / rho there), velocities by the ghost rules
    for (int l = tid; l < NH; l += T) {
      const int gi = ox + l % HX - H, gj = oy + l / HX - H;
      const long sc = field_cell(g, 2, gi, gj, 0);
      const R rho_s = (R)((const S*)A.Win)[sc];
      Ks[l] = g_div(((const R*)A.f1)[sc], rho_s);
      Os[l] = g_div(((const R*)A.f2)[sc], rho_s);
      Us[l] = g_div(Ws[NH + l], Ws[l]);
      Vs[l] = g_div(Ws[2 * NH + l], Ws[l]);
    }
    if (g.turb_model == TURB_NONE) __syncthreads();  // else the tau phase's barrier follows
  }
  // ---- tau_t of the tile and its first ring (corners unused) ---------------------------------
  if (g.turb_model != TURB_NONE) {
    for (int l = tid; l < NT; l += T) {
      const int ti = l % TX - 1, tj = l / TX - 1;
      if ((ti < 0 || ti >= X) && (tj < 0 || tj >= Y)) continue;
      const int gi = ox + ti, gj = oy + tj;
      R t;
      if (gi >= 0 && gi < n0 && gj >= 0 && gj < n1) {
        const int h0 = (tj + H) * HX + (ti + H);
        const int off[5] = {-1, 1, -HX, HX, 0};
        t = tau_gg<R, CONS>(g, kc, G, A.f1, A.f2, gi, gj, [&](int q, int v) { return Ws[v * NH + h0 + off[q]]; });
      } else {  // a ghost cell takes its source cell's value
        const long sc = field_cell(g, 2, gi, gj, 0);
        const int si = (int)(sc % n0), sj = (int)(sc / n0);
        R nb[5][4];
        const int di[5] = {-1, 1, 0, 0, 0}, dj[5] = {0, 0, -1, 1, 0};
#pragma unroll
        for (int q = 0; q < 5; ++q) load_cell<2, PREC>(g, A.Win, kc, si + di[q], sj + dj[q], 0, nb[q]);
        t = tau_gg<R, CONS>(g, kc, G, A.f1, A.f2, si, sj, [&](int q, int v) { return nb[q][v]; });
      }
      Ts[l] = t;
      if (MODE == 1 && ti >= 0 && ti < X && tj >= 0 && tj < Y && gi < n0 && gj < n1)
        ((R*)SA.tau)[(long)gj * n0 + gi] = t;
    }
    __syncthreads();
  }

  // ---- face fluxes ----------------------------------------------------------------------------
  {
    Gas<R> gas;
    gas.bK = kc.bK;
    gas.ibK = kc.ibK;
    gas.K = kc.K;
    gas.mu = kc.mu;
    gas.C_a = kc.C_a;
    const bool turb = g.turb_model != TURB_NONE;
    for (int l = tid; l < NF; l += T) {
      int li, lj, a;
      bool valid;
      if (l < NFX) {
        li = l % (X + 1);
        lj = l / (X + 1);
        a = 0;
        valid = ox + li <= n0 && oy + lj < n1;
      } else {
        const int m = l - NFX;
        li = m % X;
        lj = m / X;
        a = 1;
        valid = ox + li < n0 && oy + lj <= n1;
      }
      if (!valid) continue;
      const R nx = Gs[l], ny = Gs[NF + l], L = Gs[2 * NF + l];
      const R i01 = Gs[3 * NF + l], i12 = Gs[4 * NF + l], i23 = Gs[5 * NF + l];
      const R dl = Gs[6 * NF + l], dr = Gs[7 * NF + l];
      // stencil: cells li - 2 .. li + 1 along the face normal's grid line (WENO-5 also li - 3 and
      // li + 2), rotated into the face frame
      const int base = a == 0 ? (lj + H) * HX + li + H - 2 : (lj + H - 2) * HX + li + H;
      const int stride = a == 0 ? 1 : HX;
      auto rotated = [&](int h, R* r) {
        const R w0 = Ws[h], w1 = Ws[NH + h], w2 = Ws[2 * NH + h], w3 = Ws[3 * NH + h];
        r[0] = w0;
        r[1] = w1 * nx + w2 * ny;
        r[2] = -w1 * ny + w2 * nx;
        r[3] = w3;
      };
      R S4[4][4];
#pragma unroll
      for (int s = 0; s < 4; ++s) rotated(base + s * stride, S4[s]);
      R wl[4], wr[4], cl[4], cr[4], sl[4], sr[4];
      const bool fo = MODE == 1 && SA.first_order;
      if (RC == 0 || fo) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const R dm = (S4[1][v] - S4[0][v]) * i01, dc = (S4[2][v] - S4[1][v]) * i12,
                  dp = (S4[3][v] - S4[2][v]) * i23;
          sl[v] = fo ? R(0) : limiter<R>(g.limiter, dm, dc);
          sr[v] = fo ? R(0) : limiter<R>(g.limiter, dc, dp);
          wl[v] = S4[1][v] + dl * sl[v];
          wr[v] = S4[2][v] - dr * sr[v];
          cl[v] = S4[1][v];
          cr[v] = S4[2][v];
        }
      } else {
        R E0[4], E1[4];  // cells li - 3 and li + 2 (WENO-5)
        if (RC == 2) {
          rotated(base - stride, E0);
          rotated(base + 4 * stride, E1);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (RC == 2) {
            wl[v] = weno5<R>(E0[v], S4[0][v], S4[1][v], S4[2][v], S4[3][v]);
            wr[v] = weno5<R>(E1[v], S4[3][v], S4[2][v], S4[1][v], S4[0][v]);
          } else {
            wl[v] = muscl3_right<R>(S4[0][v], S4[1][v], S4[2][v]);
            wr[v] = muscl3_left<R>(S4[1][v], S4[2][v], S4[3][v]);
          }
          sl[v] = g_div(wl[v] - S4[1][v], dl);
          sr[v] = g_div(S4[2][v] - wr[v], dr);
          cl[v] = S4[1][v];
          cr[v] = S4[2][v];
        }
      }
      if (!physical<2, R>(kc.gamma, wl))
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          wl[v] = cl[v];
          sl[v] = R(0);
        }
      if (!physical<2, R>(kc.gamma, wr))
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          wr[v] = cr[v];
          sr[v] = R(0);
        }
      R tau_t = R(0);
      if (turb) {
        // tau of the two cells beside the face: (li - 1, lj) | (li, lj) or (li, lj - 1) | (li, lj)
        const int tr_ = (lj + 1) * TX + li + 1;
        tau_t = R(0.5) * (Ts[tr_ - (a == 0 ? 1 : TX)] + Ts[tr_]);
      }
      R tl[1][4] = {{R(0), R(0), R(0), R(0)}}, trr[1][4] = {{R(0), R(0), R(0), R(0)}};
      if (MD && !fo) {
        // tangential slopes: limited differences of the rotated states along the transverse grid
        // line over the projected centroid steps (face records tang)
        const long gf = a == 0 ? (long)(oy + lj) * (n0 + 1) + ox + li : (long)(oy + lj) * n0 + ox + li;
        const R* tg = (const R*)G.tang[a];
        const long nfa = a == 0 ? G.nf[0] : G.nf[1];
        const int step = a == 0 ? HX : 1;  // transverse neighbour in the halo
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int h0 = a == 0 ? (lj + H) * HX + li + H - 1 + side : (lj + H - 1 + side) * HX + li + H;
          const R ihm = tg[(long)(2 * side) * nfa + gf], ihp = tg[(long)(2 * side + 1) * nfa + gf];
          R rm[4], rp[4];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int h = q == 0 ? h0 - step : h0 + step;
            const R w0 = Ws[h], w1 = Ws[NH + h], w2 = Ws[2 * NH + h], w3 = Ws[3 * NH + h];
            R* r = q == 0 ? rm : rp;
            r[0] = w0;
            r[1] = w1 * nx + w2 * ny;
            r[2] = -w1 * ny + w2 * nx;
            r[3] = w3;
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const R c0 = S4[1 + side][v];
            const R t = limiter<R>(g.limiter, (c0 - rm[v]) * ihm, (rp[v] - c0) * ihp);
            if (side == 0)
              tl[0][v] = t;
            else
              trr[0][v] = t;
          }
        }
      }
      R F[4], tau;
      R win = dt, Ls = L;
      if (MODE == 1) {  // window of the face from the local steps of its two cells
        const int ai = a == 0 ? ox + li - 1 : ox + li, aj = a == 0 ? oy + lj : oy + lj - 1;
        const R* sloc = (const R*)SA.s_loc;
        win = (R)SA.cfl_flux * fmin(sloc[field_cell(g, 2, ai, aj, 0)], sloc[field_cell(g, 2, ox + li, oy + lj, 0)]);
        Ls = L / win;
      }
      if constexpr (std::is_same<R, float>::value) {
        // single precision: the two sides of the face on the paired FP32 instructions
        if (MD && !fo)
          face_flux_ps<2, true, RAR>(wl, wr, cl, cr, sl, sr, tl, trr, dl, dr, tau_t, win, gas, g.abar_t0, F, &tau);
        else
          face_flux_ps<2, false, RAR>(wl, wr, cl, cr, sl, sr, tl, trr, dl, dr, tau_t, win, gas, g.abar_t0, F, &tau);
      } else {
        if (MD && !fo)
          face_flux<2, R, true, RAR>(wl, wr, cl, cr, sl, sr, tl, trr, dl, dr, tau_t, win, gas, g.abar_t0, F, &tau);
        else
          face_flux<2, R, false, RAR>(wl, wr, cl, cr, sl, sr, tl, trr, dl, dr, tau_t, win, gas, g.abar_t0, F, &tau);
      }
      const R L_ = Ls;
      Fs[l] = F[0] * L_;
      Fs[NF + l] = (F[1] * nx - F[2] * ny) * L_;
      Fs[2 * NF + l] = (F[1] * ny + F[2] * nx) * L_;
      Fs[3 * NF + l] = F[3] * L_;
      if (TR) {
        R vk[4], vw[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          vk[t] = Ks[base + t * stride];
          vw[t] = Os[base + t * stride];
        }
        const bool kf = sizeof(R) == sizeof(float);
        const R sigk = kf ? (R)A.kw_fsigma_star : (R)A.kw_sigma_star, sigw = kf ? (R)A.kw_fsigma : (R)A.kw_sigma;
        const R fvr[7] = {Fs[l], L, i01, i12, i23, dl, dr};
        R out[2];
        kw_face<R>(vk, vw, S4[1][0], S4[2][0], fvr, dt, kc.mu, sigk, sigw, g.limiter, A.kw_diffusion, out);
        Gk[l] = out[0];
        Gw[l] = out[1];
      }
      if (SEPARATE_KW && A.mflux[0]) {  // the face's mass flux times L for a separate transport step:
                                        // time-integrated, or the rate over the residual's window
        const long gfm = a == 0 ? (long)(oy + lj) * (n0 + 1) + ox + li : (long)(oy + lj) * n0 + ox + li;
        ((R*)A.mflux[a])[gfm] = Fs[l];
      }
    }
  }
  __syncthreads();

  if (MODE == 1) {  // steady residual: sum of the outward flux rates times L, plus the forcing
    double s2 = 0.0;
    for (int l = tid; l < X * Y; l += T) {
      const int li = l % X, lj = l / X;
      const int gi = ox + li, gj = oy + lj;
      if (gi >= n0 || gj >= n1) continue;
      const long c = (long)gj * n0 + gi;
      const int fa = lj * (X + 1) + li, fc = NFX + lj * X + li;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        R r = Fs[v * NF + fa + 1] - Fs[v * NF + fa] + Fs[v * NF + fc + X] - Fs[v * NF + fc];
        if (SA.forcing) r += ((const R*)SA.forcing)[(long)v * g.ncell + c];
        ((R*)SA.R)[(long)v * g.ncell + c] = r;
        if (v == 0) {
          const double rr = (double)r / G.area[c];
          s2 += rr * rr;
        }
      }
    }
    if (SA.res_acc) {
      const double bsum = block_sum(s2, red);
      if (tid == 0) atomicAdd(SA.res_acc, bsum);
    }
    return;
  }

  // the next step may start its launch (it waits for this kernel's completion before its reads)
  if (MODE == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // ---- update, next CFL rate, physical check, residual norms ---------------------------------
  R rmax = R(0);
  unsigned bad = 0u;
  double racc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) racc[q] = 0.0;
  for (int l = tid; l < X * Y; l += T) {
    const int li = l % X, lj = l / X;
    const int gi = ox + li, gj = oy + lj;
    if (gi >= n0 || gj >= n1) continue;
    const long c = (long)gj * n0 + gi;
    const int fa = lj * (X + 1) + li, fc = NFX + lj * X + li;
    const int hidx = (lj + H) * HX + (li + H);
    const R ia = ((const R*)G.iarea)[c];
    R wn[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const R net = Fs[v * NF + fa + 1] - Fs[v * NF + fa] + Fs[v * NF + fc + X] - Fs[v * NF + fc];
      const long gidx = (long)v * g.ncell + c;
      double wd;
      if (PREC == PREC_F64) {
        const double w_old = (double)Ws[v * NH + hidx];
        const double w = w_old - (double)net / G.area[c];
        ((double*)A.Wout)[gidx] = w;
        wn[v] = (R)w;
        wd = w;
        if (A.resid) {
          const double r = (w - w_old) / dt_d;
          racc[v] += r * r;
          racc[4 + v] = fmax(racc[4 + v], fabs(r));
        }
      } else {
        const R inc = -net * ia;
        if (PREC == PREC_F32) {
          const float hi = (float)Ws[v * NH + hidx], lo = Lo[v * X * Y + l];
          const float s_ = hi + inc;
          const float bb = s_ - hi;
          const float err = (hi - (s_ - bb)) + (inc - bb);
          const float lo2 = lo + err;
          const float nhi = s_ + lo2;
          const float nlo = lo2 - (nhi - s_);
          ((float*)A.Wout)[gidx] = nhi;
          A.Wout_lo[gidx] = nlo;
          wn[v] = nhi;
          wd = (double)nhi + (double)nlo;
        } else {
          const double w = ((const double*)A.Win)[gidx] + (double)inc;
          ((double*)A.Wout)[gidx] = w;
          wn[v] = (R)w;
          wd = w;
        }
        if (A.resid) {
          const double r = (double)inc / dt_d;
          racc[v] += r * r;
          racc[4 + v] = fmax(racc[4 + v], fabs(r));
        }
      }
      if (A.resid) racc[8 + v] += wd * G.area[c];
    }
    if (!physical<2, R>(kc.gamma, wn)) bad = 1u;
    if (TR) {  // rho k, rho omega (the transport kernel's arithmetic)
      const bool kf = sizeof(R) == sizeof(float);
      const R alpha = kf ? (R)A.kw_falpha : (R)A.kw_alpha, beta0 = kf ? (R)A.kw_fbeta0 : (R)A.kw_beta0;
      const R sigma_do = kf ? (R)A.kw_fsigma_do : (R)A.kw_sigma_do, C_lim = kf ? (R)A.kw_fC_lim : (R)A.kw_C_lim;
      const R omega_floor = kf ? (R)A.kw_fomega_floor : (R)A.kw_omega_floor;
      const R Ac = (R)G.area[c];
      const R rk0 = ((const R*)A.f1)[c], rw0 = ((const R*)A.f2)[c];
      R ak = rk0 - (Gk[fa + 1] - Gk[fa] + Gk[fc + X] - Gk[fc]) / Ac;
      R aw = rw0 - (Gw[fa + 1] - Gw[fa] + Gw[fc + X] - Gw[fc]) / Ac;
      R rate_k = R(0), rate_w = R(0);
      if (A.kw_sources) {
        const int fq[4] = {fa, fa + 1, fc, fc + X};
        R gsx[4], gsy[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const R sgn = (q & 1) ? R(1) : R(-1);
          gsx[q] = sgn * Gs[fq[q]] * Gs[2 * NF + fq[q]];
          gsy[q] = sgn * Gs[NF + fq[q]] * Gs[2 * NF + fq[q]];
        }
        R Sk, Sw;
        kw_sources<R, HX>(Ks, Os, Ws, Us, Vs, hidx, gsx, gsy, Ac, alpha, kc.beta_star, sigma_do, C_lim, Sk, Sw);
        const R w0 = Os[hidx];
        ak += dt * Sk;
        aw += dt * Sw;
        rate_k = kc.beta_star * w0;
        rate_w = beta0 * w0;
      }
      ak /= R(1) + dt * rate_k;
      aw /= R(1) + dt * rate_w;
      ((R*)A.RKout)[c] = fmax(ak, R(0));
      ((R*)A.RWout)[c] = fmax(aw, wn[0] * omega_floor);
    }
    // CFL rate: sum over the four faces of (|U.n| + c) L, over 2 A
    const R ir = g_rcp(wn[0]);
    const R u = wn[1] * ir, vv = wn[2] * ir;
    const R cs = g_sqrt(g_div(kc.gamma * pressure_of<R>(2, kc.gamma, wn), wn[0]));
    const int fl[4] = {fa, fa + 1, fc, fc + X};
    R r = R(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) r += (g_abs(u * Gs[fl[q]] + vv * Gs[NF + fl[q]]) + cs) * Gs[2 * NF + fl[q]];
    rmax = fmax(rmax, R(0.5) * r * ia);
  }
  const unsigned long long bmax = block_max_rate<R>(rmax, red);
  if (tid == 0) atomicMax(&A.ctrl->rate[(A.slot + 1) % 3], bmax);
  if (__syncthreads_or(bad) && tid == 0) atomicOr(&A.ctrl->status, 1u);
  if (A.resid) {
    for (int v = 0; v < 4; ++v) {
      double s_ = block_sum(racc[v], red);
      if (tid == 0) atomicAdd(&A.ctrl->l2[v], s_);
      s_ = block_sum(racc[8 + v], red);
      if (tid == 0) atomicAdd(&A.ctrl->total[v], s_);
      const double m = block_max<double>(racc[4 + v], red);
      if (tid == 0) atomic_max_nonneg(&A.ctrl->linf[v], m);
    }
  }
}

template <int PREC, int V, int MODE = 0, bool MD = false, int RC = 0, bool TR = false, bool RAR = false>
void launch_fused(const StepArgs& A, const CurvGeom& G, cudaStream_t s, const SteadyArgs& SA = SteadyArgs{}) {
  using TG = CurvTileGeom<V, halo_for(RC)>;
  const int nt = ((A.g.n[0] + TG::X - 1) / TG::X) * ((A.g.n[1] + TG::Y - 1) / TG::Y);
  const size_t smem = TG::template smem_bytes<typename PrecT<PREC>::R, TR>();
  // time steps follow one another: on a grid of one wave of tiles or less a programmatic launch
  // lets a step's prologue (the static face records) overlap the end of the previous step; larger
  // grids (and the steady residual) launch plainly
  static int resident = 0;  // CTAs of this instantiation that fit on the GPU at once
  if (MODE == 0 && resident == 0) {
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, curv_step_kernel<PREC, V, MODE, MD, RC, TR, RAR>, TG::T,
                                                  smem);
    resident = per_sm * nsm > 0 ? per_sm * nsm : -1;
  }
  if (MODE == 1 || nt > resident) {
    curv_step_kernel<PREC, V, MODE, MD, RC, TR, RAR><<<nt, TG::T, smem, s>>>(A, G, SA);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nt);
  cfg.blockDim = dim3((unsigned)TG::T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, curv_step_kernel<PREC, V, MODE, MD, RC, TR, RAR>, A, G, SA);
}

template <int PREC, int V, int MODE, bool MD, int RC = 0, bool TR = false, bool RAR = false>
cudaError_t prepare_one() {
  using TG = CurvTileGeom<V, halo_for(RC)>;
  return cudaFuncSetAttribute(curv_step_kernel<PREC, V, MODE, MD, RC, TR, RAR>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TG::template smem_bytes<typename PrecT<PREC>::R, TR>());
}

template <int PREC, int V, int MODE = 0>
cudaError_t prepare_fused() {
  const cudaError_t a = prepare_one<PREC, V, MODE, false>(), b = prepare_one<PREC, V, MODE, true>();
  return a != cudaSuccess ? a : b;
}

}  // namespace
}  // namespace gks
