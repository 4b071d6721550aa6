// Steady-state solver on body-fitted 2D grids (Section 4: local time stepping, LU-SGS smoothing in
// the form of Yoon and Jameson, multigrid after Jameson; the readings are stated in gks.h).  One
// cycle on the device:
//   per level, down: local explicit steps s (lts_kernel), the residual R of the level's state with
//   face windows cfl_flux min(s_l, s_r) (the fused tile kernel in its residual mode; first order and
//   with the FAS forcing on coarse levels), half spectral radius times length of every face
//   (face_lambda_kernel), one LU-SGS smoothing with pseudo-time steps cfl s (lusgs_kernel: 32 x 32
//   or 16 x 16 cell tiles, one lane per tile column, hyperplane by hyperplane), then the residual
//   after smoothing restricted with the state to the next level (restrict_kernel) and the forcing
//   formed (forcing_kernel);
//   up: the coarse corrections injected (prolong_kernel).
// Every launch of a cycle is captured once in a CUDA graph; the fine residual norm of each cycle
// is appended to a device history by the last node.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "gks.h"
#include "gks_aux.cuh"
#include "gks_curv.h"
#include "gks_step.cuh"

namespace gks {
namespace {

// LU-SGS tile edge TL (16 or 32 cells; one lane per tile column)
constexpr int kST = 128;

inline unsigned nblk(long n, int t = kST) { return (unsigned)((n + t - 1) / t); }

// (single precision divides with the fast reciprocal, double precision exactly)
template <class R>
__device__ __forceinline__ void euler_normal(R gamma, const R* w, R nx, R ny, R* F) {
  const R un = g_div(w[1] * nx + w[2] * ny, w[0]);
  const R p = pressure_of<R>(2, gamma, w);
  F[0] = w[0] * un;
  F[1] = w[1] * un + p * nx;
  F[2] = w[2] * un + p * ny;
  F[3] = (w[3] + p) * un;
}

// Half spectral radius times length of every face: 1/2 L (max over the two cells of |U.n| + c +
// 2 (mu + p tau_t) / (rho d)), rho, p, tau_t face means, d the centroid distance.
template <int PREC>
__global__ void __launch_bounds__(kST) face_lambda_kernel(const __grid_constant__ StepArgs A,
                                                          const __grid_constant__ CurvGeom G, const void* tau_cell,
                                                          void* hli, void* hlj) {
  using R = typename PrecT<PREC>::R;
  const DevGrid& g = A.g;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.nf[0] + G.nf[1]) return;
  const int a = t < G.nf[0] ? 0 : 1;
  const long f = a == 0 ? t : t - G.nf[0];
  const long nf = G.nf[a];
  const int n0 = g.n[0];
  const int nfa = a == 0 ? n0 + 1 : n0;
  const int fi = (int)(f % nfa), fj = (int)(f / nfa);
  const int ia = a == 0 ? fi - 1 : fi, ja = a == 0 ? fj : fj - 1;
  const Consts<R> kc = make_consts<R>(g);
  const R* rec = (const R*)G.face[a];
  const R nx = rec[f], ny = rec[nf + f], L = rec[2 * nf + f], id = rec[4 * nf + f];
  R wa[4], wb[4];
  load_cell<2, PREC>(g, A.Win, kc, ia, ja, 0, wa);
  load_cell<2, PREC>(g, A.Win, kc, fi, fj, 0, wb);
  const R pa = pressure_of<R>(2, kc.gamma, wa), pb = pressure_of<R>(2, kc.gamma, wb);
  const R sa = g_abs((wa[1] * nx + wa[2] * ny) / wa[0]) + sqrt(kc.gamma * pa / wa[0]);
  const R sb = g_abs((wb[1] * nx + wb[2] * ny) / wb[0]) + sqrt(kc.gamma * pb / wb[0]);
  const R rho = R(0.5) * (wa[0] + wb[0]), p = R(0.5) * (pa + pb);
  R tau = R(0);
  if (g.turb_model != TURB_NONE) {
    const R* tc = (const R*)tau_cell;  // per-cell tau_t of this state
    tau = R(0.5) * (tc[field_cell(g, 2, ia, ja, 0)] + tc[field_cell(g, 2, fi, fj, 0)]);
  }
  const R lam = fmax(sa, sb) + R(2) * (kc.mu + p * tau) / (rho / id);
  ((R*)(a == 0 ? hli : hlj))[f] = R(0.5) * L * lam;
}

// dynamic shared memory of lusgs_kernel: dW, state (4 planes each) and the diagonal.  Rows are not
// padded: the lanes of a sweep step touch one anti-diagonal of a plane, (k - l) TL + l, which with a
// row pitch of TL falls into TL different banks (a pitch of TL + 1 would put them all in one).
template <class R, int TL>
constexpr size_t lusgs_smem() {
  return sizeof(R) * 9 * TL * TL;
}

struct LusgsArgs {
  const void* s_loc;  // local explicit steps; pseudo step = cfl s
  double cfl;
  const void* R;      // residual [4][ncell]
  const void* hl[2];  // 1/2 lambda L per face
  void* W;            // state, advanced by the increment
};

// Contribution 1/2 (dF - lambda dX) L of neighbour state w with increment X through normal (nx, ny).
template <class R>
__device__ __forceinline__ void offdiag(R gamma, const R* w, const R* X, R nx, R ny, R hl, R L, R* acc) {
  R wp[4], F0[4], F1[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) wp[v] = w[v] + X[v];
  euler_normal<R>(gamma, wp, nx, ny, F1);
  euler_normal<R>(gamma, w, nx, ny, F0);
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] += R(0.5) * (F1[v] - F0[v]) * L - hl * X[v];
}

// LU-SGS on one TL x TL tile per group of TL lanes: forward and backward sweeps hyperplane by
// hyperplane (lane l takes tile column l), neighbours outside the tile left out; then W += dW on the
// tile.  The tile's
// state and diagonal are staged in shared memory before the sweeps; each lane loads the residual
// and face records of its next cell while it works on the current one, so that the sweeps wait
// on shared memory and arithmetic only.
template <class R>
struct SweepIn {  // what a lane needs from global memory for one cell of a sweep
  R r[4];         // forward: the residual
  R f[2][4];      // the two faces towards the sweep's neighbours: n_x, n_y, L, 1/2 lambda L
};

template <int PREC, int TL>
__global__ void __launch_bounds__(TL) lusgs_kernel(const __grid_constant__ StepArgs A,
                                                   const __grid_constant__ CurvGeom G,
                                                   const __grid_constant__ LusgsArgs LA) {
  constexpr int kLT = TL;
  constexpr unsigned kMask = TL == 32 ? 0xffffffffu : (1u << TL) - 1u;  // the lanes of the block
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  extern __shared__ __align__(16) unsigned char lu_raw[];
  using Plane = R[kLT][kLT];
  Plane* X = (Plane*)lu_raw;  // [4]: dW* in the forward sweep, dW after the backward one
  Plane* Ws = X + 4;          // [4]: the tile's state
  Plane& Dg = Ws[4];
  const DevGrid& g = A.g;
  const int lane = threadIdx.x;
  const int n0 = g.n[0], n1 = g.n[1];
  const int ntx = (n0 + kLT - 1) / kLT;
  const int ox = (blockIdx.x % ntx) * kLT, oy = (blockIdx.x / ntx) * kLT;
  const int ex = min(kLT, n0 - ox), ey = min(kLT, n1 - oy);
  const Consts<R> kc = make_consts<R>(g);
  const R* hli = (const R*)LA.hl[0];
  const R* hlj = (const R*)LA.hl[1];
  const R* fi_rec = (const R*)G.face[0];
  const R* fj_rec = (const R*)G.face[1];
  const long nf0 = G.nf[0], nf1 = G.nf[1];
  const R* Rr = (const R*)LA.R;
  const R* sl = (const R*)LA.s_loc;
  S* Wg = (S*)LA.W;
  // stage the state and the diagonal D = A / (cfl s) + 1/2 sum lambda L
  for (int q = lane; q < ex * ey; q += kLT) {
    const int li = q % ex, lj = q / ex;
    const int i = ox + li, j = oy + lj;
    const long c = (long)j * n0 + i;
#pragma unroll
    for (int v = 0; v < 4; ++v) Ws[v][lj][li] = (R)Wg[(long)v * g.ncell + c];
    const long fa = (long)j * (n0 + 1) + i, fc = (long)j * n0 + i;
    const R dt = sl[c] * (R)LA.cfl;
    Dg[lj][li] = (R)G.area[c] / dt + hli[fa] + hli[fa + 1] + hlj[fc] + hlj[fc + n0];
  }
  __syncwarp(kMask);
  const int nk = ex + ey - 1;
  // loads of the cell of hyperplane k (forward: lower faces and the residual; backward: upper faces)
  auto fetch = [&](int k, bool fwd, SweepIn<R>& in) {
    const int li = lane, lj = k - lane;
    if (!(k >= 0 && k < nk && li < ex && lj >= 0 && lj < ey)) return;
    const int i = ox + li, j = oy + lj;
    const long c = (long)j * n0 + i;
    const long fi = (long)j * (n0 + 1) + i + (fwd ? 0 : 1), fj = (long)(j + (fwd ? 0 : 1)) * n0 + i;
    if (fwd) {
#pragma unroll
      for (int v = 0; v < 4; ++v) in.r[v] = Rr[(long)v * g.ncell + c];
    }
    in.f[0][0] = fi_rec[fi];
    in.f[0][1] = fi_rec[nf0 + fi];
    in.f[0][2] = fi_rec[2 * nf0 + fi];
    in.f[0][3] = hli[fi];
    in.f[1][0] = fj_rec[fj];
    in.f[1][1] = fj_rec[nf1 + fj];
    in.f[1][2] = fj_rec[2 * nf1 + fj];
    in.f[1][3] = hlj[fj];
  };
  auto nbr = [&](int li, int lj, R* w, R* x) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      w[v] = Ws[v][lj][li];
      x[v] = X[v][lj][li];
    }
  };
  // forward sweep
  SweepIn<R> cur, nxt;
  fetch(0, true, cur);
  for (int k = 0; k < nk; ++k) {
    fetch(k + 1, true, nxt);
    const int li = lane, lj = k - lane;
    if (li < ex && lj >= 0 && lj < ey) {
      R acc[4] = {R(0), R(0), R(0), R(0)};
      if (li > 0) {  // face i - 1/2, normal away from the cell: -n
        R w[4], x[4];
        nbr(li - 1, lj, w, x);
        offdiag<R>(kc.gamma, w, x, -cur.f[0][0], -cur.f[0][1], cur.f[0][3], cur.f[0][2], acc);
      }
      if (lj > 0) {
        R w[4], x[4];
        nbr(li, lj - 1, w, x);
        offdiag<R>(kc.gamma, w, x, -cur.f[1][0], -cur.f[1][1], cur.f[1][3], cur.f[1][2], acc);
      }
      const R D = Dg[lj][li];
#pragma unroll
      for (int v = 0; v < 4; ++v) X[v][lj][li] = g_div(-cur.r[v] - acc[v], D);
    }
    cur = nxt;
    __syncwarp(kMask);
  }
  // backward sweep
  fetch(nk - 1, false, cur);
  for (int k = nk - 1; k >= 0; --k) {
    fetch(k - 1, false, nxt);
    const int li = lane, lj = k - lane;
    if (li < ex && lj >= 0 && lj < ey) {
      R acc[4] = {R(0), R(0), R(0), R(0)};
      if (li + 1 < ex) {
        R w[4], x[4];
        nbr(li + 1, lj, w, x);
        offdiag<R>(kc.gamma, w, x, cur.f[0][0], cur.f[0][1], cur.f[0][3], cur.f[0][2], acc);
      }
      if (lj + 1 < ey) {
        R w[4], x[4];
        nbr(li, lj + 1, w, x);
        offdiag<R>(kc.gamma, w, x, cur.f[1][0], cur.f[1][1], cur.f[1][3], cur.f[1][2], acc);
      }
      const R D = Dg[lj][li];
#pragma unroll
      for (int v = 0; v < 4; ++v) X[v][lj][li] = X[v][lj][li] - g_div(acc[v], D);
    }
    cur = nxt;
    __syncwarp(kMask);
  }
  // W += dW
  for (int q = lane; q < ex * ey; q += kLT) {
    const int li = q % ex, lj = q / ex;
    const long c = (long)(oy + lj) * n0 + ox + li;
#pragma unroll
    for (int v = 0; v < 4; ++v) Wg[(long)v * g.ncell + c] = (S)(Ws[v][lj][li] + X[v][lj][li]);
  }
}

// Restriction to the next level: the state by area weights, the residual by sums.
template <class S, class R>
__global__ void restrict_kernel(int m0, int m1, int k0, long kc_, const S* Wf, const R* Rf, const double* af, S* Wc0,
                                R* Rs) {
  const long cc = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long mc = (long)m0 * m1;
  if (cc >= mc) return;
  const int I = (int)(cc % m0), J = (int)(cc / m0);
  double asum = 0.0, w[4] = {0, 0, 0, 0};
  R r[4] = {R(0), R(0), R(0), R(0)};
  for (int q = 0; q < 4; ++q) {
    const long cf = (long)(2 * J + q / 2) * k0 + 2 * I + q % 2;
    asum += af[cf];
    for (int v = 0; v < 4; ++v) {
      w[v] += af[cf] * (double)Wf[(long)v * kc_ + cf];
      r[v] += Rf[(long)v * kc_ + cf];
    }
  }
  for (int v = 0; v < 4; ++v) {
    Wc0[(long)v * mc + cc] = (S)(w[v] / asum);
    Rs[(long)v * mc + cc] = r[v];
  }
}

// FAS forcing P = (restricted residual) - R_c(W_c^0), in place over the restricted residual; the
// level's state starts from W_c^0.
template <class S, class R>
__global__ void forcing_kernel(long n, R* P, const R* Rc, const S* W0, S* W) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  P[q] = P[q] - Rc[q];
  W[q] = W0[q];
}

// W_f += W_c - W_c^0 on the four children of every coarse cell.
template <class S>
__global__ void prolong_kernel(int m0, int m1, int k0, long kc_, S* Wf, const S* Wc, const S* Wc0) {
  const long cc = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long mc = (long)m0 * m1;
  if (cc >= mc) return;
  const int I = (int)(cc % m0), J = (int)(cc / m0);
  for (int v = 0; v < 4; ++v) {
    const S d = Wc[(long)v * mc + cc] - Wc0[(long)v * mc + cc];
    for (int q = 0; q < 4; ++q) {
      const long cf = (long)(2 * J + q / 2) * k0 + 2 * I + q % 2;
      Wf[(long)v * kc_ + cf] += d;
    }
  }
}

__global__ void subsample_nodes_kernel(int m0, int m1, int k0, const double* nf, double* nc) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long)(m0 + 1) * (m1 + 1)) return;
  const int I = (int)(q % (m0 + 1)), J = (int)(q / (m0 + 1));
  for (int d = 0; d < 2; ++d) nc[q * 2 + d] = nf[((long)(2 * J) * (k0 + 1) + 2 * I) * 2 + d];
}

template <class R>
__global__ void mean4_kernel(int m0, int m1, int k0, const R* f, R* out) {
  const long cc = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cc >= (long)m0 * m1) return;
  const int I = (int)(cc % m0), J = (int)(cc / m0);
  out[cc] = R(0.25) * (f[(long)(2 * J) * k0 + 2 * I] + f[(long)(2 * J) * k0 + 2 * I + 1] +
                       f[(long)(2 * J + 1) * k0 + 2 * I] + f[(long)(2 * J + 1) * k0 + 2 * I + 1]);
}

// history[counter] = sqrt(acc / ncell); acc cleared, counter advanced (the last node of a cycle).
__global__ void store_res_kernel(double* acc, double* history, int* counter, long ncell) {
  history[*counter] = sqrt(*acc / (double)ncell);
  *counter += 1;
  *acc = 0.0;
}

template <class S>
__global__ void physical_kernel(const S* W, long n, double gamma, unsigned* bad) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double w[4];
  for (int v = 0; v < 4; ++v) w[v] = (double)W[(long)v * n + c];
  const double p = (gamma - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
  if (!(w[0] > 0.0) || !(p > 0.0)) atomicOr(bad, 1u);
}

}  // namespace
}  // namespace gks

using namespace gks;

struct SteadyLevel {
  int n0 = 0, n1 = 0;
  long ncell = 0;
  DevGrid g{};
  CurvGeom G{};
  double* nodes = nullptr;
  double* dir[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  void *W = nullptr, *W0 = nullptr, *R = nullptr, *P = nullptr, *s = nullptr, *hl[2] = {nullptr, nullptr};
  void *f1 = nullptr, *f2 = nullptr;
};

struct gks_steady {
  int dev = 0;
  int prec = PREC_F64;
  int levels = 1;
  int tile = 16;  // LU-SGS tile edge
  int multid = 0;  // multi-dimensional expansion on the finest level
  int recon = 0;   // GKS_RECON_* on the finest level (coarse levels are first order)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<SteadyLevel> L;
  double* acc = nullptr;   // fine residual accumulator of the running cycle
  int* counter = nullptr;  // cycles stored in history
  unsigned* bad = nullptr;
  double* history = nullptr;
  int history_len = 0;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  bool has_state = false, has_turb = false;
  bool transport = false;            // GKS_TURB_KOMEGA_TRANSPORT: rho k, rho omega evolved each cycle
  void *RK = nullptr, *RW = nullptr;  // finest grid, arithmetic type
  void* mflux[2] = {nullptr, nullptr};  // fine residual's face mass flux rates times L, per axis
  gks_komega kw{};
  std::map<std::pair<double, double>, cudaGraphExec_t> graphs;  // one captured cycle per (cfl, cfl_flux)
  std::string err;
};

namespace {

gks_status sfail(gks_steady* s, gks_status st, const std::string& m) {
  if (s) s->err = m;
  return st;
}

#define GKS_SCK(s, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      cudaGetLastError();                                                                         \
      return sfail((s), GKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
    }                                                                                             \
  } while (0)

size_t rbytes(int prec) { return prec == PREC_F64 ? 8 : 4; }

void free_level(SteadyLevel& l) {
  void* ps[] = {l.nodes, l.W, l.W0, l.R, l.P, l.s, l.hl[0], l.hl[1], l.f1, l.f2, l.G.face[0], l.G.face[1],
                l.G.iarea, l.G.area, l.G.tau, l.G.flux[0], l.G.flux[1], l.G.tang[0], l.G.tang[1], l.dir[0][0],
                l.dir[0][1], l.dir[1][0],
                l.dir[1][1]};
  for (void* p : ps)
    if (p) cudaFree(p);
  l = SteadyLevel{};
}

void drop_graphs(gks_steady* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

void free_steady(gks_steady* s) {
  drop_graphs(s);
  for (auto& l : s->L) free_level(l);
  s->L.clear();
  void* ps[] = {s->acc, s->counter, s->bad, s->history, s->staging, s->RK, s->RW, s->mflux[0], s->mflux[1]};
  for (void* p : ps)
    if (p) cudaFree(p);
  s->RK = s->RW = s->mflux[0] = s->mflux[1] = nullptr;
  s->acc = nullptr;
  s->counter = nullptr;
  s->bad = nullptr;
  s->history = nullptr;
  s->staging = nullptr;
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

StepArgs level_args(const gks_steady* s, int l, const void* Win) {
  StepArgs A;
  std::memset(&A, 0, sizeof(A));
  A.g = s->L[l].g;
  A.Win = Win;
  A.f1 = s->L[l].f1;
  A.f2 = s->L[l].f2;
  return A;
}

// Residual of level l's state Win into lev.R (forcing on coarse levels), with the local steps.
void residual(gks_steady* s, int l, const void* Win, const void* forcing, double cfl_flux, double* acc,
              bool mass_flux = false) {
  SteadyLevel& lev = s->L[l];
  StepArgs A = level_args(s, l, Win);
  if (mass_flux)
    for (int a = 0; a < 2; ++a) A.mflux[a] = s->mflux[a];
  launch_curv_lts(s->prec, A, lev.G, lev.s, s->stream);
  SteadyArgs SA{};
  SA.s_loc = lev.s;
  SA.cfl_flux = cfl_flux;
  SA.first_order = l > 0;
  SA.R = lev.R;
  SA.forcing = forcing;
  SA.tau = lev.G.tau;
  SA.res_acc = acc;
  SA.multid = s->multid;
  SA.recon = l == 0 ? s->recon : GKS_RECON_MUSCL2;
  if (SA.recon != GKS_RECON_MUSCL2)
    launch_curv_residual_recon(s->prec, A, lev.G, SA, s->stream);
  else if (A.g.rar)
    launch_curv_residual_rar(s->prec, A, lev.G, SA, s->stream);
  else
    launch_curv_residual(s->prec, A, lev.G, SA, s->stream);
}

// Four-cell means of the turbulence fields down the levels (f1 only for a mu_t field).
void restrict_fields(gks_steady* s) {
  const int nq = s->L[0].g.turb_model == GKS_TURB_MUT ? 1 : 2;
  for (int l = 1; l < s->levels; ++l) {
    SteadyLevel& c = s->L[l];
    SteadyLevel& p = s->L[l - 1];
    for (int q = 0; q < nq; ++q) {
      const void* src = q == 0 ? p.f1 : p.f2;
      void* dst = q == 0 ? c.f1 : c.f2;
      if (s->prec == PREC_F64)
        mean4_kernel<double><<<nblk(c.ncell), kST, 0, s->stream>>>(c.n0, c.n1, p.n0, (const double*)src, (double*)dst);
      else
        mean4_kernel<float><<<nblk(c.ncell), kST, 0, s->stream>>>(c.n0, c.n1, p.n0, (const float*)src, (float*)dst);
    }
  }
}

// Arguments of the steady k-omega update on the finest grid.
KOmegaArgs kw_args(const gks_steady* s) {
  KOmegaArgs K;
  std::memset(&K, 0, sizeof(K));
  const SteadyLevel& f = s->L[0];
  K.g = f.g;
  K.Win = f.W;
  K.Wnew = f.W;
  K.RKin = s->RK;
  K.RWin = s->RW;
  K.RKout = s->RK;
  K.RWout = s->RW;
  K.mflux[0] = s->mflux[0];
  K.mflux[1] = s->mflux[1];
  K.alpha = s->kw.alpha;
  K.beta0 = s->kw.beta0;
  K.beta_star = f.g.beta_star;
  K.sigma = s->kw.sigma;
  K.sigma_star = s->kw.sigma_star;
  K.sigma_do = s->kw.sigma_do;
  K.C_lim = s->kw.C_lim;
  K.omega_floor = s->kw.omega_floor;
  K.sources = s->kw.sources;
  K.diffusion = s->kw.diffusion;
  K.falpha = (float)K.alpha;
  K.fbeta0 = (float)K.beta0;
  K.fbeta_star = (float)K.beta_star;
  K.fsigma = (float)K.sigma;
  K.fsigma_star = (float)K.sigma_star;
  K.fsigma_do = (float)K.sigma_do;
  K.fC_lim = (float)K.C_lim;
  K.fomega_floor = (float)K.omega_floor;
  return K;
}

template <int PREC>
void cycle_prec(gks_steady* s, double cfl, double cfl_flux) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  const int nl = s->levels;
  if (s->transport) {  // k = rho k / rho, omega = rho omega / rho of the cycle's start, on every level
    SteadyLevel& f = s->L[0];
    aux::density_unscale_kernel<R, S, R><<<nblk(f.ncell), kST, 0, s->stream>>>((const R*)s->RK, (const S*)f.W,
                                                                               (R*)f.f1, f.ncell);
    aux::density_unscale_kernel<R, S, R><<<nblk(f.ncell), kST, 0, s->stream>>>((const R*)s->RW, (const S*)f.W,
                                                                               (R*)f.f2, f.ncell);
    restrict_fields(s);
  }
  for (int l = 0; l < nl; ++l) {
    SteadyLevel& lev = s->L[l];
    const void* forcing = l > 0 ? lev.P : nullptr;
    residual(s, l, lev.W, forcing, cfl_flux, l == 0 ? s->acc : nullptr, l == 0 && s->transport);
    if (l == 0 && s->transport) {  // the k-omega update from the same state, fields and residual
      const KOmegaArgs K = kw_args(s);
      launch_steady_komega(s->prec, K, lev.G, lev.f1, lev.f2, s->RK, s->RW, lev.s, cfl, s->stream);
    }
    const StepArgs A = level_args(s, l, lev.W);
    face_lambda_kernel<PREC><<<nblk(lev.G.nf[0] + lev.G.nf[1]), kST, 0, s->stream>>>(A, lev.G, lev.G.tau, lev.hl[0],
                                                                                      lev.hl[1]);
    LusgsArgs LA;
    LA.s_loc = lev.s;
    LA.cfl = cfl;
    LA.R = lev.R;
    LA.hl[0] = lev.hl[0];
    LA.hl[1] = lev.hl[1];
    LA.W = lev.W;
    const int TLs = s->tile;
    const int tiles = ((lev.n0 + TLs - 1) / TLs) * ((lev.n1 + TLs - 1) / TLs);
    if (TLs == 16)
      lusgs_kernel<PREC, 16><<<tiles, 16, lusgs_smem<R, 16>(), s->stream>>>(A, lev.G, LA);
    else
      lusgs_kernel<PREC, 32><<<tiles, 32, lusgs_smem<R, 32>(), s->stream>>>(A, lev.G, LA);
    if (l + 1 == nl) break;
    // residual after smoothing, restricted with the state; coarse residual of W_c^0; forcing
    residual(s, l, lev.W, forcing, cfl_flux, nullptr);
    SteadyLevel& c = s->L[l + 1];
    restrict_kernel<S, R><<<nblk(c.ncell), kST, 0, s->stream>>>(c.n0, c.n1, lev.n0, lev.ncell, (const S*)lev.W,
                                                                 (const R*)lev.R, lev.G.area, (S*)c.W0, (R*)c.P);
    residual(s, l + 1, c.W0, nullptr, cfl_flux, nullptr);
    forcing_kernel<S, R><<<nblk(4 * c.ncell), kST, 0, s->stream>>>(4 * c.ncell, (R*)c.P, (const R*)c.R,
                                                                    (const S*)c.W0, (S*)c.W);
  }
  for (int l = nl - 1; l >= 1; --l) {
    SteadyLevel& c = s->L[l];
    SteadyLevel& f = s->L[l - 1];
    prolong_kernel<S><<<nblk(c.ncell), kST, 0, s->stream>>>(c.n0, c.n1, f.n0, f.ncell, (S*)f.W, (const S*)c.W,
                                                           (const S*)c.W0);
  }
  store_res_kernel<<<1, 1, 0, s->stream>>>(s->acc, s->history, s->counter, s->L[0].ncell);
}

void launch_cycle(gks_steady* s, double cfl, double cfl_flux) {
  if (s->prec == PREC_F64)
    cycle_prec<PREC_F64>(s, cfl, cfl_flux);
  else
    cycle_prec<PREC_F32>(s, cfl, cfl_flux);
}

gks_status ensure_history(gks_steady* s, int n) {
  if (s->history_len >= n) return GKS_OK;
  if (s->history) cudaFree(s->history);
  s->history = nullptr;
  s->history_len = 0;
  if (cudaMalloc(&s->history, sizeof(double) * n) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, GKS_ENOMEM, "history allocation failed");
  }
  s->history_len = n;
  drop_graphs(s);  // the captured cycles name the history buffer: capture again
  return GKS_OK;
}

gks_status ensure_stage(gks_steady* s, size_t bytes) {
  if (s->staging_bytes >= bytes) return GKS_OK;
  if (s->staging) cudaFree(s->staging);
  s->staging = nullptr;
  s->staging_bytes = 0;
  if (cudaMalloc(&s->staging, bytes) != cudaSuccess) {
    cudaGetLastError();
    return sfail(s, GKS_ENOMEM, "staging allocation failed");
  }
  s->staging_bytes = bytes;
  return GKS_OK;
}

}  // namespace

extern "C" {

gks_status gks_steady_create(const gks_grid* grid, const gks_gas* gas, const gks_turb* turb,
                             const gks_numerics* num, const double* nodes, int levels, int lusgs_tile,
                             void* cuda_stream, gks_steady** out) {
  if (!out) return GKS_EINVAL;
  *out = nullptr;
  if (!grid || !gas || !num || !nodes) return GKS_EINVAL;
  if (grid->dim != 2) return GKS_EUNSUPPORTED;
  if (num->reconstruction < GKS_RECON_MUSCL2 || num->reconstruction > GKS_RECON_WENO5) return GKS_EINVAL;
  if (num->precision != GKS_FP64 && num->precision != GKS_FP32) return GKS_EUNSUPPORTED;
  const int model_in = turb ? turb->model : GKS_TURB_NONE;
  if (model_in < GKS_TURB_NONE || model_in > GKS_TURB_KOMEGA_TRANSPORT) return GKS_EUNSUPPORTED;
  const int rar = turb ? turb->rarefaction : GKS_RAR_DT;
  if (rar != GKS_RAR_DT && rar != GKS_RAR_TAUHAT) return GKS_EINVAL;
  if (rar == GKS_RAR_TAUHAT && num->reconstruction != GKS_RECON_MUSCL2) return GKS_EUNSUPPORTED;
  // with transport the levels take tau_t from the fields k, omega of each cycle's start
  const int model = model_in == GKS_TURB_KOMEGA_TRANSPORT ? (int)GKS_TURB_KOMEGA : model_in;
  if (levels < 1 || levels > 6) return GKS_EINVAL;
  if (lusgs_tile != 0 && lusgs_tile != 16 && lusgs_tile != 32) return GKS_EINVAL;
  const int n0 = grid->n[0], n1 = grid->n[1];
  if (n0 < 2 || n1 < 2) return GKS_EINVAL;
  for (int l = 1; l < levels; ++l)
    if ((n0 >> l) < 2 || (n1 >> l) < 2 || n0 % (1 << l) || n1 % (1 << l) || grid->wake_cut % (1 << l))
      return GKS_EINVAL;
  if (grid->wake_cut < 0 || 2 * grid->wake_cut > n0) return GKS_EINVAL;
  for (int d = 0; d < 2; ++d)
    for (int sd = 0; sd < 2; ++sd) {
      const int b = grid->bc[d][sd];
      if (b < GKS_BC_PERIODIC || b > GKS_BC_OUTFLOW) return GKS_EINVAL;
      if (b == GKS_BC_DIRICHLET && !grid->bc_data[d][sd]) return GKS_EINVAL;
    }
  if (!(gas->gamma > 1.0) || !(gas->mu >= 0.0)) return GKS_EINVAL;
  gks_steady* s = new (std::nothrow) gks_steady;
  if (!s) return GKS_ENOMEM;
  cudaGetDevice(&s->dev);
  s->prec = num->precision == GKS_FP64 ? PREC_F64 : PREC_F32;
  s->levels = levels;
  s->tile = lusgs_tile == 32 ? 32 : 16;
  s->multid = num->expand == GKS_EXPAND_MULTID;
  s->recon = num->reconstruction;
  s->transport = model_in == GKS_TURB_KOMEGA_TRANSPORT;
  gks_komega_defaults(&s->kw);
  auto bad = [&](gks_status st) {
    free_steady(s);
    delete s;
    return st;
  };
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return bad(GKS_ECUDA);
    }
    s->own_stream = true;
  }
  if (prepare_curv() != cudaSuccess || prepare_curv_recon() != cudaSuccess || prepare_curv_rar() != cudaSuccess ||
      cudaFuncSetAttribute(lusgs_kernel<PREC_F64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)lusgs_smem<double, 32>()) != cudaSuccess ||
      cudaFuncSetAttribute(lusgs_kernel<PREC_F32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)lusgs_smem<float, 32>()) != cudaSuccess) {
    cudaGetLastError();
    return bad(GKS_ECUDA);
  }
  const double K = 2.0 / (gas->gamma - 1.0) - 2.0;
  if (K < 0.0) return bad(GKS_EINVAL);
  const size_t rb = rbytes(s->prec);
  bool ok = true;
  auto alloc = [&](void** p, size_t b) {
    if (ok && cudaMalloc(p, b) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      ok = false;
    }
  };
  s->L.resize(levels);
  // Dirichlet primitives per level (host), the finest as given, coarser ones as pair means
  std::vector<std::vector<double>> dprim[2][2];
  for (int d = 0; d < 2; ++d)
    for (int sd = 0; sd < 2; ++sd) {
      dprim[d][sd].resize(levels);
      if (grid->bc[d][sd] != GKS_BC_DIRICHLET) continue;
      const int m = d == 0 ? n1 : n0;
      dprim[d][sd][0].assign(grid->bc_data[d][sd], grid->bc_data[d][sd] + (size_t)m * 4);
      for (int l = 1; l < levels; ++l) {
        const int mc = m >> l;
        dprim[d][sd][l].resize((size_t)mc * 4);
        for (int k = 0; k < mc; ++k)
          for (int v = 0; v < 4; ++v)
            dprim[d][sd][l][k * 4 + v] = 0.5 * (dprim[d][sd][l - 1][(2 * k) * 4 + v] + dprim[d][sd][l - 1][(2 * k + 1) * 4 + v]);
      }
    }
  for (int l = 0; l < levels; ++l) {
    SteadyLevel& lev = s->L[l];
    lev.n0 = n0 >> l;
    lev.n1 = n1 >> l;
    lev.ncell = (long)lev.n0 * lev.n1;
    CurvGeom& G = lev.G;
    G.nf[0] = (long)(lev.n0 + 1) * lev.n1;
    G.nf[1] = (long)lev.n0 * (lev.n1 + 1);
    alloc((void**)&lev.nodes, sizeof(double) * 2 * (size_t)(lev.n0 + 1) * (lev.n1 + 1));
    for (int a = 0; a < 2; ++a) {
      alloc(&G.face[a], rb * 8 * G.nf[a]);
      alloc(&G.tang[a], rb * 4 * G.nf[a]);
      alloc(&lev.hl[a], rb * G.nf[a]);
    }
    alloc(&G.iarea, rb * lev.ncell);
    alloc((void**)&G.area, sizeof(double) * lev.ncell);
    alloc(&G.tau, rb * lev.ncell);
    alloc(&lev.W, rb * 4 * lev.ncell);
    alloc(&lev.W0, rb * 4 * lev.ncell);
    alloc(&lev.R, rb * 4 * lev.ncell);
    alloc(&lev.P, rb * 4 * lev.ncell);
    alloc(&lev.s, rb * lev.ncell);
    if (model != GKS_TURB_NONE) {
      alloc(&lev.f1, rb * lev.ncell);
      alloc(&lev.f2, rb * lev.ncell);
    }
    DevGrid& g = lev.g;
    std::memset(&g, 0, sizeof(g));
    g.n[0] = lev.n0;
    g.n[1] = lev.n1;
    g.n[2] = 1;
    g.ncell = lev.ncell;
    for (int d = 0; d < 3; ++d)
      for (int sd = 0; sd < 2; ++sd) g.bc[d][sd] = d < 2 ? grid->bc[d][sd] : GKS_BC_PERIODIC;
    for (int d = 0; d < 2; ++d)
      for (int sd = 0; sd < 2; ++sd) {
        if (grid->bc[d][sd] != GKS_BC_DIRICHLET) continue;
        const std::vector<double>& pr = dprim[d][sd][l];
        const size_t m = pr.size() / 4;
        std::vector<double> cons(m * 4);
        for (size_t k = 0; k < m; ++k) {
          const double* q = &pr[k * 4];
          if (!(q[0] > 0.0) || !(q[3] > 0.0)) return bad(GKS_EINVAL);
          cons[k * 4] = q[0];
          cons[k * 4 + 1] = q[0] * q[1];
          cons[k * 4 + 2] = q[0] * q[2];
          cons[k * 4 + 3] = q[3] / (gas->gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2]);
        }
        alloc((void**)&lev.dir[d][sd], sizeof(double) * cons.size());
        if (ok) cudaMemcpy(lev.dir[d][sd], cons.data(), sizeof(double) * cons.size(), cudaMemcpyHostToDevice);
        g.dir[d][sd] = lev.dir[d][sd];
      }
    g.gamma = gas->gamma;
    g.bK = 2.0 / (gas->gamma - 1.0);
    g.K = K;
    g.mu = gas->mu;
    g.T_wall = gas->T_wall;
    g.C_a = turb ? turb->C_a : 0.0;
    g.rar = rar == GKS_RAR_TAUHAT;
    g.C_mu = turb ? turb->C_mu : 0.09;
    g.beta_star = turb ? turb->beta_star : 0.09;
    g.turb_model = model;
    g.limiter = num->limiter;
    g.abar_t0 = num->abar_mode == GKS_ABAR_T0;
    g.wake_cut = grid->wake_cut >> l;
    set_consts(g);
  }
  if (s->transport) {
    alloc(&s->RK, rb * s->L[0].ncell);
    alloc(&s->RW, rb * s->L[0].ncell);
    for (int a = 0; a < 2; ++a) alloc(&s->mflux[a], rb * s->L[0].G.nf[a]);
  }
  alloc((void**)&s->acc, sizeof(double));
  alloc((void**)&s->counter, sizeof(int));
  alloc((void**)&s->bad, sizeof(unsigned));
  if (!ok) return bad(GKS_ENOMEM);
  // nodes of every level and their metrics
  cudaMemcpy(s->L[0].nodes, nodes, sizeof(double) * 2 * (size_t)(n0 + 1) * (n1 + 1), cudaMemcpyHostToDevice);
  for (int l = 1; l < levels; ++l)
    subsample_nodes_kernel<<<nblk((long)(s->L[l].n0 + 1) * (s->L[l].n1 + 1)), kST, 0, s->stream>>>(
        s->L[l].n0, s->L[l].n1, s->L[l - 1].n0, s->L[l - 1].nodes, s->L[l].nodes);
  cudaMemsetAsync(s->bad, 0, sizeof(unsigned), s->stream);
  for (int l = 0; l < levels; ++l) {
    const bool periodic[2] = {grid->bc[0][0] == GKS_BC_PERIODIC, grid->bc[1][0] == GKS_BC_PERIODIC};
    if (curv_metrics(s->L[l].nodes, s->L[l].n0, s->L[l].n1, periodic, s->L[l].g.wake_cut, s->prec, s->L[l].G,
                     (int*)s->bad, s->stream) != cudaSuccess) {
      cudaGetLastError();
      return bad(GKS_ECUDA);
    }
  }
  unsigned badh = 0;
  if (cudaMemcpyAsync(&badh, s->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess) {
    cudaGetLastError();
    return bad(GKS_ECUDA);
  }
  if (badh) return bad(GKS_EINVAL);
  *out = s;
  return GKS_OK;
}

const char* gks_steady_last_error(const gks_steady* s) { return s ? s->err.c_str() : "null handle"; }

gks_status gks_steady_destroy(gks_steady* s) {
  if (!s) return GKS_EINVAL;
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_steady(s);
  delete s;
  return GKS_OK;
}

gks_status gks_steady_set_state(gks_steady* s, const void* W, int layout, int memspace, int dtype) {
  if (!s || !W) return sfail(s, GKS_EINVAL, "null argument");
  if (layout < GKS_LAYOUT_SOA_CONS || layout > GKS_LAYOUT_SOA_PRIM || (dtype != GKS_F64 && dtype != GKS_F32) ||
      (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return sfail(s, GKS_EINVAL, "layout, memspace or dtype");
  SteadyLevel& f = s->L[0];
  const size_t bytes = (dtype == GKS_F64 ? 8 : 4) * 4 * (size_t)f.ncell;
  const void* src = W;
  if (memspace == GKS_MEM_HOST) {
    gks_status st = ensure_stage(s, bytes);
    if (st) return st;
    GKS_SCK(s, cudaMemcpyAsync(s->staging, W, bytes, cudaMemcpyHostToDevice, s->stream));
    src = s->staging;
  }
  // the stored state of a steady handle is one word per value (no low word)
  const int prec = s->prec == PREC_F64 ? PREC_F64 : PREC_F32;
  float* lo_scratch = (float*)s->L[0].W0;  // written and ignored in single precision
  if (dtype == GKS_F64)
    aux::state_in_kernel<double><<<nblk(f.ncell, 256), 256, 0, s->stream>>>((const double*)src, layout, 2, f.ncell,
                                                                           f.g.gamma, prec, f.W, lo_scratch);
  else
    aux::state_in_kernel<float><<<nblk(f.ncell, 256), 256, 0, s->stream>>>((const float*)src, layout, 2, f.ncell,
                                                                          f.g.gamma, prec, f.W, lo_scratch);
  GKS_SCK(s, cudaGetLastError());
  s->has_state = true;
  if (s->transport) s->has_turb = false;  // rho k, rho omega belong to the previous state
  return GKS_OK;
}

gks_status gks_steady_set_turbulence(gks_steady* s, const void* f1, const void* f2, int memspace, int dtype) {
  if (!s || !f1) return sfail(s, GKS_EINVAL, "null argument");
  if (s->L[0].g.turb_model == GKS_TURB_NONE) return sfail(s, GKS_EINVAL, "no turbulence model");
  if (s->L[0].g.turb_model != GKS_TURB_MUT && !f2) return sfail(s, GKS_EINVAL, "second field missing");
  if ((dtype != GKS_F64 && dtype != GKS_F32) || (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return sfail(s, GKS_EINVAL, "memspace or dtype");
  if (s->transport && !s->has_state) return sfail(s, GKS_EINVAL, "k-omega transport: set the state first");
  SteadyLevel& f = s->L[0];
  const size_t eb = dtype == GKS_F64 ? 8 : 4, bytes = eb * (size_t)f.ncell;
  const void* srcs[2] = {f1, f2};
  void* dsts[2] = {f.f1, f.f2};
  gks_status st = ensure_stage(s, 2 * bytes);
  if (st) return st;
  for (int q = 0; q < 2; ++q) {
    if (!srcs[q]) continue;
    const void* src = srcs[q];
    if (memspace == GKS_MEM_HOST) {
      GKS_SCK(s, cudaMemcpyAsync((char*)s->staging + q * bytes, srcs[q], bytes, cudaMemcpyHostToDevice, s->stream));
      src = (char*)s->staging + q * bytes;
    }
    const unsigned blocks = nblk(f.ncell, 256);
    if (s->prec == PREC_F64 && dtype == GKS_F64)
      aux::field_kernel<double, double><<<blocks, 256, 0, s->stream>>>((const double*)src, (double*)dsts[q], f.ncell);
    else if (s->prec == PREC_F64)
      aux::field_kernel<float, double><<<blocks, 256, 0, s->stream>>>((const float*)src, (double*)dsts[q], f.ncell);
    else if (dtype == GKS_F64)
      aux::field_kernel<double, float><<<blocks, 256, 0, s->stream>>>((const double*)src, (float*)dsts[q], f.ncell);
    else
      aux::field_kernel<float, float><<<blocks, 256, 0, s->stream>>>((const float*)src, (float*)dsts[q], f.ncell);
  }
  if (s->transport) {  // rho k = k rho, rho omega = omega rho with the density of the current state
    const unsigned blocks = nblk(f.ncell, 256);
    for (int q = 0; q < 2; ++q) {
      void* dst = q == 0 ? s->RK : s->RW;
      const void* src = q == 0 ? f.f1 : f.f2;
      if (s->prec == PREC_F64) {
        aux::copy_kernel<double><<<blocks, 256, 0, s->stream>>>((const double*)src, (double*)dst, f.ncell);
        aux::density_scale_kernel<double, double><<<blocks, 256, 0, s->stream>>>((double*)dst, (const double*)f.W,
                                                                                 f.ncell);
      } else {
        aux::copy_kernel<float><<<blocks, 256, 0, s->stream>>>((const float*)src, (float*)dst, f.ncell);
        aux::density_scale_kernel<float, float><<<blocks, 256, 0, s->stream>>>((float*)dst, (const float*)f.W,
                                                                               f.ncell);
      }
    }
  }
  restrict_fields(s);
  GKS_SCK(s, cudaGetLastError());
  GKS_SCK(s, cudaStreamSynchronize(s->stream));
  s->has_turb = true;
  return GKS_OK;
}

gks_status gks_steady_set_komega(gks_steady* s, const gks_komega* c) {
  if (!s || !c) return sfail(s, GKS_EINVAL, "null argument");
  if (!s->transport) return sfail(s, GKS_EINVAL, "handle created without k-omega transport");
  s->kw = *c;
  drop_graphs(s);  // captured cycles hold the old coefficients
  return GKS_OK;
}

gks_status gks_steady_get_turbulence(gks_steady* s, void* k_out, void* omega_out, int memspace, int dtype) {
  if (!s || (!k_out && !omega_out)) return sfail(s, GKS_EINVAL, "null argument");
  if (!s->transport) return sfail(s, GKS_EINVAL, "handle created without k-omega transport");
  if (!s->has_turb) return sfail(s, GKS_EINVAL, "turbulence fields not set");
  if ((dtype != GKS_F64 && dtype != GKS_F32) || (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return sfail(s, GKS_EINVAL, "memspace or dtype");
  SteadyLevel& f = s->L[0];
  const size_t eb = dtype == GKS_F64 ? 8 : 4, bytes = eb * (size_t)f.ncell;
  gks_status st = ensure_stage(s, bytes);
  if (st) return st;
  void* outs[2] = {k_out, omega_out};
  for (int q = 0; q < 2; ++q) {
    if (!outs[q]) continue;
    void* dst = memspace == GKS_MEM_HOST ? s->staging : outs[q];
    const void* src = q == 0 ? s->RK : s->RW;
    const unsigned blocks = nblk(f.ncell, 256);
    if (s->prec == PREC_F64 && dtype == GKS_F64)
      aux::density_unscale_kernel<double, double, double><<<blocks, 256, 0, s->stream>>>(
          (const double*)src, (const double*)f.W, (double*)dst, f.ncell);
    else if (s->prec == PREC_F64)
      aux::density_unscale_kernel<double, double, float><<<blocks, 256, 0, s->stream>>>(
          (const double*)src, (const double*)f.W, (float*)dst, f.ncell);
    else if (dtype == GKS_F64)
      aux::density_unscale_kernel<float, float, double><<<blocks, 256, 0, s->stream>>>(
          (const float*)src, (const float*)f.W, (double*)dst, f.ncell);
    else
      aux::density_unscale_kernel<float, float, float><<<blocks, 256, 0, s->stream>>>(
          (const float*)src, (const float*)f.W, (float*)dst, f.ncell);
    GKS_SCK(s, cudaGetLastError());
    if (memspace == GKS_MEM_HOST) {
      GKS_SCK(s, cudaMemcpyAsync(outs[q], s->staging, bytes, cudaMemcpyDeviceToHost, s->stream));
      GKS_SCK(s, cudaStreamSynchronize(s->stream));
    }
  }
  GKS_SCK(s, cudaStreamSynchronize(s->stream));
  return GKS_OK;
}

gks_status gks_steady_cycles(gks_steady* s, int ncycles, double cfl, double cfl_flux, double* res_out) {
  if (!s || ncycles < 0 || !(cfl > 0.0) || !(cfl_flux > 0.0)) return sfail(s, GKS_EINVAL, "bad argument");
  if (!s->has_state) return sfail(s, GKS_EINVAL, "no state set");
  if (s->L[0].g.turb_model != GKS_TURB_NONE && !s->has_turb) return sfail(s, GKS_EINVAL, "turbulence fields not set");
  if (ncycles == 0) return GKS_OK;
  gks_status st = ensure_history(s, ncycles);
  if (st) return st;
  GKS_SCK(s, cudaMemsetAsync(s->acc, 0, sizeof(double), s->stream));
  GKS_SCK(s, cudaMemsetAsync(s->counter, 0, sizeof(int), s->stream));
  auto key = std::make_pair(cfl, cfl_flux);
  auto it = s->graphs.find(key);
  if (it == s->graphs.end()) {
    cudaGraph_t graph;
    GKS_SCK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    launch_cycle(s, cfl, cfl_flux);
    cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return sfail(s, GKS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return sfail(s, GKS_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
    }
    it = s->graphs.emplace(key, exec).first;
  }
  for (int k = 0; k < ncycles; ++k) GKS_SCK(s, cudaGraphLaunch(it->second, s->stream));
  GKS_SCK(s, cudaMemsetAsync(s->bad, 0, sizeof(unsigned), s->stream));
  if (s->prec == PREC_F64)
    physical_kernel<double><<<nblk(s->L[0].ncell), kST, 0, s->stream>>>((const double*)s->L[0].W, s->L[0].ncell,
                                                                        s->L[0].g.gamma, s->bad);
  else
    physical_kernel<float><<<nblk(s->L[0].ncell), kST, 0, s->stream>>>((const float*)s->L[0].W, s->L[0].ncell,
                                                                       s->L[0].g.gamma, s->bad);
  unsigned badh = 0;
  GKS_SCK(s, cudaMemcpyAsync(&badh, s->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
  if (res_out) GKS_SCK(s, cudaMemcpyAsync(res_out, s->history, sizeof(double) * ncycles, cudaMemcpyDeviceToHost, s->stream));
  GKS_SCK(s, cudaStreamSynchronize(s->stream));
  if (badh) return sfail(s, GKS_ENONPHYS, "non-physical state (rho <= 0 or p <= 0) produced");
  return GKS_OK;
}

gks_status gks_steady_residual(gks_steady* s, double cfl_flux, int first_order, double* dt_out, double* R_out) {
  if (!s || !(cfl_flux > 0.0)) return sfail(s, GKS_EINVAL, "bad argument");
  if (!s->has_state) return sfail(s, GKS_EINVAL, "no state set");
  if (s->L[0].g.turb_model != GKS_TURB_NONE && !s->has_turb) return sfail(s, GKS_EINVAL, "turbulence fields not set");
  SteadyLevel& f = s->L[0];
  const StepArgs A = level_args(s, 0, f.W);
  launch_curv_lts(s->prec, A, f.G, f.s, s->stream);
  SteadyArgs SA{};
  SA.s_loc = f.s;
  SA.cfl_flux = cfl_flux;
  SA.first_order = first_order != 0;
  SA.multid = s->multid;
  SA.recon = first_order ? GKS_RECON_MUSCL2 : s->recon;
  SA.R = f.R;
  SA.tau = f.G.tau;
  if (SA.recon != GKS_RECON_MUSCL2)
    launch_curv_residual_recon(s->prec, A, f.G, SA, s->stream);
  else if (A.g.rar)
    launch_curv_residual_rar(s->prec, A, f.G, SA, s->stream);
  else
    launch_curv_residual(s->prec, A, f.G, SA, s->stream);
  GKS_SCK(s, cudaGetLastError());
  // out in double: convert through the staging buffer in single precision
  const long n = f.ncell;
  if (s->prec == PREC_F64) {
    if (dt_out) GKS_SCK(s, cudaMemcpyAsync(dt_out, f.s, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    if (R_out) GKS_SCK(s, cudaMemcpyAsync(R_out, f.R, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s->stream));
  } else {
    gks_status st = ensure_stage(s, sizeof(double) * 5 * n);
    if (st) return st;
    double* d = (double*)s->staging;
    aux::field_kernel<float, double><<<nblk(n, 256), 256, 0, s->stream>>>((const float*)f.s, d, n);
    aux::field_kernel<float, double><<<nblk(4 * n, 256), 256, 0, s->stream>>>((const float*)f.R, d + n, 4 * n);
    if (dt_out) GKS_SCK(s, cudaMemcpyAsync(dt_out, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    if (R_out) GKS_SCK(s, cudaMemcpyAsync(R_out, d + n, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s->stream));
  }
  GKS_SCK(s, cudaStreamSynchronize(s->stream));
  return GKS_OK;
}

gks_status gks_steady_get_state(gks_steady* s, void* W_out, int layout, int memspace, int dtype) {
  if (!s || !W_out) return sfail(s, GKS_EINVAL, "null argument");
  if (!s->has_state) return sfail(s, GKS_EINVAL, "no state set");
  if (layout < GKS_LAYOUT_SOA_CONS || layout > GKS_LAYOUT_SOA_PRIM || (dtype != GKS_F64 && dtype != GKS_F32) ||
      (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return sfail(s, GKS_EINVAL, "layout, memspace or dtype");
  SteadyLevel& f = s->L[0];
  const size_t bytes = (dtype == GKS_F64 ? 8 : 4) * 4 * (size_t)f.ncell;
  void* dst = W_out;
  if (memspace == GKS_MEM_HOST) {
    gks_status st = ensure_stage(s, bytes);
    if (st) return st;
    dst = s->staging;
  }
  // a zero low word: state_out_kernel adds it in single precision
  const int prec = s->prec == PREC_F64 ? PREC_F64 : PREC_F32;
  float* zero_lo = (float*)f.W0;
  if (prec == PREC_F32) GKS_SCK(s, cudaMemsetAsync(zero_lo, 0, sizeof(float) * 4 * f.ncell, s->stream));
  if (dtype == GKS_F64)
    aux::state_out_kernel<double><<<nblk(f.ncell, 256), 256, 0, s->stream>>>((double*)dst, layout, 2, f.ncell,
                                                                           f.g.gamma, prec, f.W, zero_lo);
  else
    aux::state_out_kernel<float><<<nblk(f.ncell, 256), 256, 0, s->stream>>>((float*)dst, layout, 2, f.ncell,
                                                                          f.g.gamma, prec, f.W, zero_lo);
  GKS_SCK(s, cudaGetLastError());
  if (memspace == GKS_MEM_HOST) {
    GKS_SCK(s, cudaMemcpyAsync(W_out, s->staging, bytes, cudaMemcpyDeviceToHost, s->stream));
    GKS_SCK(s, cudaStreamSynchronize(s->stream));
  }
  return GKS_OK;
}

}  // extern "C"
