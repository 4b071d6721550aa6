// C ABI of the gas-kinetic library (include/gks.h): handle, device buffers, state conversion,
// time stepping with captured CUDA graphs, diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gks.h"
#include "gks_curv.h"
#include "gks_dispatch.h"
#include "gks_step.cuh"
#include "gks_aux.cuh"

using namespace gks;
using namespace gks::aux;

struct gks_handle {
  int dev = 0;
  int D = 1, nv = 3;
  int n[3] = {1, 1, 1};
  long ncell = 0;
  int prec = PREC_F64;
  bool multid = false;
  int recon = 0;  // GKS_RECON_*
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* W[2] = {nullptr, nullptr};
  float* Wlo[2] = {nullptr, nullptr};
  void* f1 = nullptr;
  void* f2 = nullptr;
  bool transport = false;            // GKS_TURB_KOMEGA_TRANSPORT: k and omega evolve with the flow
  void* RK[2] = {nullptr, nullptr};  // rho k, rho omega (arithmetic type), buffered like the state
  void* RW[2] = {nullptr, nullptr};
  void* mflux[3] = {nullptr, nullptr, nullptr};  // face mass fluxes of the last flow step
  gks_komega kw{};
  bool curv = false;  // body-fitted 2D grid set by gks_set_nodes
  CurvGeom cg{};
  double* widths[3] = {nullptr, nullptr, nullptr};
  double* dir[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  Ctrl* ctrl = nullptr;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  long long step = 0;
  bool has_state = false, has_turb = false;
  bool rate_stale = false;  // a step call with t_end ran: steps past t_end leave the next CFL rate unset
  int nblocks = 0;
  int tile_variant = 0;   // 2D FP32: tile shape chosen by the autotuner
  bool tuned = false;
  StepArgs base;
  std::map<int, cudaGraphExec_t> graphs;
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  double ms_total = 0.0;
  long long launches = 0;
  std::string err;
};

namespace {

const int kGraphChunk = 48;  // steps per captured graph; a multiple of 6 keeps buffer and slot phases fixed

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

gks_status fail(gks_handle* h, gks_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

gks_status cuda_fail(gks_handle* h, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(h, GKS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GKS_CK(h, call)                                          \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);     \
  } while (0)

size_t stored_bytes(int prec) { return prec == PREC_F32 ? sizeof(float) : sizeof(double); }
size_t arith_bytes(int prec) { return prec == PREC_F64 ? sizeof(double) : sizeof(float); }

// ------------------------------------------------------------------------------------------------
// Kernels for state conversion, CFL rate and diagnostics
// ------------------------------------------------------------------------------------------------
// Per-cell turbulent relaxation time and rarefaction diagnostic, from the same cell formula the
// step kernel uses (neighbourhood staged in registers with the boundary rules applied).
template <int D, int PREC>
__global__ void __launch_bounds__(kThreads) diag_kernel(const __grid_constant__ StepArgs A, int what, void* out,
                                                        int out_dtype) {
  using R = typename PrecT<PREC>::R;
  constexpr int nv = D + 2;
  constexpr int S3 = D >= 3 ? 3 : 1, S2 = D >= 2 ? 3 : 1;
  const DevGrid& g = A.g;
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const Consts<R> kc = make_consts<R>(g);
  const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((long)g.n[0] * g.n[1]));
  R Wn[nv * 3 * S2 * S3];
  const int NN = 3 * S2 * S3;
  for (int l = 0; l < NN; ++l) {
    const int di = l % 3 - 1, dj = D >= 2 ? (l / 3) % 3 - 1 : 0, dk = D >= 3 ? l / 9 - 1 : 0;
    const bool on_axis = (di != 0) + (dj != 0) + (dk != 0) <= 1;
    R w[nv];
    if (on_axis) {
      load_cell<D, PREC>(A.g, A.Win, kc, i + di, j + dj, k + dk, w);
    } else {
      for (int v = 0; v < nv; ++v) w[v] = R(1);
    }
    for (int v = 0; v < nv; ++v) Wn[v * NN + l] = w[v];
  }
  R wx[3], wy[3], wz[3];
  for (int q = 0; q < 3; ++q) {
    wx[q] = (R)g.w[0][i + kWG - 1 + q];
    wy[q] = D >= 2 ? (R)g.w[1][j + kWG - 1 + q] : R(1);
    wz[q] = D >= 3 ? (R)g.w[2][k + kWG - 1 + q] : R(1);
  }
  const int strides[3] = {1, 3, 9};
  const R* widths[3] = {wx, wy, wz};
  // inverse distance between the centres of the two neighbours along each axis (position 1)
  R igx[3], igy[3], igz[3];
  igx[1] = g_rcp(R(0.5) * wx[0] + wx[1] + R(0.5) * wx[2]);
  igy[1] = g_rcp(R(0.5) * wy[0] + wy[1] + R(0.5) * wy[2]);
  igz[1] = g_rcp(R(0.5) * wz[0] + wz[1] + R(0.5) * wz[2]);
  igx[0] = igx[2] = igy[0] = igy[2] = igz[0] = igz[2] = R(1);
  const R* igrad[3] = {igx, igy, igz};
  const int pos[3] = {1, 1, 1};
  const int idx = 1 + (D >= 2 ? 3 : 0) + (D >= 3 ? 9 : 0);
  R f1 = R(0), f2 = R(0);
  if (g.turb_model != TURB_NONE) {
    f1 = ((const R*)A.f1)[c];
    if (g.turb_model != TURB_MUT) f2 = ((const R*)A.f2)[c];
  }
  R val = tau_turb_cell<D, R>(g.turb_model, g.turb_cons != 0, kc, Wn, NN, idx, strides, igrad, pos, f1, f2);
  if (what == 1) {  // rarefaction: (mu/p + tau_t) |div U|
    R w[nv];
    for (int v = 0; v < nv; ++v) w[v] = Wn[v * NN + idx];
    const R p = pressure_of<R>(D, kc.gamma, w);
    R div = R(0);
    for (int a = 0; a < D; ++a) {
      const R* wd = widths[a];
      const R dist = R(0.5) * wd[0] + wd[1] + R(0.5) * wd[2];
      const int im = idx - strides[a], ip = idx + strides[a];
      div += (Wn[(1 + a) * NN + ip] / Wn[ip] - Wn[(1 + a) * NN + im] / Wn[im]) / dist;
    }
    val = (kc.mu / p + val) * g_abs(div);
  }
  if (out_dtype == GKS_F64)
    ((double*)out)[c] = (double)val;
  else
    ((float*)out)[c] = (float)val;
}

__global__ void set_time_kernel(Ctrl* c, int slot, double t) { c->t[slot] = t; }

inline unsigned grid_for(long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int tiles_for(const gks_handle* h, int variant) {
  int t[3];
  tile_shape(h->D, variant, &t[0], &t[1], &t[2]);
  long n = 1;
  for (int d = 0; d < 3; ++d) n *= (h->n[d] + t[d] - 1) / t[d];
  return (int)n;
}

// k-omega transport fused into the body-fitted step (MUSCL-2, FP64 or the FP32 float-pair form);
// other combinations run the step and the transport kernel one after the other.
bool fused_transport(const gks_handle* h) {
  return h->curv && h->transport && h->recon == GKS_RECON_MUSCL2 && h->prec != PREC_F32D && !h->base.g.rar;
}

void launch_step_variant(gks_handle* h, const StepArgs& A, int variant) {
  if (h->base.g.rar) {  // the rarefaction option: one tile shape per grid kind
    if (h->curv)
      launch_curv_step_rar(h->prec, A, h->cg, h->multid, h->stream);
    else
      launch_step_rar(h->D, h->prec, h->multid, A, tiles_for(h, 0), h->stream);
    return;
  }
  if (fused_transport(h)) {
    launch_curv_step_transport(h->prec, A, h->cg, variant, h->multid, h->stream);
    return;
  }
  if (h->curv) {
    if (h->recon != GKS_RECON_MUSCL2)
      launch_curv_step_recon(h->prec, h->recon, A, h->cg, variant, h->multid, h->stream);
    else
      launch_curv_step(h->prec, A, h->cg, variant, h->multid, h->stream);
    return;
  }
  if (h->recon == GKS_RECON_MUSCL3) {
    launch_step_muscl3(h->D, h->prec, h->multid, variant, A, tiles_for(h, variant), h->stream);
    return;
  }
  if (h->recon == GKS_RECON_WENO5) {
    launch_step_weno5(h->D, h->prec, h->multid, variant, A, tiles_for(h, variant), h->stream);
    return;
  }
  if (h->D == 1 && variant > 0)
    launch_step_d1_variant(variant, h->prec, A, tiles_for(h, variant), h->stream);
  else if (h->D == 1)
    launch_step_d1(h->prec, false, A, tiles_for(h, 0), h->stream);
  else if (h->D >= 2 && variant > 0 && h->prec == PREC_F32D)
    launch_step_acc64_variant(h->D, variant, h->multid, A, tiles_for(h, variant), h->stream);
  else if (h->D == 2 && variant > 0)
    launch_step_d2_variant(variant, h->multid, A, tiles_for(h, variant), h->stream);
  else if (h->D == 3 && variant > 0)
    launch_step_d3_variant(variant, h->multid, A, tiles_for(h, variant), h->stream);
  else if (h->D == 2)
    launch_step_d2(h->prec, h->multid, A, tiles_for(h, 0), h->stream);
  else
    launch_step_d3(h->prec, h->multid, A, h->nblocks, h->stream);
}

// One full step: the flow step and, with k-omega transport, the transport step of rho k and
// rho omega (into the other buffer pair) with the same dt and the flow step's mass fluxes.
void launch_step(gks_handle* h, const StepArgs& A) {
  launch_step_variant(h, A, h->tile_variant);
  if (!h->transport || fused_transport(h)) return;
  const int cur = A.Win == h->W[0] ? 0 : 1;
  KOmegaArgs K;
  std::memset(&K, 0, sizeof(K));
  K.g = A.g;
  K.Win = A.Win;
  K.Wnew = A.Wout;
  K.RKin = h->RK[cur];
  K.RWin = h->RW[cur];
  K.RKout = h->RK[cur ^ 1];
  K.RWout = h->RW[cur ^ 1];
  for (int d = 0; d < 3; ++d) K.mflux[d] = h->mflux[d];
  K.ctrl = h->ctrl;
  K.alpha = h->kw.alpha;
  K.beta0 = h->kw.beta0;
  K.beta_star = A.g.beta_star;
  K.sigma = h->kw.sigma;
  K.sigma_star = h->kw.sigma_star;
  K.sigma_do = h->kw.sigma_do;
  K.C_lim = h->kw.C_lim;
  K.omega_floor = h->kw.omega_floor;
  K.sources = h->kw.sources;
  K.diffusion = h->kw.diffusion;
  K.falpha = (float)K.alpha;
  K.fbeta0 = (float)K.beta0;
  K.fbeta_star = (float)K.beta_star;
  K.fsigma = (float)K.sigma;
  K.fsigma_star = (float)K.sigma_star;
  K.fsigma_do = (float)K.sigma_do;
  K.fC_lim = (float)K.C_lim;
  K.fomega_floor = (float)K.omega_floor;
  if (h->curv)
    launch_curv_komega(h->prec, K, h->cg, h->stream);
  else
    launch_komega(h->D, h->prec, K, h->stream);
}

// Arguments of the step that starts at absolute step index s.
StepArgs step_args(const gks_handle* h, long long s, int resid) {
  StepArgs A = h->base;
  const int cur = (int)(s & 1);
  A.Win = h->W[cur];
  A.Wout = h->W[cur ^ 1];
  A.Win_lo = h->Wlo[cur];
  A.Wout_lo = h->Wlo[cur ^ 1];
  A.slot = (int)(s % 3);
  A.tslot = cur;
  A.resid = resid;
  if (h->transport) {
    A.f1 = h->RK[cur];
    A.f2 = h->RW[cur];
    if (fused_transport(h)) {  // the step advances rho k, rho omega itself
      A.RKout = h->RK[cur ^ 1];
      A.RWout = h->RW[cur ^ 1];
      A.kw_alpha = h->kw.alpha;
      A.kw_beta0 = h->kw.beta0;
      A.kw_sigma = h->kw.sigma;
      A.kw_sigma_star = h->kw.sigma_star;
      A.kw_sigma_do = h->kw.sigma_do;
      A.kw_C_lim = h->kw.C_lim;
      A.kw_omega_floor = h->kw.omega_floor;
      A.kw_falpha = (float)h->kw.alpha;
      A.kw_fbeta0 = (float)h->kw.beta0;
      A.kw_fsigma = (float)h->kw.sigma;
      A.kw_fsigma_star = (float)h->kw.sigma_star;
      A.kw_fsigma_do = (float)h->kw.sigma_do;
      A.kw_fC_lim = (float)h->kw.C_lim;
      A.kw_fomega_floor = (float)h->kw.omega_floor;
      A.kw_sources = h->kw.sources;
      A.kw_diffusion = h->kw.diffusion;
    } else {
      for (int d = 0; d < 3; ++d) A.mflux[d] = h->mflux[d];
    }
  }
  return A;
}

template <int D>
void launch_rate_d(gks_handle* h, const StepArgs& A, unsigned blocks) {
  if (h->prec == PREC_F64)
    rate_kernel<D, PREC_F64><<<blocks, kThreads, 0, h->stream>>>(A);
  else if (h->prec == PREC_F32)
    rate_kernel<D, PREC_F32><<<blocks, kThreads, 0, h->stream>>>(A);
  else
    rate_kernel<D, PREC_F32D><<<blocks, kThreads, 0, h->stream>>>(A);
}

gks_status launch_rate(gks_handle* h) {
  StepArgs A = step_args(h, h->step, 0);
  if (h->curv) {
    launch_curv_rate(h->prec, A, h->cg, h->stream);
    GKS_CK(h, cudaGetLastError());
    return GKS_OK;
  }
  const unsigned blocks = std::min<unsigned>(grid_for(h->ncell, kThreads), 152u * 8u);
  if (h->D == 1)
    launch_rate_d<1>(h, A, blocks);
  else if (h->D == 2)
    launch_rate_d<2>(h, A, blocks);
  else
    launch_rate_d<3>(h, A, blocks);
  GKS_CK(h, cudaGetLastError());
  return GKS_OK;
}

template <int D>
void launch_diag_d(gks_handle* h, const StepArgs& A, int what, void* out, int dtype) {
  const unsigned blocks = grid_for(h->ncell, kThreads);
  if (h->prec == PREC_F64)
    diag_kernel<D, PREC_F64><<<blocks, kThreads, 0, h->stream>>>(A, what, out, dtype);
  else if (h->prec == PREC_F32)
    diag_kernel<D, PREC_F32><<<blocks, kThreads, 0, h->stream>>>(A, what, out, dtype);
  else
    diag_kernel<D, PREC_F32D><<<blocks, kThreads, 0, h->stream>>>(A, what, out, dtype);
}

gks_status ensure_staging(gks_handle* h, size_t bytes) {
  if (h->staging_bytes >= bytes) return GKS_OK;
  if (h->staging) cudaFree(h->staging);
  h->staging = nullptr;
  h->staging_bytes = 0;
  if (cudaMalloc(&h->staging, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, GKS_ENOMEM, "staging buffer allocation failed");
  }
  h->staging_bytes = bytes;
  return GKS_OK;
}

bool valid_bc(int b) { return b >= GKS_BC_PERIODIC && b <= GKS_BC_OUTFLOW; }

void free_curv(gks_handle* h) {
  CurvGeom& G = h->cg;
  for (int a = 0; a < 2; ++a) {
    if (G.face[a]) cudaFree(G.face[a]);
    if (G.tang[a]) cudaFree(G.tang[a]);
    if (G.flux[a]) cudaFree(G.flux[a]);
  }
  if (G.iarea) cudaFree(G.iarea);
  if (G.area) cudaFree(G.area);
  if (G.tau) cudaFree(G.tau);
  G = CurvGeom{};
  if (h->curv) {  // back to the rectilinear step: its tile shape is chosen again
    h->tile_variant = 0;
    h->tuned = false;
  }
  h->curv = false;
}

void free_all(gks_handle* h) {
  free_curv(h);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
  for (int b = 0; b < 2; ++b) {
    if (h->W[b]) cudaFree(h->W[b]);
    if (h->Wlo[b]) cudaFree(h->Wlo[b]);
  }
  if (h->f1) cudaFree(h->f1);
  if (h->f2) cudaFree(h->f2);
  for (int b = 0; b < 2; ++b) {
    if (h->RK[b]) cudaFree(h->RK[b]);
    if (h->RW[b]) cudaFree(h->RW[b]);
  }
  for (int d = 0; d < 3; ++d)
    if (h->mflux[d]) cudaFree(h->mflux[d]);
  for (int d = 0; d < 3; ++d) {
    if (h->widths[d]) cudaFree(h->widths[d]);
    for (int s = 0; s < 2; ++s)
      if (h->dir[d][s]) cudaFree(h->dir[d][s]);
  }
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->staging) cudaFree(h->staging);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

gks_status sticky_status(gks_handle* h) {
  unsigned int st = 0;
  GKS_CK(h, cudaMemcpyAsync(&st, &h->ctrl->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  if (st & 1u) return fail(h, GKS_ENONPHYS, "non-physical state (rho <= 0 or p <= 0) produced");
  return GKS_OK;
}

// Tile-shape autotuner: each candidate shape runs the step that is about to be taken from the current
// state (the results are identical, and the step is then taken for real) five times, round robin
// over the shapes, each launch timed with CUDA events; the shape with the fastest launch is kept for
// the handle and for later handles of the same grid.
struct TuneKey {
  int n0, n1, multid;
  bool operator<(const TuneKey& o) const {
    return n0 != o.n0 ? n0 < o.n0 : (n1 != o.n1 ? n1 < o.n1 : multid < o.multid);
  }
};
std::map<TuneKey, int> g_tuned;
std::mutex g_tuned_mutex;

// Tile variants the autotuner tries for a handle (variant indices of tile_shape).
std::vector<int> tile_candidates(const gks_handle* h) {
  std::vector<int> c;
  if (h->base.g.rar) return {h->curv ? 2 : 0};  // the tile the rarefaction kernels are built for
  if (h->curv) {
    // the tiles the reconstruction and fused-transport kernels are built for
    if (h->recon != GKS_RECON_MUSCL2 || fused_transport(h)) return {0, 2};
    for (int v = 0; v < kCurvVariants; ++v) c.push_back(v);
    return c;
  }
  if (h->recon != GKS_RECON_MUSCL2) {
    c.push_back(0);
    if (h->D == 2 && h->prec == PREC_F32 && h->multid) c.push_back(3);  // 32 x 27 (four full waves at 1024^2)
    return c;
  }
  const bool f32 = h->prec == PREC_F32 || h->prec == PREC_F32D;
  const int n = h->D == 1 ? kTileVariants1D
                          : (h->D == 2 && f32 ? kTileVariants2D : (h->D == 3 && f32 ? kTileVariants3D : 1));
  for (int v = 0; v < n; ++v) c.push_back(v);
  return c;
}

int n_variants(const gks_handle* h) {
  if (h->base.g.rar) return 1;
  if (h->curv) return (h->recon != GKS_RECON_MUSCL2 || fused_transport(h)) ? 2 : kCurvVariants;
  if (h->recon != GKS_RECON_MUSCL2) return (int)tile_candidates(h).size();
  if (h->D == 1) return kTileVariants1D;
  if (h->D == 2 && (h->prec == PREC_F32 || h->prec == PREC_F32D)) return kTileVariants2D;
  if (h->D == 3 && (h->prec == PREC_F32 || h->prec == PREC_F32D)) return kTileVariants3D;
  return 1;
}

gks_status autotune(gks_handle* h) {
  h->tuned = true;
  const int nvar = n_variants(h);
  if (nvar == 1) {
    h->tile_variant = tile_candidates(h)[0];
    return GKS_OK;
  }
  const char* force = std::getenv("GKS_TILE_VARIANT");
  if (force) {
    const int v = std::atoi(force);
    for (int c : tile_candidates(h))
      if (c == v) h->tile_variant = v;
    return GKS_OK;
  }
  const TuneKey key{h->n[0] + 100000 * h->prec, h->n[1] * 4 + h->D,
                    h->curv ? 2 + 4 * h->recon + 16 * (int)fused_transport(h) : (int)h->multid};
  {
    std::lock_guard<std::mutex> lk(g_tuned_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      h->tile_variant = it->second;
      return GKS_OK;
    }
  }
  cudaEvent_t e0, e1;
  GKS_CK(h, cudaEventCreate(&e0));
  GKS_CK(h, cudaEventCreate(&e1));
  const StepArgs A = step_args(h, h->step, 0);
  const std::vector<int> cand = tile_candidates(h);
  std::vector<float> fastest(cand.size(), 1e30f);
  for (int v : cand) launch_step_variant(h, A, v);  // warm-up
  // round robin, each launch timed alone, the fastest launch of each shape kept: a clock that is
  // still ramping up penalises no shape in particular
  for (int r = 0; r < 5; ++r)
    for (size_t k = 0; k < cand.size(); ++k) {
      GKS_CK(h, cudaEventRecord(e0, h->stream));
      launch_step_variant(h, A, cand[k]);
      GKS_CK(h, cudaEventRecord(e1, h->stream));
      GKS_CK(h, cudaEventSynchronize(e1));
      float ms = 0.0f;
      GKS_CK(h, cudaEventElapsedTime(&ms, e0, e1));
      fastest[k] = std::min(fastest[k], ms);
    }
  int best_v = cand[0];
  float best = fastest[0];
  for (size_t k = 1; k < cand.size(); ++k)
    if (fastest[k] < best) {
      best = fastest[k];
      best_v = cand[k];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the trials max-wrote the next step's CFL-rate slot: clear it so that the real step alone sets it
  GKS_CK(h, cudaMemsetAsync(&h->ctrl->rate[(h->step + 1) % 3], 0, sizeof(unsigned long long), h->stream));
  h->tile_variant = best_v;
  std::lock_guard<std::mutex> lk(g_tuned_mutex);
  g_tuned[key] = best_v;
  return GKS_OK;
}

}  // namespace

// ================================================================================================
extern "C" {

gks_status gks_create(const gks_grid* grid, const gks_gas* gas, const gks_turb* turb, const gks_numerics* num,
                      void* cuda_stream, gks_handle** out) {
  if (!out) return GKS_EINVAL;
  *out = nullptr;
  if (!grid || !gas || !num) return GKS_EINVAL;
  gks_handle* h = new (std::nothrow) gks_handle();
  if (!h) return GKS_ENOMEM;
  auto bad = [&](gks_status s, const char* m) {
    h->err = m;
    *out = h;  // return the handle so that the caller can read the message
    return s;
  };
  const int D = grid->dim;
  if (D < 1 || D > 3) return bad(GKS_EINVAL, "dim must be 1, 2 or 3");
  h->D = D;
  h->nv = D + 2;
  h->ncell = 1;
  for (int d = 0; d < 3; ++d) {
    h->n[d] = d < D ? grid->n[d] : 1;
    if (d < D && h->n[d] < 2) return bad(GKS_EINVAL, "at least two cells per active axis");
    // the cell count is bounded before it is formed, so that it and every byte count taken from it
    // stay exact (GKS_MAX_CELLS cells hold more state than any device's memory)
    if (h->n[d] > GKS_MAX_CELLS / h->ncell) return bad(GKS_EINVAL, "more than GKS_MAX_CELLS cells");
    h->ncell *= h->n[d];
  }
  if (!(gas->gamma > 1.0)) return bad(GKS_EINVAL, "gamma must exceed 1");
  if (grid->wake_cut < 0 || (grid->wake_cut > 0 && (D != 2 || 2 * grid->wake_cut > h->n[0])))
    return bad(GKS_EINVAL, "a wake cut needs 2D and at most half the j-lo side on each end");
  const double bK = 2.0 / (gas->gamma - 1.0), K = bK - D;
  if (K < 0.0) return bad(GKS_EINVAL, "gamma leaves a negative number of internal degrees of freedom");
  if (!(gas->mu >= 0.0)) return bad(GKS_EINVAL, "mu must be >= 0");
  if (gas->prandtl != 0.0 && gas->prandtl != 1.0) return bad(GKS_EUNSUPPORTED, "only Pr = 1 is built");
  if (num->precision < GKS_FP64 || num->precision > GKS_FP32_ACC64) return bad(GKS_EINVAL, "precision");
  if (num->limiter != GKS_LIM_MINMOD && num->limiter != GKS_LIM_VANLEER) return bad(GKS_EINVAL, "limiter");
  if (num->expand != GKS_EXPAND_DIRECTIONAL && num->expand != GKS_EXPAND_MULTID) return bad(GKS_EINVAL, "expand");
  if (num->abar_mode != GKS_ABAR_TIMEINT && num->abar_mode != GKS_ABAR_T0) return bad(GKS_EINVAL, "abar_mode");
  const int model = turb ? turb->model : GKS_TURB_NONE;
  if (model < GKS_TURB_NONE || model > GKS_TURB_KOMEGA_TRANSPORT) return bad(GKS_EINVAL, "turbulence model");
  const int rar = turb ? turb->rarefaction : GKS_RAR_DT;
  if (rar != GKS_RAR_DT && rar != GKS_RAR_TAUHAT) return bad(GKS_EINVAL, "rarefaction");
  if (rar == GKS_RAR_TAUHAT && num->reconstruction != GKS_RECON_MUSCL2)
    return bad(GKS_EUNSUPPORTED, "the rarefaction option is built for MUSCL2");
  h->transport = model == GKS_TURB_KOMEGA_TRANSPORT;
  for (int d = 0; d < D; ++d) {
    for (int s = 0; s < 2; ++s) {
      if (!valid_bc(grid->bc[d][s])) return bad(GKS_EINVAL, "boundary condition code");
      if (grid->bc[d][s] == GKS_BC_DIRICHLET && !grid->bc_data[d][s]) return bad(GKS_EINVAL, "Dirichlet data missing");
    }
    if ((grid->bc[d][0] == GKS_BC_PERIODIC) != (grid->bc[d][1] == GKS_BC_PERIODIC))
      return bad(GKS_EINVAL, "periodic boundaries must be set on both sides of an axis");
    if (!grid->dx[d] && !(grid->hi[d] > grid->lo[d])) return bad(GKS_EINVAL, "extent hi > lo required");
    if (grid->dx[d])
      for (int i = 0; i < h->n[d]; ++i)
        if (!(grid->dx[d][i] > 0.0)) return bad(GKS_EINVAL, "cell widths must be positive");
  }
  if (grid->bc[0][0] == GKS_BC_WALL || grid->bc[0][1] == GKS_BC_WALL || (D > 1 && (grid->bc[1][0] == GKS_BC_WALL ||
      grid->bc[1][1] == GKS_BC_WALL)) || (D > 2 && (grid->bc[2][0] == GKS_BC_WALL || grid->bc[2][1] == GKS_BC_WALL)))
    if (!(gas->T_wall > 0.0)) return bad(GKS_EINVAL, "T_wall must be positive with wall boundaries");
  h->prec = num->precision;
  h->multid = D > 1 && num->expand == GKS_EXPAND_MULTID;
  h->recon = num->reconstruction;
  if (h->recon < GKS_RECON_MUSCL2 || h->recon > GKS_RECON_WENO5) return bad(GKS_EINVAL, "reconstruction");
  if (h->recon != GKS_RECON_MUSCL2 && (h->prec == PREC_F32D || (D == 3 && !h->multid)))
    return bad(GKS_EUNSUPPORTED, "higher-order reconstruction needs GKS_FP64 or GKS_FP32 (and multi-D in 3D)");
  for (int d = 0; d < D; ++d)
    if (h->recon == GKS_RECON_WENO5 && h->n[d] < 3) return bad(GKS_EINVAL, "WENO5 needs at least 3 cells per axis");

  if (cudaGetDevice(&h->dev) != cudaSuccess) {
    cudaGetLastError();
    return bad(GKS_ECUDA, "no CUDA device");
  }
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return bad(GKS_ECUDA, "stream creation failed");
    }
    h->own_stream = true;
  }
  static bool prepared[4] = {false, false, false, false};
  if (!prepared[D]) {
    cudaError_t e = D == 1 ? prepare_step_d1() : (D == 2 ? prepare_step_d2() : prepare_step_d3());
    if (e == cudaSuccess && D == 2) e = prepare_step_d2_variants();
    if (e == cudaSuccess && D == 2) e = prepare_curv();
    if (e == cudaSuccess && D == 2) e = prepare_curv_recon();
    if (e == cudaSuccess && D == 2) e = prepare_curv_transport();
    if (e == cudaSuccess && D == 1) e = prepare_step_d1_variants();
    if (e == cudaSuccess && D == 3) e = prepare_step_d3_variants();
    if (e == cudaSuccess && D >= 2) e = prepare_step_acc64();
    if (e == cudaSuccess && D >= 2) e = prepare_step_pair();
    if (e == cudaSuccess) e = prepare_step_rar();
    if (e == cudaSuccess && D == 2) e = prepare_curv_rar();
    if (e == cudaSuccess) e = prepare_komega();
    if (e == cudaSuccess) e = prepare_step_muscl3();
    if (e == cudaSuccess) e = prepare_step_weno5();
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bad(GKS_ECUDA, "kernel attribute setup failed");
    }
    prepared[D] = true;
  }

  const size_t sb = stored_bytes(h->prec), nbytes = sb * h->nv * h->ncell;
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  for (int b = 0; b < 2; ++b) {
    if (!alloc(&h->W[b], nbytes)) return bad(GKS_ENOMEM, "state allocation failed");
    if (h->prec == PREC_F32 && !alloc((void**)&h->Wlo[b], sizeof(float) * h->nv * h->ncell))
      return bad(GKS_ENOMEM, "state allocation failed");
  }
  if (!alloc((void**)&h->ctrl, sizeof(Ctrl))) return bad(GKS_ENOMEM, "control block allocation failed");
  cudaMemset(h->ctrl, 0, sizeof(Ctrl));
  if (h->transport) {
    const size_t fb = arith_bytes(h->prec) * h->ncell;
    for (int b = 0; b < 2; ++b) {
      if (!alloc(&h->RK[b], fb) || !alloc(&h->RW[b], fb)) return bad(GKS_ENOMEM, "field allocation failed");
      cudaMemset(h->RK[b], 0, fb);
      cudaMemset(h->RW[b], 0, fb);
    }
    for (int d = 0; d < D; ++d) {
      long nf = 1;
      for (int b = 0; b < D; ++b) nf *= h->n[b] + (b == d ? 1 : 0);
      if (!alloc(&h->mflux[d], arith_bytes(h->prec) * nf)) return bad(GKS_ENOMEM, "mass-flux allocation failed");
    }
    gks_komega_defaults(&h->kw);
  } else if (model != GKS_TURB_NONE) {
    const size_t fb = arith_bytes(h->prec) * h->ncell;
    if (!alloc(&h->f1, fb) || !alloc(&h->f2, fb)) return bad(GKS_ENOMEM, "field allocation failed");
    cudaMemset(h->f1, 0, fb);
    cudaMemset(h->f2, 0, fb);
  }
  // widths with kWG ghosts per side: periodic axes wrap, other axes mirror
  for (int d = 0; d < 3; ++d) {
    const int n = d < D ? h->n[d] : 1;
    std::vector<double> w(n + 2 * kWG, 1.0), in(n, 1.0);
    if (d < D) {
      for (int i = 0; i < n; ++i) in[i] = grid->dx[d] ? grid->dx[d][i] : (grid->hi[d] - grid->lo[d]) / n;
      const bool per = grid->bc[d][0] == GKS_BC_PERIODIC;
      for (int i = 0; i < n; ++i) w[i + kWG] = in[i];
      for (int gi = 1; gi <= kWG; ++gi) {
        w[kWG - gi] = per ? in[(n - gi % n) % n] : in[std::min(gi - 1, n - 1)];
        w[n + kWG - 1 + gi] = per ? in[(gi - 1) % n] : in[std::max(n - gi, 0)];
      }
    }
    const size_t wb = sizeof(double) * (n + 2 * kWG);
    if (!alloc((void**)&h->widths[d], wb)) return bad(GKS_ENOMEM, "width allocation failed");
    cudaMemcpy(h->widths[d], w.data(), wb, cudaMemcpyHostToDevice);
  }
  // Dirichlet states, converted to conservative variables
  for (int d = 0; d < D; ++d)
    for (int s = 0; s < 2; ++s) {
      if (grid->bc[d][s] != GKS_BC_DIRICHLET) continue;
      long cnt = 1;
      for (int b = 0; b < D; ++b)
        if (b != d) cnt *= h->n[b];
      std::vector<double> cons(cnt * h->nv);
      for (long c = 0; c < cnt; ++c) {
        const double* pr = grid->bc_data[d][s] + c * h->nv;
        if (!(pr[0] > 0.0) || !(pr[D + 1] > 0.0)) return bad(GKS_EINVAL, "Dirichlet state must have rho, p > 0");
        double q = 0.0;
        cons[c * h->nv] = pr[0];
        for (int i = 0; i < D; ++i) {
          cons[c * h->nv + 1 + i] = pr[0] * pr[1 + i];
          q += pr[1 + i] * pr[1 + i];
        }
        cons[c * h->nv + D + 1] = pr[D + 1] / (gas->gamma - 1.0) + 0.5 * pr[0] * q;
      }
      if (!alloc((void**)&h->dir[d][s], sizeof(double) * cons.size())) return bad(GKS_ENOMEM, "allocation failed");
      cudaMemcpy(h->dir[d][s], cons.data(), sizeof(double) * cons.size(), cudaMemcpyHostToDevice);
    }
  if (cudaGetLastError() != cudaSuccess) return bad(GKS_ECUDA, "device set-up failed");

  DevGrid& g = h->base.g;
  std::memset(&h->base, 0, sizeof(h->base));
  for (int d = 0; d < 3; ++d) {
    g.n[d] = h->n[d];
    g.w[d] = h->widths[d];
    for (int s = 0; s < 2; ++s) {
      g.bc[d][s] = d < D ? grid->bc[d][s] : GKS_BC_PERIODIC;
      g.dir[d][s] = h->dir[d][s];
    }
  }
  g.ncell = h->ncell;
  g.gamma = gas->gamma;
  g.bK = bK;
  g.K = K;
  g.mu = gas->mu;
  g.T_wall = gas->T_wall;
  g.C_a = turb ? turb->C_a : 0.0;
  g.C_mu = turb ? turb->C_mu : 0.09;
  g.beta_star = turb ? turb->beta_star : 0.09;
  g.turb_model = h->transport ? (int)GKS_TURB_KOMEGA : model;
  g.turb_cons = h->transport ? 1 : 0;
  g.limiter = num->limiter;
  g.abar_t0 = num->abar_mode == GKS_ABAR_T0;
  g.wake_cut = grid->wake_cut;
  g.rar = rar == GKS_RAR_TAUHAT;
  set_consts(g);
  h->base.f1 = h->f1;
  h->base.f2 = h->f2;
  h->base.ctrl = h->ctrl;
  long tiles = 1;
  const int T[3] = {D == 1 ? Tile<1>::X : (D == 2 ? Tile<2>::X : Tile<3>::X),
                    D == 1 ? 1 : (D == 2 ? Tile<2>::Y : Tile<3>::Y), D == 3 ? Tile<3>::Z : 1};
  for (int d = 0; d < 3; ++d) tiles *= (h->n[d] + T[d] - 1) / T[d];
  h->nblocks = (int)tiles;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return bad(GKS_ECUDA, "device set-up failed");
  }
  *out = h;
  return GKS_OK;
}

gks_status gks_destroy(gks_handle* h) {
  if (!h) return GKS_EINVAL;
  {
    DeviceGuard dg(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
  }
  delete h;
  return GKS_OK;
}

const char* gks_last_error(const gks_handle* h) { return h ? h->err.c_str() : "null handle"; }

gks_status gks_set_state(gks_handle* h, const void* W, int layout, int memspace, int dtype) {
  if (!h || !W) return fail(h, GKS_EINVAL, "null argument");
  if (layout < GKS_LAYOUT_SOA_CONS || layout > GKS_LAYOUT_SOA_PRIM || (dtype != GKS_F64 && dtype != GKS_F32) ||
      (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return fail(h, GKS_EINVAL, "layout, memspace or dtype");
  DeviceGuard dg(h->dev);
  const size_t eb = dtype == GKS_F64 ? 8 : 4, bytes = eb * h->nv * h->ncell;
  const void* src = W;
  if (memspace == GKS_MEM_HOST) {
    gks_status s = ensure_staging(h, bytes);
    if (s) return s;
    GKS_CK(h, cudaMemcpyAsync(h->staging, W, bytes, cudaMemcpyHostToDevice, h->stream));
    src = h->staging;
  }
  h->step = 0;
  GKS_CK(h, cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));
  const unsigned blocks = grid_for(h->ncell, 256);
  if (dtype == GKS_F64)
    state_in_kernel<double><<<blocks, 256, 0, h->stream>>>((const double*)src, layout, h->D, h->ncell,
                                                          h->base.g.gamma, h->prec, h->W[0], h->Wlo[0]);
  else
    state_in_kernel<float><<<blocks, 256, 0, h->stream>>>((const float*)src, layout, h->D, h->ncell,
                                                         h->base.g.gamma, h->prec, h->W[0], h->Wlo[0]);
  GKS_CK(h, cudaGetLastError());
  h->has_state = true;
  h->rate_stale = false;
  if (h->transport) h->has_turb = false;  // rho k, rho omega belong to the previous state
  return launch_rate(h);
}

gks_status gks_get_state(gks_handle* h, void* W_out, int layout, int memspace, int dtype) {
  if (!h || !W_out) return fail(h, GKS_EINVAL, "null argument");
  if (!h->has_state) return fail(h, GKS_EINVAL, "no state set");
  if (layout < GKS_LAYOUT_SOA_CONS || layout > GKS_LAYOUT_SOA_PRIM || (dtype != GKS_F64 && dtype != GKS_F32) ||
      (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return fail(h, GKS_EINVAL, "layout, memspace or dtype");
  DeviceGuard dg(h->dev);
  const size_t eb = dtype == GKS_F64 ? 8 : 4, bytes = eb * h->nv * h->ncell;
  void* dst = W_out;
  if (memspace == GKS_MEM_HOST) {
    gks_status s = ensure_staging(h, bytes);
    if (s) return s;
    dst = h->staging;
  }
  const int cur = (int)(h->step & 1);
  const unsigned blocks = grid_for(h->ncell, 256);
  if (dtype == GKS_F64)
    state_out_kernel<double><<<blocks, 256, 0, h->stream>>>((double*)dst, layout, h->D, h->ncell, h->base.g.gamma,
                                                           h->prec, h->W[cur], h->Wlo[cur]);
  else
    state_out_kernel<float><<<blocks, 256, 0, h->stream>>>((float*)dst, layout, h->D, h->ncell, h->base.g.gamma,
                                                          h->prec, h->W[cur], h->Wlo[cur]);
  GKS_CK(h, cudaGetLastError());
  if (memspace == GKS_MEM_HOST) {
    GKS_CK(h, cudaMemcpyAsync(W_out, h->staging, bytes, cudaMemcpyDeviceToHost, h->stream));
    GKS_CK(h, cudaStreamSynchronize(h->stream));
    return sticky_status(h);
  }
  return GKS_OK;
}

gks_status gks_set_turbulence(gks_handle* h, const void* f1, const void* f2, int memspace, int dtype) {
  if (!h || !f1) return fail(h, GKS_EINVAL, "null argument");
  if (h->base.g.turb_model == GKS_TURB_NONE) return fail(h, GKS_EINVAL, "handle created without a turbulence model");
  if (h->base.g.turb_model != GKS_TURB_MUT && !f2) return fail(h, GKS_EINVAL, "second turbulence field missing");
  if ((dtype != GKS_F64 && dtype != GKS_F32) || (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return fail(h, GKS_EINVAL, "memspace or dtype");
  if (h->transport && !h->has_state) return fail(h, GKS_EINVAL, "k-omega transport: set the state first");
  DeviceGuard dg(h->dev);
  const size_t eb = dtype == GKS_F64 ? 8 : 4, bytes = eb * h->ncell;
  const void* srcs[2] = {f1, f2};
  const int cur = (int)(h->step & 1);
  void* dsts[2] = {h->transport ? h->RK[cur] : h->f1, h->transport ? h->RW[cur] : h->f2};
  for (int q = 0; q < 2; ++q) {
    if (!srcs[q]) continue;
    const void* src = srcs[q];
    if (memspace == GKS_MEM_HOST) {
      gks_status s = ensure_staging(h, bytes);
      if (s) return s;
      GKS_CK(h, cudaMemcpyAsync(h->staging, src, bytes, cudaMemcpyHostToDevice, h->stream));
      src = h->staging;
    }
    const unsigned blocks = grid_for(h->ncell, 256);
    const bool f64 = h->prec == PREC_F64;
    if (dtype == GKS_F64 && f64)
      field_kernel<double, double><<<blocks, 256, 0, h->stream>>>((const double*)src, (double*)dsts[q], h->ncell);
    else if (dtype == GKS_F64)
      field_kernel<double, float><<<blocks, 256, 0, h->stream>>>((const double*)src, (float*)dsts[q], h->ncell);
    else if (f64)
      field_kernel<float, double><<<blocks, 256, 0, h->stream>>>((const float*)src, (double*)dsts[q], h->ncell);
    else
      field_kernel<float, float><<<blocks, 256, 0, h->stream>>>((const float*)src, (float*)dsts[q], h->ncell);
    GKS_CK(h, cudaGetLastError());
    if (h->transport) {  // k, omega -> rho k, rho omega with the density of the current state
      if (f64)
        density_scale_kernel<double, double><<<blocks, 256, 0, h->stream>>>((double*)dsts[q], (const double*)h->W[cur],
                                                                            h->ncell);
      else if (h->prec == PREC_F32)
        density_scale_kernel<float, float><<<blocks, 256, 0, h->stream>>>((float*)dsts[q], (const float*)h->W[cur],
                                                                          h->ncell);
      else
        density_scale_kernel<float, double><<<blocks, 256, 0, h->stream>>>((float*)dsts[q], (const double*)h->W[cur],
                                                                           h->ncell);
      GKS_CK(h, cudaGetLastError());
    }
    if (memspace == GKS_MEM_HOST) GKS_CK(h, cudaStreamSynchronize(h->stream));  // staging is reused
  }
  h->has_turb = true;
  return GKS_OK;
}

gks_status gks_komega_defaults(gks_komega* c) {
  if (!c) return GKS_EINVAL;
  c->alpha = 13.0 / 25.0;
  c->beta0 = 0.0708;
  c->sigma = 0.5;
  c->sigma_star = 0.6;
  c->sigma_do = 0.125;
  c->C_lim = 7.0 / 8.0;
  c->omega_floor = 1e-12;
  c->sources = 1;
  c->diffusion = 1;
  return GKS_OK;
}

gks_status gks_set_komega(gks_handle* h, const gks_komega* c) {
  if (!h || !c) return fail(h, GKS_EINVAL, "null argument");
  if (!h->transport) return fail(h, GKS_EINVAL, "handle not created with GKS_TURB_KOMEGA_TRANSPORT");
  if (!(c->omega_floor > 0.0)) return fail(h, GKS_EINVAL, "omega_floor must be positive");
  h->kw = *c;
  // captured graphs hold the old coefficients in their kernel parameters
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  return GKS_OK;
}

gks_status gks_get_turbulence(gks_handle* h, void* k_out, void* omega_out, int memspace, int dtype) {
  if (!h || !k_out || !omega_out) return fail(h, GKS_EINVAL, "null argument");
  if (!h->transport) return fail(h, GKS_EINVAL, "handle not created with GKS_TURB_KOMEGA_TRANSPORT");
  if (!h->has_turb) return fail(h, GKS_EINVAL, "turbulence fields not set");
  if ((dtype != GKS_F64 && dtype != GKS_F32) || (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return fail(h, GKS_EINVAL, "memspace or dtype");
  DeviceGuard dg(h->dev);
  const size_t eb = dtype == GKS_F64 ? 8 : 4, bytes = eb * h->ncell;
  const int cur = (int)(h->step & 1);
  const unsigned blocks = grid_for(h->ncell, 256);
  void* outs[2] = {k_out, omega_out};
  const void* srcs[2] = {h->RK[cur], h->RW[cur]};
  for (int q = 0; q < 2; ++q) {
    void* dst = outs[q];
    if (memspace == GKS_MEM_HOST) {
      gks_status s = ensure_staging(h, bytes);
      if (s) return s;
      dst = h->staging;
    }
    if (h->prec == PREC_F64) {
      if (dtype == GKS_F64)
        density_unscale_kernel<double, double, double><<<blocks, 256, 0, h->stream>>>(
            (const double*)srcs[q], (const double*)h->W[cur], (double*)dst, h->ncell);
      else
        density_unscale_kernel<double, double, float><<<blocks, 256, 0, h->stream>>>(
            (const double*)srcs[q], (const double*)h->W[cur], (float*)dst, h->ncell);
    } else if (h->prec == PREC_F32) {
      if (dtype == GKS_F64)
        density_unscale_kernel<float, float, double><<<blocks, 256, 0, h->stream>>>(
            (const float*)srcs[q], (const float*)h->W[cur], (double*)dst, h->ncell);
      else
        density_unscale_kernel<float, float, float><<<blocks, 256, 0, h->stream>>>(
            (const float*)srcs[q], (const float*)h->W[cur], (float*)dst, h->ncell);
    } else {
      if (dtype == GKS_F64)
        density_unscale_kernel<float, double, double><<<blocks, 256, 0, h->stream>>>(
            (const float*)srcs[q], (const double*)h->W[cur], (double*)dst, h->ncell);
      else
        density_unscale_kernel<float, double, float><<<blocks, 256, 0, h->stream>>>(
            (const float*)srcs[q], (const double*)h->W[cur], (float*)dst, h->ncell);
    }
    GKS_CK(h, cudaGetLastError());
    if (memspace == GKS_MEM_HOST) {
      GKS_CK(h, cudaMemcpyAsync(outs[q], h->staging, bytes, cudaMemcpyDeviceToHost, h->stream));
      GKS_CK(h, cudaStreamSynchronize(h->stream));
    }
  }
  return GKS_OK;
}

// Steps taken at or past t_end carry the state over without computing the CFL rate of the next
// step; before the next use of that rate it is computed from the stored state.
gks_status refresh_rate(gks_handle* h) {
  if (!h->rate_stale) return GKS_OK;
  h->rate_stale = false;
  GKS_CK(h, cudaMemsetAsync(&h->ctrl->rate[h->step % 3], 0, sizeof(unsigned long long), h->stream));
  return launch_rate(h);
}

gks_status gks_compute_dt(gks_handle* h, double cfl, double* dt_out) {
  if (!h || !dt_out || !(cfl > 0.0)) return fail(h, GKS_EINVAL, "bad argument");
  if (!h->has_state) return fail(h, GKS_EINVAL, "no state set");
  DeviceGuard dg(h->dev);
  {
    const gks_status rs = refresh_rate(h);
    if (rs != GKS_OK) return rs;
  }
  unsigned long long bits = 0;
  GKS_CK(h, cudaMemcpyAsync(&bits, &h->ctrl->rate[h->step % 3], sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  double r;
  std::memcpy(&r, &bits, sizeof(r));
  *dt_out = cfl / r;
  return sticky_status(h);
}

gks_status gks_step(gks_handle* h, double dt, double cfl, int nsteps, double t_end) {
  if (!h || nsteps < 0) return fail(h, GKS_EINVAL, "bad argument");
  if (!h->has_state) return fail(h, GKS_EINVAL, "no state set");
  if (!(dt > 0.0) && !(cfl > 0.0)) return fail(h, GKS_EINVAL, "need dt > 0 or cfl > 0");
  if (h->base.g.turb_model != GKS_TURB_NONE && !h->has_turb) return fail(h, GKS_EINVAL, "turbulence fields not set");
  if (h->base.g.wake_cut > 0 && !h->curv) return fail(h, GKS_EINVAL, "a wake cut needs a body-fitted grid");
  if (nsteps == 0) return GKS_OK;
  DeviceGuard dg(h->dev);
  {
    const gks_status rs = refresh_rate(h);
    if (rs != GKS_OK) return rs;
  }
  set_params_kernel<0><<<1, 1, 0, h->stream>>>(h->ctrl, dt > 0.0 ? dt : 0.0, cfl, t_end);
  GKS_CK(h, cudaGetLastError());
  if (t_end > 0.0) h->rate_stale = true;
  if (!h->tuned) {
    const gks_status st = autotune(h);
    if (st != GKS_OK) return st;
  }
  int remaining = nsteps;
  while (remaining > 0) {
    if (!h->timing && remaining - 1 >= kGraphChunk && h->step % 6 == 0) {
      auto it = h->graphs.find(kGraphChunk);
      if (it == h->graphs.end()) {
        cudaGraph_t graph;
        GKS_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kGraphChunk; ++k) launch_step(h, step_args(h, k, 0));
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiation");
        it = h->graphs.emplace(kGraphChunk, exec).first;
      }
      GKS_CK(h, cudaGraphLaunch(it->second, h->stream));
      h->step += kGraphChunk;
      remaining -= kGraphChunk;
      continue;
    }
    const StepArgs A = step_args(h, h->step, remaining == 1);
    if (h->timing) {
      cudaEvent_t e0, e1;
      GKS_CK(h, cudaEventCreate(&e0));
      GKS_CK(h, cudaEventCreate(&e1));
      h->ev.push_back(e0);
      h->ev.push_back(e1);
      GKS_CK(h, cudaEventRecord(e0, h->stream));
      launch_step(h, A);
      GKS_CK(h, cudaEventRecord(e1, h->stream));
    } else {
      launch_step(h, A);
    }
    GKS_CK(h, cudaGetLastError());
    h->step += 1;
    remaining -= 1;
  }
  return GKS_OK;
}

gks_status gks_get_time(gks_handle* h, double* t, long long* steps) {
  if (!h) return GKS_EINVAL;
  DeviceGuard dg(h->dev);
  double tv = 0.0;
  GKS_CK(h, cudaMemcpyAsync(&tv, &h->ctrl->t[h->step & 1], sizeof(tv), cudaMemcpyDeviceToHost, h->stream));
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  if (t) *t = tv;
  if (steps) *steps = h->step;
  return GKS_OK;
}

gks_status gks_set_time(gks_handle* h, double t) {
  if (!h) return GKS_EINVAL;
  DeviceGuard dg(h->dev);
  set_time_kernel<<<1, 1, 0, h->stream>>>(h->ctrl, (int)(h->step & 1), t);
  GKS_CK(h, cudaGetLastError());
  return GKS_OK;
}

gks_status gks_residual(gks_handle* h, double* l2, double* linf, double* total) {
  if (!h) return GKS_EINVAL;
  DeviceGuard dg(h->dev);
  Ctrl c;
  GKS_CK(h, cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  for (int v = 0; v < h->nv; ++v) {
    if (l2) l2[v] = std::sqrt(c.l2[v] / (double)h->ncell);
    if (linf) std::memcpy(&linf[v], &c.linf[v], sizeof(double));
    if (total) total[v] = c.total[v];
  }
  if (c.status & 1u) return fail(h, GKS_ENONPHYS, "non-physical state (rho <= 0 or p <= 0) produced");
  return GKS_OK;
}

gks_status gks_status_word(gks_handle* h, unsigned int* bits, double* last_dt) {
  if (!h) return GKS_EINVAL;
  DeviceGuard dg(h->dev);
  Ctrl c;
  GKS_CK(h, cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  if (bits) *bits = c.status;
  if (last_dt) *last_dt = c.last_dt;
  return GKS_OK;
}

static gks_status get_diag(gks_handle* h, int what, void* out, int memspace, int dtype) {
  if (!h || !out) return fail(h, GKS_EINVAL, "null argument");
  if (!h->has_state) return fail(h, GKS_EINVAL, "no state set");
  if (h->base.g.turb_model != GKS_TURB_NONE && !h->has_turb) return fail(h, GKS_EINVAL, "turbulence fields not set");
  if ((dtype != GKS_F64 && dtype != GKS_F32) || (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE))
    return fail(h, GKS_EINVAL, "memspace or dtype");
  DeviceGuard dg(h->dev);
  const size_t bytes = (dtype == GKS_F64 ? 8 : 4) * h->ncell;
  void* dst = out;
  if (memspace == GKS_MEM_HOST) {
    gks_status s = ensure_staging(h, bytes);
    if (s) return s;
    dst = h->staging;
  }
  const StepArgs A = step_args(h, h->step, 0);
  if (h->curv) {
    if (what == 0 && h->base.g.turb_model == GKS_TURB_NONE) {
      GKS_CK(h, cudaMemsetAsync(dst, 0, bytes, h->stream));
    } else {
      launch_curv_tau(h->prec, A, h->cg, h->cg.tau, h->stream, what);
      const unsigned blocks = grid_for(h->ncell, 256);
      if (h->prec == PREC_F64 && dtype == GKS_F64)
        field_kernel<double, double><<<blocks, 256, 0, h->stream>>>((const double*)h->cg.tau, (double*)dst, h->ncell);
      else if (h->prec == PREC_F64)
        field_kernel<double, float><<<blocks, 256, 0, h->stream>>>((const double*)h->cg.tau, (float*)dst, h->ncell);
      else if (dtype == GKS_F64)
        field_kernel<float, double><<<blocks, 256, 0, h->stream>>>((const float*)h->cg.tau, (double*)dst, h->ncell);
      else
        field_kernel<float, float><<<blocks, 256, 0, h->stream>>>((const float*)h->cg.tau, (float*)dst, h->ncell);
    }
  } else if (h->D == 1)
    launch_diag_d<1>(h, A, what, dst, dtype);
  else if (h->D == 2)
    launch_diag_d<2>(h, A, what, dst, dtype);
  else
    launch_diag_d<3>(h, A, what, dst, dtype);
  GKS_CK(h, cudaGetLastError());
  if (memspace == GKS_MEM_HOST) {
    GKS_CK(h, cudaMemcpyAsync(out, h->staging, bytes, cudaMemcpyDeviceToHost, h->stream));
    GKS_CK(h, cudaStreamSynchronize(h->stream));
  }
  return GKS_OK;
}

gks_status gks_get_rarefaction(gks_handle* h, void* eps_out, int memspace, int dtype) {
  return get_diag(h, 1, eps_out, memspace, dtype);
}

gks_status gks_get_tau_turb(gks_handle* h, void* tau_out, int memspace, int dtype) {
  return get_diag(h, 0, tau_out, memspace, dtype);
}

gks_status gks_set_nodes(gks_handle* h, const double* nodes, int memspace) {
  if (!h || !nodes) return fail(h, GKS_EINVAL, "null argument");
  if (memspace != GKS_MEM_HOST && memspace != GKS_MEM_DEVICE) return fail(h, GKS_EINVAL, "memspace");
  if (h->D != 2) return fail(h, GKS_EUNSUPPORTED, "curvilinear grids are built in 2D");
  if (h->base.g.rar && h->prec == PREC_F32D)
    return fail(h, GKS_EUNSUPPORTED, "the rarefaction option on body-fitted grids is built for GKS_FP64 and GKS_FP32");
  DeviceGuard dg(h->dev);
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  free_curv(h);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  const int n0 = h->n[0], n1 = h->n[1];
  CurvGeom& G = h->cg;
  G.nf[0] = (long)(n0 + 1) * n1;
  G.nf[1] = (long)n0 * (n1 + 1);
  const size_t rb = arith_bytes(h->prec);
  bool ok = true;
  auto alloc = [&](void** p, size_t b) {
    if (ok && cudaMalloc(p, b) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      ok = false;
    }
  };
  for (int a = 0; a < 2; ++a) {
    alloc(&G.face[a], rb * 8 * G.nf[a]);
    alloc(&G.tang[a], rb * 4 * G.nf[a]);
    alloc(&G.flux[a], rb * 4 * G.nf[a]);
  }
  alloc(&G.iarea, rb * h->ncell);
  alloc((void**)&G.area, sizeof(double) * h->ncell);
  alloc(&G.tau, rb * h->ncell);
  if (!ok) {
    free_curv(h);
    return fail(h, GKS_ENOMEM, "curvilinear grid allocation failed");
  }
  const size_t nb = sizeof(double) * 2 * (size_t)(n0 + 1) * (n1 + 1);
  gks_status st = ensure_staging(h, nb + 16);
  if (st) {
    free_curv(h);
    return st;
  }
  const double* src = nodes;
  if (memspace == GKS_MEM_HOST) {
    GKS_CK(h, cudaMemcpyAsync(h->staging, nodes, nb, cudaMemcpyHostToDevice, h->stream));
    src = (const double*)h->staging;
  }
  int* bad_dev = (int*)((char*)h->staging + ((nb + 7) / 8) * 8);
  GKS_CK(h, cudaMemsetAsync(bad_dev, 0, sizeof(int), h->stream));
  const bool periodic[2] = {h->base.g.bc[0][0] == GKS_BC_PERIODIC, h->base.g.bc[1][0] == GKS_BC_PERIODIC};
  cudaError_t e = curv_metrics(src, n0, n1, periodic, h->base.g.wake_cut, h->prec, G, bad_dev, h->stream);
  if (e != cudaSuccess) {
    free_curv(h);
    return cuda_fail(h, e, "curvilinear metrics");
  }
  int bad_host = 0;
  GKS_CK(h, cudaMemcpyAsync(&bad_host, bad_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  if (bad_host) {
    free_curv(h);
    return fail(h, GKS_EINVAL, "a cell is not a convex counter-clockwise quadrilateral");
  }
  h->curv = true;
  h->tile_variant = 0;
  h->tuned = false;  // the tile shape of the curvilinear step is chosen at the first step
  if (h->has_state) {
    GKS_CK(h, cudaMemsetAsync(&h->ctrl->rate[h->step % 3], 0, sizeof(unsigned long long), h->stream));
    return launch_rate(h);
  }
  return GKS_OK;
}

gks_status gks_enable_timing(gks_handle* h, int enable) {
  if (!h) return GKS_EINVAL;
  h->timing = enable != 0;
  return GKS_OK;
}

gks_status gks_kernel_time(gks_handle* h, double* ms_total, long long* launches) {
  if (!h) return GKS_EINVAL;
  DeviceGuard dg(h->dev);
  GKS_CK(h, cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i + 1 < h->ev.size(); i += 2) {
    float ms = 0.0f;
    GKS_CK(h, cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
    h->ms_total += ms;
    h->launches += 1;
  }
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
  if (ms_total) *ms_total = h->ms_total;
  if (launches) *launches = h->launches;
  h->ms_total = 0.0;
  h->launches = 0;
  return GKS_OK;
}

gks_status gks_tile_shape(gks_handle* h, int* variant, int* tx, int* ty, int* tz) {
  if (!h) return GKS_EINVAL;
  int t[3];
  if (h->curv) {
    curv_tile_shape(h->tile_variant, &t[0], &t[1]);
    t[2] = 1;
  } else {
    tile_shape(h->D, h->tile_variant, &t[0], &t[1], &t[2]);
  }
  if (variant) *variant = h->tile_variant;
  if (tx) *tx = t[0];
  if (ty) *ty = t[1];
  if (tz) *tz = t[2];
  return GKS_OK;
}

int gks_face_record_len(int dim) {
  if (dim < 1 || dim > 3) return -1;
  const int nv = dim + 2;
  return 6 * nv + 2 * (dim - 1) * nv + 3;
}

gks_status gks_face_flux(int dim, int precision, int expand, int abar_mode, int rarefaction, double gamma, double mu,
                         double C_a, double dt, const double* faces, long nfaces, double* F_out, double* tau_out,
                         void* cuda_stream) {
  if (dim < 1 || dim > 3 || !faces || !F_out || nfaces < 0) return GKS_EINVAL;
  if (precision != GKS_FP64 && precision != GKS_FP32) return GKS_EINVAL;
  if (rarefaction != GKS_RAR_DT && rarefaction != GKS_RAR_TAUHAT) return GKS_EINVAL;
  if (!(gamma > 1.0) || 2.0 / (gamma - 1.0) - dim < 0.0 || !(dt > 0.0)) return GKS_EINVAL;
  if (nfaces == 0) return GKS_OK;
  launch_face_flux(dim, precision == GKS_FP64 ? 0 : 1, dim > 1 && expand == GKS_EXPAND_MULTID,
                   abar_mode == GKS_ABAR_T0, rarefaction == GKS_RAR_TAUHAT, gamma, mu, C_a, dt, faces, nfaces, F_out,
                   tau_out, (cudaStream_t)cuda_stream);
  if (cudaGetLastError() != cudaSuccess) return GKS_ECUDA;
  return GKS_OK;
}

}  // extern "C"
