// Fused time step of the gas-kinetic finite-volume scheme on a structured grid.
//
// One launch advances the whole grid by one step.  Each CTA owns a tile of cells; it stages the
// tile with two halo layers in shared memory (boundary cells are resolved while loading: periodic,
// transmissive/outflow, isothermal no-slip wall, Dirichlet), computes the turbulent relaxation
// time of the tile and its first halo ring (Eqs. tautchen, tautchenadjusted, tauttrivial), the
// MUSCL-reconstructed face states and the time-integrated flux of every face of the tile
// (Eq. fluxesf), then updates its cells W <- W - sum_d dF_d / dx_d and folds the CFL rate of the
// new state into the control block for the next step.  Faces on a tile border are evaluated by
// both neighbouring tiles (same inputs, same result), so no flux leaves the CTA.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "gks_flux.cuh"

namespace gks {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_WALL = 2, BC_DIRICHLET = 3, BC_OUTFLOW = 4 };
enum { TURB_NONE = 0, TURB_MUT = 1, TURB_KEPS = 2, TURB_KOMEGA = 3 };
// arithmetic / storage of a run
enum { PREC_F64 = 0,    // double flux, double state
       PREC_F32 = 1,    // float flux, state as a pair of floats (hi + lo)
       PREC_F32D = 2 };  // float flux, double state

constexpr int kThreads = 256;   // threads of the auxiliary kernels and of tile variant 0
constexpr int kWG = 3;          // ghost entries per side of the cell-width arrays (index cell + kWG)
// face reconstruction: second-order MUSCL (limited slopes), third-order MUSCL (kappa = 1/3),
// fifth-order WENO (three halo layers)
enum { RECON_MUSCL2 = 0, RECON_MUSCL3 = 1, RECON_WENO5 = 2 };
__host__ __device__ constexpr int halo_of(int recon) { return recon == RECON_WENO5 ? 3 : 2; }
constexpr int kMaxWarps = 16;   // largest CTA of any tile variant: 512 threads

// Tile of cells owned by one CTA (variant 0 is the default; 2D has four more, chosen by the
// autotuner).  Each 2D shape makes the face count of a tile fill whole rounds of its threads:
// 32x15: 1007 faces / 256 threads, 64x7: 967 / 256, 32x31: 2047 / 512.
template <int D, int V = 0> struct Tile;
template <> struct Tile<1, 0> { static constexpr int X = 256, Y = 1, Z = 1, T = 256; };
// narrow 1D tiles spread small grids over more SMs: 31 cells (32 faces) per warp, 63 per two warps
template <> struct Tile<1, 1> { static constexpr int X = 31, Y = 1, Z = 1, T = 32; };
template <> struct Tile<1, 2> { static constexpr int X = 63, Y = 1, Z = 1, T = 64; };
template <> struct Tile<2, 0> { static constexpr int X = 32, Y = 15, Z = 1, T = 256; };
template <> struct Tile<2, 1> { static constexpr int X = 64, Y = 7, Z = 1, T = 256; };
template <> struct Tile<2, 2> { static constexpr int X = 32, Y = 31, Z = 1, T = 512; };
// 32x27: 1787 faces in 7 rounds of 256 (99.7%), 1216 tiles on a 1024^2 grid = 4 full waves of two
// CTAs per SM; 32x18: 1202 faces in 5 rounds (94%), 1824 tiles = 6 full waves
template <> struct Tile<2, 3> { static constexpr int X = 32, Y = 27, Z = 1, T = 256; };
template <> struct Tile<2, 4> { static constexpr int X = 32, Y = 18, Z = 1, T = 256; };
// 64x27 on one 512-thread CTA per SM: 3547 faces in 7 rounds (99%), 608 tiles = 4 full waves; all
// warps of an SM work in the same phase of one tile
template <> struct Tile<2, 5> { static constexpr int X = 64, Y = 27, Z = 1, T = 512; };
// Paired tiles (FP32 forms): each thread evaluates two faces at once with the paired FP32 instructions
// (two operations per issue slot); the face body then needs up to 255 registers, so 32x27 runs 128
// threads (two CTAs per SM) and 64x27 256 threads (one CTA per SM), both in 7 rounds of face pairs.
template <> struct Tile<2, 6> { static constexpr int X = 32, Y = 27, Z = 1, T = 128; };
template <> struct Tile<2, 7> { static constexpr int X = 64, Y = 27, Z = 1, T = 256; };
template <> struct Tile<3, 3> { static constexpr int X = 16, Y = 8, Z = 2, T = 128; };
// 32 x 21 on two 256-thread CTAs per SM: 1397 faces in 6 rounds; 1024 x 384 gives 608 tiles, two
// full waves on 152 SMs
template <> struct Tile<2, 8> { static constexpr int X = 32, Y = 21, Z = 1, T = 256; };
template <int D, int V> __host__ __device__ constexpr bool paired_tile() {
  return (D == 2 && (V == 6 || V == 7)) || (D == 3 && V == 3);
}
template <> struct Tile<3, 0> { static constexpr int X = 16, Y = 8, Z = 4, T = 256; };
// 256-cell 3D tiles with the per-cell slope table (two CTAs per SM): 944 and 896 faces
template <> struct Tile<3, 1> { static constexpr int X = 16, Y = 8, Z = 2, T = 256; };
template <> struct Tile<3, 2> { static constexpr int X = 8, Y = 8, Z = 4, T = 256; };

template <int D, int V = 0, int H = 2> struct TileGeom {
  static constexpr int X = Tile<D, V>::X, Y = Tile<D, V>::Y, Z = Tile<D, V>::Z, T = Tile<D, V>::T;
  static constexpr int HALO = H;  // halo layers staged around the tile
  static constexpr int HX = X + 2 * H, HY = D >= 2 ? Y + 2 * H : 1, HZ = D >= 3 ? Z + 2 * H : 1;
  static constexpr int NH = HX * HY * HZ;  // cells with halo
  static constexpr int RX = X + 2, RY = D >= 2 ? Y + 2 : 1, RZ = D >= 3 ? Z + 2 : 1;
  static constexpr int NR = RX * RY * RZ;  // cells with the first halo ring
  static constexpr int NC = X * Y * Z;
  static constexpr int NFX = (X + 1) * Y * Z;
  static constexpr int NFY = D >= 2 ? X * (Y + 1) * Z : 0;
  static constexpr int NFZ = D >= 3 ? X * Y * (Z + 1) : 0;
  static constexpr int NF = NFX + NFY + NFZ;
  static constexpr int nv = D + 2;
  // Shared memory, in elements of the arithmetic type R: the staged state [nv][NH], tau_t of the
  // ring [NR], the width tables 4 (HX + HY + HZ), then (from a 16-byte boundary) the face fluxes
  // [nv][NF] and, with pre, the limited slopes of the first halo ring per cell and axis [D][nv][NR];
  // then the two turbulence fields of the ring and, for the float-pair state, the low words of the
  // tile's own cells (staged with the state so that the tile waits on global memory once).
  template <class R> __host__ __device__ static constexpr size_t fs_offset() {
    return ((size_t)nv * NH + NR + 4 * (HX + HY + HZ) + (16 / sizeof(R) - 1)) / (16 / sizeof(R)) * (16 / sizeof(R));
  }
  template <class R> __host__ __device__ static constexpr size_t smem_bytes(bool pre, bool lo) {
    return sizeof(R) * (fs_offset<R>() + (size_t)nv * NF + (pre ? (size_t)D * nv * NR : 0) + 2 * (size_t)NR) +
           (lo ? sizeof(float) * (size_t)nv * NC : 0);
  }
  // The double-state form stages the tile's doubles in the space of the face fluxes and slopes (free
  // until the ring phase) and converts them to float there; true if they fit.
  __host__ __device__ static constexpr bool dstage_fits(bool pre) {
    return sizeof(double) * (size_t)nv * NH <= sizeof(float) * ((size_t)nv * NF + (pre ? (size_t)D * nv * NR : 0));
  }
};

struct Ctrl {
  unsigned long long rate[3];  // bits of a non-negative double: max_cells sum_d (|U_d| + c)/dx_d
  double t[2];
  double dt_fixed, cfl, t_end;
  double last_dt;
  unsigned int status;  // bit 0: non-physical state after an update
  unsigned int pad;
  double l2[5], total[5];
  unsigned long long linf[5];
};

// Gas and model constants in the arithmetic type.
template <class R> struct Consts {
  R gamma, mu, C_mu, beta_star, T_wall, bK, K, C_a, ibK;
};

struct DevGrid {
  int n[3];
  long ncell;
  int bc[3][2];
  const double* w[3];       // cell widths with kWG ghosts per side, index i + kWG
  const double* dir[3][2];  // Dirichlet conservative states, [transverse cell][nv]
  double gamma, bK, K, mu, C_a, T_wall, C_mu, beta_star;
  int turb_model, limiter, abar_t0;
  int turb_cons;  // the turbulence fields hold rho k and rho omega (k-omega transport), not k and omega
  int wake_cut;   // 2D C-grids: the first and last wake_cut cells of the j-lo side form a wake cut
  int rar;        // the rarefaction option (eps = tau/tauhat in the time coefficients): kernels built with RAR
  // the constants above in each arithmetic type, filled by set_consts on the host (kernels read
  // them from the parameter bank instead of converting)
  Consts<float> kf;
  Consts<double> kd;
};

template <class R>
inline void fill_consts(const DevGrid& g, Consts<R>& c) {
  c.gamma = (R)g.gamma;
  c.mu = (R)g.mu;
  c.C_mu = (R)g.C_mu;
  c.beta_star = (R)g.beta_star;
  c.T_wall = (R)g.T_wall;
  c.bK = (R)g.bK;
  c.ibK = (R)(1.0 / g.bK);
  c.K = (R)g.K;
  c.C_a = (R)g.C_a;
}

// Host: derive the per-type constants once the double-precision ones are set.
inline void set_consts(DevGrid& g) {
  fill_consts<float>(g, g.kf);
  fill_consts<double>(g, g.kd);
}

template <class R>
__device__ __forceinline__ Consts<R> make_consts(const DevGrid& g) {
  if constexpr (sizeof(R) == sizeof(float))
    return g.kf;
  else
    return g.kd;
}

struct StepArgs {
  DevGrid g;
  const void* Win;
  void* Wout;
  const float* Win_lo;  // PREC_F32 only
  float* Wout_lo;
  const void* f1;  // turbulence fields in the arithmetic type, or null
  const void* f2;
  Ctrl* ctrl;
  void* mflux[3];  // if set: time-integrated mass flux of every face along each axis, faces j - 1/2
                   // for j = 0 .. n_d (x fastest), in the arithmetic type (k-omega transport input)
  int slot;    // rate slot read by this step (step index mod 3)
  int tslot;   // time slot read by this step (step index mod 2)
  int resid;   // accumulate residual norms in this step
  // k-omega transport fused into the body-fitted step (f1, f2 are then rho k, rho omega): outputs
  // and the closure coefficients (double, and float for the single-precision kernels)
  void* RKout;
  void* RWout;
  double kw_alpha, kw_beta0, kw_sigma, kw_sigma_star, kw_sigma_do, kw_C_lim, kw_omega_floor;
  float kw_falpha, kw_fbeta0, kw_fsigma, kw_fsigma_star, kw_fsigma_do, kw_fC_lim, kw_fomega_floor;
  int kw_sources, kw_diffusion;
};

// Arguments of the k-omega transport step that follows a flow step (closure coefficients in
// double; the kernel converts them to its arithmetic type).
struct KOmegaArgs {
  DevGrid g;
  const void* Win;   // flow state at the start of the step (stored type)
  const void* Wnew;  // flow state after the step: its density scales the omega floor
  const void* RKin;  // rho k, rho omega at the start of the step (arithmetic type)
  const void* RWin;
  void* RKout;
  void* RWout;
  const void* mflux[3];  // the flow step's time-integrated face mass fluxes (StepArgs::mflux)
  const Ctrl* ctrl;      // last_dt: the step's dt
  double alpha, beta0, beta_star, sigma, sigma_star, sigma_do, C_lim, omega_floor;
  float falpha, fbeta0, fbeta_star, fsigma, fsigma_star, fsigma_do, fC_lim, fomega_floor;  // same, float
  int sources, diffusion;
};


template <int PREC> struct PrecT;

// Cell slopes are precomputed in shared memory in 1D, 2D and for the small 3D tiles (variants 1, 2:
// 256 cells); the 15 slopes per ring cell of the 512-cell 3D tile would hold it to one CTA per SM,
// so its faces recompute them (two CTAs per SM in FP32).
template <int D, int PREC, int V = 0> __host__ __device__ constexpr bool pre_slopes() { return D < 3 || V > 0; }

// Axis order of the face frame of a face normal to axis ax: the normal first, then the tangential
// axes in increasing order (entries past D are 0).
template <int D> __host__ __device__ constexpr int face_perm_c(int ax, int k) {
  return k == 0 ? ax : (D == 2 ? (k == 1 ? 1 - ax : 0) : (D == 3 ? (k == 1 ? (ax == 0 ? 1 : 0) : (ax == 2 ? 1 : 2)) : 0));
}
template <> struct PrecT<PREC_F64> { using R = double; using S = double; };
template <> struct PrecT<PREC_F32> { using R = float; using S = float; };
template <> struct PrecT<PREC_F32D> { using R = float; using S = double; };

__device__ __forceinline__ long cell_index(const DevGrid& g, int i, int j, int k) {
  return ((long)k * g.n[1] + j) * g.n[0] + i;
}

// Conversions between the double state and the float arithmetic of the double-state form, on the
// integer pipe: this part converts at the FP64 rate (gks_probe_cvt: about 2 conversions per clock per
// SM, 1/64 of the FP32 rate), while these take about ten full-rate integer instructions.
// d2f rounds toward zero (the FP32 flux inputs carry 2^-23 relative error either way); magnitudes
// below 2^-126 give a signed zero, 2^128 and above, infinities and NaN give NaN (so that a non-physical
// state stays visible).
__device__ __forceinline__ float d2f(double x) {
  const unsigned int H = (unsigned int)__double2hiint(x), L = (unsigned int)__double2loint(x);
  const unsigned int e = (H >> 20) & 0x7ffu;  // biased double exponent
  // bits 29..60 of the double: 23 mantissa bits and the low 9 exponent bits; rebias 1023 -> 127
  unsigned int f = ((__funnelshift_r(L, H, 29) + 0x40000000u) & 0x7fffffffu) | (H & 0x80000000u);
  f = e <= 896u ? (H & 0x80000000u) : f;
  f = e >= 1151u ? 0x7fffffffu : f;
  return __uint_as_float(f);
}
// Exact float -> double (a subnormal float gives a signed zero; infinities and NaN give NaN).
__device__ __forceinline__ double f2d(float x) {
  const unsigned int f = __float_as_uint(x), a = f & 0x7fffffffu, sg = f & 0x80000000u;
  unsigned int H = ((a >> 3) + (896u << 20)) | sg, L = f << 29;
  H = a < 0x00800000u ? sg : H;
  L = a < 0x00800000u ? 0u : L;
  H = a >= 0x7f800000u ? 0x7ff80000u : H;
  return __hiloint2double((int)H, (int)L);
}

// Asynchronous global -> shared copy of one 4- or 8-byte element (cp.async, completed by
// cp_async_wait_all); the thread's registers are not involved, so all of a tile's loads are in
// flight together.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "element copies of 4, 8 or 16 bytes");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (BYTES == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else if (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ bool in_grid(const DevGrid& g, int D, int i, int j, int k) {
  return i >= 0 && i < g.n[0] && (D < 2 || (j >= 0 && j < g.n[1])) && (D < 3 || (k >= 0 && k < g.n[2]));
}

template <class R>
__device__ __forceinline__ R pressure_of(int D, R gamma, const R* w) {
  R q = R(0);
  for (int i = 0; i < D; ++i) q += w[1 + i] * w[1 + i];
  return (gamma - R(1)) * (w[D + 1] - R(0.5) * g_div(q, w[0]));
}

// rho > 0 and p > 0 for a conservative state.  Single precision tests 2 rho (rho E) > |rho U|^2 (the
// same condition once rho > 0, without a quotient); double precision evaluates p as the oracle does.
template <int D, class R>
__device__ __forceinline__ bool physical(R gamma, const R* w) {
  if constexpr (sizeof(R) == sizeof(float)) {
    R q = R(0);
#pragma unroll
    for (int i = 0; i < D; ++i) q += w[1 + i] * w[1 + i];
    return w[0] > R(0) && R(2) * w[0] * w[D + 1] > q;
  } else {
    return w[0] > R(0) && pressure_of<R>(D, gamma, w) > R(0);
  }
}

// Isothermal no-slip wall image: velocity reversed, same pressure, T_g = T_w^2 / T_i (T = p/rho).
template <int D, class R>
__device__ __forceinline__ void wall_image(const Consts<R>& k, R* w) {
  const R gamma = k.gamma, Tw = k.T_wall;
  R U[D], q = R(0);
#pragma unroll
  for (int i = 0; i < D; ++i) U[i] = g_div(w[1 + i], w[0]);
  const R p = pressure_of<R>(D, gamma, w);
  const R Ti = g_div(p, w[0]);
  const R Tg = g_div(Tw * Tw, Ti);
  const R rho = g_div(p, Tg);
  w[0] = rho;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    w[1 + i] = rho * -U[i];
    q += U[i] * U[i];
  }
  w[D + 1] = g_div(p, gamma - R(1)) + R(0.5) * rho * q;
}

template <int D, int PREC>
__device__ __forceinline__ void load_stored(const DevGrid& g, const void* Win, long c, typename PrecT<PREC>::R* out) {
  using S = typename PrecT<PREC>::S;
  using R = typename PrecT<PREC>::R;
  const S* W = (const S*)Win;
#pragma unroll
  for (int v = 0; v < D + 2; ++v) out[v] = (R)W[(long)v * g.ncell + c];
}

// State of cell (i, j, k), possibly outside the grid: ghost cells follow the boundary rules, the
// transform of the last axis applied first.
template <int D, int PREC>
__device__ void load_cell(const DevGrid& g, const void* Win, const Consts<typename PrecT<PREC>::R>& kc, int i, int j,
                          int k, typename PrecT<PREC>::R* out) {
  using R = typename PrecT<PREC>::R;
  int c[3] = {i, j, k}, xf[3] = {0, 0, 0}, side[3] = {0, 0, 0};
  bool inside = true;
  // cells further out than the three ghost layers only feed faces of cells outside the grid
#pragma unroll
  for (int a = 0; a < D; ++a) c[a] = min(max(c[a], -3), g.n[a] + 2);
  int src[3] = {c[0], c[1], c[2]};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int n = g.n[a];
    if (c[a] < 0 || c[a] >= n) {
      inside = false;
      const int s = c[a] < 0 ? 0 : 1;
      side[a] = s;
      const int bc = g.bc[a][s];
      if (bc == BC_PERIODIC) {
        src[a] = s == 0 ? c[a] + n : c[a] - n;
      } else if (bc == BC_WALL) {
        src[a] = s == 0 ? -c[a] - 1 : 2 * n - 1 - c[a];
        xf[a] = 1;
      } else if (bc == BC_DIRICHLET) {
        src[a] = s == 0 ? 0 : n - 1;
        xf[a] = 2;
      } else {
        src[a] = s == 0 ? 0 : n - 1;
      }
    }
  }
  // C-grid wake cut: the cell across it (for a corner, across from the column the i rule picks)
  if (D == 2 && g.wake_cut > 0 && c[1] < 0 && (src[0] < g.wake_cut || src[0] >= g.n[0] - g.wake_cut)) {
    src[0] = g.n[0] - 1 - src[0];
    src[1] = -c[1] - 1;
    xf[1] = 0;
  }
  load_stored<D, PREC>(g, Win, cell_index(g, src[0], src[1], src[2]), out);
  if (inside) return;
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    if (xf[a] == 1) {
      wall_image<D, R>(kc, out);
    } else if (xf[a] == 2) {
      long off = 0, stride = 1;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        if (b == a) continue;
        int cb = b < a ? src[b] : min(max(c[b], 0), g.n[b] - 1);
        off += cb * stride;
        stride *= g.n[b];
      }
      const double* d = g.dir[a][side[a]] + off * (D + 2);
#pragma unroll
      for (int v = 0; v < D + 2; ++v) out[v] = (R)d[v];
    }
  }
}

// A (possibly ghost) cell whose state is a plain copy of one cell of the grid -- in the grid, or a
// ghost cell of periodic, transmissive or outflow sides or across a C-grid wake cut, the same rules as
// load_cell -- gets that cell's index in *src (the copy can then be asynchronous); false for ghost
// cells that a wall image or Dirichlet data transform.
__device__ __forceinline__ bool plain_source(const DevGrid& g, int D, int i, int j, int k, long* src) {
  int c[3] = {i, j, k}, xf[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) c[a] = min(max(c[a], -3), g.n[a] + 2);
  int s[3] = {c[0], c[1], c[2]};
  for (int a = 0; a < D; ++a) {
    const int n = g.n[a];
    if (c[a] < 0 || c[a] >= n) {
      const int sd = c[a] < 0 ? 0 : 1;
      const int bc = g.bc[a][sd];
      if (bc == BC_PERIODIC) {
        s[a] = sd == 0 ? c[a] + n : c[a] - n;
      } else if (bc == BC_WALL) {
        s[a] = sd == 0 ? -c[a] - 1 : 2 * n - 1 - c[a];
        xf[a] = 1;
      } else {
        s[a] = sd == 0 ? 0 : n - 1;
        if (bc == BC_DIRICHLET) xf[a] = 1;
      }
    }
  }
  if (D == 2 && g.wake_cut > 0 && c[1] < 0 && (s[0] < g.wake_cut || s[0] >= g.n[0] - g.wake_cut)) {
    s[0] = g.n[0] - 1 - s[0];
    s[1] = -c[1] - 1;
    xf[1] = 0;
  }
  if (xf[0] || xf[1] || xf[2]) return false;
  *src = cell_index(g, s[0], s[1], s[2]);
  return true;
}

// Cell whose turbulence field value a (possibly ghost) cell takes: periodic axes wrap, other axes
// the nearest interior cell, a C-grid wake cut the cell across the cut.
__device__ __forceinline__ long field_cell(const DevGrid& g, int D, int i, int j, int k) {
  if (D == 2 && g.wake_cut > 0 && j < 0 && i >= 0 && i < g.n[0] && (i < g.wake_cut || i >= g.n[0] - g.wake_cut))
    return cell_index(g, g.n[0] - 1 - i, -j - 1, 0);  // across a C-grid wake cut
  int c[3] = {i, j, k};
  for (int a = 0; a < D; ++a) {
    const int n = g.n[a];
    if (c[a] < 0 || c[a] >= n) {
      if (g.bc[a][0] == BC_PERIODIC)
        c[a] = (c[a] + n) % n;
      else
        c[a] = min(max(c[a], 0), n - 1);
    }
  }
  return cell_index(g, c[0], c[1], c[2]);
}

template <class R>
__device__ __forceinline__ R load_field(const StepArgs& A, const void* f, int D, int i, int j, int k) {
  return ((const R*)f)[field_cell(A.g, D, i, j, k)];
}

// Turbulent part of the relaxation time of one cell (Eqs. tauttrivial, tautchen, tautchenadjusted
// with T = p/rho); S = sqrt(2 S_ij S_ij) from central differences of the velocity.
// igrad[a][p] = 1 / (distance between the centres of halo cells p - 1 and p + 1 along axis a).
template <int D, class R>
__device__ __forceinline__ R tau_turb_cell(int turb_model, bool cons, const Consts<R>& kc, const R* Ws, int stride_v,
                                           int idx, const int* strides, const R* const* igrad, const int* pos,
                                           R f1, R f2) {
  if (turb_model == TURB_NONE) return R(0);
  R w[D + 2];
#pragma unroll
  for (int v = 0; v < D + 2; ++v) w[v] = Ws[v * stride_v + idx];
  if (cons) {  // rho k, rho omega -> k, omega
    f1 = g_div(f1, w[0]);
    f2 = g_div(f2, w[0]);
  }
  const R p = pressure_of<R>(D, kc.gamma, w);
  if (turb_model == TURB_MUT) return g_div(f1, p);
  if (!(f1 > R(0)) || !(f2 > R(0))) return R(0);
  R grad[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int im = idx - strides[a], ip = idx + strides[a];
    const R id = igrad[a][pos[a]];
    const R irm = g_rcp(Ws[im]), irp = g_rcp(Ws[ip]);
#pragma unroll
    for (int b = 0; b < D; ++b)
      grad[a][b] = (Ws[(1 + b) * stride_v + ip] * irp - Ws[(1 + b) * stride_v + im] * irm) * id;
  }
  R s2 = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const R sab = R(0.5) * (grad[a][b] + grad[b][a]);
      s2 += sab * sab;
    }
  const R S = g_sqrt(R(2) * s2);
  R nu, eta;
  if (turb_model == TURB_KEPS) {
    nu = g_div(kc.C_mu * f1 * f1, f2);
    eta = g_div(S * f1, f2);
  } else {
    nu = g_div(f1, f2);
    eta = g_div(S, kc.beta_star * f2);
  }
  return g_div(w[0] * nu, p * g_sqrt(R(1) + eta * eta));
}

// The k-epsilon / k-omega branch of tau_turb_cell written without early returns, so that several
// cells can be evaluated side by side: the same arithmetic, with the non-positive k or
// epsilon|omega case selected to zero at the end.
template <int D, class R>
__device__ __forceinline__ R tau_turb_two_eq(bool keps, bool cons, const Consts<R>& kc, const R* Ws, int stride_v,
                                             int idx, const int* strides, const R* const* igrad, const int* pos,
                                             R f1, R f2) {
  R w[D + 2];
#pragma unroll
  for (int v = 0; v < D + 2; ++v) w[v] = Ws[v * stride_v + idx];
  if (cons) {  // rho k, rho omega -> k, omega
    f1 = g_div(f1, w[0]);
    f2 = g_div(f2, w[0]);
  }
  const R p = pressure_of<R>(D, kc.gamma, w);
  R grad[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int im = idx - strides[a], ip = idx + strides[a];
    const R id = igrad[a][pos[a]];
    const R irm = g_rcp(Ws[im]), irp = g_rcp(Ws[ip]);
#pragma unroll
    for (int b = 0; b < D; ++b)
      grad[a][b] = (Ws[(1 + b) * stride_v + ip] * irp - Ws[(1 + b) * stride_v + im] * irm) * id;
  }
  R s2 = R(0);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const R sab = R(0.5) * (grad[a][b] + grad[b][a]);
      s2 += sab * sab;
    }
  const R S = g_sqrt(R(2) * s2);
  // k-epsilon: nu = C_mu k^2/eps, eta = S k/eps; k-omega: nu = k/omega, eta = S/(beta* omega)
  const R nu = keps ? g_div(kc.C_mu * f1 * f1, f2) : g_div(f1, f2);
  const R eta = keps ? g_div(S * f1, f2) : g_div(S, kc.beta_star * f2);
  const R t = g_div(w[0] * nu, p * g_sqrt(R(1) + eta * eta));
  return (f1 > R(0) && f2 > R(0)) ? t : R(0);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <class R>
__device__ __forceinline__ R block_max(R v, R* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : R(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

// Block maximum of a non-negative CFL rate, returned (in thread 0) as the bit pattern of the double
// that atomicMax folds into the control block.  Single precision reduces in float; double precision
// reduces the bit patterns as unsigned integers (non-negative doubles order like their bits), which
// keeps the reduction off the FP64 pipe.  A NaN rate counts as zero, as fmax would treat it.
template <class R>
__device__ __forceinline__ unsigned long long block_max_rate(R v, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (sizeof(R) == sizeof(float)) {
    float* rf = (float*)red;
    float m = v == v ? (float)v : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) rf[warp] = m;
    __syncthreads();
    if (warp == 0) {
      m = lane < (int)(blockDim.x >> 5) ? rf[lane] : 0.0f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    return (unsigned long long)__double_as_longlong((double)m);
  } else {
    unsigned long long* ru = (unsigned long long*)red;
    unsigned long long m = v == v ? (unsigned long long)__double_as_longlong((double)v) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
      m = t > m ? t : m;
    }
    __syncthreads();
    if (lane == 0) ru[warp] = m;
    __syncthreads();
    if (warp == 0) {
      m = lane < (int)(blockDim.x >> 5) ? ru[lane] : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
      }
    }
    return m;
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// CFL rate of one cell: sum_d (|U_d| + c) / dx_d, c = sqrt(gamma p / rho).
template <int D, class R>
__device__ __forceinline__ R cell_rate(const R* w, R gamma, const R* h) {
  const R p = pressure_of<R>(D, gamma, w);
  const R cs = g_sqrt(g_div(gamma * p, w[0]));
  R r = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) r += g_div(g_abs(g_div(w[1 + d], w[0])) + cs, h[d]);
  return r;
}

// The same rate from the inverse cell widths, with one reciprocal of the density and one square root.
template <int D, class R>
__device__ __forceinline__ R cell_rate_inv(const R* w, R gamma, const R* ih) {
  const R ir = g_rcp(w[0]);
  const R cs = g_sqrt(gamma * pressure_of<R>(D, gamma, w) * ir);
  R r = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) r += (g_abs(w[1 + d] * ir) + cs) * ih[d];
  return r;
}

// Ring cells that the faces of a tile read: in 3D the tile and its six face layers (the edge and
// corner cells of the ring box border no face of the tile), otherwise the whole ring box.  ring_used
// is their number, ring_slot(s) the ring index of the s-th (tile cells first, then the x, y and z
// layers, low side before high side).
template <int D, class G> __host__ __device__ constexpr int ring_used() {
  return D == 3 ? G::X * G::Y * G::Z + 2 * (G::Y * G::Z + G::X * G::Z + G::X * G::Y) : G::NR;
}
template <int D, class G> __host__ __device__ __forceinline__ int ring_slot(int s) {
  if constexpr (D < 3) {
    return s;
  } else {
    constexpr int X = G::X, Y = G::Y, Z = G::Z;
    int ri, rj, rk;
    if (s < X * Y * Z) {
      ri = s % X + 1;
      rj = (s / X) % Y + 1;
      rk = s / (X * Y) + 1;
    } else if (s < X * Y * Z + 2 * Y * Z) {
      const int t = s - X * Y * Z;
      ri = t < Y * Z ? 0 : X + 1;
      rj = (t % (Y * Z)) % Y + 1;
      rk = (t % (Y * Z)) / Y + 1;
    } else if (s < X * Y * Z + 2 * Y * Z + 2 * X * Z) {
      const int t = s - X * Y * Z - 2 * Y * Z;
      rj = t < X * Z ? 0 : Y + 1;
      ri = (t % (X * Z)) % X + 1;
      rk = (t % (X * Z)) / X + 1;
    } else {
      const int t = s - X * Y * Z - 2 * Y * Z - 2 * X * Z;
      rk = t < X * Y ? 0 : Z + 1;
      ri = (t % (X * Y)) % X + 1;
      rj = (t % (X * Y)) / X + 1;
    }
    return (rk * G::RY + rj) * G::RX + ri;
  }
}

// Turbulent relaxation time (Eqs. tautchen, tautchenadjusted, tauttrivial) and, with PRE, the
// limited MUSCL slope along each axis of every cell of the tile's first halo ring.  A function of its
// own (not inlined) so that its register allocation is separate from the face loop's: each thread
// evaluates its ring cells tid + q T side by side, results in registers and stored afterwards, so
// that their shared-memory and MUFU latencies overlap.  A slot past the ring repeats the last cell
// and is not stored.  The model and limiter branches are taken once, outside the cells.
template <int D, int PREC, int V, int H>
__device__ __noinline__ void ring_phase(const Consts<typename PrecT<PREC>::R> kc, int turb_model, bool cons, int lim,
                                        const typename PrecT<PREC>::R* Ws, const typename PrecT<PREC>::R* Fl,
                                        typename PrecT<PREC>::R* taus, typename PrecT<PREC>::R* Ss,
                                        const typename PrecT<PREC>::R* icx, const typename PrecT<PREC>::R* icy,
                                        const typename PrecT<PREC>::R* icz, const typename PrecT<PREC>::R* igx,
                                        const typename PrecT<PREC>::R* igy, const typename PrecT<PREC>::R* igz) {
  using R = typename PrecT<PREC>::R;
  using G = TileGeom<D, V, H>;
  constexpr int kThreads = G::T, nv = D + 2, HX = G::HX, HY = G::HY;
  constexpr bool PRE = pre_slopes<D, PREC, V>();
  const int tid = threadIdx.x;
  const int strides[3] = {1, HX, HX * HY};
  const R* igrad[3] = {igx, igy, igz};
  const R* icent[3] = {icx, icy, icz};
  constexpr int NU = ring_used<D, G>();
  constexpr int NIT = (NU + kThreads - 1) / kThreads;
  // groups of at most four ring cells per thread, as even as the count allows (5 -> 3 + 3, not 4 + 4)
  constexpr int GRP = D == 3 ? 2 : (NIT + (NIT + 3) / 4 - 1) / ((NIT + 3) / 4);
  constexpr int NS = PRE ? D * nv : 1;
  auto ring = [&](auto two_eq_tag, auto lim_tag, auto keps_tag) {
    constexpr bool TWO_EQ = decltype(two_eq_tag)::value;
    constexpr int LIM = decltype(lim_tag)::value;
    constexpr bool KEPS = decltype(keps_tag)::value;
    // single precision, van Leer: the slopes along x and y of each variable limited together on the
    // paired FP32 instructions (reciprocals per lane)
    constexpr bool PAIRXY = std::is_same<R, float>::value && D >= 2 && LIM == LIM_VANLEER;
    (void)LIM;
    for (int i0 = 0; i0 < NIT; i0 += GRP) {
      R tv[GRP], sv[GRP][NS];
      (void)sv;
#pragma unroll
      for (int q = 0; q < GRP; ++q) {
        const int l = ring_slot<D, G>(min(tid + (i0 + q) * kThreads, NU - 1));
        const int ri = l % G::RX, rj = (l / G::RX) % G::RY, rk = l / (G::RX * G::RY);
        const int hi = ri + H - 1, hj = D >= 2 ? rj + H - 1 : 0, hk = D >= 3 ? rk + H - 1 : 0;
        const int idx = (hk * HY + hj) * HX + hi;
        const int pos[3] = {hi, hj, hk};
        if constexpr (TWO_EQ)
          tv[q] = tau_turb_two_eq<D, R>(KEPS, cons, kc, Ws, G::NH, idx, strides, igrad, pos, Fl[l],
                                        Fl[G::NR + l]);
        else
          tv[q] = tau_turb_cell<D, R>(turb_model, cons, kc, Ws, G::NH, idx, strides, igrad, pos,
                                      turb_model == TURB_NONE ? R(0) : Fl[l], R(0));
        if constexpr (PRE && PAIRXY) {
          const F2 im2(icent[0][pos[0]], icent[1][pos[1]]), ip2(icent[0][pos[0] + 1], icent[1][pos[1] + 1]);
#pragma unroll
          for (int v = 0; v < nv; ++v) {
            const R* pc = Ws + v * G::NH + idx;
            const F2 c(pc[0]);
            const F2 dm = F2((c - F2(pc[-strides[0]], pc[-strides[1]])) * im2);
            const F2 dp = F2((F2(pc[strides[0]], pc[strides[1]]) - c) * ip2);
            const F2 ab = F2(dm * dp), den = dm + dp;
            const F2 lim = F2((ab + ab) * g_rcp(den));
            sv[q][v] = ab.v.x > 0.0f ? lim.v.x : 0.0f;
            sv[q][nv + v] = ab.v.y > 0.0f ? lim.v.y : 0.0f;
          }
          if constexpr (D == 3) {
            const R im = icent[2][pos[2]], ip = icent[2][pos[2] + 1];
#pragma unroll
            for (int v = 0; v < nv; ++v) {
              const R* pc = Ws + v * G::NH + idx;
              sv[q][2 * nv + v] = limiter<R>(LIM, (pc[0] - pc[-strides[2]]) * im, (pc[strides[2]] - pc[0]) * ip);
            }
          }
        } else if constexpr (PRE) {
          // slope along each axis: normal slope of the faces along that axis, tangential slope of
          // the faces along the others
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const R im = icent[a][pos[a]], ip = icent[a][pos[a] + 1];
#pragma unroll
            for (int v = 0; v < nv; ++v) {
              const R* pc = Ws + v * G::NH + idx;
              sv[q][a * nv + v] = limiter<R>(LIM, (pc[0] - pc[-strides[a]]) * im, (pc[strides[a]] - pc[0]) * ip);
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < GRP; ++q) {
        const int su = tid + (i0 + q) * kThreads;
        if (i0 + q >= NIT || su >= NU) continue;
        const int l = ring_slot<D, G>(su);
        taus[l] = tv[q];
        if constexpr (PRE) {
#pragma unroll
          for (int j = 0; j < NS; ++j) Ss[j * G::NR + l] = sv[q][j];
        }
      }
    }
  };
  using T1 = std::integral_constant<bool, true>;
  using T0 = std::integral_constant<bool, false>;
  using LV = std::integral_constant<int, LIM_VANLEER>;
  using LM = std::integral_constant<int, LIM_MINMOD>;
  const bool two_eq = turb_model == TURB_KEPS || turb_model == TURB_KOMEGA;
  const bool keps = turb_model == TURB_KEPS;
  if (lim == LIM_VANLEER) {
    if (two_eq && keps) ring(T1{}, LV{}, T1{}); else if (two_eq) ring(T1{}, LV{}, T0{}); else ring(T0{}, LV{}, T0{});
  } else {
    if (two_eq && keps) ring(T1{}, LM{}, T1{}); else if (two_eq) ring(T1{}, LM{}, T0{}); else ring(T0{}, LM{}, T0{});
  }
}

// One tile of one step: every thread of the CTA calls it with the same arguments.  RAR: the time
// coefficients of the faces take the degree of rarefaction tau/tauhat (gks_turb.rarefaction).
template <int D, int PREC, bool MULTID, int V = 0, int RECON = RECON_MUSCL2, bool RAR = false>
__device__ __forceinline__ void step_tile(const StepArgs& A, const int b) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  constexpr int H = halo_of(RECON);
  using G = TileGeom<D, V, H>;
  constexpr int kThreads = G::T;
  constexpr int nv = D + 2;
  constexpr int X = G::X, Y = G::Y, Z = G::Z, HX = G::HX, HY = G::HY, HZ = G::HZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* Ws = (R*)smem_raw;                    // [nv][HZ][HY][HX]
  constexpr bool PRE = pre_slopes<D, PREC, V>();
  constexpr bool PAIR = paired_tile<D, V>() && std::is_same<R, float>::value && RECON == RECON_MUSCL2 && !RAR;
  R* taus = Ws + (size_t)nv * G::NH;       // [RZ][RY][RX]
  R* wsx = taus + G::NR;                   // widths with halo
  R* wsy = wsx + HX;
  R* wsz = wsy + HY;
  R* icx = wsz + HZ;  // 1 / centre distance between halo cells p - 1 and p, per axis
  R* icy = icx + HX;
  R* icz = icy + HY;
  R* igx = icz + HZ;  // 1 / (distance between the centres of p - 1 and p + 1), per axis
  R* igy = igx + HX;
  R* igz = igy + HY;
  R* iwx = igz + HZ;  // 1 / width, per axis
  R* iwy = iwx + HX;
  R* iwz = iwy + HY;
  R* Fs = Ws + G::template fs_offset<R>();  // [nv][NF], 8-byte aligned
  R* Ss = Fs + (size_t)nv * G::NF;          // PRE: [D][nv][NR] limited slopes of the ring cells along each axis
  R* Fl = Ss + (PRE ? (size_t)D * nv * G::NR : 0);  // [2][NR] turbulence fields of the ring cells
  float* Lo = (float*)(Fl + 2 * G::NR);             // PREC_F32: [nv][NC] low words of the tile's cells
  // the stored type is the arithmetic type (FP64, FP32 pair): cells that are plain copies of grid
  // cells are copied as they are
  constexpr bool ASYNC = sizeof(S) == sizeof(R);
  // double state, float arithmetic: the doubles are copied to the flux/slope space [nv][NH] and
  // converted to float once the copies have landed
  constexpr bool DSTAGE = PREC == PREC_F32D && G::dstage_fits(PRE);
  double* Wd = (double*)Fs;
  __shared__ double red[kMaxWarps];

  const DevGrid& g = A.g;
  const int tiles_x = (g.n[0] + X - 1) / X;
  const int tiles_y = D >= 2 ? (g.n[1] + Y - 1) / Y : 1;
  const int ox = (b % tiles_x) * X;
  const int oy = D >= 2 ? ((b / tiles_x) % tiles_y) * Y : 0;
  const int oz = D >= 3 ? (b / (tiles_x * tiles_y)) * Z : 0;
  const int tid = threadIdx.x;
  const Consts<R> kc = make_consts<R>(g);
  __shared__ R s_dtr;   // the time step in the arithmetic type, converted once per CTA
  __shared__ int s_end;  // the time step is zero (t_end reached)
  __shared__ double s_dt;

  // ---- stage the tile with two halo layers, the ring's turbulence fields and the low words ------
  // In-grid cells are copied asynchronously; ghost cells are resolved by the boundary rules.  A tile
  // whose halo lies inside the grid copies two cells along x per instruction (both elements of a
  // pair are in-grid and adjacent in memory; the pair starts on an even cell, hence on a boundary of
  // twice the element size, when the halo origin, the row length and the state pointer allow it).
  // The widths of this thread's width-table entry (threads 0 .. HX + HY + HZ - 1) and the control
  // words of the time step (one thread without a table entry) are loaded before the copies are
  // issued, so that their memory latency overlaps the copies instead of following them.
  constexpr bool WT1 = HX + HY + HZ < kThreads;  // at most one table entry per thread
  constexpr int kDtThread = WT1 ? kThreads - 1 : 0;
  double wtab[3] = {1.0, 1.0, 1.0};
  if constexpr (WT1) {
    if (tid < HX + HY + HZ) {
      const int a = tid < HX ? 0 : (tid < HX + HY ? 1 : 2);
      const int p = a == 0 ? tid : (a == 1 ? tid - HX : tid - HX - HY);
      if (a < D) {
        const int o = a == 0 ? ox : (a == 1 ? oy : oz), top = g.n[a] + 2 * kWG - 1;
        const int iw = o + p - H + kWG;
        wtab[0] = g.w[a][min(max(iw - 1, 0), top)];
        wtab[1] = g.w[a][min(max(iw, 0), top)];
        wtab[2] = g.w[a][min(max(iw + 1, 0), top)];
      }
    }
  }
  double c_dtf = 0.0, c_cfl = 0.0, c_tend = 0.0, c_t = 0.0;
  unsigned long long c_rate = 0ull;
  if (tid == kDtThread) {
    const Ctrl* c = A.ctrl;
    c_dtf = c->dt_fixed;
    c_cfl = c->cfl;
    c_tend = c->t_end;
    c_t = c->t[A.tslot];
    c_rate = c->rate[A.slot];
  }
  constexpr bool PAIRCOPY = (ASYNC || DSTAGE) && HX % 2 == 0;
  const bool inner = ox >= H && ox + X + H <= g.n[0] && (D < 2 || (oy >= H && oy + Y + H <= g.n[1])) &&
                     (D < 3 || (oz >= H && oz + Z + H <= g.n[2]));
  const bool pairs = PAIRCOPY && inner && (ox - H) % 2 == 0 && g.n[0] % 2 == 0 &&
                     ((size_t)A.Win % (2 * sizeof(S))) == 0;
  if (pairs) {
    for (int l2 = tid; l2 < G::NH / 2; l2 += kThreads) {
      const int l = 2 * l2;
      const int hi = l % HX, hj = (l / HX) % HY, hk = l / (HX * HY);
      const S* src = (const S*)A.Win + cell_index(g, ox + hi - H, D >= 2 ? oy + hj - H : 0, D >= 3 ? oz + hk - H : 0);
#pragma unroll
      for (int v = 0; v < nv; ++v) {
        if constexpr (DSTAGE)
          cp_async<16>(&Wd[v * G::NH + l], src + (long)v * g.ncell);
        else
          cp_async<2 * sizeof(S)>(&Ws[v * G::NH + l], src + (long)v * g.ncell);
      }
    }
  }
  for (int l = pairs ? G::NH : tid; l < G::NH; l += kThreads) {
    const int hi = l % HX, hj = (l / HX) % HY, hk = l / (HX * HY);
    const int gi = ox + hi - H, gj = D >= 2 ? oy + hj - H : 0, gk = D >= 3 ? oz + hk - H : 0;
    long sc;
    const bool plain = (ASYNC || DSTAGE) && plain_source(g, D, gi, gj, gk, &sc);
    if (plain) {
      const S* src = (const S*)A.Win + sc;
      if constexpr (DSTAGE) {
#pragma unroll
        for (int v = 0; v < nv; ++v) cp_async<8>(&Wd[v * G::NH + l], src + (long)v * g.ncell);
      } else {
#pragma unroll
        for (int v = 0; v < nv; ++v) cp_async<sizeof(S)>(&Ws[v * G::NH + l], src + (long)v * g.ncell);
      }
    } else if constexpr (DSTAGE) {
      // wall image or Dirichlet ghost: the boundary rule in double precision, converted with the rest
      double w[nv];
      load_cell<D, PREC_F64>(g, A.Win, g.kd, gi, gj, gk, w);
#pragma unroll
      for (int v = 0; v < nv; ++v) Wd[v * G::NH + l] = w[v];
    } else {
      R w[nv];
      load_cell<D, PREC>(g, A.Win, kc, gi, gj, gk, w);
#pragma unroll
      for (int v = 0; v < nv; ++v) Ws[v * G::NH + l] = w[v];
    }
  }
  if (g.turb_model != TURB_NONE) {
    const bool two = g.turb_model != TURB_MUT;
    for (int l = tid; l < G::NR; l += kThreads) {
      const int ri = l % G::RX, rj = (l / G::RX) % G::RY, rk = l / (G::RX * G::RY);
      const int gi = ox + ri - 1, gj = D >= 2 ? oy + rj - 1 : 0, gk = D >= 3 ? oz + rk - 1 : 0;
      if (in_grid(g, D, gi, gj, gk)) {
        const long c = cell_index(g, gi, gj, gk);
        cp_async<sizeof(R)>(&Fl[l], (const R*)A.f1 + c);
        if (two) cp_async<sizeof(R)>(&Fl[G::NR + l], (const R*)A.f2 + c);
      } else {
        R v1 = load_field<R>(A, A.f1, D, gi, gj, gk), v2 = two ? load_field<R>(A, A.f2, D, gi, gj, gk) : R(0);
        if (g.turb_cons) {
          // a ghost cell takes k and omega of its source cell; the ring phase divides rho k, rho omega
          // by this cell's own (boundary-rule) density, so carry the ratio of the two densities
          R wg[nv];
          load_cell<D, PREC>(g, A.Win, kc, gi, gj, gk, wg);
          const R sc = g_div(wg[0], (R)((const S*)A.Win)[field_cell(g, D, gi, gj, gk)]);
          v1 *= sc;
          v2 *= sc;
        }
        Fl[l] = v1;
        if (two) Fl[G::NR + l] = v2;
      }
    }
  }
  if (PREC == PREC_F32) {
    for (int l = tid; l < G::NC; l += kThreads) {
      const int li = l % X, lj = (l / X) % Y, lk = l / (X * Y);
      const int gi = ox + li, gj = oy + lj, gk = oz + lk;
      if (!in_grid(g, D, gi, gj, gk)) continue;
      const float* src = A.Win_lo + cell_index(g, gi, gj, gk);
#pragma unroll
      for (int v = 0; v < nv; ++v) cp_async<4>(&Lo[v * G::NC + l], src + (long)v * g.ncell);
    }
  }
  if constexpr (WT1) {
    // this thread's width-table entry, from the widths loaded before the copies
    if (tid < HX + HY + HZ) {
      const int a = tid < HX ? 0 : (tid < HX + HY ? 1 : 2);
      const int p = a == 0 ? tid : (a == 1 ? tid - HX : tid - HX - HY);
      R* wd = a == 0 ? wsx : (a == 1 ? wsy : wsz);
      R* ic = a == 0 ? icx : (a == 1 ? icy : icz);
      R* ig = a == 0 ? igx : (a == 1 ? igy : igz);
      R* iwd = a == 0 ? iwx : (a == 1 ? iwy : iwz);
      const R wm = (R)wtab[0], w0 = (R)wtab[1], wp = (R)wtab[2];
      wd[p] = w0;
      ic[p] = a < D ? g_rcp(R(0.5) * (wm + w0)) : R(1);
      ig[p] = a < D ? g_rcp(R(0.5) * wm + w0 + R(0.5) * wp) : R(1);
      iwd[p] = a < D ? g_rcp(w0) : R(1);
    }
  } else {
    for (int l = tid; l < HX + HY + HZ; l += kThreads) {
      // halo position p is the cell origin + p - H, width index cell + kWG (clamped to the ghosts);
      // the inverse distances make the slope and gradient quotients products
      const int a = l < HX ? 0 : (l < HX + HY ? 1 : 2);
      const int p = a == 0 ? l : (a == 1 ? l - HX : l - HX - HY);
      R* wd = a == 0 ? wsx : (a == 1 ? wsy : wsz);
      R* ic = a == 0 ? icx : (a == 1 ? icy : icz);
      R* ig = a == 0 ? igx : (a == 1 ? igy : igz);
      R* iwd = a == 0 ? iwx : (a == 1 ? iwy : iwz);
      if (a < D) {
        const int o = a == 0 ? ox : (a == 1 ? oy : oz), top = g.n[a] + 2 * kWG - 1;
        const int iw = o + p - H + kWG;
        const R wm = (R)g.w[a][min(max(iw - 1, 0), top)];
        const R w0 = (R)g.w[a][min(max(iw, 0), top)];
        const R wp = (R)g.w[a][min(max(iw + 1, 0), top)];
        wd[p] = w0;
        ic[p] = g_rcp(R(0.5) * (wm + w0));
        ig[p] = g_rcp(R(0.5) * wm + w0 + R(0.5) * wp);
        iwd[p] = g_rcp(w0);
      } else {
        wd[p] = R(1);
        ic[p] = R(1);
        ig[p] = R(1);
        iwd[p] = R(1);
      }
    }
  }
  // the time step of this step, from the control words read before the copies
  if (tid == kDtThread) {
    double dtv = c_dtf > 0.0 ? c_dtf : c_cfl / __longlong_as_double((long long)c_rate);
    if (c_tend > 0.0) dtv = (c_t >= c_tend) ? 0.0 : fmin(dtv, c_tend - c_t);
    s_dtr = (R)dtv;
    s_end = dtv == 0.0;
    s_dt = dtv;
    if (b == 0) {
      Ctrl* c = A.ctrl;
      c->t[A.tslot ^ 1] = c_t + dtv;
      c->rate[(A.slot + 2) % 3] = 0ull;
      c->last_dt = dtv;
    }
  }
  cp_async_wait_all();
  if constexpr (DSTAGE) {
    // each thread converts the cells it staged: its own copies have landed, so no barrier is needed
    // before the conversion (the same cell-to-thread assignment as the staging loops above)
    if (pairs) {
      for (int l2 = tid; l2 < G::NH / 2; l2 += kThreads) {
#pragma unroll
        for (int v = 0; v < nv; ++v) {
          Ws[v * G::NH + 2 * l2] = d2f(Wd[v * G::NH + 2 * l2]);
          Ws[v * G::NH + 2 * l2 + 1] = d2f(Wd[v * G::NH + 2 * l2 + 1]);
        }
      }
    } else {
      for (int l = tid; l < G::NH; l += kThreads) {
#pragma unroll
        for (int v = 0; v < nv; ++v) Ws[v * G::NH + l] = d2f(Wd[v * G::NH + l]);
      }
    }
  }
  __syncthreads();
  const double dt_d = s_dt;
  if (s_end) {  // t_end reached: carry the state over
    for (int l = tid; l < G::NC; l += kThreads) {
      const int li = l % X, lj = (l / X) % Y, lk = l / (X * Y);
      const int gi = ox + li, gj = oy + lj, gk = oz + lk;
      if (gi >= g.n[0] || (D >= 2 && gj >= g.n[1]) || (D >= 3 && gk >= g.n[2])) continue;
      const long c = cell_index(g, gi, gj, gk);
      for (int v = 0; v < nv; ++v) {
        ((S*)A.Wout)[(long)v * g.ncell + c] = ((const S*)A.Win)[(long)v * g.ncell + c];
        if (PREC == PREC_F32) A.Wout_lo[(long)v * g.ncell + c] = A.Win_lo[(long)v * g.ncell + c];
      }
    }
    return;
  }
  const R dt = s_dtr;

  // ---- turbulent relaxation time and limited slopes on the tile and its first halo ring -------
  ring_phase<D, PREC, V, H>(kc, g.turb_model, g.turb_cons != 0, g.limiter, Ws, Fl, taus, Ss, icx, icy, icz, igx, igy,
                         igz);
  __syncthreads();

  // ---- fluxes of every face of the tile ----------------------------------------------------
  {
    Gas<R> gas;
    gas.bK = kc.bK;
    gas.ibK = kc.ibK;
    gas.K = kc.K;
    gas.mu = kc.mu;
    gas.C_a = kc.C_a;
    const R gamma = kc.gamma;
    // Inputs of one face in its frame (velocity order: normal first, then tangential axes).
    struct FaceIn {
      R wl[nv], wr[nv], cl[nv], cr[nv], sl[nv], sr[nv], tl[Dims<D>::nt][nv], tr[Dims<D>::nt][nv];
      R dxl, dxr, idxl, idxr, tau_t;
      int ax, ci, cj, ck, perm[3];
    };
    // AX: the face's axis when the caller knows it at compile time (the frame permutation, strides
    // and shared-memory offsets below then fold to constants), -1 when it is found from f here
    auto prep = [&](int f, FaceIn& in, auto ax_tag) {
      constexpr int AX = decltype(ax_tag)::value;
      int ax, ci, cj, ck;  // face between cell (c - e_ax) and c, tile coordinates
      if (AX == 0 || (AX < 0 && f < G::NFX)) {
        ax = 0;
        ci = f % (X + 1);
        cj = (f / (X + 1)) % Y;
        ck = f / ((X + 1) * Y);
      } else if (AX == 1 || (AX < 0 && D >= 2 && f < G::NFX + G::NFY)) {
        const int q = f - G::NFX;
        ax = 1;
        ci = q % X;
        cj = (q / X) % (Y + 1);
        ck = q / (X * (Y + 1));
      } else {
        const int q = f - G::NFX - G::NFY;
        ax = 2;
        ci = q % X;
        cj = (q / X) % Y;
        ck = q / (X * Y);
      }
      in.ax = ax;
      in.ci = ci;
      in.cj = cj;
      in.ck = ck;
      const int st[3] = {1, HX, HX * HY};
      const int sn = st[ax];
      const int hc = ((ck + (D >= 3 ? H : 0)) * HY + (cj + (D >= 2 ? H : 0))) * HX + (ci + H);
      int* perm = in.perm;
      perm[0] = ax;
      if (D == 2) perm[1] = 1 - ax;
      if (D == 3) {
        perm[1] = ax == 0 ? 1 : 0;
        perm[2] = ax == 2 ? 1 : 2;
      }
      const R* wn = ax == 0 ? wsx : (ax == 1 ? wsy : wsz);
      const int pn = ax == 0 ? ci + H : (ax == 1 ? cj + H : ck + H);  // halo coordinate of cell c
      const R h1 = wn[pn - 1], h2 = wn[pn];
      [[maybe_unused]] R i2h1 = R(0), i2h2 = R(0);  // 2 / width of the two cells (higher-order slopes)
      if constexpr (RECON != RECON_MUSCL2) {
        i2h1 = g_rcp(R(0.5) * h1);
        i2h2 = g_rcp(R(0.5) * h2);
      }
      const R* icn = ax == 0 ? icx : (ax == 1 ? icy : icz);
      (void)icn;
      // ring indices of the two cells
      const int rc = ((ck + (D >= 3 ? 1 : 0)) * G::RY + (cj + (D >= 2 ? 1 : 0))) * G::RX + (ci + 1);
      const int rst[3] = {1, G::RX, G::RX * G::RY};
      const int rl = rc - rst[ax];
      R* wl = in.wl;
      R* wr = in.wr;
      R* cl = in.cl;
      R* cr = in.cr;
      R* sl = in.sl;
      R* sr = in.sr;
#pragma unroll
      for (int v = 0; v < nv; ++v) {
        const int sv = (v >= 1 && v <= D) ? 1 + perm[v - 1] : v;
        const R* p = Ws + sv * G::NH + hc;
        const R s1 = p[-sn], s2 = p[0];
        if constexpr (RECON != RECON_MUSCL2) {
          // higher-order face values from the normal stencil (cells pn-3 .. pn+2); the normal
          // slopes are the one-sided differences to them
          if constexpr (RECON == RECON_WENO5) {
            wl[v] = weno5<R>(p[-3 * sn], p[-2 * sn], s1, s2, p[sn]);
            wr[v] = weno5<R>(p[2 * sn], p[sn], s2, s1, p[-2 * sn]);
          } else {
            wl[v] = muscl3_right<R>(p[-2 * sn], s1, s2);
            wr[v] = muscl3_left<R>(s1, s2, p[sn]);
          }
          sl[v] = (wl[v] - s1) * i2h1;
          sr[v] = (s2 - wr[v]) * i2h2;
        } else if (PRE) {
          sl[v] = Ss[(ax * nv + sv) * G::NR + rl];
          sr[v] = Ss[(ax * nv + sv) * G::NR + rc];
          wl[v] = s1 + R(0.5) * h1 * sl[v];
          wr[v] = s2 - R(0.5) * h2 * sr[v];
        } else {
          // MUSCL with the tabulated inverse centre distances (cells pn-2 .. pn+1 along the normal)
          const R dm = (s1 - p[-2 * sn]) * icn[pn - 1], dc = (s2 - s1) * icn[pn], dp = (p[sn] - s2) * icn[pn + 1];
          sl[v] = limiter<R>(g.limiter, dm, dc);
          sr[v] = limiter<R>(g.limiter, dc, dp);
          wl[v] = s1 + R(0.5) * h1 * sl[v];
          wr[v] = s2 - R(0.5) * h2 * sr[v];
        }
        cl[v] = s1;
        cr[v] = s2;
      }
      if (!physical<D, R>(gamma, wl)) {
#pragma unroll
        for (int v = 0; v < nv; ++v) {
          wl[v] = cl[v];
          sl[v] = R(0);
        }
      }
      if (!physical<D, R>(gamma, wr)) {
#pragma unroll
        for (int v = 0; v < nv; ++v) {
          wr[v] = cr[v];
          sr[v] = R(0);
        }
      }
      if (MULTID && PRE) {
#pragma unroll
        for (int s = 0; s < D - 1; ++s) {
          const int ta = perm[1 + s];
#pragma unroll
          for (int v = 0; v < nv; ++v) {
            const int sv = (v >= 1 && v <= D) ? 1 + perm[v - 1] : v;
            in.tl[s][v] = Ss[(ta * nv + sv) * G::NR + rl];
            in.tr[s][v] = Ss[(ta * nv + sv) * G::NR + rc];
          }
        }
      } else if (MULTID) {
#pragma unroll
        for (int s = 0; s < D - 1; ++s) {
          const int ta = perm[1 + s];
          const int stt = st[ta];
          const R* ict = ta == 0 ? icx : (ta == 1 ? icy : icz);
          const int hcell[3] = {ci + H, cj + (D >= 2 ? H : 0), ck + (D >= 3 ? H : 0)};
          const int pt = hcell[ta];
          const R im = ict[pt], ip = ict[pt + 1];
#pragma unroll
          for (int v = 0; v < nv; ++v) {
            const int sv = (v >= 1 && v <= D) ? 1 + perm[v - 1] : v;
            const R* pc = Ws + sv * G::NH + hc;
            const R* pl = pc - sn;
            in.tl[s][v] = limiter<R>(g.limiter, (pl[0] - pl[-stt]) * im, (pl[stt] - pl[0]) * ip);
            in.tr[s][v] = limiter<R>(g.limiter, (pc[0] - pc[-stt]) * im, (pc[stt] - pc[0]) * ip);
          }
        }
      }
      in.dxl = R(0.5) * h1;
      in.dxr = R(0.5) * h2;
      {
        const R* iwn = ax == 0 ? iwx : (ax == 1 ? iwy : iwz);
        in.idxl = R(2) * iwn[pn - 1];
        in.idxr = R(2) * iwn[pn];
      }
      in.tau_t = R(0.5) * (taus[rl] + taus[rc]);
    };
    // the flux of face f back in the grid frame; with a mass-flux output (k-omega transport) also
    // the face's time-integrated mass flux
    auto store = [&](int f, const FaceIn& in, const R* F, auto ax_tag) {
      constexpr int AX = decltype(ax_tag)::value;  // the face's axis if known at compile time, else -1
      Fs[0 * G::NF + f] = F[0];
#pragma unroll
      for (int k = 0; k < D; ++k) Fs[(1 + (AX >= 0 ? face_perm_c<D>(AX, k) : in.perm[k])) * G::NF + f] = F[1 + k];
      Fs[(D + 1) * G::NF + f] = F[D + 1];
      if (A.mflux[0]) {
        // global face (cell c = tile origin + (ci, cj, ck), face c - 1/2 along ax)
        const int gc[3] = {ox + in.ci, oy + in.cj, oz + in.ck};
        int nf[3] = {g.n[0], g.n[1], g.n[2]};
        nf[in.ax] += 1;
        if (gc[0] < nf[0] && gc[1] < nf[1] && gc[2] < nf[2])
          ((R*)A.mflux[in.ax])[((long)gc[2] * nf[1] + gc[1]) * nf[0] + gc[0]] = F[0];
      }
    };
    // Rounds of kThreads faces (of 2 kThreads faces, two per thread, on the paired tiles).  On the
    // paired tiles, whose face body is about twice as long, the warps of every 128-thread group meet
    // at a named barrier after each round, so that the warps sharing an SM sub-partition run the body
    // close together and share its instruction fetches (every thread runs every round).  With one
    // face per thread and the two sides paired, the body is short enough that such a barrier costs
    // more than it saves (2% on the 1024^2 workload), so those rounds run free.
    if constexpr (PAIR) {
      // two faces per thread, fa and fb = fa + kThreads, evaluated together with paired FP32
      // instructions (lane x: fa, lane y: fb; a missing fb repeats fa and is not stored)
      Gas<F2> gas2;
      gas2.bK = F2(kc.bK);
      gas2.ibK = F2(kc.ibK);
      gas2.K = F2(kc.K);
      gas2.mu = F2(kc.mu);
      gas2.C_a = F2(kc.C_a);
      constexpr int kRounds2 = (G::NF + 2 * kThreads - 1) / (2 * kThreads);
      for (int it = 0; it < kRounds2; ++it) {
        const int fa = tid + 2 * it * kThreads, fb = fa + kThreads;
        if (fa < G::NF) {
          FaceIn a, b;
          prep(fa, a, std::integral_constant<int, -1>{});
          prep(fb < G::NF ? fb : fa, b, std::integral_constant<int, -1>{});
          F2 wl[nv], wr[nv], cl[nv], cr[nv], sl[nv], sr[nv], tl[Dims<D>::nt][nv], tr[Dims<D>::nt][nv];
#pragma unroll
          for (int v = 0; v < nv; ++v) {
            wl[v] = F2(a.wl[v], b.wl[v]);
            wr[v] = F2(a.wr[v], b.wr[v]);
            cl[v] = F2(a.cl[v], b.cl[v]);
            cr[v] = F2(a.cr[v], b.cr[v]);
            sl[v] = F2(a.sl[v], b.sl[v]);
            sr[v] = F2(a.sr[v], b.sr[v]);
#pragma unroll
            for (int s = 0; s < Dims<D>::nt; ++s) {
              tl[s][v] = F2(a.tl[s][v], b.tl[s][v]);
              tr[s][v] = F2(a.tr[s][v], b.tr[s][v]);
            }
          }
          F2 F[nv], tau;
          face_flux<D, F2, MULTID, false>(wl, wr, cl, cr, sl, sr, tl, tr, F2(a.dxl, b.dxl), F2(a.dxr, b.dxr),
                                          F2(a.tau_t, b.tau_t), F2(dt), gas2, g.abar_t0, F, &tau);
          R Fa[nv], Fb[nv];
#pragma unroll
          for (int v = 0; v < nv; ++v) {
            Fa[v] = F[v].v.x;
            Fb[v] = F[v].v.y;
          }
          store(fa, a, Fa, std::integral_constant<int, -1>{});
          if (fb < G::NF) store(fb, b, Fb, std::integral_constant<int, -1>{});
        }
        if constexpr (kThreads % 128 == 0)
          asm volatile("bar.sync %0, 128;" ::"r"(1 + (tid >> 7)) : "memory");
        else
          __syncwarp();
      }
    } else {
      constexpr int kRounds = (G::NF + kThreads - 1) / kThreads;
      for (int it = 0; it < kRounds; ++it) {
        const int f = tid + it * kThreads;
        if (f < G::NF) {
          FaceIn in;
          if (f < G::NFX)
            prep(f, in, std::integral_constant<int, 0>{});
          else if (D < 3 || f < G::NFX + G::NFY)
            prep(f, in, std::integral_constant<int, D >= 2 ? 1 : 0>{});
          else
            prep(f, in, std::integral_constant<int, D >= 3 ? 2 : 0>{});
          R F[nv], tau;
          if constexpr (std::is_same<R, float>::value && D <= 2) {
            // single precision: the two sides of the face on the paired FP32 instructions (in 3D the
            // paired body does not fit the register budget of two CTAs per SM)
            face_flux_ps<D, MULTID, RAR>(in.wl, in.wr, in.cl, in.cr, in.sl, in.sr, in.tl, in.tr, in.dxl, in.dxr,
                                         in.idxl, in.idxr, in.tau_t, dt, gas, g.abar_t0, F, &tau);
          } else {
            face_flux<D, R, MULTID, RAR>(in.wl, in.wr, in.cl, in.cr, in.sl, in.sr, in.tl, in.tr, in.dxl, in.dxr,
                                         in.tau_t, dt, gas, g.abar_t0, F, &tau);
          }
          if (f < G::NFX)
            store(f, in, F, std::integral_constant<int, 0>{});
          else if (D < 3 || f < G::NFX + G::NFY)
            store(f, in, F, std::integral_constant<int, D >= 2 ? 1 : 0>{});
          else
            store(f, in, F, std::integral_constant<int, D >= 3 ? 2 : 0>{});
        }
      }
    }
  }
  // double state: the old doubles of this thread's cells are loaded while the CTA meets at the barrier
  constexpr int NCI = (G::NC + kThreads - 1) / kThreads;
  double wold[PREC == PREC_F32D ? NCI : 1][nv];
  if constexpr (PREC == PREC_F32D) {
#pragma unroll
    for (int q = 0; q < NCI; ++q) {
      const int l = tid + q * kThreads;
      const int li = l % X, lj = (l / X) % Y, lk = l / (X * Y);
      const int gi = ox + li, gj = oy + lj, gk = oz + lk;
      if (l >= G::NC || gi >= g.n[0] || (D >= 2 && gj >= g.n[1]) || (D >= 3 && gk >= g.n[2])) continue;
      const long c = cell_index(g, gi, gj, gk);
#pragma unroll
      for (int v = 0; v < nv; ++v) wold[q][v] = __ldg((const double*)A.Win + (long)v * g.ncell + c);
    }
  }
  __syncthreads();

  // ---- conservative update, CFL rate of the new state, residual norms --------------------------
  R rmax = R(0);
  double racc[3 * 5];
#pragma unroll
  for (int q = 0; q < 15; ++q) racc[q] = 0.0;
  unsigned int bad = 0;
#pragma unroll
  for (int qc = 0; qc < NCI; ++qc) {
    const int l = tid + qc * kThreads;
    const int li = l % X, lj = (l / X) % Y, lk = l / (X * Y);
    const int gi = ox + li, gj = oy + lj, gk = oz + lk;
    if (l >= G::NC || gi >= g.n[0] || (D >= 2 && gj >= g.n[1]) || (D >= 3 && gk >= g.n[2])) continue;
    const long c = cell_index(g, gi, gj, gk);
    // faces below/above the cell along each axis
    int fm[3], fp[3];
    R h[3];
    fm[0] = (lk * Y + lj) * (X + 1) + li;
    fp[0] = fm[0] + 1;
    h[0] = wsx[li + H];
    if (D >= 2) {
      fm[1] = G::NFX + (lk * (Y + 1) + lj) * X + li;
      fp[1] = fm[1] + X;
      h[1] = wsy[lj + H];
    }
    if (D >= 3) {
      fm[2] = G::NFX + G::NFY + (lk * Y + lj) * X + li;
      fp[2] = fm[2] + X * Y;
      h[2] = wsz[lk + H];
    }
    R ih[3];
#pragma unroll
    for (int d = 0; d < D; ++d) ih[d] = (d == 0 ? iwx[li + H] : (d == 1 ? iwy[lj + H] : iwz[lk + H]));
    R wn[nv];
    double vol = 1.0;
    if (A.resid) {  // cell volume from the double-precision widths
      const int gc[3] = {gi, gj, gk};
      for (int d = 0; d < D; ++d) vol *= g.w[d][gc[d] + kWG];
    }
    // the cell's old state: staged in shared memory (FP64, float pair), else loaded into wold above
    const int hidx = ((lk + (D >= 3 ? H : 0)) * HY + (lj + (D >= 2 ? H : 0))) * HX + (li + H);
#pragma unroll
    for (int v = 0; v < nv; ++v) {
      const long gidx = (long)v * g.ncell + c;
      if constexpr (PREC == PREC_F64) {
        double w = (double)Ws[v * G::NH + hidx];
        const double w_old = w;
#pragma unroll
        for (int d = 0; d < D; ++d) w -= ((double)Fs[v * G::NF + fp[d]] - (double)Fs[v * G::NF + fm[d]]) / (double)h[d];
        ((double*)A.Wout)[gidx] = w;
        wn[v] = (R)w;
        if (A.resid) {
          const double r = (w - w_old) / dt_d;
          racc[v] += r * r;
          racc[5 + v] = fmax(racc[5 + v], fabs(r));
          racc[10 + v] += w * vol;
        }
      } else {
        R inc = R(0);
#pragma unroll
        for (int d = 0; d < D; ++d) inc -= (Fs[v * G::NF + fp[d]] - Fs[v * G::NF + fm[d]]) * ih[d];
        double wd = 0.0;
        if constexpr (PREC == PREC_F32) {
          // (hi, lo) += inc with an error-free sum, then renormalise
          const float hi = (float)Ws[v * G::NH + hidx], lo = Lo[v * G::NC + l];
          const float s = hi + inc;
          const float bb = s - hi;
          const float err = (hi - (s - bb)) + (inc - bb);
          const float lo2 = lo + err;
          const float nhi = s + lo2;
          const float nlo = lo2 - (nhi - s);
          ((float*)A.Wout)[gidx] = nhi;
          A.Wout_lo[gidx] = nlo;
          wn[v] = nhi;
          if (A.resid) wd = (double)nhi + (double)nlo;
        } else {
          const double w = wold[qc][v] + f2d(inc);
          ((double*)A.Wout)[gidx] = w;
          wn[v] = (float)Ws[v * G::NH + hidx] + inc;  // the new state in float, for the rate and status
          wd = w;
        }
        if (A.resid) {
          const double r = (double)inc / dt_d;
          racc[v] += r * r;
          racc[5 + v] = fmax(racc[5 + v], fabs(r));
          racc[10 + v] += wd * vol;
        }
      }
    }
    const R p = pressure_of<R>(D, kc.gamma, wn);
    if (!(wn[0] > R(0)) || !(p > R(0))) bad = 1u;
    rmax = fmax(rmax, cell_rate_inv<D, R>(wn, kc.gamma, ih));
  }
  const unsigned long long bmax = block_max_rate<R>(rmax, red);
  if (tid == 0) atomicMax(&A.ctrl->rate[(A.slot + 1) % 3], bmax);
  if (__syncthreads_or(bad) && tid == 0) atomicOr(&A.ctrl->status, 1u);
  if (A.resid) {
    for (int v = 0; v < nv; ++v) {
      double s = block_sum(racc[v], red);
      if (tid == 0) atomicAdd(&A.ctrl->l2[v], s);
      s = block_sum(racc[10 + v], red);
      if (tid == 0) atomicAdd(&A.ctrl->total[v], s);
      const double m = block_max<double>(racc[5 + v], red);
      if (tid == 0) atomic_max_nonneg(&A.ctrl->linf[v], m);
    }
  }
}

template <int D, int V = 0> constexpr int min_blocks(int prec) {
  return prec != PREC_F64 ? (paired_tile<D, V>() ? 256 : 512) / Tile<D, V>::T : 1;
}

template <int D, int PREC, bool MULTID, int V = 0, int RECON = RECON_MUSCL2, bool RAR = false>
__global__ void __launch_bounds__(Tile<D, V>::T, min_blocks<D, V>(PREC))
    step_kernel(const __grid_constant__ StepArgs A) {
  step_tile<D, PREC, MULTID, V, RECON, RAR>(A, blockIdx.x);
}

// ---- batches of independent solves --------------------------------------------------------------
// A batch advances many solves of one dimension and arithmetic by one step per launch.  The
// arguments of a solve depend on the batch step k only through k mod 6 (buffer k mod 2, rate slot
// k mod 3), so each solve carries six precomputed argument sets.  A solve takes part while
// k < stop_at; afterwards its state rests in buffer stop_at mod 2.
struct BatchSolve {
  StepArgs args[6];
  long long stop_at;
  int tiles;
  int pad;
};

struct BatchArgs {
  const BatchSolve* solves;
  const int2* items;        // (solve, tile) work items
  const int* nitems;        // device: number of valid items
  long long* counter;       // batch step index, two slots
  int phase;                // k mod 6 of the launch (fixed by the position in a captured chunk)
};

// Persistent CTAs stride over the work items of one step.  V: the tile shape (the items are tiles of
// that shape; the server picks one per group).
template <int D, int PREC, bool MULTID, int V = 0>
__global__ void __launch_bounds__(Tile<D, V>::T, min_blocks<D, V>(PREC)) batch_step_kernel(const __grid_constant__ BatchArgs B) {
  const int tslot = B.phase & 1;
  const long long k = B.counter[tslot];
  if (blockIdx.x == 0 && threadIdx.x == 0) B.counter[tslot ^ 1] = k + 1;
  const int n = *B.nitems;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const int2 w = B.items[it];
    const BatchSolve& S = B.solves[w.x];
    if (k < S.stop_at) step_tile<D, PREC, MULTID, V>(S.args[B.phase], w.y);
    __syncthreads();
  }
}

template <int D, int PREC, bool MULTID, int V = 0>
size_t batch_smem() {
  using R = typename PrecT<PREC>::R;
  return TileGeom<D, V>::template smem_bytes<R>(pre_slopes<D, PREC, V>(), PREC == PREC_F32);
}

template <int D, int PREC, bool MULTID, int V = 0>
void launch_batch(const BatchArgs& B, int nblocks, cudaStream_t s) {
  batch_step_kernel<D, PREC, MULTID, V><<<nblocks, Tile<D, V>::T, batch_smem<D, PREC, MULTID, V>(), s>>>(B);
}

// Sets the kernel's shared-memory limit; *resident (if given) receives the CTAs per SM that fit.
template <int D, int PREC, bool MULTID, int V = 0>
cudaError_t prepare_batch(int* resident = nullptr) {
  const size_t sm = batch_smem<D, PREC, MULTID, V>();
  cudaError_t e = cudaFuncSetAttribute(batch_step_kernel<D, PREC, MULTID, V>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess && resident)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, batch_step_kernel<D, PREC, MULTID, V>, Tile<D, V>::T,
                                                      sm);
  return e;
}

template <int D, int PREC, bool MULTID, int V = 0, int RECON = RECON_MUSCL2, bool RAR = false>
void launch_step(const StepArgs& A, int nblocks, cudaStream_t s) {
  using R = typename PrecT<PREC>::R;
  const size_t sm =
      TileGeom<D, V, halo_of(RECON)>::template smem_bytes<R>(pre_slopes<D, PREC, V>(), PREC == PREC_F32);
  step_kernel<D, PREC, MULTID, V, RECON, RAR><<<nblocks, Tile<D, V>::T, sm, s>>>(A);
}

template <int D, int PREC, bool MULTID, int V = 0, int RECON = RECON_MUSCL2, bool RAR = false>
cudaError_t prepare_step() {
  using R = typename PrecT<PREC>::R;
  const size_t sm =
      TileGeom<D, V, halo_of(RECON)>::template smem_bytes<R>(pre_slopes<D, PREC, V>(), PREC == PREC_F32);
  return cudaFuncSetAttribute(step_kernel<D, PREC, MULTID, V, RECON, RAR>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

}  // namespace gks
