// Body-fitted 2D grids with the directional expansion (the paper's C-type and channel grids,
// Section 5, Table 2).  The cells are the quadrilaterals of a structured node lattice; each face
// evaluates the gas-kinetic flux of Section 4 in its own (normal, tangent) frame:
//   - metrics (once per grid, double precision): per face the unit normal n pointing to increasing
//     index, the length L, and the distances of the face's MUSCL stencil (centroid to centroid along
//     the grid line, centroid to face midpoint); per cell the area.  Centroids are vertex averages;
//     a ghost centroid is its source cell translated by the period on a periodic axis, else the
//     mirror image of the interior cell through the boundary face midpoint;
//   - per step, one fused kernel over tiles of cells: the tile's state with two halo layers and the
//     geometry records of its faces staged in shared memory; the turbulent relaxation time of the
//     tile and its first ring from Green-Gauss velocity gradients (face value the mean of the two
//     cells); the face fluxes: the four cells of the stencil rotated into the face frame (rho,
//     rho u_n, rho u_t, rho E), limited slopes over the centroid distances, the flux of face_flux
//     with the centroid-to-midpoint distances, the momentum flux rotated back and weighted by L;
//     then the update of each cell by its four face fluxes divided by its area, the CFL rate
//     sum_faces (|U.n| + c) L / (2 A) of the new state for the next step, the physical-state check
//     and the residual norms.
// Ghost cells follow the boundary rules of the index lattice (load_cell); a ghost cell's
// turbulent relaxation time is that of its source cell.
#include <algorithm>

#include "gks_curv.h"
#include "gks_curv_step.cuh"
#include "gks_flux.cuh"
#include "gks_step.cuh"

namespace gks {

namespace {

constexpr int kCurvThreads = 128;

__device__ __forceinline__ double node_x(const double* nodes, int n0, int i, int j) {
  return nodes[((long)j * (n0 + 1) + i) * 2];
}
__device__ __forceinline__ double node_y(const double* nodes, int n0, int i, int j) {
  return nodes[((long)j * (n0 + 1) + i) * 2 + 1];
}

// Vertex-average centroid of interior cell (i, j).
__device__ void centroid_in(const double* nodes, int n0, int i, int j, double& x, double& y) {
  x = 0.25 * (node_x(nodes, n0, i, j) + node_x(nodes, n0, i + 1, j) + node_x(nodes, n0, i + 1, j + 1) +
              node_x(nodes, n0, i, j + 1));
  y = 0.25 * (node_y(nodes, n0, i, j) + node_y(nodes, n0, i + 1, j) + node_y(nodes, n0, i + 1, j + 1) +
              node_y(nodes, n0, i, j + 1));
}

// Midpoint of the face between nodes (i0, j0) and (i1, j1).
__device__ void mid(const double* nodes, int n0, int i0, int j0, int i1, int j1, double& x, double& y) {
  x = 0.5 * (node_x(nodes, n0, i0, j0) + node_x(nodes, n0, i1, j1));
  y = 0.5 * (node_y(nodes, n0, i0, j0) + node_y(nodes, n0, i1, j1));
}

// Centroid of cell (i, j) of a stencil along axis a: at most two layers outside the grid along a,
// the other index inside.
__device__ void centroid(const double* nodes, int n0, int n1, int a, bool periodic, int cut, int i, int j,
                         double& x, double& y) {
  const int n = a == 0 ? n0 : n1;
  const int c = a == 0 ? i : j;
  if (c >= 0 && c < n) {
    centroid_in(nodes, n0, i, j, x, y);
    return;
  }
  if (a == 1 && c < 0 && cut > 0 && (i < cut || i >= n0 - cut)) {  // across a C-grid wake cut
    centroid_in(nodes, n0, n0 - 1 - i, -c - 1, x, y);
    return;
  }
  double lx, ly, hx, hy;  // midpoints of the low and high boundary faces of this grid line
  if (a == 0) {
    mid(nodes, n0, 0, j, 0, j + 1, lx, ly);
    mid(nodes, n0, n0, j, n0, j + 1, hx, hy);
  } else {
    mid(nodes, n0, i, 0, i + 1, 0, lx, ly);
    mid(nodes, n0, i, n1, i + 1, n1, hx, hy);
  }
  const bool lo = c < 0;
  const int k = lo ? -c : c - n + 1;  // ghost layer 1 or 2
  double sx, sy;
  if (periodic) {
    const int s = lo ? n - k : k - 1;
    if (a == 0)
      centroid_in(nodes, n0, s, j, sx, sy);
    else
      centroid_in(nodes, n0, i, s, sx, sy);
    x = sx + (lo ? lx - hx : hx - lx);
    y = sy + (lo ? ly - hy : hy - ly);
  } else {
    const int s = lo ? k - 1 : n - k;
    if (a == 0)
      centroid_in(nodes, n0, s, j, sx, sy);
    else
      centroid_in(nodes, n0, i, s, sx, sy);
    x = 2.0 * (lo ? lx : hx) - sx;
    y = 2.0 * (lo ? ly : hy) - sy;
  }
}

// Centroid of any cell at most two layers outside the grid: along one axis as above; a corner by the
// parallelogram of its i ghost, its j ghost and their common source cell.
__device__ int ghost_source(int c, int n, bool per) {
  const int k = c < 0 ? -c : c - n + 1;
  return per ? (c < 0 ? n - k : k - 1) : (c < 0 ? k - 1 : n - k);
}
__device__ void centroid_any(const double* nodes, int n0, int n1, bool per0, bool per1, int cut, int i, int j,
                             double& x, double& y) {
  const bool iin = i >= 0 && i < n0, jin = j >= 0 && j < n1;
  if (jin) {
    centroid(nodes, n0, n1, 0, per0, cut, i, j, x, y);
    return;
  }
  if (iin) {
    centroid(nodes, n0, n1, 1, per1, cut, i, j, x, y);
    return;
  }
  const int is = ghost_source(i, n0, per0), js = ghost_source(j, n1, per1);
  double ax, ay, bx, by, cx, cy;
  centroid(nodes, n0, n1, 0, per0, cut, i, js, ax, ay);
  centroid(nodes, n0, n1, 1, per1, cut, is, j, bx, by);
  centroid_in(nodes, n0, is, js, cx, cy);
  x = ax + bx - cx;
  y = ay + by - cy;
}

__device__ __forceinline__ double dist(double ax, double ay, double bx, double by) {
  return sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
}

// Per-cell metrics: area (double and the inverse in the arithmetic type) and the convexity check.
template <class R>
__global__ void metrics_cell_kernel(const double* nodes, int n0, int n1, double* area, R* iarea, int* bad) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (long)n0 * n1) return;
  const int i = (int)(c % n0), j = (int)(c / n0);
  const double qx[4] = {node_x(nodes, n0, i, j), node_x(nodes, n0, i + 1, j), node_x(nodes, n0, i + 1, j + 1),
                        node_x(nodes, n0, i, j + 1)};
  const double qy[4] = {node_y(nodes, n0, i, j), node_y(nodes, n0, i + 1, j), node_y(nodes, n0, i + 1, j + 1),
                        node_y(nodes, n0, i, j + 1)};
  const double A = 0.5 * ((qx[2] - qx[0]) * (qy[3] - qy[1]) - (qx[3] - qx[1]) * (qy[2] - qy[0]));
  bool ok = A > 0.0;
  for (int q = 0; q < 4; ++q) {
    const int a = (q + 3) % 4, b = (q + 1) % 4;
    if (!((qx[q] - qx[a]) * (qy[b] - qy[q]) - (qy[q] - qy[a]) * (qx[b] - qx[q]) > 0.0)) ok = false;
  }
  if (!ok) atomicOr(bad, 1);
  area[c] = A;
  iarea[c] = (R)(1.0 / A);
}

// Per-face metrics along axis a, in the order of CurvGeom::face.
template <class R>
__global__ void metrics_face_kernel(const double* nodes, int n0, int n1, int a, bool per0, bool per1, int cut,
                                    R* out, R* tang, long nf) {
  const bool periodic = a == 0 ? per0 : per1;
  const long f = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int nfa = a == 0 ? n0 + 1 : n0;
  const int fi = (int)(f % nfa), fj = (int)(f / nfa);
  // face end points: i-face from node (fi, fj) to (fi, fj + 1), j-face from (fi, fj) to (fi + 1, fj)
  const int ei = a == 0 ? fi : fi + 1, ej = a == 0 ? fj + 1 : fj;
  const double ex = node_x(nodes, n0, ei, ej) - node_x(nodes, n0, fi, fj);
  const double ey = node_y(nodes, n0, ei, ej) - node_y(nodes, n0, fi, fj);
  const double L = sqrt(ex * ex + ey * ey);
  const double nx = a == 0 ? ey / L : -ey / L, ny = a == 0 ? -ex / L : ex / L;
  double mx, my;
  mid(nodes, n0, fi, fj, ei, ej, mx, my);
  double cx[4], cy[4];
  for (int s = 0; s < 4; ++s) {
    const int ci = a == 0 ? fi - 2 + s : fi, cj = a == 0 ? fj : fj - 2 + s;
    centroid(nodes, n0, n1, a, periodic, cut, ci, cj, cx[s], cy[s]);
  }
  const double g[8] = {nx,
                       ny,
                       L,
                       1.0 / dist(cx[0], cy[0], cx[1], cy[1]),
                       1.0 / dist(cx[1], cy[1], cx[2], cy[2]),
                       1.0 / dist(cx[2], cy[2], cx[3], cy[3]),
                       dist(mx, my, cx[1], cy[1]),
                       dist(mx, my, cx[2], cy[2])};
  for (int q = 0; q < 8; ++q) out[(long)q * nf + f] = (R)g[q];
  // tangential steps of the two cells beside the face: centroid steps to the transverse neighbours
  // projected on the tangent t = (-n_y, n_x), inverted (the multi-dimensional expansion)
  const double tx = -ny, ty = nx;
  for (int side = 0; side < 2; ++side) {
    const int i0 = a == 0 ? fi - 1 + side : fi, j0 = a == 0 ? fj : fj - 1 + side;
    const int di = a == 0 ? 0 : 1, dj = a == 0 ? 1 : 0;
    double mxx, myy, c0x, c0y, pxx, pyy;
    centroid_any(nodes, n0, n1, per0, per1, cut, i0 - di, j0 - dj, mxx, myy);
    centroid_any(nodes, n0, n1, per0, per1, cut, i0, j0, c0x, c0y);
    centroid_any(nodes, n0, n1, per0, per1, cut, i0 + di, j0 + dj, pxx, pyy);
    tang[(long)(2 * side) * nf + f] = (R)(1.0 / ((c0x - mxx) * tx + (c0y - myy) * ty));
    tang[(long)(2 * side + 1) * nf + f] = (R)(1.0 / ((pxx - c0x) * tx + (pyy - c0y) * ty));
  }
}

// Per-cell diagnostics: what = 0 the turbulent relaxation time (gks_get_tau_turb), what = 1 the
// rarefaction eps = (mu / p + tau_t) |div U| with the Green-Gauss divergence (face values the means of
// the two cells; gks_get_rarefaction).
template <int PREC>
__global__ void __launch_bounds__(kCurvThreads) curv_tau_kernel(const __grid_constant__ StepArgs A,
                                                                const __grid_constant__ CurvGeom G, void* out,
                                                                int what) {
  using R = typename PrecT<PREC>::R;
  const DevGrid& g = A.g;
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const Consts<R> kc = make_consts<R>(g);
  const int n0 = g.n[0];
  const int i = (int)(c % n0), j = (int)(c / n0);
  R nb[5][4];
  const int di[5] = {-1, 1, 0, 0, 0}, dj[5] = {0, 0, -1, 1, 0};
#pragma unroll
  for (int q = 0; q < 5; ++q) load_cell<2, PREC>(g, A.Win, kc, i + di[q], j + dj[q], 0, nb[q]);
  const R tau_t = g.turb_model == TURB_NONE
                      ? R(0)
                      : tau_gg<R>(g, kc, G, A.f1, A.f2, i, j, [&](int q, int v) { return nb[q][v]; });
  if (what == 0) {
    ((R*)out)[c] = tau_t;
    return;
  }
  const FaceView<R> fi{(const R*)G.face[0], G.nf[0]}, fj{(const R*)G.face[1], G.nf[1]};
  const long fa = (long)j * (n0 + 1) + i, fc = (long)j * n0 + i;
  const long fid[4] = {fa, fa + 1, fc, fc + n0};
  const R* w = nb[4];
  R div = R(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const FaceView<R>& fv = q < 2 ? fi : fj;
    const R sgn = (q & 1) ? R(1) : R(-1);
    const R ux = R(0.5) * (g_div(w[1], w[0]) + g_div(nb[q][1], nb[q][0]));
    const R uy = R(0.5) * (g_div(w[2], w[0]) + g_div(nb[q][2], nb[q][0]));
    div += sgn * (ux * fv(0, fid[q]) + uy * fv(1, fid[q])) * fv(2, fid[q]);
  }
  div = g_div(div, (R)G.area[c]);
  const R p = pressure_of<R>(2, kc.gamma, w);
  ((R*)out)[c] = (g_div(kc.mu, p) + tau_t) * g_abs(div);
}

// CFL rate of a cell on the curvilinear grid: sum over its faces of (|U.n| + c) L / (2 A).
template <class R>
__device__ __forceinline__ R curv_rate(const R* w, R gamma, const CurvGeom& G, int n0, int i, int j, long c) {
  const FaceView<R> fi{(const R*)G.face[0], G.nf[0]}, fj{(const R*)G.face[1], G.nf[1]};
  const R ir = g_rcp(w[0]);
  const R u = w[1] * ir, v = w[2] * ir;
  const R p = pressure_of<R>(2, gamma, w);
  const R cs = g_sqrt(g_div(gamma * p, w[0]));
  const long fa = (long)j * (n0 + 1) + i, fc = (long)j * n0 + i;
  R r = R(0);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    r += (g_abs(u * fi(0, fa + s) + v * fi(1, fa + s)) + cs) * fi(2, fa + s);
    r += (g_abs(u * fj(0, fc + s * n0) + v * fj(1, fc + s * n0)) + cs) * fj(2, fc + s * n0);
  }
  return R(0.5) * r * ((const R*)G.iarea)[c];
}

// CFL rate of the stored state into ctrl->rate[slot].
template <int PREC>
__global__ void __launch_bounds__(kCurvThreads) curv_rate_kernel(const __grid_constant__ StepArgs A,
                                                                 const __grid_constant__ CurvGeom G) {
  using R = typename PrecT<PREC>::R;
  __shared__ double red[kMaxWarps];
  const DevGrid& g = A.g;
  const Consts<R> kc = make_consts<R>(g);
  R rmax = R(0);
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += (long)gridDim.x * blockDim.x) {
    R w[4];
    load_stored<2, PREC>(g, A.Win, c, w);
    rmax = fmax(rmax, curv_rate<R>(w, kc.gamma, G, g.n[0], (int)(c % g.n[0]), (int)(c / g.n[0]), c));
  }
  const double m = block_max<double>((double)rmax, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&A.ctrl->rate[A.slot], m);
}

// ---- k-omega transport after a flow step --------------------------------------------------------
// One CTA per tile of KwTile::X x KwTile::Y cells in four phases: stage k, omega (of each cell's
// source cell) and the ghost-rule density and velocity of the tile and its two-cell halo (corners
// left out: no face stencil or neighbour reaches them); the convective-diffusive fluxes of rho k
// and rho omega through every face of the tile, once per face; per cell the divergence, Wilcox's
// sources with Green-Gauss gradients, the point-implicit destruction and the floors.

struct KwTile {
  static constexpr int X = 32, Y = 8, T = X * Y;
  static constexpr int SX = X + 4, SY = Y + 4;  // staged cells with the halo
};

// k and omega of a (possibly ghost) cell: those of its source cell (rho k / rho of that cell).
template <int PREC>
__device__ __forceinline__ void cell_kw(const KOmegaArgs& K, int i, int j, typename PrecT<PREC>::R& k,
                                        typename PrecT<PREC>::R& om) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  const long c = field_cell(K.g, 2, i, j, 0);
  const R rho = (R)((const S*)K.Win)[c];
  k = g_div(((const R*)K.RKin)[c], rho);
  om = g_div(((const R*)K.RWin)[c], rho);
}

template <int PREC>
__global__ void __launch_bounds__(KwTile::T) curv_komega_kernel(const __grid_constant__ KOmegaArgs K,
                                                                const __grid_constant__ CurvGeom G) {
  using R = typename PrecT<PREC>::R;
  using S = typename PrecT<PREC>::S;
  constexpr int TX = KwTile::X, TY = KwTile::Y, SX = KwTile::SX, NS = KwTile::SX * KwTile::SY;
  constexpr int NFI = (TX + 1) * TY, NFJ = TX * (TY + 1);
  __shared__ R sk[NS], sw[NS], sr[NS], su[NS], sv[NS];
  __shared__ R fi_k[NFI], fi_w[NFI], fj_k[NFJ], fj_w[NFJ];
  const DevGrid& g = K.g;
  const int n0 = g.n[0], n1 = g.n[1];
  const int tiles_x = (n0 + TX - 1) / TX;
  const int i0 = (blockIdx.x % tiles_x) * TX, j0 = (blockIdx.x / tiles_x) * TY;
  const int tid = threadIdx.x;
  const R* RKi = (const R*)K.RKin;
  const R* RWi = (const R*)K.RWin;
  const int li = tid % TX, lj = tid / TX;
  const int i = i0 + li, j = j0 + lj;
  const bool mine = i < n0 && j < n1;
  const long c = (long)j * n0 + i;
  const R dt = (R)K.ctrl->last_dt;  // in flight during the staging
  // the face data of this thread's faces and the cell data of its cell, loaded before the staging
  // so that their latency overlaps it
  constexpr int FPT = (NFI + NFJ + KwTile::T - 1) / KwTile::T;
  R fv[FPT][7];
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    const int q = tid + u * KwTile::T;
    const bool ia = q < NFI;
    const int r = ia ? q : q - NFI;
    const int fl = ia ? r % (TX + 1) : r % TX, fm = ia ? r / (TX + 1) : r / TX;
    const int fi = i0 + fl, fj = j0 + fm;
    if (q >= NFI + NFJ || (ia ? (fi > n0 || fj >= n1) : (fi >= n0 || fj > n1))) continue;
    const int a = ia ? 0 : 1;
    const long nf = G.nf[a];
    const long f = ia ? (long)fj * (n0 + 1) + fi : (long)fj * n0 + fi;
    const R* rec = (const R*)G.face[a];
    fv[u][0] = ((const R*)K.mflux[a])[f];
#pragma unroll
    for (int v = 1; v < 7; ++v) fv[u][v] = rec[(v + 1) * nf + f];
  }
  const long fa = (long)j * (n0 + 1) + i, fc = (long)j * n0 + i;
  const long fid[4] = {fa, fa + 1, fc, fc + n0};
  R A = R(1), rk0 = R(0), rw0 = R(0), gsx[4], gsy[4];
  if (mine) {
    A = (R)G.area[c];
    rk0 = RKi[c];
    rw0 = RWi[c];
    if (K.sources) {
      const FaceView<R> fvi{(const R*)G.face[0], G.nf[0]}, fvj{(const R*)G.face[1], G.nf[1]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const FaceView<R>& fw = q < 2 ? fvi : fvj;
        const R sgn = (q & 1) ? R(1) : R(-1);
        gsx[q] = sgn * fw(0, fid[q]) * fw(2, fid[q]);
        gsy[q] = sgn * fw(1, fid[q]) * fw(2, fid[q]);
      }
    }
  }
  const Consts<R> kc = make_consts<R>(g);
  // phase 1: stage the tile with its halo
  for (int q = tid; q < NS; q += KwTile::T) {
    const int qi = q % SX, qj = q / SX;
    const bool corner = (qi < 2 || qi >= TX + 2) && (qj < 2 || qj >= TY + 2);
    const int gi = i0 - 2 + qi, gj = j0 - 2 + qj;
    if (corner || gi > n0 + 1 || gj > n1 + 1) continue;
    R w[4], k, om;
    load_cell<2, PREC>(g, K.Win, kc, gi, gj, 0, w);
    cell_kw<PREC>(K, gi, gj, k, om);
    sk[q] = k;
    sw[q] = om;
    sr[q] = w[0];
    su[q] = g_div(w[1], w[0]);
    sv[q] = g_div(w[2], w[0]);
  }
  if (dt == R(0)) {  // t_end reached: carry the fields over (dt is the same for every CTA)
    if (mine) {
      ((R*)K.RKout)[c] = rk0;
      ((R*)K.RWout)[c] = rw0;
    }
    return;
  }
  __syncthreads();
  // phase 2: every face of the tile once
  const bool kf = sizeof(R) == sizeof(float);
  const R sigk = kf ? (R)K.fsigma_star : (R)K.sigma_star, sigw = kf ? (R)K.fsigma : (R)K.sigma;
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    const int q = tid + u * KwTile::T;
    const bool ia = q < NFI;
    const int r = ia ? q : q - NFI;
    const int fl = ia ? r % (TX + 1) : r % TX, fm = ia ? r / (TX + 1) : r / TX;  // local face index
    const int fi = i0 + fl, fj = j0 + fm;
    if (q >= NFI + NFJ || (ia ? (fi > n0 || fj >= n1) : (fi >= n0 || fj > n1))) continue;
    // staged index of the first stencil cell (fi - 2 or fj - 2) and the step along the grid line
    const int s0 = ia ? (fm + 2) * SX + fl : fm * SX + fl + 2, st = ia ? 1 : SX;
    R vk[4], vw[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      vk[t] = sk[s0 + t * st];
      vw[t] = sw[s0 + t * st];
    }
    R out[2];
    kw_face<R>(vk, vw, sr[s0 + st], sr[s0 + 2 * st], fv[u], dt, kc.mu, sigk, sigw, g.limiter, K.diffusion, out);
    (ia ? fi_k : fj_k)[r] = out[0];
    (ia ? fi_w : fj_w)[r] = out[1];
  }
  __syncthreads();
  if (!mine) return;
  // phase 3: divergence, sources, point-implicit destruction
  const R alpha = kf ? (R)K.falpha : (R)K.alpha, beta0 = kf ? (R)K.fbeta0 : (R)K.beta0;
  const R beta_star = kf ? (R)K.fbeta_star : (R)K.beta_star, sigma_do = kf ? (R)K.fsigma_do : (R)K.sigma_do;
  const R C_lim = kf ? (R)K.fC_lim : (R)K.C_lim, omega_floor = kf ? (R)K.fomega_floor : (R)K.omega_floor;
  const int ra = lj * (TX + 1) + li, rc = lj * TX + li;
  R ak = rk0 - (fi_k[ra + 1] - fi_k[ra] + fj_k[rc + TX] - fj_k[rc]) / A;
  R aw = rw0 - (fi_w[ra + 1] - fi_w[ra] + fj_w[rc + TX] - fj_w[rc]) / A;
  R rate_k = R(0), rate_w = R(0);
  if (K.sources) {
    const int sc = (lj + 2) * SX + li + 2;
    R Sk, Sw;
    kw_sources<R, SX>(sk, sw, sr, su, sv, sc, gsx, gsy, A, alpha, beta_star, sigma_do, C_lim, Sk, Sw);
    const R w0 = sw[sc];
    ak += dt * Sk;
    aw += dt * Sw;
    rate_k = beta_star * w0;
    rate_w = beta0 * w0;
  }
  ak /= R(1) + dt * rate_k;
  aw /= R(1) + dt * rate_w;
  const R rho_new = (R)((const S*)K.Wnew)[c];
  ((R*)K.RKout)[c] = fmax(ak, R(0));
  ((R*)K.RWout)[c] = fmax(aw, rho_new * omega_floor);
}

// ---- steady k-omega update ---------------------------------------------------------------------
// One diagonal-implicit step of the steady k-omega equations on the finest grid of the steady solver,
// in place, with the fine residual's face mass flux rates (times L) and local steps: per face the
// rates G = m phi_upwind - (mu + sigma rho k / omega |face) L / d12 (phi_r - phi_l); per cell
// R = sum G (outward) - A (S - beta omega RK), RK -= R / D, D = A / (cfl s_loc) + sum_faces
// (max(m_out, 0) + conductance) / rho + A beta omega; then the floors.  Tiles and staging as the
// transport kernel; k and omega come from the field arrays (RK / rho of the cycle's start), so the
// in-place update reads no value another thread writes.
struct SteadyKw {
  const void* k;      // k, omega per cell (arithmetic type)
  const void* om;
  void* RK;           // rho k, rho omega, updated in place
  void* RW;
  const void* s_loc;  // local explicit steps
  double cfl;         // pseudo-time steps cfl s_loc
};

template <int PREC>
__global__ void __launch_bounds__(KwTile::T) steady_komega_kernel(const __grid_constant__ KOmegaArgs K,
                                                                  const __grid_constant__ CurvGeom G,
                                                                  const __grid_constant__ SteadyKw Q) {
  using R = typename PrecT<PREC>::R;
  constexpr int TX = KwTile::X, TY = KwTile::Y, SX = KwTile::SX, NS = KwTile::SX * KwTile::SY;
  constexpr int NFI = (TX + 1) * TY, NFJ = TX * (TY + 1);
  __shared__ R sk[NS], sw[NS], sr[NS], su[NS], sv[NS];
  // per face: rates of rho k and rho omega, mass rate, conductances of k and omega
  __shared__ R fg[5][NFI + NFJ];
  const DevGrid& g = K.g;
  const int n0 = g.n[0], n1 = g.n[1];
  const int tiles_x = (n0 + TX - 1) / TX;
  const int i0 = (blockIdx.x % tiles_x) * TX, j0 = (blockIdx.x / tiles_x) * TY;
  const int tid = threadIdx.x;
  const int li = tid % TX, lj = tid / TX;
  const int i = i0 + li, j = j0 + lj;
  const bool mine = i < n0 && j < n1;
  const long c = (long)j * n0 + i;
  R* RK = (R*)Q.RK;
  R* RW = (R*)Q.RW;
  constexpr int FPT = (NFI + NFJ + KwTile::T - 1) / KwTile::T;
  R fv[FPT][7];
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    const int q = tid + u * KwTile::T;
    const bool ia = q < NFI;
    const int r = ia ? q : q - NFI;
    const int fl = ia ? r % (TX + 1) : r % TX, fm = ia ? r / (TX + 1) : r / TX;
    const int fi = i0 + fl, fj = j0 + fm;
    if (q >= NFI + NFJ || (ia ? (fi > n0 || fj >= n1) : (fi >= n0 || fj > n1))) continue;
    const int a = ia ? 0 : 1;
    const long nf = G.nf[a];
    const long f = ia ? (long)fj * (n0 + 1) + fi : (long)fj * n0 + fi;
    const R* rec = (const R*)G.face[a];
    fv[u][0] = ((const R*)K.mflux[a])[f];
#pragma unroll
    for (int v = 1; v < 7; ++v) fv[u][v] = rec[(v + 1) * nf + f];
  }
  const long fa = (long)j * (n0 + 1) + i, fc = (long)j * n0 + i;
  const long fid[4] = {fa, fa + 1, fc, fc + n0};
  R A = R(1), rk0 = R(0), rw0 = R(0), sl = R(1), gsx[4], gsy[4];
  if (mine) {
    A = (R)G.area[c];
    rk0 = RK[c];
    rw0 = RW[c];
    sl = ((const R*)Q.s_loc)[c];
    const FaceView<R> fvi{(const R*)G.face[0], G.nf[0]}, fvj{(const R*)G.face[1], G.nf[1]};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const FaceView<R>& fw = q < 2 ? fvi : fvj;
      const R sgn = (q & 1) ? R(1) : R(-1);
      gsx[q] = sgn * fw(0, fid[q]) * fw(2, fid[q]);
      gsy[q] = sgn * fw(1, fid[q]) * fw(2, fid[q]);
    }
  }
  const Consts<R> kc = make_consts<R>(g);
  for (int q = tid; q < NS; q += KwTile::T) {
    const int qi = q % SX, qj = q / SX;
    const bool corner = (qi < 2 || qi >= TX + 2) && (qj < 2 || qj >= TY + 2);
    const int gi = i0 - 2 + qi, gj = j0 - 2 + qj;
    if (corner || gi > n0 + 1 || gj > n1 + 1) continue;
    R w[4];
    load_cell<2, PREC>(g, K.Win, kc, gi, gj, 0, w);
    const long src = field_cell(g, 2, gi, gj, 0);
    sk[q] = ((const R*)Q.k)[src];
    sw[q] = ((const R*)Q.om)[src];
    sr[q] = w[0];
    su[q] = g_div(w[1], w[0]);
    sv[q] = g_div(w[2], w[0]);
  }
  __syncthreads();
  const bool kf = sizeof(R) == sizeof(float);
  const R sigk = kf ? (R)K.fsigma_star : (R)K.sigma_star, sigw = kf ? (R)K.fsigma : (R)K.sigma;
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    const int q = tid + u * KwTile::T;
    const bool ia = q < NFI;
    const int r = ia ? q : q - NFI;
    const int fl = ia ? r % (TX + 1) : r % TX, fm = ia ? r / (TX + 1) : r / TX;
    const int fi = i0 + fl, fj = j0 + fm;
    if (q >= NFI + NFJ || (ia ? (fi > n0 || fj >= n1) : (fi >= n0 || fj > n1))) continue;
    const int s0 = ia ? (fm + 2) * SX + fl : fm * SX + fl + 2, st = ia ? 1 : SX;
    const R m = fv[u][0], L = fv[u][1], i01 = fv[u][2], i12 = fv[u][3], i23 = fv[u][4], dl = fv[u][5],
            dr = fv[u][6];
    const R rl = sr[s0 + st], rr = sr[s0 + 2 * st];
    R vk[4], vw[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      vk[t] = sk[s0 + t * st];
      vw[t] = sw[s0 + t * st];
    }
    R cond[2] = {R(0), R(0)}, gq[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const R* v = e == 0 ? vk : vw;
      const R sa = limiter<R>(g.limiter, (v[1] - v[0]) * i01, (v[2] - v[1]) * i12);
      const R sb = limiter<R>(g.limiter, (v[2] - v[1]) * i12, (v[3] - v[2]) * i23);
      const R phiL = v[1] + sa * dl, phiR = v[2] - sb * dr;
      gq[e] = m * (m >= R(0) ? phiL : phiR);
      if (K.diffusion) {
        const R mdl = g_div(rl * vk[1], vw[1]), mdr = g_div(rr * vk[2], vw[2]);
        cond[e] = (kc.mu + (e == 0 ? sigk : sigw) * R(0.5) * (mdl + mdr)) * L * i12;
        gq[e] -= cond[e] * (v[2] - v[1]);
      }
    }
    fg[0][q] = gq[0];
    fg[1][q] = gq[1];
    fg[2][q] = m;
    fg[3][q] = cond[0];
    fg[4][q] = cond[1];
  }
  __syncthreads();
  if (!mine) return;
  const R alpha = kf ? (R)K.falpha : (R)K.alpha, beta0 = kf ? (R)K.fbeta0 : (R)K.beta0;
  const R beta_star = kf ? (R)K.fbeta_star : (R)K.beta_star, sigma_do = kf ? (R)K.fsigma_do : (R)K.sigma_do;
  const R C_lim = kf ? (R)K.fC_lim : (R)K.C_lim, omega_floor = kf ? (R)K.fomega_floor : (R)K.omega_floor;
  // faces i-1/2, i+1/2, j-1/2, j+1/2 in the face arrays, and the outward sign
  const int ra = lj * (TX + 1) + li, rc = NFI + lj * TX + li;
  const int fq[4] = {ra, ra + 1, rc, rc + TX};
  const int sc = (lj + 2) * SX + li + 2;
  const R rho = sr[sc];
  R rk = fg[0][fq[1]] - fg[0][fq[0]] + fg[0][fq[3]] - fg[0][fq[2]];
  R rw = fg[1][fq[1]] - fg[1][fq[0]] + fg[1][fq[3]] - fg[1][fq[2]];
  R dk = R(0), dw = R(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R mo = (q & 1) ? fg[2][fq[q]] : -fg[2][fq[q]];
    dk += fmax(mo, R(0)) + fg[3][fq[q]];
    dw += fmax(mo, R(0)) + fg[4][fq[q]];
  }
  const R base = A / ((R)Q.cfl * sl);
  dk = base + dk / rho;
  dw = base + dw / rho;
  if (K.sources) {
    R Sk, Sw;
    kw_sources<R, SX>(sk, sw, sr, su, sv, sc, gsx, gsy, A, alpha, beta_star, sigma_do, C_lim, Sk, Sw);
    const R w0 = sw[sc];
    rk -= A * (Sk - beta_star * w0 * rk0);
    rw -= A * (Sw - beta0 * w0 * rw0);
    dk += A * beta_star * w0;
    dw += A * beta0 * w0;
  }
  RK[c] = fmax(rk0 - rk / dk, R(0));
  RW[c] = fmax(rw0 - rw / dw, rho * omega_floor);
}

// Local explicit step (CFL 1) of every cell: 2 A / sum_faces (|U.n| + c) L.
template <int PREC>
__global__ void __launch_bounds__(kCurvThreads) lts_kernel(const __grid_constant__ StepArgs A,
                                                           const __grid_constant__ CurvGeom G, void* s_out) {
  using R = typename PrecT<PREC>::R;
  const DevGrid& g = A.g;
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const Consts<R> kc = make_consts<R>(g);
  R w[4];
  load_stored<2, PREC>(g, A.Win, c, w);
  ((R*)s_out)[c] = g_rcp(curv_rate<R>(w, kc.gamma, G, g.n[0], (int)(c % g.n[0]), (int)(c / g.n[0]), c));
}

inline unsigned blocks_for(long n) { return (unsigned)((n + kCurvThreads - 1) / kCurvThreads); }

inline unsigned kw_tiles(const DevGrid& g) {
  return (unsigned)(((g.n[0] + KwTile::X - 1) / KwTile::X) * ((g.n[1] + KwTile::Y - 1) / KwTile::Y));
}

template <int PREC, bool MD>
void step_prec_md(const StepArgs& A, const CurvGeom& G, int variant, cudaStream_t s) {
  if (variant == 0)
    launch_fused<PREC, 0, 0, MD>(A, G, s);
  else if (variant == 1)
    launch_fused<PREC, 1, 0, MD>(A, G, s);
  else
    launch_fused<PREC, 2, 0, MD>(A, G, s);
}

template <int PREC>
void step_prec(const StepArgs& A, const CurvGeom& G, int variant, bool md, cudaStream_t s) {
  if (md)
    step_prec_md<PREC, true>(A, G, variant, s);
  else
    step_prec_md<PREC, false>(A, G, variant, s);
}

}  // namespace

cudaError_t curv_metrics(const double* nodes, int n0, int n1, const bool periodic[2], int cut, int prec,
                         CurvGeom& G, int* bad, cudaStream_t s) {
  const long nc = (long)n0 * n1;
  if (prec == PREC_F64) {
    metrics_cell_kernel<double><<<blocks_for(nc), kCurvThreads, 0, s>>>(nodes, n0, n1, G.area, (double*)G.iarea, bad);
    for (int a = 0; a < 2; ++a)
      metrics_face_kernel<double><<<blocks_for(G.nf[a]), kCurvThreads, 0, s>>>(
          nodes, n0, n1, a, periodic[0], periodic[1], cut, (double*)G.face[a], (double*)G.tang[a], G.nf[a]);
  } else {
    metrics_cell_kernel<float><<<blocks_for(nc), kCurvThreads, 0, s>>>(nodes, n0, n1, G.area, (float*)G.iarea, bad);
    for (int a = 0; a < 2; ++a)
      metrics_face_kernel<float><<<blocks_for(G.nf[a]), kCurvThreads, 0, s>>>(
          nodes, n0, n1, a, periodic[0], periodic[1], cut, (float*)G.face[a], (float*)G.tang[a], G.nf[a]);
  }
  return cudaGetLastError();
}

cudaError_t prepare_curv() {
  cudaError_t e = cudaSuccess;
  const cudaError_t r[13] = {prepare_fused<PREC_F64, 0>(),   prepare_fused<PREC_F64, 1>(),
                            prepare_fused<PREC_F32, 0>(),    prepare_fused<PREC_F32, 1>(),
                            prepare_fused<PREC_F32D, 0>(),   prepare_fused<PREC_F32D, 1>(),
                            prepare_fused<PREC_F64, 2>(),    prepare_fused<PREC_F32, 2>(),
                            prepare_fused<PREC_F32D, 2>(),   prepare_fused<PREC_F64, 2, 1>(),
                            prepare_fused<PREC_F32, 2, 1>(),
                            prepare_fused<PREC_F64, 0, 1>(), prepare_fused<PREC_F32, 0, 1>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) e = x;
  return e;
}

void launch_curv_step(int prec, const StepArgs& A, const CurvGeom& G, int variant, bool multid, cudaStream_t s) {
  if (prec == PREC_F64)
    step_prec<PREC_F64>(A, G, variant, multid, s);
  else if (prec == PREC_F32)
    step_prec<PREC_F32>(A, G, variant, multid, s);
  else
    step_prec<PREC_F32D>(A, G, variant, multid, s);
}

void launch_steady_komega(int prec, const KOmegaArgs& K, const CurvGeom& G, const void* k, const void* om, void* RK,
                          void* RW, const void* s_loc, double cfl, cudaStream_t s) {
  const SteadyKw Q{k, om, RK, RW, s_loc, cfl};
  if (prec == PREC_F64)
    steady_komega_kernel<PREC_F64><<<kw_tiles(K.g), KwTile::T, 0, s>>>(K, G, Q);
  else
    steady_komega_kernel<PREC_F32><<<kw_tiles(K.g), KwTile::T, 0, s>>>(K, G, Q);
}

void curv_tile_shape(int variant, int* x, int* y) {
  *x = variant == 0 ? CurvTile<0>::X : (variant == 1 ? CurvTile<1>::X : CurvTile<2>::X);
  *y = variant == 0 ? CurvTile<0>::Y : (variant == 1 ? CurvTile<1>::Y : CurvTile<2>::Y);
}

void launch_curv_rate(int prec, const StepArgs& A, const CurvGeom& G, cudaStream_t s) {
  const unsigned blocks = std::min<unsigned>(blocks_for(A.g.ncell), 152u * 16u);
  if (prec == PREC_F64)
    curv_rate_kernel<PREC_F64><<<blocks, kCurvThreads, 0, s>>>(A, G);
  else if (prec == PREC_F32)
    curv_rate_kernel<PREC_F32><<<blocks, kCurvThreads, 0, s>>>(A, G);
  else
    curv_rate_kernel<PREC_F32D><<<blocks, kCurvThreads, 0, s>>>(A, G);
}

void launch_curv_residual(int prec, const StepArgs& A, const CurvGeom& G, const SteadyArgs& SA, cudaStream_t s) {
  // 32 x 15 tiles on grids of two or more waves of them, 16 x 11 tiles (one wave of four CTAs per SM
  // covers 107k cells) on the smaller grids and coarse multigrid levels
  const bool big = A.g.ncell >= 300000;
  if (SA.multid) {
    if (prec == PREC_F64)
      big ? launch_fused<PREC_F64, 0, 1, true>(A, G, s, SA) : launch_fused<PREC_F64, 2, 1, true>(A, G, s, SA);
    else
      big ? launch_fused<PREC_F32, 0, 1, true>(A, G, s, SA) : launch_fused<PREC_F32, 2, 1, true>(A, G, s, SA);
  } else {
    if (prec == PREC_F64)
      big ? launch_fused<PREC_F64, 0, 1>(A, G, s, SA) : launch_fused<PREC_F64, 2, 1>(A, G, s, SA);
    else
      big ? launch_fused<PREC_F32, 0, 1>(A, G, s, SA) : launch_fused<PREC_F32, 2, 1>(A, G, s, SA);
  }
}

void launch_curv_lts(int prec, const StepArgs& A, const CurvGeom& G, void* s_out, cudaStream_t s) {
  if (prec == PREC_F64)
    lts_kernel<PREC_F64><<<blocks_for(A.g.ncell), kCurvThreads, 0, s>>>(A, G, s_out);
  else
    lts_kernel<PREC_F32><<<blocks_for(A.g.ncell), kCurvThreads, 0, s>>>(A, G, s_out);
}

void launch_curv_komega(int prec, const KOmegaArgs& K, const CurvGeom& G, cudaStream_t s) {
  if (prec == PREC_F64)
    curv_komega_kernel<PREC_F64><<<kw_tiles(K.g), KwTile::T, 0, s>>>(K, G);
  else if (prec == PREC_F32)
    curv_komega_kernel<PREC_F32><<<kw_tiles(K.g), KwTile::T, 0, s>>>(K, G);
  else
    curv_komega_kernel<PREC_F32D><<<kw_tiles(K.g), KwTile::T, 0, s>>>(K, G);
}

void launch_curv_tau(int prec, const StepArgs& A, const CurvGeom& G, void* out, cudaStream_t s, int what) {
  if (prec == PREC_F64)
    curv_tau_kernel<PREC_F64><<<blocks_for(A.g.ncell), kCurvThreads, 0, s>>>(A, G, out, what);
  else if (prec == PREC_F32)
    curv_tau_kernel<PREC_F32><<<blocks_for(A.g.ncell), kCurvThreads, 0, s>>>(A, G, out, what);
  else
    curv_tau_kernel<PREC_F32D><<<blocks_for(A.g.ncell), kCurvThreads, 0, s>>>(A, G, out, what);
}

}  // namespace gks
